// Allocation-free fused SpTRSV -> SpMV (k = 1) for callers that cannot allocate device
// memory when they call (a custom allocator's own callbacks, code whose device memory is fixed
// in advance by a pool or a budget, latency-critical loops that must not wait for the
// device-wide synchronisation an allocation can cause): the scratch of the fused executor (the
// intermediate x, the launch state and the pattern-check words) lives in one file-scope device
// array, and the rows run in their natural order, so no inspector schedule is needed.
#include <algorithm>
#include <cstring>
#include <mutex>

#include "sf_exec.cuh"
#include "sf_inspect.cuh"

#define SF_API extern "C" __attribute__((visibility("default")))

namespace sf {
namespace {

constexpr size_t kHeaderBytes = 256;
static_assert(SF_NOALLOC_SCRATCH_BYTES == kHeaderBytes + 8ull * SF_NOALLOC_MAX_ROWS, "scratch layout");

struct NoallocHeader {
    ExecState st;                       // abort / error words of the launch
    unsigned long long pattern_L;       // first pattern violation of L, all ones when none
    unsigned long long pattern_M;
};
static_assert(sizeof(NoallocHeader) <= kHeaderBytes, "header fits its slot");

// The scratch: header, then x (n doubles or floats). Shared by every call on a device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[SF_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 256;
std::mutex g_mu;
void *g_scratch_addr[kMaxDevices] = {};
unsigned long long g_scratch_ctx[kMaxDevices] = {};

// Identifier of the current CUDA context (0 when the driver cannot tell): a reset of the device
// creates a new context, in which the array has a new address.
unsigned long long current_context_id() {
    using get_ctx_t = int (*)(void **);
    using get_id_t = int (*)(void *, unsigned long long *);
    static get_ctx_t get_ctx = nullptr;
    static get_id_t get_id = nullptr;
    static bool looked = false;
    if (!looked) {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_ctx = (get_ctx_t)f;
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = (get_id_t)f;
        cudaGetLastError();
        looked = true;
    }
    void *ctx = nullptr;
    unsigned long long id = 0;
    if (get_ctx && get_id && get_ctx(&ctx) == 0 && ctx && get_id(ctx, &id) == 0) return id;
    return 0;
}

// Device address of the scratch array for the current device: looked up (cudaGetSymbolAddress,
// with that device current) at the first call on the device, and again when the device's
// context has changed since (after a device reset).
cudaError_t scratch_address(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    const unsigned long long ctx = current_context_id();
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[dev] || g_scratch_ctx[dev] != ctx) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = p;
        g_scratch_ctx[dev] = ctx;
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

constexpr int kChunk = 8;   // items per partition of the natural order

// Variant of the SpTRSV -> SpMV executor (value flags, one lane per row) whose order is
// implicit: position q < n is SpTRSV row q, position n + i is SpMV row i. Partitions of
// kChunk positions go round robin to the warps of a cooperative launch. Nothing runs if
// the pattern check failed.
template <typename T>
__global__ void __launch_bounds__(kExecThreads) k_trsv_spmv_noalloc(const ExecArgs a, const NoallocHeader *h) {
    if (h->pattern_L != ~0ull || h->pattern_M != ~0ull) return;
    const int lane = threadIdx.x & 31;
    const unsigned gmask = 1u << lane;
    const long long nitems = 2LL * a.n;
    const long long nparts = (nitems + kChunk - 1) / kChunk;
    const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
    bool ok = true;
    for (long long p = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); p < nparts; p += nwarps) {
        const long long q = p * kChunk + lane;
        if (lane < kChunk && q < nitems && ok) {
            if (q < a.n) ok = item_trsv<T, 1, true>(a, (int)q, 0u, 0, gmask, (T *)a.xs);
            else ok = item_spmv_dep<T, 1, true>(a, (int)(q - a.n), 0u, 0, gmask, (const T *)a.xs);
        }
        if (!__all_sync(0xffffffffu, ok) || ld_relaxed_u32(&a.st->abort)) break;
    }
}

sf_status nfail(sf_status st, const char *msg) {
    set_error_detail(msg);
    return st;
}

}  // namespace
}  // namespace sf

using namespace sf;

SF_API sf_status sf_trsv_spmv_noalloc(sf_dtype dt, const sf_csr *L, const sf_csr *M, const void *L_vals,
                                      const void *M_vals, const void *b, void *y, void *stream) {
    if (dt != SF_F64 && dt != SF_F32) return nfail(SF_ERR_INVALID_ARG, "sf_trsv_spmv_noalloc: unknown dtype");
    if (!L || !M || !L_vals || !M_vals || !b || !y)
        return nfail(SF_ERR_INVALID_ARG, "sf_trsv_spmv_noalloc: NULL argument");
    const int n = L->n_rows;
    if (n < 1 || L->n_cols != n || M->n_rows != n || M->n_cols != n)
        return nfail(SF_ERR_INVALID_ARG, "sf_trsv_spmv_noalloc: L and M must be n x n with n >= 1");
    if (n > SF_NOALLOC_MAX_ROWS)
        return nfail(SF_ERR_INVALID_ARG, "sf_trsv_spmv_noalloc: n exceeds SF_NOALLOC_MAX_ROWS (1048576)");
    if (L->nnz < n || L->nnz >= (1LL << 31) || M->nnz < 0 || M->nnz >= (1LL << 31) || !L->rowptr || !L->colidx ||
        !M->rowptr || (M->nnz > 0 && !M->colidx))
        return nfail(SF_ERR_INVALID_ARG, "sf_trsv_spmv_noalloc: bad pattern sizes or NULL pattern arrays");
    cudaStream_t s = (cudaStream_t)stream;
    void *base = nullptr;
    cudaError_t e = scratch_address(&base);
    if (e != cudaSuccess) return nfail(SF_ERR_CUDA, "sf_trsv_spmv_noalloc: scratch address lookup failed");
    NoallocHeader *h = (NoallocHeader *)base;
    void *x = (unsigned char *)base + kHeaderBytes;
    const size_t es = dt == SF_F64 ? 8 : 4;
    // clear the state, mark "no pattern violation", reset x to the not-yet-produced pattern
    if ((e = cudaMemsetAsync(&h->st, 0, sizeof(ExecState), s)) != cudaSuccess ||
        (e = cudaMemsetAsync(&h->pattern_L, 0xff, 2 * sizeof(unsigned long long), s)) != cudaSuccess ||
        (e = cudaMemsetAsync(x, 0xff, (size_t)n * es, s)) != cudaSuccess)
        return nfail(SF_ERR_CUDA, "sf_trsv_spmv_noalloc: scratch reset failed");
    const unsigned cb = (unsigned)((n + 255) / 256);
    k_check_csr<<<cb, 256, 0, s>>>(n, n, L->nnz, L->rowptr, L->colidx, 1, &h->pattern_L);
    k_check_csr<<<cb, 256, 0, s>>>(n, n, M->nnz, M->rowptr, M->colidx, 0, &h->pattern_M);
    ExecArgs a;
    memset(&a, 0, sizeof a);
    a.n = n;
    a.k = 1;
    a.kt = 1;
    a.st = &h->st;
    a.timeout_ns = 2000000000ull;
    a.Lrp = L->rowptr;
    a.Lci = L->colidx;
    a.Mrp = M->rowptr;
    a.Mci = M->colidx;
    a.Lv = L_vals;
    a.Mv = M_vals;
    a.b = b;
    a.y = y;
    a.xs = x;
    int dev = 0, sms = 1, occ = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const void *f = dt == SF_F64 ? (const void *)k_trsv_spmv_noalloc<double> : (const void *)k_trsv_spmv_noalloc<float>;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, f, kExecThreads, 0)) != cudaSuccess)
        return nfail(SF_ERR_CUDA, "sf_trsv_spmv_noalloc: occupancy query failed");
    const long long parts = (2LL * n + kChunk - 1) / kChunk;
    long long blocks = std::min<long long>((long long)std::max(occ, 1) * sms, (parts + 7) / 8);
    blocks = std::max<long long>(blocks, 1);
    const NoallocHeader *hc = h;
    void *args[] = {(void *)&a, (void *)&hc};
    if ((e = cudaLaunchCooperativeKernel(f, dim3((unsigned)blocks), dim3(kExecThreads), args, 0, s)) != cudaSuccess)
        return nfail(SF_ERR_CUDA, "sf_trsv_spmv_noalloc: launch failed");
    NoallocHeader hh;
    if ((e = cudaMemcpyAsync(&hh, h, sizeof hh, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return nfail(SF_ERR_CUDA, "sf_trsv_spmv_noalloc: execution failed");
    if (hh.pattern_L != ~0ull) return nfail(SF_ERR_BAD_PATTERN, "sf_trsv_spmv_noalloc: invalid pattern of L");
    if (hh.pattern_M != ~0ull) return nfail(SF_ERR_BAD_PATTERN, "sf_trsv_spmv_noalloc: invalid pattern of M");
    if (hh.st.err_code) return nfail((sf_status)hh.st.err_code, "sf_trsv_spmv_noalloc: device-side failure");
    return SF_OK;
}
