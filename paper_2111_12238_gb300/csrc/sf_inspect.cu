// GPU inspector (§2.2, §3): pattern checks, CSR transposes (successor lists of the DAGs),
// wavefront levels of the joint DAG by parallel Kahn peeling, the linear order by
// (level, kernel, row) and the cut of that order into cost-balanced partitions.
//
// Building blocks are hand-written: a three-phase exclusive scan, a stable LSD radix sort
// (8-bit digits, per-block histograms, in-tile ranking with warp match), a count/scan/
// sort transpose and a cooperative persistent Kahn kernel with a bounded grid barrier.
#include <algorithm>
#include <mutex>
#include <vector>

#include "sf_inspect.cuh"

namespace sf {

// ------------------------------------------------------------------------------ arena
namespace {
constexpr int kPoolDevices = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pool[kPoolDevices];

// The library's memory pool of the current device (created on first use), or NULL.
cudaMemPool_t library_pool() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kPoolDevices) return nullptr;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pool[dev]) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t p = nullptr;
        if (cudaMemPoolCreate(&p, &props) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        unsigned long long keep = 1ull << 30;
        cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
        g_pool[dev] = p;
    }
    return g_pool[dev];
}
}  // namespace

void *Arena::alloc(size_t bytes) {
    void *p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaMemPool_t pool = pooled ? library_pool() : nullptr;
    const cudaError_t e = pool ? cudaMallocFromPoolAsync(&p, bytes, pool, stream) : cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        oom = true;
        return nullptr;
    }
    ptrs.push_back(p);
    return p;
}
Arena::~Arena() {
    // pooled memory is returned in stream order, after the work that used it
    for (void *p : ptrs) {
        if (pooled && library_pool()) cudaFreeAsync(p, stream);
        else cudaFree(p);
    }
}

static inline unsigned grid_for(long long n, int threads, long long cap = 1 << 20) {
    long long b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (unsigned)b;
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// ------------------------------------------------------------------------------ scan
constexpr int kScanT = 256, kScanI = 8, kScanTile = kScanT * kScanI;

template <typename T>
__device__ T block_excl_scan(T v, T *total) {
    __shared__ T wtot[kScanT / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    T inc = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const T t = __shfl_up_sync(0xffffffffu, inc, off);
        if (lane >= off) inc += t;
    }
    if (lane == 31) wtot[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        T w = lane < kScanT / 32 ? wtot[lane] : T(0);
#pragma unroll
        for (int off = 1; off < kScanT / 32; off <<= 1) {
            const T t = __shfl_up_sync(0xffffffffu, w, off);
            if (lane >= off) w += t;
        }
        if (lane < kScanT / 32) wtot[lane] = w;
    }
    __syncthreads();
    *total = wtot[kScanT / 32 - 1];
    return (wid > 0 ? wtot[wid - 1] : T(0)) + inc - v;
}

template <typename T>
__global__ void __launch_bounds__(kScanT) k_scan_reduce(const T *__restrict__ in, long long n, T *__restrict__ sums) {
    const long long base = (long long)blockIdx.x * kScanTile;
    T s = T(0);
#pragma unroll
    for (int i = 0; i < kScanI; ++i) {
        const long long idx = base + i * kScanT + threadIdx.x;
        if (idx < n) s += in[idx];
    }
    T tot;
    block_excl_scan<T>(s, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// exclusive scan of sums[0..nb) in place, one block
template <typename T>
__global__ void __launch_bounds__(kScanT) k_scan_top(T *sums, long long nb) {
    T carry = T(0);
    for (long long c0 = 0; c0 < nb; c0 += kScanTile) {
        T loc[kScanI];
        T s = T(0);
#pragma unroll
        for (int i = 0; i < kScanI; ++i) {
            const long long idx = c0 + (long long)threadIdx.x * kScanI + i;
            loc[i] = idx < nb ? sums[idx] : T(0);
            s += loc[i];
        }
        T tot;
        T pre = block_excl_scan<T>(s, &tot) + carry;
#pragma unroll
        for (int i = 0; i < kScanI; ++i) {
            const long long idx = c0 + (long long)threadIdx.x * kScanI + i;
            if (idx < nb) sums[idx] = pre;
            pre += loc[i];
        }
        carry += tot;
    }
}

template <typename T>
__global__ void __launch_bounds__(kScanT) k_scan_down(const T *__restrict__ in, T *__restrict__ out, long long n,
                                                      const T *__restrict__ sums) {
    const long long base = (long long)blockIdx.x * kScanTile;
    T loc[kScanI];
    T s = T(0);
#pragma unroll
    for (int i = 0; i < kScanI; ++i) {
        const long long idx = base + (long long)threadIdx.x * kScanI + i;
        loc[i] = idx < n ? in[idx] : T(0);
        s += loc[i];
    }
    T tot;
    T pre = block_excl_scan<T>(s, &tot) + sums[blockIdx.x];
#pragma unroll
    for (int i = 0; i < kScanI; ++i) {
        const long long idx = base + (long long)threadIdx.x * kScanI + i;
        if (idx < n) out[idx] = pre;
        pre += loc[i];
        if (idx == n - 1) out[n] = pre;
    }
}

template <typename T>
__global__ void k_set_zero1(T *out) { out[0] = T(0); }

template <typename T>
cudaError_t scan_excl(const T *in, T *out, long long n, cudaStream_t s, Arena &ar) {
    if (n <= 0) {
        k_set_zero1<T><<<1, 1, 0, s>>>(out);
        return cudaGetLastError();
    }
    const long long nb = (n + kScanTile - 1) / kScanTile;
    T *sums = (T *)ar.alloc(sizeof(T) * nb);
    if (!sums) return cudaErrorMemoryAllocation;
    k_scan_reduce<T><<<(unsigned)nb, kScanT, 0, s>>>(in, n, sums);
    k_scan_top<T><<<1, kScanT, 0, s>>>(sums, nb);
    k_scan_down<T><<<(unsigned)nb, kScanT, 0, s>>>(in, out, n, sums);
    return cudaGetLastError();
}
template cudaError_t scan_excl<int>(const int *, int *, long long, cudaStream_t, Arena &);
template cudaError_t scan_excl<long long>(const long long *, long long *, long long, cudaStream_t, Arena &);

// ------------------------------------------------------------------------------ radix sort
constexpr int kRsT = 256, kRsR = 16, kRsTile = kRsT * kRsR;

__global__ void __launch_bounds__(kRsT) k_radix_hist(const unsigned *__restrict__ keys, long long n, int shift,
                                                     int *__restrict__ hist, int nb) {
    __shared__ unsigned h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const long long base = (long long)blockIdx.x * kRsTile;
#pragma unroll 4
    for (int r = 0; r < kRsR; ++r) {
        const long long idx = base + r * kRsT + threadIdx.x;
        if (idx < n) atomicAdd(&h[(keys[idx] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(long long)threadIdx.x * nb + blockIdx.x] = (int)h[threadIdx.x];
}

// Stable scatter: element order inside a tile is (round, warp, lane); the rank of an
// element among equal digits is the count of earlier rounds, earlier warps of this round
// and lower lanes of this warp.
__global__ void __launch_bounds__(kRsT) k_radix_scatter(const unsigned *__restrict__ kin,
                                                        const unsigned *__restrict__ vin,
                                                        unsigned *__restrict__ kout, unsigned *__restrict__ vout,
                                                        long long n, int shift, const int *__restrict__ hscan,
                                                        int nb) {
    __shared__ unsigned run[256];
    __shared__ unsigned wcnt[kRsT / 32][256];
    __shared__ unsigned gofs[256];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    gofs[tid] = (unsigned)hscan[(long long)tid * nb + blockIdx.x];
    run[tid] = 0;
#pragma unroll
    for (int w = 0; w < kRsT / 32; ++w) wcnt[w][tid] = 0;
    __syncthreads();
    const long long base = (long long)blockIdx.x * kRsTile;
    for (int r = 0; r < kRsR; ++r) {
        const long long idx = base + r * kRsT + tid;
        const bool valid = idx < n;
        const unsigned key = valid ? kin[idx] : 0u;
        const unsigned d = (key >> shift) & 255u;
        const unsigned peers = __match_any_sync(0xffffffffu, valid ? d : 256u + lane);
        const unsigned rank = __popc(peers & lanemask_lt());
        if (valid && rank == 0) wcnt[wid][d] = __popc(peers);
        __syncthreads();
        if (valid) {
            unsigned off = run[d] + rank;
            for (int w = 0; w < wid; ++w) off += wcnt[w][d];
            const unsigned pos = gofs[d] + off;
            kout[pos] = key;
            vout[pos] = vin[idx];
        }
        __syncthreads();
        unsigned t = 0;
#pragma unroll
        for (int w = 0; w < kRsT / 32; ++w) {
            t += wcnt[w][tid];
            wcnt[w][tid] = 0;
        }
        run[tid] += t;
        __syncthreads();
    }
}

int bits_for(unsigned long long maxval) {
    int b = 0;
    while (b < 64 && (maxval >> b) != 0) ++b;
    return b;
}

cudaError_t radix_sort_pairs(unsigned *keys, unsigned *vals, long long n, int bits, cudaStream_t s, Arena &ar) {
    if (n <= 1 || bits <= 0) return cudaSuccess;
    const int nb = (int)((n + kRsTile - 1) / kRsTile);
    unsigned *k2 = (unsigned *)ar.alloc(sizeof(unsigned) * n);
    unsigned *v2 = (unsigned *)ar.alloc(sizeof(unsigned) * n);
    int *hist = (int *)ar.alloc(sizeof(int) * 256 * (size_t)nb);
    int *hscan = (int *)ar.alloc(sizeof(int) * (256 * (size_t)nb + 1));
    if (!k2 || !v2 || !hist || !hscan) return cudaErrorMemoryAllocation;
    unsigned *ki = keys, *vi = vals, *ko = k2, *vo = v2;
    for (int shift = 0; shift < bits; shift += 8) {
        k_radix_hist<<<nb, kRsT, 0, s>>>(ki, n, shift, hist, nb);
        cudaError_t e = scan_excl<int>(hist, hscan, 256LL * nb, s, ar);
        if (e != cudaSuccess) return e;
        k_radix_scatter<<<nb, kRsT, 0, s>>>(ki, vi, ko, vo, n, shift, hscan, nb);
        unsigned *t = ki; ki = ko; ko = t;
        t = vi; vi = vo; vo = t;
    }
    if (ki != keys) {
        cudaMemcpyAsync(keys, ki, sizeof(unsigned) * n, cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(vals, vi, sizeof(unsigned) * n, cudaMemcpyDeviceToDevice, s);
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------ patterns
// First violation per matrix as (code << 32 | row), minimised over rows.
__device__ __forceinline__ void report_pattern(unsigned long long *status, unsigned code, int row) {
    atomicMin(status, ((unsigned long long)code << 32) | (unsigned)row);
}

__global__ void k_check_csr(int n_rows, int n_cols, long long nnz, const int *__restrict__ rp,
                            const int *__restrict__ ci, int lower, unsigned long long *status) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_rows) return;
    if (i == 0 && rp[0] != 0) report_pattern(status, PAT_ROWPTR0, 0);
    if (i == n_rows - 1 && rp[n_rows] != nnz) report_pattern(status, PAT_NNZ, (int)i);
    const int a = rp[i], b = rp[i + 1];
    if (b < a || a < 0 || b > nnz) {
        report_pattern(status, PAT_ROWPTR, (int)i);
        return;
    }
    for (int e = a; e < b; ++e) {
        const int c = ci[e];
        if (c < 0 || c >= n_cols) { report_pattern(status, PAT_COL_RANGE, (int)i); return; }
        if (e > a && ci[e - 1] >= c) { report_pattern(status, PAT_UNSORTED, (int)i); return; }
    }
    if (lower && (b == a || ci[b - 1] != i)) report_pattern(status, PAT_DIAG, (int)i);
}

__global__ void k_row_of(int n, const int *__restrict__ rp, int *__restrict__ row_of) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int e = rp[i]; e < rp[i + 1]; ++e) row_of[e] = (int)i;
}

__global__ void k_count_cols(long long nnz, const int *__restrict__ ci, int *__restrict__ cnt) {
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (long long)gridDim.x * blockDim.x)
        atomicAdd(&cnt[ci[e]], 1);
}

__global__ void k_iota(long long n, unsigned *__restrict__ v) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        v[i] = (unsigned)i;
}

__global__ void k_gather_rows(long long nnz, const unsigned *__restrict__ perm, const int *__restrict__ row_of,
                              int *__restrict__ tci, int *__restrict__ tperm) {
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < nnz; t += (long long)gridDim.x * blockDim.x) {
        const unsigned e = perm[t];
        tci[t] = row_of[e];
        tperm[t] = (int)e;
    }
}

cudaError_t transpose_csr(const DevCsr &src, DevCsrT &dst, cudaStream_t s, Arena &ar, Arena &keep) {
    const long long nnz = src.nnz;
    dst.t.n_rows = src.n_cols;
    dst.t.n_cols = src.n_rows;
    dst.t.nnz = nnz;
    dst.t.rowptr = (int *)keep.alloc(sizeof(int) * ((size_t)src.n_cols + 1));
    dst.t.colidx = (int *)keep.alloc(sizeof(int) * (size_t)(nnz > 0 ? nnz : 1));
    dst.perm = (int *)keep.alloc(sizeof(int) * (size_t)(nnz > 0 ? nnz : 1));
    int *cnt = (int *)ar.alloc(sizeof(int) * ((size_t)src.n_cols + 1));
    int *row_of = (int *)ar.alloc(sizeof(int) * (size_t)(nnz > 0 ? nnz : 1));
    unsigned *keys = (unsigned *)ar.alloc(sizeof(unsigned) * (size_t)(nnz > 0 ? nnz : 1));
    unsigned *vals = (unsigned *)ar.alloc(sizeof(unsigned) * (size_t)(nnz > 0 ? nnz : 1));
    if (!dst.t.rowptr || !dst.t.colidx || !dst.perm || !cnt || !row_of || !keys || !vals)
        return cudaErrorMemoryAllocation;
    cudaMemsetAsync(cnt, 0, sizeof(int) * ((size_t)src.n_cols + 1), s);
    if (nnz > 0) {
        k_count_cols<<<grid_for(nnz, 256, 4096), 256, 0, s>>>(nnz, src.colidx, cnt);
        k_row_of<<<grid_for(src.n_rows, 256), 256, 0, s>>>(src.n_rows, src.rowptr, row_of);
    }
    cudaError_t e = scan_excl<int>(cnt, dst.t.rowptr, src.n_cols, s, ar);
    if (e != cudaSuccess) return e;
    if (nnz > 0) {
        cudaMemcpyAsync(keys, src.colidx, sizeof(int) * nnz, cudaMemcpyDeviceToDevice, s);
        k_iota<<<grid_for(nnz, 256, 4096), 256, 0, s>>>(nnz, vals);
        e = radix_sort_pairs(keys, vals, nnz, bits_for(src.n_cols > 0 ? (unsigned long long)src.n_cols - 1 : 0), s, ar);
        if (e != cudaSuccess) return e;
        k_gather_rows<<<grid_for(nnz, 256, 4096), 256, 0, s>>>(nnz, vals, row_of, dst.t.colidx, dst.perm);
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------ Kahn
// In-degree of every joint-DAG vertex: one count per edge of the successor lists.
__global__ void k_indeg(int n1, const int *__restrict__ s1rp, const int *__restrict__ s1ci,
                        const int *__restrict__ s2rp, const int *__restrict__ s2ci, int *__restrict__ indeg) {
    const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n1) return;
    for (int e = s1rp[v]; e < s1rp[v + 1]; ++e) {
        const int t = s1ci[e];
        if (t != v) atomicAdd(&indeg[t], 1);
    }
    if (s2rp)
        for (int e = s2rp[v]; e < s2rp[v + 1]; ++e) atomicAdd(&indeg[n1 + s2ci[e]], 1);
}

__global__ void k_sources(long long nv, const int *__restrict__ indeg, int *__restrict__ queue, KahnCtl *ctl) {
    const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool src = v < nv && indeg[v] == 0;
    const unsigned m = __ballot_sync(0xffffffffu, src);
    if (!m) return;
    const int lane = threadIdx.x & 31;
    unsigned base = 0;
    if (lane == __ffs(m) - 1) base = atomicAdd(&ctl->nsrc, (unsigned)__popc(m));
    base = __shfl_sync(0xffffffffu, base, __ffs(m) - 1);
    if (src) queue[base + __popc(m & lanemask_lt())] = (int)v;
}

// Grid-wide barrier for a cooperative launch, bounded by a spin limit: returns false
// (and sets ctl->err) if the other blocks do not arrive in time.
__device__ bool grid_barrier(KahnCtl *ctl, unsigned nblocks, unsigned long long tmo) {
    __syncthreads();
    bool ok = true;
    if (threadIdx.x == 0) {
        const unsigned gen = ld_acquire_u32(&ctl->bar_gen);
        const unsigned arrived = atom_add_acq_rel_u32(&ctl->bar_count, 1u);
        if (arrived == nblocks - 1u) {
            st_relaxed_u32(&ctl->bar_count, 0u);
            st_release_u32(&ctl->bar_gen, gen + 1u);
        } else {
            const unsigned long long t0 = global_ns();
            unsigned it = 0, ns = 32;
            while (ld_acquire_u32(&ctl->bar_gen) == gen) {
                __nanosleep(ns);
                if (ns < 256) ns *= 2;
                if ((++it & 63u) == 0u && global_ns() - t0 > tmo) {
                    atomicExch(&ctl->err, 1u);
                    ok = false;
                    break;
                }
            }
        }
    }
    return __syncthreads_and(ok) != 0;
}

constexpr int kKahnBatch = 8;      // successors per thread whose in-degree atomics are in flight together
constexpr int kKahnThreads = 256;
constexpr int kKahnGroup = 8;      // lanes per frontier vertex (a warp expands four at a time)
constexpr int kKahnLongDeg = 32 * kKahnBatch;   // longer successor lists are expanded by the whole block
constexpr int kKahnMaxLong = 64;   // long vertices a block collects per round (more: expanded by their warp)

// One batch of a frontier vertex's successors: entries k = k_first + stride * u (u <
// kKahnBatch, k < deg) of the concatenated successor lists (first s1ci[a1 .. a1 + deg1), the
// diagonal entry `self` skipped; then s2ci[a2 ..], offset by n1). Decrements each successor's
// in-degree (all atomics in flight before any result is looked at) and appends those that
// reach zero to the next frontier; the appends of a warp share one atomic on the frontier
// counter. Every lane of the calling warp takes part.
__device__ __forceinline__ void kahn_batch(int k_first, int stride, int deg1, int deg, const int *__restrict__ s1ci,
                                           int a1, int self, const int *__restrict__ s2ci, int a2, int n1,
                                           int *__restrict__ indeg, int *__restrict__ queue, long long fe,
                                           unsigned *cnt) {
    const int lane = threadIdx.x & 31;
    int t[kKahnBatch];
#pragma unroll
    for (int u = 0; u < kKahnBatch; ++u) {
        const int k = k_first + stride * u;
        t[u] = -1;
        if (k < deg1) {
            const int c = s1ci[a1 + k];
            if (c != self) t[u] = c;
        } else if (k < deg) {
            t[u] = n1 + s2ci[a2 + k - deg1];
        }
    }
    bool rd[kKahnBatch];
#pragma unroll
    for (int u = 0; u < kKahnBatch; ++u) rd[u] = t[u] >= 0 && atomicSub(&indeg[t[u]], 1) == 1;
    int mine = 0;
#pragma unroll
    for (int u = 0; u < kKahnBatch; ++u) mine += rd[u] ? 1 : 0;
    // inclusive prefix sum of `mine` over the warp, one append per batch
    int incl = mine;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += y;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    if (total == 0) return;
    unsigned base = 0;
    if (lane == 31) base = atomicAdd(cnt, (unsigned)total);
    base = __shfl_sync(0xffffffffu, base, 31);
    long long pos = fe + base + (incl - mine);
#pragma unroll
    for (int u = 0; u < kKahnBatch; ++u)
        if (rd[u]) queue[pos++] = t[u];
}

// Frontier peeling: round r owns the vertices whose last predecessor was removed in
// round r-1 (its level is r); removing a vertex decrements its successors' in-degrees and
// appends those that reach zero to the next frontier. A warp expands four frontier vertices at
// a time, eight lanes splitting each successor list; a vertex with more than kKahnLongDeg
// successors is set aside and expanded by all the threads of the block once the block's warps
// are done, so one long row costs a few atomic round trips instead of one per 64 successors. Counters of
// the next frontier are triple-buffered so that no block reads a count while another resets it.
__global__ void __launch_bounds__(kKahnThreads) k_kahn(int n1, const int *__restrict__ s1rp, const int *__restrict__ s1ci,
                                                       const int *__restrict__ s2rp, const int *__restrict__ s2ci,
                                                       int *__restrict__ indeg, int *__restrict__ queue,
                                                       int *__restrict__ level, KahnCtl *ctl, unsigned long long tmo) {
    __shared__ int s_long[kKahnMaxLong];
    __shared__ int s_nlong;
    const unsigned nblocks = gridDim.x;
    const int lane = threadIdx.x & 31;
    const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long gwarp = gtid >> 5;
    const long long nwarp = ((long long)gridDim.x * blockDim.x) >> 5;
    long long fs = 0, fe = (long long)ld_acquire_u32(&ctl->nsrc);
    int round = 0;
    if (threadIdx.x == 0) s_nlong = 0;
    __syncthreads();
    while (fs < fe) {
        unsigned *cnt = &ctl->cnt[round % 3];
        // a warp takes 32 / G frontier vertices at a time, G lanes each; every warp-wide
        // operation below (the shuffles, kahn_batch) is reached by all 32 lanes
        constexpr int G = kKahnGroup, VPW = 32 / G;
        const int sub = lane / G, gl = lane % G;
        for (long long base = fs + gwarp * VPW; base < fe; base += nwarp * VPW) {
            const long long idx = base + sub;
            int v = -1, a1 = 0, deg1 = 0, a2 = 0, deg = 0;
            if (idx < fe) {
                v = queue[idx];
                if (gl == 0) level[v] = round;
                if (v < n1) {
                    a1 = s1rp[v];
                    deg1 = s1rp[v + 1] - a1;
                    deg = deg1;
                    if (s2rp) {
                        a2 = s2rp[v];
                        deg += s2rp[v + 1] - a2;
                    }
                }
            }
            // a long list goes to the whole block: the group's first lane claims a slot, and
            // the group then expands nothing of it
            int slot = kKahnMaxLong;
            if (deg > kKahnLongDeg && gl == 0) {
                slot = atomicAdd(&s_nlong, 1);
                if (slot < kKahnMaxLong) s_long[slot] = v;
            }
            slot = __shfl_sync(0xffffffffu, slot, sub * G);
            if (deg > kKahnLongDeg && slot < kKahnMaxLong) deg = deg1 = 0;
            int maxdeg = deg;
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) maxdeg = max(maxdeg, __shfl_xor_sync(0xffffffffu, maxdeg, o));
            for (int k0 = 0; k0 < maxdeg; k0 += G * kKahnBatch)
                kahn_batch(k0 + gl, G, deg1, deg, s1ci, a1, v, s2ci, a2, n1, indeg, queue, fe, cnt);
        }
        __syncthreads();
        const int nl = min(s_nlong, kKahnMaxLong);
        for (int i = 0; i < nl; ++i) {
            const int v = s_long[i];
            const int a1 = s1rp[v], deg1 = s1rp[v + 1] - a1;
            const int a2 = s2rp ? s2rp[v] : 0, deg = deg1 + (s2rp ? s2rp[v + 1] - a2 : 0);
            for (int k0 = 0; k0 < deg; k0 += kKahnThreads * kKahnBatch)
                kahn_batch(k0 + (int)threadIdx.x, kKahnThreads, deg1, deg, s1ci, a1, v, s2ci, a2, n1, indeg, queue, fe,
                           cnt);
        }
        __syncthreads();
        if (threadIdx.x == 0) s_nlong = 0;
        if (gtid == 0) ctl->cnt[(round + 1) % 3] = 0u;
        if (!grid_barrier(ctl, nblocks, tmo)) return;
        const long long nf = (long long)ld_acquire_u32(cnt);
        fs = fe;
        fe += nf;
        ++round;
    }
    if (gtid == 0) {
        ctl->depth = (unsigned)round;
        ctl->processed = (unsigned)fe;
    }
}

cudaError_t kahn_levels(long long nv, int n1, const int *s1rp, const int *s1ci, const int *s2rp, const int *s2ci,
                        int *level, int *depth_out, cudaStream_t s, Arena &ar, bool *timed_out) {
    *timed_out = false;
    int *indeg = (int *)ar.alloc(sizeof(int) * nv);
    int *queue = (int *)ar.alloc(sizeof(int) * nv);
    KahnCtl *ctl = (KahnCtl *)ar.alloc(sizeof(KahnCtl));
    if (!indeg || !queue || !ctl) return cudaErrorMemoryAllocation;
    cudaMemsetAsync(indeg, 0, sizeof(int) * nv, s);
    cudaMemsetAsync(ctl, 0, sizeof(KahnCtl), s);
    k_indeg<<<grid_for(n1, 256), 256, 0, s>>>(n1, s1rp, s1ci, s2rp, s2ci, indeg);
    k_sources<<<grid_for(nv, 256), 256, 0, s>>>(nv, indeg, queue, ctl);
    int dev = 0, sms = 0, occ = 0, coop = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (!coop) return cudaErrorNotSupported;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_kahn, 256, 0);
    if (e != cudaSuccess) return e;
    if (occ < 1) occ = 1;
    long long want = (nv + 255) / 256;
    long long blocks = (long long)sms * std::min(occ, 2);   // fewer arrivals per barrier
    if (blocks > want) blocks = want;
    if (blocks < 1) blocks = 1;
    unsigned long long tmo = 5000000000ull;   // 5 s per barrier
    void *args[] = {(void *)&n1, (void *)&s1rp, (void *)&s1ci, (void *)&s2rp, (void *)&s2ci, (void *)&indeg,
                    (void *)&queue, (void *)&level, (void *)&ctl, (void *)&tmo};
    e = cudaLaunchCooperativeKernel((const void *)k_kahn, dim3((unsigned)blocks), dim3(256), args, 0, s);
    if (e != cudaSuccess) return e;
    KahnCtl h;
    e = cudaMemcpyAsync(&h, ctl, sizeof(KahnCtl), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return e;
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    if (h.err) {
        *timed_out = true;
        return cudaSuccess;
    }
    if ((long long)h.processed != nv) return cudaErrorInvalidValue;   // a cycle: impossible for valid input
    *depth_out = (int)h.depth;
    return cudaSuccess;
}

// ------------------------------------------------------------------------------ order, costs, cut
__global__ void k_level_keys(long long nv, const int *__restrict__ level, unsigned *__restrict__ keys,
                             unsigned *__restrict__ vals) {
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += (long long)gridDim.x * blockDim.x) {
        keys[v] = (unsigned)level[v];
        vals[v] = (unsigned)v;
    }
}

__global__ void k_encode_order(long long nv, int n1, const unsigned *__restrict__ vids, int *__restrict__ order) {
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < nv; q += (long long)gridDim.x * blockDim.x) {
        const unsigned v = vids[q];
        order[q] = (int)(v < (unsigned)n1 ? v : ((v - (unsigned)n1) | 0x80000000u));
    }
}

// c(v) of §3.1 (nonzeros touched by the iteration) + 1 (adjoint items exclude the value
// gradients, which run as a separate streaming pass); formulas per `what`:
// 0 SEP, 1 PAIRED_T, 2 SEP_T, 3 SpMV->SpTRSV, 4 SpIC0->SpTRSV, 5 SpTRSV, 6 SpIC0,
// 7 SpTRSV->SpTRSV (the row of L twice), 8 SpILU0->SpTRSV (row i of A, the rows of A it
// eliminates with, and the solve row).
__global__ void k_costs(int what, int n, const int *__restrict__ Lrp, const int *__restrict__ Lci,
                        const int *__restrict__ Mrp, const int *__restrict__ LTrp, const int *__restrict__ MTrp,
                        int *__restrict__ cost) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int nl = Lrp[i + 1] - Lrp[i];
    const int nm = Mrp ? Mrp[i + 1] - Mrp[i] : 0;
    const int cl = LTrp ? LTrp[i + 1] - LTrp[i] : 0;
    const int cm = MTrp ? MTrp[i + 1] - MTrp[i] : 0;
    int sj = 0;
    if (what == 4 || what == 6)
        for (int e = Lrp[i]; e < Lrp[i + 1] - 1; ++e) {
            const int j = Lci[e];
            sj += Lrp[j + 1] - Lrp[j];
        }
    if (what == 8)
        for (int e = Lrp[i]; e < Lrp[i + 1] - 1; ++e) {
            const int j = Lci[e];
            sj += Mrp[j + 1] - Mrp[j];
        }
    switch (what) {
        case 0: cost[i] = nl + 1; cost[n + i] = nm + 1; break;
        case 1: cost[i] = cm + cl + 1; break;
        case 2: cost[i] = cl + 1; cost[n + i] = cm + 1; break;
        case 3: cost[i] = nm + nl + 1; break;
        case 4: cost[i] = 2 * nl + sj + 1; break;
        case 5: cost[i] = nl + 1; break;
        case 7: cost[i] = 2 * nl + 1; break;
        case 8: cost[i] = nm + sj + nl + 1; break;
        default: cost[i] = nl + sj + 1; break;
    }
}

__global__ void k_gather_cost(long long nv, int n1, const int *__restrict__ order, const int *__restrict__ cost,
                              long long *__restrict__ cs) {
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < nv; q += (long long)gridDim.x * blockDim.x) {
        const unsigned o = (unsigned)order[q];
        cs[q] = cost[(long long)(o >> 31) * n1 + (o & 0x7fffffffu)];
    }
}

// A partition starts where floor(S_q / C) changes, and around every wide item (cost > W,
// W > 0), which gets a partition of its own.
__global__ void k_cut_flags(long long nv, const long long *__restrict__ S, const long long *__restrict__ cs,
                            long long C, long long W, int *__restrict__ f) {
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < nv; q += (long long)gridDim.x * blockDim.x) {
        const bool wide = W > 0 && cs[q] > W;
        const bool prev_wide = q > 0 && W > 0 && cs[q - 1] > W;
        f[q] = (q == 0 || S[q] / C != S[q - 1] / C || wide || prev_wide) ? 1 : 0;
    }
}

__global__ void k_cut_scatter(long long nv, const int *__restrict__ f, const int *__restrict__ idx,
                              const long long *__restrict__ cs, long long W, int *__restrict__ part_ptr,
                              unsigned char *__restrict__ part_wide) {
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < nv; q += (long long)gridDim.x * blockDim.x) {
        if (f[q]) {
            part_ptr[idx[q]] = (int)q;
            part_wide[idx[q]] = (W > 0 && cs[q] > W) ? 1 : 0;
        }
        if (q == 0) part_ptr[idx[nv]] = (int)nv;
    }
}

cudaError_t build_order(long long nv, int n1, const int *level, int depth, int *order, cudaStream_t s, Arena &ar) {
    unsigned *keys = (unsigned *)ar.alloc(sizeof(unsigned) * nv);
    unsigned *vals = (unsigned *)ar.alloc(sizeof(unsigned) * nv);
    if (!keys || !vals) return cudaErrorMemoryAllocation;
    k_level_keys<<<grid_for(nv, 256, 4096), 256, 0, s>>>(nv, level, keys, vals);
    cudaError_t e = radix_sort_pairs(keys, vals, nv, bits_for(depth > 0 ? (unsigned long long)depth - 1 : 0), s, ar);
    if (e != cudaSuccess) return e;
    k_encode_order<<<grid_for(nv, 256, 4096), 256, 0, s>>>(nv, n1, vals, order);
    return cudaGetLastError();
}

cudaError_t vertex_costs(int what, int n, const DevCsr &L, const DevCsr *M, const DevCsrT *LT, const DevCsrT *MT,
                         int *cost, cudaStream_t s) {
    k_costs<<<grid_for(n, 256), 256, 0, s>>>(what, n, L.rowptr, L.colidx, M ? M->rowptr : nullptr,
                                             LT ? LT->t.rowptr : nullptr, MT ? MT->t.rowptr : nullptr, cost);
    return cudaGetLastError();
}

cudaError_t prefix_costs(long long nv, int n1, const int *order, const int *cost, long long *cs, long long *S,
                         long long *total, cudaStream_t s, Arena &ar) {
    k_gather_cost<<<grid_for(nv, 256, 4096), 256, 0, s>>>(nv, n1, order, cost, cs);
    cudaError_t e = scan_excl<long long>(cs, S, nv, s, ar);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(total, S + nv, sizeof(long long), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(s);
}

cudaError_t cut_partitions(long long nv, const long long *S, const long long *cs, long long C, long long W,
                           int *part_ptr_out_capacity_nv1, unsigned char *part_wide, int *n_parts, cudaStream_t s,
                           Arena &ar) {
    int *f = (int *)ar.alloc(sizeof(int) * nv);
    int *idx = (int *)ar.alloc(sizeof(int) * (nv + 1));
    if (!f || !idx) return cudaErrorMemoryAllocation;
    k_cut_flags<<<grid_for(nv, 256, 4096), 256, 0, s>>>(nv, S, cs, C, W, f);
    cudaError_t e = scan_excl<int>(f, idx, nv, s, ar);
    if (e != cudaSuccess) return e;
    k_cut_scatter<<<grid_for(nv, 256, 4096), 256, 0, s>>>(nv, f, idx, cs, W, part_ptr_out_capacity_nv1, part_wide);
    e = cudaMemcpyAsync(n_parts, idx + nv, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(s);
}

// Placement of the second kernel's vertices of a separated schedule by their slack (§3.2.2):
// they are sinks of the joint DAG, so mode < 0 moves them to the last wavefront, mode d > 0
// delays them by d wavefronts (at most to the last); the first kernel's levels stay.
__global__ void k_place_g2(int n, int depth, int mode, int *__restrict__ level) {
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        int *l = level + n + t;
        const long long v = mode < 0 ? (long long)depth - 1 : (long long)*l + mode;
        *l = (int)(v < depth - 1 ? v : depth - 1);
    }
}

cudaError_t place_g2(int n, int depth, int mode, int *level, cudaStream_t s) {
    if (mode == 0) return cudaSuccess;
    k_place_g2<<<grid_for(n, 256, 4096), 256, 0, s>>>(n, depth, mode, level);
    return cudaGetLastError();
}

// Zero-fill IC0 (§2.1, up-looking form): entry (i, j), j < i, subtracts the sum of L_ik L_jk
// over the columns k < j present in both rows i and j. Those columns follow from the pattern
// alone, so the inspector lists them once: for every entry t = (i, j), the pairs (p, q) of
// entry positions with column k in row i (p < t) and in row j (q before row j's diagonal),
// in increasing k. One warp per row, lanes over the row's off-diagonal entries, each a merge
// of two sorted column lists.
template <bool FILL>
__global__ void k_ic0_pairs(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                            long long *__restrict__ cnt, const long long *__restrict__ off, int2 *__restrict__ pairs) {
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long i = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += warps) {
        const int rs = rp[i], dg = rp[i + 1] - 1;
        for (int t = rs + lane; t < dg; t += 32) {
            const int j = ci[t];
            int p = rs, q = rp[j];
            const int qe = rp[j + 1] - 1;   // row j's diagonal is its last entry
            long long c = 0, w = FILL ? off[t] : 0;
            while (p < t && q < qe) {
                const int cp = ci[p], cq = ci[q];
                if (cp == cq) {
                    if (FILL) pairs[w++] = make_int2(p, q);
                    else ++c;
                    ++p;
                    ++q;
                } else if (cp < cq) {
                    ++p;
                } else {
                    ++q;
                }
            }
            if (!FILL) cnt[t] = c;
        }
        if (!FILL && lane == 0) cnt[dg] = 0;
    }
}

__global__ void k_narrow_offsets(long long m, const long long *__restrict__ in, int *__restrict__ out) {
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < m; t += (long long)gridDim.x * blockDim.x)
        out[t] = (int)in[t];
}

cudaError_t build_ic0_pairs(const DevCsr &L, long long max_pairs, int **pp_out, int2 **pairs_out, long long *np_out,
                            cudaStream_t s, Arena &ar, Arena &keep) {
    *pp_out = nullptr;
    *pairs_out = nullptr;
    *np_out = 0;
    const long long nnz = L.nnz;
    if (L.n_rows <= 0 || nnz <= 0) return cudaSuccess;
    long long *cnt = (long long *)ar.alloc(sizeof(long long) * (nnz + 1));
    long long *off = (long long *)ar.alloc(sizeof(long long) * (nnz + 1));
    if (!cnt || !off) return cudaErrorMemoryAllocation;
    const unsigned g = grid_for((long long)L.n_rows * 32, 256, 8192);
    k_ic0_pairs<false><<<g, 256, 0, s>>>(L.n_rows, L.rowptr, L.colidx, cnt, nullptr, nullptr);
    cudaError_t e = cudaMemsetAsync(cnt + nnz, 0, sizeof(long long), s);
    if (e != cudaSuccess) return e;
    e = scan_excl<long long>(cnt, off, nnz + 1, s, ar);
    if (e != cudaSuccess) return e;
    long long total = 0;
    e = cudaMemcpyAsync(&total, off + nnz, sizeof(long long), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    *np_out = total;
    if (total > max_pairs || total > 0x7fffffffLL) return cudaSuccess;   // too many: searched per call instead
    int *pp = (int *)keep.alloc(sizeof(int) * (nnz + 1));
    int2 *pairs = (int2 *)keep.alloc(sizeof(int2) * std::max<long long>(total, 1));
    if (!pp || !pairs) return cudaErrorMemoryAllocation;
    k_narrow_offsets<<<grid_for(nnz + 1, 256, 4096), 256, 0, s>>>(nnz + 1, off, pp);
    if (total > 0) k_ic0_pairs<true><<<g, 256, 0, s>>>(L.n_rows, L.rowptr, L.colidx, nullptr, off, pairs);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    *pp_out = pp;
    *pairs_out = pairs;
    return cudaStreamSynchronize(s);
}

// Partition classes of a separated schedule: class 1 when the partition's first vertex is a
// second-kernel row (a sink of the joint DAG), else class 0. plist lists the class-0
// partitions in increasing order, then the class-1 partitions in increasing order.
__global__ void k_part_class(int P, const int *__restrict__ part_ptr, const int *__restrict__ order, int *__restrict__ f0) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x)
        f0[p] = ((unsigned)order[part_ptr[p]] >> 31) ? 0 : 1;
}

__global__ void k_part_list(int P, const int *__restrict__ f0, const int *__restrict__ pos0, int *__restrict__ plist) {
    const int P0 = pos0[P];
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x)
        plist[f0[p] ? pos0[p] : P0 + (p - pos0[p])] = p;
}

cudaError_t split_partition_classes(int P, const int *part_ptr, const int *order, int *plist, int *n_class0,
                                    cudaStream_t s, Arena &ar) {
    int *f0 = (int *)ar.alloc(sizeof(int) * ((size_t)P + 1));
    int *pos0 = (int *)ar.alloc(sizeof(int) * ((size_t)P + 1));
    if (!f0 || !pos0) return cudaErrorMemoryAllocation;
    k_part_class<<<grid_for(P, 256, 4096), 256, 0, s>>>(P, part_ptr, order, f0);
    cudaError_t e = scan_excl<int>(f0, pos0, P, s, ar);
    if (e != cudaSuccess) return e;
    k_part_list<<<grid_for(P, 256, 4096), 256, 0, s>>>(P, f0, pos0, plist);
    e = cudaMemcpyAsync(n_class0, pos0 + P, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(s);
}

// ------------------------------------------------------------------------------ row blocks
// Instance of row i: the t with inst_ptr[t] <= i < inst_ptr[t + 1].
__device__ __forceinline__ int instance_of(int i, const int *__restrict__ inst_ptr, int n_inst) {
    int lo = 0, hi = n_inst - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (inst_ptr[mid] <= i) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Block of every vertex for the row-block executor: first-kernel rows by their own row
// (decreasing row order for the transposed kinds), second-kernel rows by the latest block
// among the rows they read (columns ascend, so that is the last column of an M row, or the
// first row of an A^T row when blocks run in decreasing row order). With inst_ptr, the blocks
// are the independent instances of a block-diagonal system instead, every vertex in the block
// of its row's instance. key = block*depth+level.
__global__ void k_block_keys(int kind, int n, long long nv, int B, int nb, int depth, const int *__restrict__ level,
                             const int *__restrict__ Mrp, const int *__restrict__ Mci,
                             const int *__restrict__ MTrp, const int *__restrict__ MTci,
                             const int *__restrict__ inst_ptr, unsigned *__restrict__ keys,
                             unsigned *__restrict__ vals) {
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += (long long)gridDim.x * blockDim.x) {
        const bool rev = kind == K_PAIRED_T || kind == K_SEP_T;
        long long b;
        if (inst_ptr) {
            b = instance_of((int)(v < n ? v : v - n), inst_ptr, nb);
        } else if (v < n) {
            b = rev ? nb - 1 - v / B : v / B;
        } else {
            const int i = (int)(v - n);
            if (kind == K_SEP) {
                const int e0 = Mrp[i], e1 = Mrp[i + 1];
                b = e1 > e0 ? Mci[e1 - 1] / B : 0;
            } else {   // K_SEP_T
                const int e0 = MTrp[i], e1 = MTrp[i + 1];
                b = e1 > e0 ? nb - 1 - MTci[e0] / B : 0;
            }
        }
        keys[v] = (unsigned)(b * depth + level[v]);
        vals[v] = (unsigned)v;
    }
}

// First position of every block in the sorted keys (block b's keys are b*depth .. b*depth +
// depth - 1): a binary search per block, block_ptr[nb] = nv.
__global__ void k_block_ptr(int nb, long long nv, unsigned depth, const unsigned *__restrict__ keys,
                            int *__restrict__ block_ptr) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b <= nb; b += gridDim.x * blockDim.x) {
        if (b == nb) {
            block_ptr[b] = (int)nv;
            continue;
        }
        const unsigned key = (unsigned)b * depth;
        long long lo = 0, hi = nv;
        while (lo < hi) {
            const long long mid = (lo + hi) >> 1;
            if (keys[mid] < key) lo = mid + 1;
            else hi = mid;
        }
        block_ptr[b] = (int)lo;
    }
}

// Level segments of the row-block order: maximal runs of positions with the same (block,
// level) key. A segment's vertices are independent of one another, so the row-block
// executor runs a segment with all its threads and then crosses one CTA barrier.
__global__ void k_seg_flags(long long nv, const unsigned *__restrict__ keys, int *__restrict__ flag) {
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < nv; q += (long long)gridDim.x * blockDim.x)
        flag[q] = (q == 0 || keys[q] != keys[q - 1]) ? 1 : 0;
}

__global__ void k_seg_ptr(long long nv, const int *__restrict__ flag, const int *__restrict__ segidx,
                          int *__restrict__ seg_ptr) {
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < nv; q += (long long)gridDim.x * blockDim.x) {
        if (flag[q]) seg_ptr[segidx[q]] = (int)q;
        if (q == nv - 1) seg_ptr[segidx[nv]] = (int)nv;
    }
}

__global__ void k_seg_width(long long nv, const int *__restrict__ segidx, const int *__restrict__ seg_ptr,
                            int *__restrict__ maxw) {
    const int ns = segidx[nv];
    int w = 0;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < ns; t += (long long)gridDim.x * blockDim.x)
        w = max(w, seg_ptr[t + 1] - seg_ptr[t]);
    for (int off = 16; off >= 1; off >>= 1) w = max(w, __shfl_xor_sync(0xffffffffu, w, off));
    if ((threadIdx.x & 31) == 0 && w > 0) atomicMax(maxw, w);
}

__global__ void k_block_seg(int nb, long long nv, const int *__restrict__ block_ptr, const int *__restrict__ segidx,
                            int *__restrict__ block_seg, int *__restrict__ out2) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b <= nb; b += gridDim.x * blockDim.x) {
        block_seg[b] = b < nb ? segidx[block_ptr[b]] : segidx[nv];
        if (b == nb) out2[0] = segidx[nv];
    }
}

cudaError_t build_block_order(int kind, int n, long long nv, int B, int depth, const int *level, const DevCsr *M,
                              const DevCsrT *MT, const int *inst_ptr, int n_inst, int *order, int *block_ptr,
                              int *seg_ptr, int *block_seg, int *nb_out, int *n_segs_out, int *max_width_out,
                              cudaStream_t s, Arena &ar) {
    const int nb = inst_ptr ? n_inst : (int)((n + (long long)B - 1) / B);
    if ((unsigned long long)nb * (unsigned long long)std::max(depth, 1) > 0xffffffffull) return cudaErrorInvalidValue;
    unsigned *keys = (unsigned *)ar.alloc(sizeof(unsigned) * nv);
    unsigned *vals = (unsigned *)ar.alloc(sizeof(unsigned) * nv);
    int *flag = (int *)ar.alloc(sizeof(int) * (size_t)nv);
    int *segidx = (int *)ar.alloc(sizeof(int) * ((size_t)nv + 1));
    int *out2 = (int *)ar.alloc(sizeof(int) * 2);
    if (!keys || !vals || !flag || !segidx || !out2) return cudaErrorMemoryAllocation;
    cudaMemsetAsync(out2, 0, sizeof(int) * 2, s);
    k_block_keys<<<grid_for(nv, 256, 4096), 256, 0, s>>>(kind, n, nv, B, nb, depth, level, M ? M->rowptr : nullptr,
                                                         M ? M->colidx : nullptr, MT ? MT->t.rowptr : nullptr,
                                                         MT ? MT->t.colidx : nullptr, inst_ptr, keys, vals);
    cudaError_t e = radix_sort_pairs(keys, vals, nv, bits_for((unsigned long long)nb * depth - 1), s, ar);
    if (e != cudaSuccess) return e;
    k_encode_order<<<grid_for(nv, 256, 4096), 256, 0, s>>>(nv, n, vals, order);
    k_block_ptr<<<grid_for((long long)nb + 1, 256, 4096), 256, 0, s>>>(nb, nv, (unsigned)depth, keys, block_ptr);
    k_seg_flags<<<grid_for(nv, 256, 4096), 256, 0, s>>>(nv, keys, flag);
    e = scan_excl<int>(flag, segidx, nv, s, ar);
    if (e != cudaSuccess) return e;
    k_seg_ptr<<<grid_for(nv, 256, 4096), 256, 0, s>>>(nv, flag, segidx, seg_ptr);
    k_seg_width<<<grid_for(nv, 256, 4096), 256, 0, s>>>(nv, segidx, seg_ptr, out2 + 1);
    k_block_seg<<<grid_for((long long)nb + 1, 256, 4096), 256, 0, s>>>(nb, nv, block_ptr, segidx, block_seg, out2);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    int h[2] = {0, 0};
    e = cudaMemcpyAsync(h, out2, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return e;
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    *nb_out = nb;
    *n_segs_out = h[0];
    *max_width_out = h[1];
    return cudaSuccess;
}

// Per-position descriptor of the row-block order: the entry range [rs, re) of the row whose
// entries are waited on (strict lower part of L_i; M_i for a second-kernel row of a forward
// schedule; strict part of (L^T)_j, i.e. after the diagonal, or (A^T)_j for the transposed
// ones), so that a round of the row-block executor reads its metadata in one coalesced load.
__global__ void k_block_desc(int kind, long long nv, const int *__restrict__ order, const int *__restrict__ Lrp,
                             const int *__restrict__ Mrp, const int *__restrict__ LTrp, const int *__restrict__ MTrp,
                             int2 *__restrict__ desc) {
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < nv; q += (long long)gridDim.x * blockDim.x) {
        const unsigned o = (unsigned)order[q];
        const int row = (int)(o & 0x7fffffffu);
        const bool tag = (o >> 31) != 0;
        int2 d;
        if (kind == K_SEP || kind == K_PAIRED) {
            if (!tag) d = make_int2(Lrp[row], Lrp[row + 1] - 1);
            else d = make_int2(Mrp[row], Mrp[row + 1]);
        } else {
            if (!tag) d = make_int2(LTrp[row] + 1, LTrp[row + 1]);
            else d = make_int2(MTrp[row], MTrp[row + 1]);
        }
        desc[q] = d;
    }
}

cudaError_t build_block_desc(int kind, long long nv, const int *order, const DevCsr &L, const DevCsr *M,
                             const DevCsrT &LT, const DevCsrT *MT, int2 *desc, cudaStream_t s) {
    k_block_desc<<<grid_for(nv, 256, 4096), 256, 0, s>>>(kind, nv, order, L.rowptr, M ? M->rowptr : nullptr,
                                                         LT.t.rowptr, MT ? MT->t.rowptr : nullptr, desc);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------ batching
__global__ void k_concat(const InstDesc *__restrict__ d, int *__restrict__ rp_out, int *__restrict__ ci_out) {
    const InstDesc in = d[blockIdx.y];
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < in.n; i += (long long)gridDim.x * blockDim.x)
        rp_out[in.row_off + i] = in.rowptr[i] + in.nnz_off;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < in.nnz; e += (long long)gridDim.x * blockDim.x)
        ci_out[in.nnz_off + e] = in.colidx[e] + in.row_off;
}

cudaError_t concat_patterns(const std::vector<InstDesc> &h, int *rp_out, int *ci_out, long long total_nnz,
                            int total_rows, cudaStream_t s, Arena &ar) {
    if (h.empty()) return cudaErrorInvalidValue;
    InstDesc *d = (InstDesc *)ar.alloc(sizeof(InstDesc) * h.size());
    if (!d) return cudaErrorMemoryAllocation;
    cudaError_t e = cudaMemcpyAsync(d, h.data(), sizeof(InstDesc) * h.size(), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    unsigned gy = (unsigned)h.size();
    k_concat<<<dim3(64, gy), 256, 0, s>>>(d, rp_out, ci_out);
    const int last = (int)total_nnz;
    e = cudaMemcpyAsync(rp_out + total_rows, &last, sizeof(int), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(s);   // `last` and `h` live on this stack frame
}

cudaError_t row_of_entries(const DevCsr &m, int *row_of, cudaStream_t s) {
    if (m.n_rows > 0 && m.nnz > 0) k_row_of<<<grid_for(m.n_rows, 256), 256, 0, s>>>(m.n_rows, m.rowptr, row_of);
    return cudaGetLastError();
}

// Diagonal positions of A's rows and a comparison of L with tril(A): a_diag[i] = position of
// A_ii (or -1); bit 0 of *bad: a row of A misses its diagonal; bit 1: L's row differs from
// the lower part of A's row (diagonal included).
__global__ void k_tril_map(int n, const int *__restrict__ Arp, const int *__restrict__ Aci,
                           const int *__restrict__ Lrp, const int *__restrict__ Lci, int *__restrict__ a_diag,
                           unsigned *bad) {
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)t;
        const int ra = Arp[i], re = Arp[i + 1];
        int lo = ra, hi = re;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (Aci[mid] < i) lo = mid + 1; else hi = mid;
        }
        const int dp = (lo < re && Aci[lo] == i) ? lo : -1;
        a_diag[i] = dp;
        if (dp < 0) {
            atomicOr(bad, 1u);
            continue;
        }
        const int ls = Lrp[i], le = Lrp[i + 1];
        bool same = le - ls == dp - ra + 1;
        for (int u = 0; same && u < le - ls; ++u) same = Lci[ls + u] == Aci[ra + u];
        if (!same) atomicOr(bad, 2u);
    }
}

cudaError_t tril_map(const DevCsr &A, const DevCsr &L, int *a_diag, unsigned *bad_host, cudaStream_t s, Arena &ar) {
    unsigned *bad = (unsigned *)ar.alloc(sizeof(unsigned));
    if (!bad) return cudaErrorMemoryAllocation;
    cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    k_tril_map<<<grid_for(A.n_rows, 256), 256, 0, s>>>(A.n_rows, A.rowptr, A.colidx, L.rowptr, L.colidx, a_diag, bad);
    e = cudaMemcpyAsync(bad_host, bad, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(s);
}

cudaError_t check_pattern(const DevCsr &m, int lower, unsigned long long *status_host, cudaStream_t s, Arena &ar) {
    unsigned long long *st = (unsigned long long *)ar.alloc(sizeof(unsigned long long));
    if (!st) return cudaErrorMemoryAllocation;
    cudaMemsetAsync(st, 0xff, sizeof(unsigned long long), s);
    if (m.n_rows > 0)
        k_check_csr<<<grid_for(m.n_rows, 256), 256, 0, s>>>(m.n_rows, m.n_cols, m.nnz, m.rowptr, m.colidx, lower, st);
    cudaError_t e = cudaMemcpyAsync(status_host, st, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(s);
}

}  // namespace sf
