// C ABI of libsparsefusion.so: argument validation, the schedule object, the inspector
// driver (the runtime half of the paper's Figure 3b driver: DAGs, F, reuse ratio,
// scheduling) and executor launches. No call here traps or throws across the ABI.
#include <algorithm>
#include <chrono>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "sf_inspect.cuh"

#define SF_API extern "C" __attribute__((visibility("default")))

using namespace sf;

namespace {

thread_local char g_detail[512] = "";

sf_status fail(sf_status st, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_detail, sizeof g_detail, fmt, ap);
    va_end(ap);
    return st;
}

sf_status from_cuda(cudaError_t e, const char *what) {
    cudaGetLastError();
    if (e == cudaErrorMemoryAllocation) return fail(SF_ERR_OOM, "%s: out of device memory", what);
    return fail(SF_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define SF_CK(call, what)                                  \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return from_cuda(e_, what); \
    } while (0)

const char *pat_name(unsigned code) {
    switch (code) {
        case PAT_ROWPTR0: return "rowptr[0] != 0";
        case PAT_NNZ: return "rowptr[n_rows] != nnz";
        case PAT_ROWPTR: return "rowptr not monotone or out of range";
        case PAT_COL_RANGE: return "column index out of range";
        case PAT_UNSORTED: return "columns not strictly ascending";
        case PAT_DIAG: return "diagonal missing or not the last entry of the row";
        default: return "invalid pattern";
    }
}

struct Dir {
    bool present = false;
    int kind = 0;
    long long nv = 0;
    int depth = 0;
    int n_parts = 0;
    long long C = 0;
    int *level = nullptr;
    int *order = nullptr;
    int *part_ptr = nullptr;
    unsigned char *part_wide = nullptr;
    long long W = 0;            // items of cost > W run on a whole warp (0: none)
    int lpr = 1;                // lanes per row of this direction's launches
    int team = 8;               // lanes of a team (the unit that runs a partition)
    int *plist = nullptr;       // separated kinds: class-0 then class-1 partitions
    int n_parts0 = 0;           // class-0 partitions (first vertex in the first kernel)
    int split_pct = 0;          // percent of teams that run class 0 (0: one class for all)
    int g2 = 0;                 // placement of second-kernel vertices (separated kinds)
    int minb = 1;               // 1: register-rich executor kernels; 3: occupancy variants
    int *level_asap = nullptr;  // separated kinds: the earliest (Kahn) levels, kept for re-placement
    cudaEvent_t ev_start = nullptr, ev_stop = nullptr;   // recorded around the executor kernel
    int *cost = nullptr;        // c(v) of every vertex (kept for re-cutting)
    long long cost_total = 0;
    // row-block schedule (k = 1 executor with shared-memory dependences)
    int B = 0, nb = 0;
    int blpr = 1;               // lanes per row of the row-block executor (1, 4 or 32)
    int exec_mode = 0;          // 0 automatic (partitions), 1 partitions, 2-4 row blocks, 5 one CTA per instance
    int *border = nullptr;      // order by (block, level, kernel, row)
    int2 *bdesc = nullptr;      // per position: entry range of the row waited on
    int *block_ptr = nullptr;
    int *seg_ptr = nullptr;     // level segments of the row-block order (n_segs + 1)
    int *block_seg = nullptr;   // first segment of every block (nb + 1)
    int n_segs = 0, max_seg = 0;
    bool per_inst = false;      // blocks are the instances (single-CTA executor), not B rows
    int *bperm = nullptr;       // per-instance blocks: launch order, costliest block first
    int cta_per_sm = 0;         // single-CTA executor: CTAs per SM (0 automatic)
    void *cta_vbuf = nullptr;   // single-CTA executor: x handed to the helper CTAs (n doubles, reset)
    void *rsep = nullptr;       // SpMV -> SpTRSV with separated packing: r (value flags), rsep_bytes
    size_t rsep_bytes = 0;
    void *aux = nullptr;        // (c_i, 1 / L_ii) per row, written by the row-block pre-pass
    // packed records of the row-block order (exec_mode 4), built when that mode is chosen
    void *pmeta = nullptr, *pvals = nullptr, *paux = nullptr;
    int *pcols = nullptr;
    int nvp = 0, packed_B = 0;
    unsigned *flags = nullptr;
    ExecState *st = nullptr;
    // long rows split at execution time (sf_schedule_set_slices): queue units, partial slots
    long long slice_cost = 0;   // cost per slice (0: off)
    int kt = 0;                 // right-hand-side tile of this direction (0: the schedule's)
    int4 *xlist = nullptr;      // owned (cudaMalloc), rebuilt with every cut
    int nx = 0, max_m = 1;
    long long n_slots = 0;
};

const ExecState kInitState = {0u, 0u, 1u, 0u, 0u, 0, 0u, 0u};

int pow2_ceil(long long v) {
    int p = 1;
    while (p < v && p < (1 << 30)) p <<= 1;
    return p;
}
bool is_pow2_upto32(int v) { return v >= 1 && v <= 32 && (v & (v - 1)) == 0; }

double reuse_ratio(sf_pair pair, long long n, long long sl, long long sm) {
    // Table 2 / §2.2: common accesses over the larger kernel's accesses
    switch (pair) {
        case SF_TRSV_SPMV: return (double)(2 * n) / (double)std::max(sl + 2 * n, sm + 2 * n);
        case SF_IC0_TRSV: return (double)(2 * sl) / (double)std::max(sl, sl + 2 * n);
        case SF_SPMV_TRSV: return (double)(2 * n) / (double)std::max(sm + 2 * n, sl + 2 * n);
        case SF_TRSV_TRSV: return (double)(2 * n + 2 * sl) / (double)std::max(2 * n + sl, sl + 2 * n);
        case SF_ILU0_TRSV: return (double)(2 * sm) / (double)std::max(sm, sl + 2 * n);
        default: return 0.0;
    }
}

}  // namespace

void sf::set_error_detail(const char *msg) { snprintf(g_detail, sizeof g_detail, "%s", msg); }

struct sf_schedule {
    sf_pair pair = SF_TRSV;
    int n = 0;
    int instances = 1;
    std::vector<int> inst_rows;   // first row of every instance, then n (instances + 1)
    int *inst_ptr = nullptr;      // the same on the device
    Arena keep;
    DevCsr L, M;
    bool hasM = false;
    DevCsrT LT, MT;
    bool hasLT = false, hasMT = false;
    void *LTv = nullptr, *MTv = nullptr;   // adjoint: values in transposed order (8 B per entry)
    Dir fwd, adj;
    int lpr = 4, kt = 0;
    int blocks_per_sm = 0;
    int team = 0;               // 0: automatic (whole-warp teams)
    int block_rows = 0;         // rows per block of the row-block executor (0: automatic)
    int exec_mode = 0;          // 0 automatic, 1 partitions, 2 row blocks
    int g2 = 0;                 // placement of second-kernel vertices at inspection
    bool epoch_flags = false;
    bool dynamic_queue = false;
    unsigned long long timeout_ns = 2000000000ull;
    double reuse = 0.0, inspect_ms = 0.0;
    int packing = 0;
    // IC0 intersection pairs listed by the inspector (NULL when there were too many)
    int *ic0_pp = nullptr;
    int2 *ic0_pairs = nullptr;
    long long ic0_npairs = 0;
    bool ic0_use_pairs = true;
    void *ic0_rinv = nullptr;   // 1 / L_ii of the factor, n values of the widest element type
    // pairs with A (SpMV -> SpTRSV, SpILU0 -> SpTRSV): position of the diagonal in each row of A,
    // and whether L's pattern is tril(A)'s (then SpMV -> SpTRSV may read L from A's storage)
    int *a_diag = nullptr;
    bool tril_ok = false;
    // adjoint schedules: the row of every entry of L and of M (value-gradient passes)
    int *L_row = nullptr, *M_row = nullptr;
    std::mutex mu;
    void *scratch = nullptr;
    size_t scratch_bytes = 0;
    void *scratch2 = nullptr;   // partial sums of split rows
    size_t scratch2_bytes = 0;
    int device = 0;
    int sms = 1;
};

namespace {

sf_status validate_options(const sf_options *o) {
    if (!o) return SF_OK;
    if (o->part_cost_target < 0) return fail(SF_ERR_INVALID_ARG, "part_cost_target must be >= 0");
    if (o->lanes_per_row != 0 && !is_pow2_upto32(o->lanes_per_row))
        return fail(SF_ERR_INVALID_ARG, "lanes_per_row must be 0 or a power of two in [1, 32]");
    if (o->rhs_tile != 0 && !is_pow2_upto32(o->rhs_tile))
        return fail(SF_ERR_INVALID_ARG, "rhs_tile must be 0 or a power of two in [1, 32]");
    if (o->team_lanes != 0 && o->team_lanes != 8 && o->team_lanes != 32)
        return fail(SF_ERR_INVALID_ARG, "team_lanes must be 0, 8 or 32");
    if (o->block_rows < 0 || o->block_rows > (1 << 20))
        return fail(SF_ERR_INVALID_ARG, "block_rows must be in [0, 2^20]");
    if (o->exec_mode < 0 || o->exec_mode > 5) return fail(SF_ERR_INVALID_ARG, "exec_mode must be 0 .. 5");
    if (o->blocks_per_sm < 0) return fail(SF_ERR_INVALID_ARG, "blocks_per_sm must be >= 0");
    if (o->flags & ~(SF_WANT_ADJOINT | SF_EPOCH_FLAGS | SF_DYNAMIC_QUEUE))
        return fail(SF_ERR_INVALID_ARG, "unknown option flags 0x%x", o->flags);
    return SF_OK;
}

bool pair_has_M(sf_pair p) { return p == SF_TRSV_SPMV || p == SF_SPMV_TRSV || p == SF_ILU0_TRSV; }
bool pair_valid(sf_pair p) { return p >= SF_TRSV_SPMV && p <= SF_ILU0_TRSV; }

sf_status check_csr_args(const sf_csr *m, const char *name, bool square) {
    if (!m) return fail(SF_ERR_INVALID_ARG, "%s is NULL", name);
    if (m->n_rows < 1 || m->n_cols < 1) return fail(SF_ERR_INVALID_ARG, "%s: empty matrix", name);
    if (square && m->n_rows != m->n_cols) return fail(SF_ERR_INVALID_ARG, "%s must be square", name);
    if (m->nnz < 0 || m->nnz >= (1LL << 31)) return fail(SF_ERR_INVALID_ARG, "%s: nnz out of range", name);
    if (!m->rowptr || (m->nnz > 0 && !m->colidx)) return fail(SF_ERR_INVALID_ARG, "%s: NULL pattern array", name);
    return SF_OK;
}

sf_status copy_pattern(sf_schedule *S, const sf_csr *src, DevCsr &dst, cudaStream_t s) {
    dst.n_rows = src->n_rows;
    dst.n_cols = src->n_cols;
    dst.nnz = src->nnz;
    dst.rowptr = (int *)S->keep.alloc(sizeof(int) * ((size_t)src->n_rows + 1));
    dst.colidx = (int *)S->keep.alloc(sizeof(int) * (size_t)std::max<long long>(src->nnz, 1));
    if (!dst.rowptr || !dst.colidx) return fail(SF_ERR_OOM, "pattern copy: out of device memory");
    SF_CK(cudaMemcpyAsync(dst.rowptr, src->rowptr, sizeof(int) * ((size_t)src->n_rows + 1), cudaMemcpyDeviceToDevice, s),
          "pattern copy");
    if (src->nnz > 0)
        SF_CK(cudaMemcpyAsync(dst.colidx, src->colidx, sizeof(int) * (size_t)src->nnz, cudaMemcpyDeviceToDevice, s),
              "pattern copy");
    return SF_OK;
}

// Execution-time split of long rows (one direction): every partition holding a single vertex
// of cost above d.slice_cost whose kind the executor can split (SpTRSV rows, SpMV -> SpTRSV
// rows, the transposed solve rows of the adjoints) becomes m = ceil(cost / slice_cost) <= 32
// queue units, its helpers first and its owner last; other partitions stay one unit each.
// The units and partial-sum slots go to d.xlist / d.n_slots; nothing to split clears them.
sf_status slice_dir(sf_schedule *S, Dir &d) {
    if (d.xlist) {
        cudaFree(d.xlist);
        d.xlist = nullptr;
    }
    d.nx = 0;
    d.n_slots = 0;
    d.max_m = 1;
    if (d.slice_cost <= 0) return SF_OK;
    const bool fwd_ok = S->pair == SF_TRSV || S->pair == SF_SPMV_TRSV || S->pair == SF_TRSV_SPMV;
    const bool ok_kind = (&d == &S->adj) ? true : fwd_ok;
    if (!ok_kind) return SF_OK;
    const int P = d.n_parts;
    std::vector<int> pp((size_t)P + 1), order((size_t)d.nv), cost((size_t)d.nv);
    SF_CK(cudaMemcpy(pp.data(), d.part_ptr, sizeof(int) * pp.size(), cudaMemcpyDeviceToHost), "slices");
    SF_CK(cudaMemcpy(order.data(), d.order, sizeof(int) * order.size(), cudaMemcpyDeviceToHost), "slices");
    SF_CK(cudaMemcpy(cost.data(), d.cost, sizeof(int) * cost.size(), cudaMemcpyDeviceToHost), "slices");
    std::vector<int4> xl;
    xl.reserve((size_t)P);
    long long slot = 0;
    for (int p = 0; p < P; ++p) {
        int m = 1;
        if (pp[p + 1] - pp[p] == 1) {
            const unsigned o = (unsigned)order[pp[p]];
            const int tag = (int)(o >> 31), row = (int)(o & 0x7fffffffu);
            const long long c = cost[(size_t)tag * S->n + row];
            if (tag == 0 && c > d.slice_cost) m = (int)std::min<long long>(32, (c + d.slice_cost - 1) / d.slice_cost);
        }
        if (m > 1) {
            if (slot + m > (1LL << 30)) return fail(SF_ERR_UNSUPPORTED, "too many row slices");
            for (int sl = 0; sl < m; ++sl) xl.push_back(make_int4(p, sl, m, (int)slot));
            slot += m - 1;
            d.max_m = std::max(d.max_m, m);
        } else {
            xl.push_back(make_int4(p, 0, 1, 0));
        }
    }
    if (slot == 0) return SF_OK;
    if (xl.size() >= (size_t)(1LL << 31)) return fail(SF_ERR_UNSUPPORTED, "too many queue units");
    SF_CK(cudaMalloc(&d.xlist, sizeof(int4) * xl.size()), "slices");
    SF_CK(cudaMemcpy(d.xlist, xl.data(), sizeof(int4) * xl.size(), cudaMemcpyHostToDevice), "slices");
    d.nx = (int)xl.size();
    d.n_slots = slot;
    return SF_OK;
}

// Cost prefix and partition cut of one direction (the part of the inspection that the
// launch shape influences): C_user > 0 is the cost target, else about one round of a
// team's groups (at most eight items).
sf_status cut_dir(sf_schedule *S, Dir &d, long long C_user, cudaStream_t s, Arena &tmp) {
    const long long nv = d.nv;
    long long *cs = (long long *)tmp.alloc(sizeof(long long) * nv);
    long long *Sx = (long long *)tmp.alloc(sizeof(long long) * (nv + 1));
    if (!cs || !Sx) return fail(SF_ERR_OOM, "inspector: out of device memory");
    long long total = 0;
    cudaError_t e = prefix_costs(nv, S->n, d.order, d.cost, cs, Sx, &total, s, tmp);
    if (e != cudaSuccess) return from_cuda(e, "cost prefix");
    d.cost_total = total;
    long long C = C_user;
    if (C <= 0) {   // about one round of a team's groups, at most eight items
        const long long mean = std::max<long long>(1, (total + nv - 1) / nv);
        C = (long long)std::max(1, std::min(d.team / d.lpr, 8)) * mean;
    }
    d.C = C;
    // rows much longer than a group's lanes can cover quickly get the whole warp, and rows to be
    // split over several teams (cost above the slice cost) a partition of their own
    d.W = d.lpr < 32 ? 16LL * d.lpr + 1 : 0;
    if (d.slice_cost > 0) d.W = d.W ? std::min(d.W, d.slice_cost) : d.slice_cost;
    e = cut_partitions(nv, Sx, cs, C, d.W, d.part_ptr, d.part_wide, &d.n_parts, s, tmp);
    if (e != cudaSuccess) return from_cuda(e, "partition cut");
    if (d.kind == K_SEP || d.kind == K_SEP_T) {
        if (!d.plist) {
            d.plist = (int *)S->keep.alloc(sizeof(int) * ((size_t)nv + 1));
            if (!d.plist) return fail(SF_ERR_OOM, "inspector: out of device memory");
        }
        e = split_partition_classes(d.n_parts, d.part_ptr, d.order, d.plist, &d.n_parts0, s, tmp);
        if (e != cudaSuccess) return from_cuda(e, "partition classes");
    }
    return slice_dir(S, d);
}

// Row-block order of one direction for blocks of B rows (0: automatic, 8192 rows or n; -1: one
// block per instance, launched costliest first).
sf_status block_dir(sf_schedule *S, Dir &d, int B, cudaStream_t s, Arena &tmp) {
    const bool per_inst = B < 0;
    if (B == 0) B = (int)std::min<long long>(8192, ((long long)S->n + 31) / 32 * 32);
    const int nb_new = per_inst ? S->instances : (int)(((long long)S->n + B - 1) / B);
    if (!d.block_ptr || nb_new > d.nb) {
        d.block_ptr = (int *)S->keep.alloc(sizeof(int) * ((size_t)nb_new + 1));
        d.block_seg = (int *)S->keep.alloc(sizeof(int) * ((size_t)nb_new + 1));
        if (!d.block_ptr || !d.block_seg) return fail(SF_ERR_OOM, "inspector: out of device memory");
    }
    if (!d.seg_ptr) {
        d.seg_ptr = (int *)S->keep.alloc(sizeof(int) * ((size_t)d.nv + 1));
        d.aux = S->keep.alloc(sizeof(double) * 2 * (size_t)S->n);
        if (!d.seg_ptr || !d.aux) return fail(SF_ERR_OOM, "inspector: out of device memory");
    }
    const bool sep = d.kind == K_SEP || d.kind == K_SEP_T;
    cudaError_t e = build_block_order(d.kind, S->n, d.nv, B, d.depth, d.level, sep ? &S->M : nullptr,
                                      (d.kind == K_SEP_T) ? &S->MT : nullptr, per_inst ? S->inst_ptr : nullptr,
                                      S->instances, d.border, d.block_ptr, d.seg_ptr, d.block_seg, &d.nb, &d.n_segs,
                                      &d.max_seg, s, tmp);
    if (e != cudaSuccess) return from_cuda(e, "row-block order");
    if (per_inst) {
        // launch order: most level segments first (they bound a CTA's time), then most rows
        std::vector<int> bs((size_t)d.nb + 1), perm((size_t)d.nb);
        SF_CK(cudaMemcpyAsync(bs.data(), d.block_seg, sizeof(int) * bs.size(), cudaMemcpyDeviceToHost, s), "block order");
        SF_CK(cudaStreamSynchronize(s), "block order");
        for (int b = 0; b < d.nb; ++b) perm[(size_t)b] = b;
        auto cost = [&](int b) {
            return (long long)(bs[(size_t)b + 1] - bs[(size_t)b]) * 4096 +
                   (S->inst_rows[(size_t)b + 1] - S->inst_rows[(size_t)b]);
        };
        std::stable_sort(perm.begin(), perm.end(), [&](int x, int y) { return cost(x) > cost(y); });
        if (!d.bperm) {
            d.bperm = (int *)S->keep.alloc(sizeof(int) * (size_t)std::max(d.nb, 1));
            if (!d.bperm) return fail(SF_ERR_OOM, "inspector: out of device memory");
        }
        SF_CK(cudaMemcpyAsync(d.bperm, perm.data(), sizeof(int) * perm.size(), cudaMemcpyHostToDevice, s), "block order");
        SF_CK(cudaStreamSynchronize(s), "block order");   // perm lives on this stack frame
        B = 0;
    }
    d.per_inst = per_inst;
    if (!d.bdesc) {
        d.bdesc = (int2 *)S->keep.alloc(sizeof(int2) * d.nv);
        if (!d.bdesc) return fail(SF_ERR_OOM, "inspector: out of device memory");
    }
    e = build_block_desc(d.kind, d.nv, d.border, S->L, sep ? &S->M : nullptr, S->LT,
                         (d.kind == K_SEP_T) ? &S->MT : nullptr, d.bdesc, s);
    if (e != cudaSuccess) return from_cuda(e, "row-block descriptors");
    d.B = B;
    d.packed_B = 0;   // packed records follow the block order
    return SF_OK;
}

// Packed records of a direction's row-block order (exec_mode 4): allocated once, rebuilt when
// the block order changes.
sf_status pack_dir(sf_schedule *S, Dir &d, cudaStream_t s) {
    if (d.pmeta && d.packed_B == d.B) return SF_OK;
    const long long nvp = (d.nv + 3) / 4 * 4;
    if (nvp >= (1LL << 31)) return fail(SF_ERR_UNSUPPORTED, "too many positions for packed records");
    if (!d.pmeta) {
        d.pmeta = S->keep.alloc(16 * (size_t)nvp);
        d.pcols = (int *)S->keep.alloc(sizeof(int) * 8 * (size_t)nvp);
        d.pvals = S->keep.alloc(sizeof(double) * 8 * (size_t)nvp);
        d.paux = S->keep.alloc(sizeof(double) * 2 * (size_t)nvp);
        if (!d.pmeta || !d.pcols || !d.pvals || !d.paux) return fail(SF_ERR_OOM, "packed records: out of device memory");
    }
    d.nvp = (int)nvp;
    SF_CK(pack_pattern(d.kind, d.nv, d.nvp, d.border, d.bdesc, S->L.colidx, S->hasM ? S->M.colidx : nullptr,
                       S->LT.t.colidx, S->hasMT ? S->MT.t.colidx : nullptr, d.pmeta, d.pcols, s),
          "packed records");
    d.packed_B = d.B;
    return SF_OK;
}

// Threads of a row-block CTA: enough groups for the widest level segment, 64 to 512.
int block_threads(const Dir &d) {
    const long long want = ((long long)std::max(d.max_seg, 1) * d.blpr + 31) / 32 * 32;
    return (int)std::min<long long>(kBlockMaxThreads, std::max<long long>(64, want));
}

sf_status build_dir(sf_schedule *S, Dir &d, int kind, int what, long long C_user, cudaStream_t s, Arena &tmp) {
    const int n = S->n;
    d.kind = kind;
    d.lpr = S->lpr;
    d.team = S->team ? std::max(S->team, d.lpr) : 32;
    d.nv = (kind == K_SEP || kind == K_SEP_T) ? 2LL * n : (long long)n;
    const long long nv = d.nv;
    d.level = (int *)S->keep.alloc(sizeof(int) * nv);
    d.order = (int *)S->keep.alloc(sizeof(int) * nv);
    d.part_ptr = (int *)S->keep.alloc(sizeof(int) * (nv + 1));
    d.part_wide = (unsigned char *)S->keep.alloc((size_t)nv + 1);
    d.flags = (unsigned *)S->keep.alloc(sizeof(unsigned) * (size_t)n);
    d.st = (ExecState *)S->keep.alloc(sizeof(ExecState));
    d.cost = (int *)S->keep.alloc(sizeof(int) * nv);
    if (!d.level || !d.order || !d.part_ptr || !d.part_wide || !d.flags || !d.st || !d.cost)
        return fail(SF_ERR_OOM, "inspector: out of device memory");
    SF_CK(cudaMemsetAsync(d.flags, 0, sizeof(unsigned) * (size_t)n, s), "inspector");
    SF_CK(cudaMemcpyAsync(d.st, &kInitState, sizeof(ExecState), cudaMemcpyHostToDevice, s), "inspector");
    // successor lists of the joint DAG (§2.2): forward DAG edges j -> i come from the
    // transposed L (column j of L), F edges from the transposed M; the reversed DAGs of
    // the adjoint use the rows of L (and of A) directly
    const int *s1rp, *s1ci, *s2rp = nullptr, *s2ci = nullptr;
    if (kind == K_SEP || kind == K_PAIRED) {
        s1rp = S->LT.t.rowptr;
        s1ci = S->LT.t.colidx;
        if (kind == K_SEP) {
            s2rp = S->MT.t.rowptr;
            s2ci = S->MT.t.colidx;
        }
    } else {
        s1rp = S->L.rowptr;
        s1ci = S->L.colidx;
        if (kind == K_SEP_T) {
            s2rp = S->M.rowptr;
            s2ci = S->M.colidx;
        }
    }
    bool timed_out = false;
    cudaError_t e = kahn_levels(nv, n, s1rp, s1ci, s2rp, s2ci, d.level, &d.depth, s, tmp, &timed_out);
    if (e == cudaErrorInvalidValue) return fail(SF_ERR_BAD_PATTERN, "inspector: the joint DAG has a cycle");
    if (e != cudaSuccess) return from_cuda(e, "Kahn peeling");
    if (timed_out) return fail(SF_ERR_TIMEOUT, "Kahn peeling: grid barrier timed out");
    if (kind == K_SEP || kind == K_SEP_T) {
        d.level_asap = (int *)S->keep.alloc(sizeof(int) * nv);
        if (!d.level_asap) return fail(SF_ERR_OOM, "inspector: out of device memory");
        SF_CK(cudaMemcpyAsync(d.level_asap, d.level, sizeof(int) * nv, cudaMemcpyDeviceToDevice, s), "inspector");
        d.g2 = S->g2;
        SF_CK(place_g2(n, d.depth, d.g2, d.level, s), "second-kernel placement");
    }
    e = build_order(nv, n, d.level, d.depth, d.order, s, tmp);
    if (e != cudaSuccess) return from_cuda(e, "ordering");
    e = vertex_costs(what, n, S->L, S->hasM ? &S->M : nullptr, S->hasLT ? &S->LT : nullptr,
                     S->hasMT ? &S->MT : nullptr, d.cost, s);
    if (e != cudaSuccess) return from_cuda(e, "vertex costs");
    sf_status st = cut_dir(S, d, C_user, s, tmp);
    if (st != SF_OK) return st;
    d.border = (int *)S->keep.alloc(sizeof(int) * nv);
    if (!d.border) return fail(SF_ERR_OOM, "inspector: out of device memory");
    st = block_dir(S, d, S->exec_mode == 5 ? -1 : S->block_rows, s, tmp);
    if (st != SF_OK) return st;
    d.exec_mode = S->exec_mode;
    d.blpr = d.lpr <= 1 ? 1 : (d.lpr <= 2 ? 2 : (d.lpr <= 16 ? 4 : 32));
    if (d.exec_mode == 4) {
        st = pack_dir(S, d, s);
        if (st != SF_OK) return st;
    }
    d.present = true;
    return SF_OK;
}

sf_status build_schedule(sf_schedule *S, const sf_options &o, cudaStream_t s) {
    Arena tmp(s);
    unsigned long long pst = 0;
    SF_CK(check_pattern(S->L, 1, &pst, s, tmp), "pattern check");
    if (pst != ~0ull)
        return fail(SF_ERR_BAD_PATTERN, "L: %s (row %d)", pat_name((unsigned)(pst >> 32)), (int)(pst & 0xffffffffu));
    if (S->hasM) {
        SF_CK(check_pattern(S->M, 0, &pst, s, tmp), "pattern check");
        if (pst != ~0ull)
            return fail(SF_ERR_BAD_PATTERN, "M: %s (row %d)", pat_name((unsigned)(pst >> 32)), (int)(pst & 0xffffffffu));
    }
    const bool want_adj = (o.flags & SF_WANT_ADJOINT) != 0;
    if (S->pair == SF_SPMV_TRSV || S->pair == SF_ILU0_TRSV) {
        S->a_diag = (int *)S->keep.alloc(sizeof(int) * (size_t)S->n);
        if (!S->a_diag) return fail(SF_ERR_OOM, "inspector: out of device memory");
        unsigned bad = 0;
        SF_CK(tril_map(S->M, S->L, S->a_diag, &bad, s, tmp), "diagonal positions of A");
        S->tril_ok = bad == 0;
        if (S->pair == SF_ILU0_TRSV) {
            if (bad & 1u) return fail(SF_ERR_BAD_PATTERN, "A: a row misses its diagonal");
            if (bad & 2u) return fail(SF_ERR_BAD_PATTERN, "L must be the pattern of tril(A)");
            std::vector<int> rp((size_t)S->n + 1);
            SF_CK(cudaMemcpy(rp.data(), S->M.rowptr, sizeof(int) * rp.size(), cudaMemcpyDeviceToHost), "inspector");
            for (int i = 0; i < S->n; ++i)
                if (rp[i + 1] - rp[i] > kIluMaxRow)
                    return fail(SF_ERR_UNSUPPORTED, "ILU0 rows of A hold at most %d entries (row %d has %d)", kIluMaxRow,
                                i, rp[i + 1] - rp[i]);
        }
    }
    SF_CK(transpose_csr(S->L, S->LT, s, tmp, S->keep), "transpose of L");
    S->hasLT = true;
    if (S->pair == SF_TRSV_SPMV || (S->pair == SF_SPMV_TRSV && want_adj)) {
        SF_CK(transpose_csr(S->M, S->MT, s, tmp, S->keep), "transpose of M");
        S->hasMT = true;
    }
    // launch shape: one lane per row while rows are short (each lane then keeps several
    // rows in flight); wider groups for long rows, and at least the right-hand-side tile
    if (o.lanes_per_row) {
        S->lpr = o.lanes_per_row;
    } else {
        const long long nnz = S->L.nnz + (S->hasM ? S->M.nnz : 0);
        const long long nv = (S->pair == SF_TRSV_SPMV) ? 2LL * S->n : S->n;
        const long long mean = std::max<long long>(1, (nnz + nv - 1) / nv);
        S->lpr = std::min(32, pow2_ceil((mean + 31) / 32));
    }
    S->kt = o.rhs_tile;
    if (S->kt > S->lpr) S->lpr = S->kt;
    S->team = o.team_lanes;
    S->block_rows = o.block_rows;
    S->exec_mode = o.exec_mode;
    S->g2 = o.g2_placement;
    int kind = K_PAIRED, what = 5;
    switch (S->pair) {
        case SF_TRSV_SPMV: kind = K_SEP; what = 0; break;
        case SF_IC0_TRSV: kind = K_PAIRED; what = 4; break;
        case SF_SPMV_TRSV: kind = K_PAIRED; what = 3; break;
        case SF_TRSV: kind = K_PAIRED; what = 5; break;
        case SF_IC0: kind = K_PAIRED; what = 6; break;
        case SF_TRSV_TRSV: kind = K_PAIRED; what = 7; break;
        case SF_ILU0_TRSV: kind = K_PAIRED; what = 8; break;
    }
    S->packing = (kind == K_SEP) ? 0 : 1;
    sf_status st = build_dir(S, S->fwd, kind, what, o.part_cost_target, s, tmp);
    if (st != SF_OK) return st;
    if (S->pair == SF_IC0_TRSV || S->pair == SF_IC0) {
        // room for four pairs per entry on average before the factor searches per call
        const long long cap = 4 * S->L.nnz + (1LL << 20);
        SF_CK(build_ic0_pairs(S->L, cap, &S->ic0_pp, &S->ic0_pairs, &S->ic0_npairs, s, tmp, S->keep),
              "inspector: IC0 intersection pairs");
        S->ic0_rinv = S->keep.alloc(sizeof(double) * (size_t)std::max(S->n, 1));
        if (S->keep.oom || !S->ic0_rinv) return fail(SF_ERR_OOM, "inspector: out of device memory");
    }
    if (want_adj) {
        if (S->pair == SF_TRSV_SPMV) st = build_dir(S, S->adj, K_PAIRED_T, 1, o.part_cost_target, s, tmp);
        else st = build_dir(S, S->adj, K_SEP_T, 2, o.part_cost_target, s, tmp);
        if (st != SF_OK) return st;
        S->LTv = S->keep.alloc(8 * (size_t)std::max<long long>(S->L.nnz, 1));
        S->MTv = S->keep.alloc(8 * (size_t)std::max<long long>(S->M.nnz, 1));
        S->L_row = (int *)S->keep.alloc(sizeof(int) * (size_t)std::max<long long>(S->L.nnz, 1));
        S->M_row = (int *)S->keep.alloc(sizeof(int) * (size_t)std::max<long long>(S->M.nnz, 1));
        if (!S->LTv || !S->MTv || !S->L_row || !S->M_row) return fail(SF_ERR_OOM, "inspector: out of device memory");
        SF_CK(row_of_entries(S->L, S->L_row, s), "inspector: rows of entries");
        SF_CK(row_of_entries(S->M, S->M_row, s), "inspector: rows of entries");
    }
    S->reuse = reuse_ratio(S->pair, S->n, S->L.nnz, S->hasM ? S->M.nnz : 0);
    SF_CK(cudaStreamSynchronize(s), "inspector");
    return SF_OK;
}

sf_status finish_inspect(sf_schedule *S, const sf_options &o, cudaStream_t s, sf_schedule **out,
                         std::chrono::steady_clock::time_point t0) {
    // instance boundaries on the device (one instance for sf_inspect)
    if (S->inst_rows.empty()) S->inst_rows = {0, S->n};
    S->inst_ptr = (int *)S->keep.alloc(sizeof(int) * S->inst_rows.size());
    sf_status st = S->inst_ptr ? SF_OK : fail(SF_ERR_OOM, "inspector: out of device memory");
    if (st == SF_OK && (cudaMemcpyAsync(S->inst_ptr, S->inst_rows.data(), sizeof(int) * S->inst_rows.size(),
                                        cudaMemcpyHostToDevice, s) != cudaSuccess ||
                        cudaStreamSynchronize(s) != cudaSuccess))
        st = fail(SF_ERR_CUDA, "inspector: instance boundaries");
    if (st == SF_OK) st = build_schedule(S, o, s);
    if (st != SF_OK) {
        cudaStreamSynchronize(s);
        cudaGetLastError();
        delete S;
        return st;
    }
    if (o.timeout_ns) S->timeout_ns = o.timeout_ns;
    S->blocks_per_sm = o.blocks_per_sm;
    S->epoch_flags = (o.flags & SF_EPOCH_FLAGS) != 0;
    S->dynamic_queue = (o.flags & SF_DYNAMIC_QUEUE) != 0;
    S->inspect_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    *out = S;
    return SF_OK;
}

sf_schedule *new_schedule(sf_pair pair) {
    sf_schedule *S = new (std::nothrow) sf_schedule();
    if (!S) return nullptr;
    S->pair = pair;
    cudaGetDevice(&S->device);
    cudaDeviceGetAttribute(&S->sms, cudaDevAttrMultiProcessorCount, S->device);
    if (S->sms < 1) S->sms = 1;
    return S;
}

sf_status get_scratch(const sf_schedule *Sc, size_t bytes, cudaStream_t s, void **out, int which = 0) {
    sf_schedule *S = const_cast<sf_schedule *>(Sc);
    std::lock_guard<std::mutex> lk(S->mu);
    void *&buf = which ? S->scratch2 : S->scratch;
    size_t &have = which ? S->scratch2_bytes : S->scratch_bytes;
    if (have >= bytes) {
        *out = buf;
        return SF_OK;
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(s, &cs);
    if (cs != cudaStreamCaptureStatusNone)
        return fail(SF_ERR_INVALID_ARG, "this call needs a library-owned buffer that is allocated on first use; "
                                        "make one such call before capturing the stream");
    if (buf) {
        cudaFree(buf);
        buf = nullptr;
        have = 0;
    }
    SF_CK(cudaMalloc(&buf, bytes), "scratch allocation");
    have = bytes;
    *out = buf;
    return SF_OK;
}

int occupancy(int mode, int dtype, int lpr, bool vf, int team, int minb) {
    static std::mutex mu;
    static int cache[M_COUNT][2][6][2][2][4] = {};
    int li = 0;
    while ((1 << li) < lpr) ++li;
    std::lock_guard<std::mutex> lk(mu);
    int &c = cache[mode][dtype][li][vf ? 1 : 0][team == 8 ? 0 : 1][std::min(std::max(minb, 1), 3)];
    if (!c) {
        if (mode == M_TRSV_SPMV || mode == M_TRSV) c = occupancy_fwd(mode, dtype, lpr, vf, team, minb);
        else if (mode == M_TRSV_TRSV || mode == M_ILU0_TRSV) c = occupancy_next(mode, dtype, lpr, vf, team, minb);
        else if (mode == M_ADJ_TRSV_SPMV || mode == M_ADJ_SPMV_TRSV)
            c = occupancy_adj(mode, dtype, lpr, vf, team, minb);
        else c = occupancy_pair(mode, dtype, lpr, vf, team, minb);
    }
    return c;
}

// Buffer through which a value-flag launch publishes its rows (k = 1), or NULL.
void *value_flag_buffer(int mode, const ExecArgs &a) {
    switch (mode) {
        case M_TRSV_SPMV: return a.xs;
        case M_TRSV_TRSV: return a.xs;
        case M_TRSV:
        case M_SPMV_TRSV: return a.y;
        case M_ADJ_TRSV_SPMV:
        case M_ADJ_SPMV_TRSV: return a.gb;
        default: return nullptr;
    }
}

sf_status launch(const sf_schedule *S, const Dir &d, int mode, sf_dtype dt, int k, ExecArgs &a, cudaStream_t s) {
    const int kt_s = d.kt ? d.kt : S->kt;
    const int kt = kt_s ? std::min(kt_s, 32) : std::min(pow2_ceil(k), 32);
    const int lpr = std::max(d.lpr, kt);
    const int team = lpr <= 8 ? d.team : 32;
    a.order = d.order;
    a.part_ptr = d.part_ptr;
    a.part_wide = d.part_wide;
    a.LTv = S->LTv;
    a.MTv = S->MTv;
    a.n_parts = d.n_parts;
    a.n = S->n;
    a.k = k;
    a.kt = kt;
    a.dynamic = S->dynamic_queue ? 1 : 0;
    a.flags = d.flags;
    a.st = d.st;
    a.timeout_ns = S->timeout_ns;
    a.Lrp = S->L.rowptr;
    a.Lci = S->L.colidx;
    a.Mrp = S->hasM ? S->M.rowptr : nullptr;
    a.Mci = S->hasM ? S->M.colidx : nullptr;
    a.LTrp = S->LT.t.rowptr;
    a.LTci = S->LT.t.colidx;
    a.LTperm = S->LT.perm;
    a.MTrp = S->hasMT ? S->MT.t.rowptr : nullptr;
    a.MTci = S->hasMT ? S->MT.t.colidx : nullptr;
    a.MTperm = S->hasMT ? S->MT.perm : nullptr;
    a.ic0_pp = S->ic0_use_pairs ? S->ic0_pp : nullptr;
    a.ic0_pairs = S->ic0_use_pairs ? S->ic0_pairs : nullptr;
    a.ic0_rinv = S->ic0_rinv;
    a.a_diag = S->a_diag;
    const int dtype = dt == SF_F64 ? 0 : 1;
    void *vbuf = value_flag_buffer(mode, a);
    const bool ic0 = mode == M_IC0_TRSV || mode == M_IC0;
    // IC0 rows publish through their values when the pair lists exist (any k; the flat
    // index row * k + column of y must fit in an int)
    const bool vf = ic0 ? (!S->epoch_flags && a.ic0_pp != nullptr && (long long)S->n * k <= 0x7fffffffLL)
                        : (!S->epoch_flags && vbuf != nullptr && (long long)S->n * k <= 0x7fffffffLL &&
                           (k == 1 || lpr >= 16));
    // shared storage (SpMV -> SpTRSV with L read from A's rows) is a partition-executor path
    // that publishes through values
    const bool shared = mode == M_SPMV_TRSV && a.Lv == nullptr;
    if (shared && !vf)
        return fail(SF_ERR_UNSUPPORTED, "L read from A's rows needs value flags: k = 1, or at least 16 lanes per row");
    // separated packing of SpMV -> SpTRSV (the forward): r = b - A x_in is computed by every group
    // of the partition executor before it takes partitions, published by value (reset here)
    const bool sep = mode == M_SPMV_TRSV && S->packing == 0;
    a.rsep = nullptr;
    if (sep) {
        if (!vf) return fail(SF_ERR_UNSUPPORTED, "separated packing needs value flags: k = 1, or at least 16 lanes per row");
        if (d.minb >= 3) return fail(SF_ERR_UNSUPPORTED, "separated packing runs on the one- and two-block kernels");
        const size_t bytes = (size_t)S->n * (size_t)k * (dt == SF_F64 ? 8 : 4);
        if (bytes > d.rsep_bytes) {
            sf_schedule *Sm = const_cast<sf_schedule *>(S);
            std::lock_guard<std::mutex> lk(Sm->mu);
            Dir &dm = const_cast<Dir &>(d);
            dm.rsep = Sm->keep.alloc(std::max<size_t>(bytes, 16));
            if (!dm.rsep) return fail(SF_ERR_OOM, "separated packing: out of device memory");
            dm.rsep_bytes = bytes;
        }
        SF_CK(cudaMemsetAsync(d.rsep, 0xff, bytes, s), "separated packing");
        a.rsep = d.rsep;
    }
    // the row-block executors serve one right-hand side
    const bool rows1 = vf && !ic0 && k == 1 && !shared && !sep;
    // single-CTA executor: small systems whose whole row-block order is one block
    if (d.exec_mode == 5) {
        if ((mode != M_TRSV_SPMV && mode != M_TRSV) || k != 1 || a.Lv == nullptr)
            return fail(SF_ERR_UNSUPPORTED, "the single-CTA executor runs SpTRSV -> SpMV and SpTRSV with k = 1");
        if (!d.per_inst) return fail(SF_ERR_UNSUPPORTED, "the single-CTA executor needs one block per instance");
        a.order = d.border;
        a.seg_ptr = d.seg_ptr;
        a.block_seg = d.block_seg;
        a.block_ptr = d.block_ptr;
        a.n_blocks = d.nb;
        // a single SpTRSV -> SpMV system hands x to helper CTAs through a flag buffer that every
        // launch leaves reset (all bits set)
        if (mode == M_TRSV_SPMV && d.nb == 1 && !d.cta_vbuf) {
            sf_schedule *Sm = const_cast<sf_schedule *>(S);
            std::lock_guard<std::mutex> lk(Sm->mu);
            Dir &dm = const_cast<Dir &>(d);
            dm.cta_vbuf = Sm->keep.alloc(sizeof(double) * (size_t)std::max(S->n, 1));
            if (!dm.cta_vbuf) return fail(SF_ERR_OOM, "single-CTA executor: out of device memory");
            SF_CK(cudaMemsetAsync(dm.cta_vbuf, 0xff, sizeof(double) * (size_t)std::max(S->n, 1), s), "single-CTA executor");
        }
        const cudaError_t e = launch_cta_exec(mode, dtype, S->inst_ptr, d.bperm, d.cta_per_sm, S->sms,
                                              mode == M_TRSV_SPMV ? d.cta_vbuf : nullptr, s, a, d.ev_start,
                                              d.ev_stop);
        if (e != cudaSuccess) return from_cuda(e, "single-CTA executor launch");
        return SF_OK;
    }
    // row-block executor with packed records and bulk copies
    if (rows1 && d.exec_mode == 4 && d.nb > 0) {
        const int nc = std::min(256, std::max(32, pow2_ceil(std::max(d.max_seg, 1))));
        const int rows = std::min(d.B, S->n);
        const int occ = block_tma_fits(mode, dtype, rows, nc);
        if (occ <= 0) return fail(SF_ERR_UNSUPPORTED, "row blocks of %d rows do not fit in shared memory", d.B);
        if (!d.pmeta || d.packed_B != d.B) return fail(SF_ERR_UNSUPPORTED, "packed records are missing");
        a.aux = d.aux;
        a.order = d.border;
        a.bdesc = d.bdesc;
        a.block_ptr = d.block_ptr;
        a.seg_ptr = d.seg_ptr;
        a.block_seg = d.block_seg;
        a.block_rows = d.B;
        a.n_blocks = d.nb;
        a.block_rev = (d.kind == K_PAIRED_T || d.kind == K_SEP_T) ? 1 : 0;
        a.pack_meta = d.pmeta;
        a.pack_cols = d.pcols;
        a.pack_vals = d.pvals;
        a.pack_aux = d.paux;
        a.pack_stride = d.nvp;
        long long blocks = std::min<long long>((long long)occ * S->sms, d.nb);
        blocks = std::max<long long>(blocks, 1);
        cudaError_t e = launch_block_tma(mode, dtype, (int)blocks, nc, s, a, d.ev_start, d.ev_stop);
        if (e != cudaSuccess) return from_cuda(e, "row-block executor launch");
        return SF_OK;
    }
    // warp-specialised row-block executor
    if (rows1 && d.exec_mode == 3 && d.nb > 0) {
        // consumer threads: one per position of the widest segment, a power of two in [32, 256]
        const int nc = std::min(256, std::max(32, pow2_ceil(std::max(d.max_seg, 1))));
        const int rows = std::min(d.B, S->n);
        const int occ = block_ws_fits(mode, dtype, rows, nc);
        if (occ <= 0) return fail(SF_ERR_UNSUPPORTED, "row blocks of %d rows do not fit in shared memory", d.B);
        a.aux = d.aux;
        a.order = d.border;
        a.bdesc = d.bdesc;
        a.block_ptr = d.block_ptr;
        a.seg_ptr = d.seg_ptr;
        a.block_seg = d.block_seg;
        a.block_rows = d.B;
        a.n_blocks = d.nb;
        a.block_rev = (d.kind == K_PAIRED_T || d.kind == K_SEP_T) ? 1 : 0;
        long long blocks = std::min<long long>((long long)occ * S->sms, d.nb);
        blocks = std::max<long long>(blocks, 1);
        cudaError_t e = launch_block_ws(mode, dtype, (int)blocks, nc, s, a, d.ev_start, d.ev_stop);
        if (e != cudaSuccess) return from_cuda(e, "row-block executor launch");
        return SF_OK;
    }
    // the row-block executor serves one right-hand side with value flags (its pre-pass
    // resets the published vector)
    if (rows1 && d.exec_mode == 2 && d.nb > 0) {
        const int threads = block_threads(d);
        const int occ = block_exec_occupancy(mode, dtype, d.blpr, std::min(d.B, S->n), threads);
        if (occ > 0) {
            a.aux = d.aux;
            a.order = d.border;
            a.bdesc = d.bdesc;
            a.block_ptr = d.block_ptr;
            a.seg_ptr = d.seg_ptr;
            a.block_seg = d.block_seg;
            a.block_rows = d.B;
            a.n_blocks = d.nb;
            a.block_rev = (d.kind == K_PAIRED_T || d.kind == K_SEP_T) ? 1 : 0;
            int per_sm = occ;
            if (S->blocks_per_sm > 0) per_sm = std::min(per_sm, S->blocks_per_sm);
            long long blocks = std::min<long long>((long long)per_sm * S->sms, d.nb);
            blocks = std::max<long long>(blocks, 1);
            cudaError_t e = launch_block_exec(mode, dtype, d.blpr, (int)blocks, threads, s, a, d.ev_start, d.ev_stop);
            if (e != cudaSuccess) return from_cuda(e, "row-block executor launch");
            return SF_OK;
        }
        return fail(SF_ERR_UNSUPPORTED, "row blocks of %d rows do not fit in shared memory", d.B);
    }
    const bool ilu0 = mode == M_ILU0_TRSV;
    if (ilu0) {
        // value flags only: the factor and y start as the all-ones pattern; whole-warp rows
        const size_t es = dt == SF_F64 ? 8 : 4;
        SF_CK(cudaMemsetAsync(a.y, 0xff, es * (size_t)S->n * (size_t)k, s), "value-flag reset");
        SF_CK(cudaMemsetAsync(a.xs, 0xff, es * (size_t)S->M.nnz, s), "value-flag reset");
    } else if (vf && ic0) {
        // value-flag reset (all bits set): y, 1 / L_ii, and the factor when pairs read it
        const size_t es = dt == SF_F64 ? 8 : 4;
        if (a.y) SF_CK(cudaMemsetAsync(a.y, 0xff, es * (size_t)S->n * (size_t)k, s), "value-flag reset");
        SF_CK(cudaMemsetAsync(a.ic0_rinv, 0xff, es * (size_t)S->n, s), "value-flag reset");
        if (S->ic0_npairs > 0) SF_CK(cudaMemsetAsync(a.xs, 0xff, es * (size_t)S->L.nnz, s), "value-flag reset");
    } else if (vf) {
        // value-flag reset and reciprocal diagonals in one pass
        a.rdiag = d.aux;
        // shared storage: the diagonal of L is A's
        SF_CK(launch_rdiag(dtype, S->n, k, S->L.rowptr, shared ? a.Mv : a.Lv, vbuf, d.aux, d.st, s,
                           shared ? S->a_diag : nullptr, mode == M_TRSV_TRSV ? a.y : nullptr),
              "value-flag reset");
    }
    // long rows split over several teams (value flags; the kinds slice_dir selected)
    const bool sliced = vf && d.nx > 0 &&
                        (mode == M_TRSV || mode == M_TRSV_SPMV || mode == M_SPMV_TRSV || mode == M_ADJ_SPMV_TRSV ||
                         mode == M_ADJ_TRSV_SPMV);
    const int minb = d.minb;
    const int lpr_l = ilu0 ? 32 : lpr, team_l = ilu0 ? 32 : team;
    const bool vf_l = ilu0 ? true : vf;
    int per_sm = occupancy(mode, dtype, lpr_l, vf_l, team_l, minb);
    if (S->blocks_per_sm > 0) per_sm = std::min(per_sm, S->blocks_per_sm);
    long long blocks = (long long)per_sm * S->sms;
    const long long teams_per_block = 8LL * (32 / team_l);
    const long long units = sliced ? d.nx : d.n_parts;
    blocks = std::min<long long>(blocks, (units + teams_per_block - 1) / teams_per_block);
    blocks = std::max<long long>(blocks, 1);
    a.xlist = nullptr;
    a.nx = 0;
    a.parts = nullptr;
    if (sliced && blocks * teams_per_block >= d.max_m && d.n_slots * (long long)k <= 0x7fffffffLL) {
        // the helpers' partial sums start as the all-ones pattern
        const size_t es = dt == SF_F64 ? 8 : 4;
        const size_t bytes = es * (size_t)d.n_slots * (size_t)k;
        sf_status st = get_scratch(S, bytes, s, &a.parts, 1);
        if (st != SF_OK) return st;
        SF_CK(cudaMemsetAsync(a.parts, 0xff, bytes, s), "value-flag reset");
        a.xlist = d.xlist;
        a.nx = d.nx;
    }
    // two partition classes when a split is set: split_pct percent of the teams run the
    // partitions that open with a first-kernel row, the others the second-kernel ones
    const long long nteams = blocks * teams_per_block;
    a.plist = nullptr;
    if (d.split_pct > 0 && d.plist && d.n_parts0 > 0 && d.n_parts0 < d.n_parts && nteams >= 2 &&
        !S->dynamic_queue && !a.xlist) {
        a.plist = d.plist;
        a.n_parts0 = d.n_parts0;
        const long long t0 = (nteams * d.split_pct + 50) / 100;
        a.teams0 = (int)std::min<long long>(std::max<long long>(t0, 1), nteams - 1);
    }
    cudaError_t e;
    if (d.ev_start) SF_CK(cudaEventRecord(d.ev_start, s), "timing event");
    if (mode == M_TRSV_SPMV || mode == M_TRSV) e = launch_exec_fwd(mode, dtype, lpr, vf, team, minb, (int)blocks, s, a);
    else if (mode == M_TRSV_TRSV || mode == M_ILU0_TRSV)
        e = launch_exec_next(mode, dtype, lpr_l, vf_l, team_l, minb, (int)blocks, s, a);
    else if (mode == M_ADJ_TRSV_SPMV || mode == M_ADJ_SPMV_TRSV)
        e = launch_exec_adj(mode, dtype, lpr, vf, team, minb, (int)blocks, s, a);
    else e = launch_exec_pair(mode, dtype, lpr, vf, team, minb, (int)blocks, s, a);
    if (e != cudaSuccess) return from_cuda(e, "executor launch");
    if (d.ev_stop) SF_CK(cudaEventRecord(d.ev_stop, s), "timing event");
    return SF_OK;
}

}  // namespace

// =========================================================================== ABI
SF_API sf_status sf_inspect(sf_pair pair, const sf_csr *L, const sf_csr *M, const sf_options *opt, void *stream,
                            sf_schedule **out) {
    const auto t0 = std::chrono::steady_clock::now();
    if (!out) return fail(SF_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!pair_valid(pair)) return fail(SF_ERR_INVALID_ARG, "unknown pair %d", (int)pair);
    sf_status st = validate_options(opt);
    if (st != SF_OK) return st;
    sf_options o = opt ? *opt : sf_options{};
    if ((o.flags & SF_WANT_ADJOINT) && pair != SF_TRSV_SPMV && pair != SF_SPMV_TRSV)
        return fail(SF_ERR_UNSUPPORTED, "adjoint schedules exist for SF_TRSV_SPMV and SF_SPMV_TRSV only");
    if ((st = check_csr_args(L, "L", true)) != SF_OK) return st;
    if (pair_has_M(pair)) {
        if ((st = check_csr_args(M, "M", true)) != SF_OK) return st;
        if (M->n_rows != L->n_rows) return fail(SF_ERR_INVALID_ARG, "M must be n x n with n = L.n_rows");
    } else if (M) {
        return fail(SF_ERR_INVALID_ARG, "M must be NULL for this pair");
    }
    cudaStream_t s = (cudaStream_t)stream;
    sf_schedule *S = new_schedule(pair);
    if (!S) return fail(SF_ERR_OOM, "host allocation failed");
    S->n = L->n_rows;
    if ((st = copy_pattern(S, L, S->L, s)) != SF_OK) { delete S; return st; }
    if (pair_has_M(pair)) {
        S->hasM = true;
        if ((st = copy_pattern(S, M, S->M, s)) != SF_OK) { delete S; return st; }
    }
    return finish_inspect(S, o, s, out, t0);
}

SF_API sf_status sf_inspect_batched(sf_pair pair, int32_t count, const sf_csr *Ls, const sf_csr *Ms,
                                    const sf_options *opt, void *stream, sf_schedule **out) {
    const auto t0 = std::chrono::steady_clock::now();
    if (!out) return fail(SF_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!pair_valid(pair)) return fail(SF_ERR_INVALID_ARG, "unknown pair %d", (int)pair);
    if (count < 1 || !Ls) return fail(SF_ERR_INVALID_ARG, "need count >= 1 instances");
    if (pair_has_M(pair) && !Ms) return fail(SF_ERR_INVALID_ARG, "Ms is NULL");
    sf_status st = validate_options(opt);
    if (st != SF_OK) return st;
    sf_options o = opt ? *opt : sf_options{};
    if ((o.flags & SF_WANT_ADJOINT) && pair != SF_TRSV_SPMV && pair != SF_SPMV_TRSV)
        return fail(SF_ERR_UNSUPPORTED, "adjoint schedules exist for SF_TRSV_SPMV and SF_SPMV_TRSV only");
    long long n = 0, nnzL = 0, nnzM = 0;
    std::vector<InstDesc> dl((size_t)count), dm(pair_has_M(pair) ? (size_t)count : 0);
    for (int t = 0; t < count; ++t) {
        char nm[32];
        snprintf(nm, sizeof nm, "L[%d]", t);
        if ((st = check_csr_args(&Ls[t], nm, true)) != SF_OK) return st;
        if (pair_has_M(pair)) {
            snprintf(nm, sizeof nm, "M[%d]", t);
            if ((st = check_csr_args(&Ms[t], nm, true)) != SF_OK) return st;
            if (Ms[t].n_rows != Ls[t].n_rows) return fail(SF_ERR_INVALID_ARG, "M[%d] size differs from L[%d]", t, t);
            dm[t] = InstDesc{Ms[t].rowptr, Ms[t].colidx, Ms[t].n_rows, (int)n, (int)Ms[t].nnz, (int)nnzM};
            nnzM += Ms[t].nnz;
        }
        dl[t] = InstDesc{Ls[t].rowptr, Ls[t].colidx, Ls[t].n_rows, (int)n, (int)Ls[t].nnz, (int)nnzL};
        n += Ls[t].n_rows;
        nnzL += Ls[t].nnz;
        if (n >= (1LL << 31) - 1 || nnzL >= (1LL << 31) || nnzM >= (1LL << 31))
            return fail(SF_ERR_INVALID_ARG, "batched total size exceeds int32 indexing");
    }
    cudaStream_t s = (cudaStream_t)stream;
    sf_schedule *S = new_schedule(pair);
    if (!S) return fail(SF_ERR_OOM, "host allocation failed");
    S->n = (int)n;
    S->instances = count;
    S->inst_rows.resize((size_t)count + 1);
    for (int t = 0; t < count; ++t) S->inst_rows[(size_t)t] = dl[(size_t)t].row_off;
    S->inst_rows[(size_t)count] = (int)n;
    Arena tmp(s);
    auto alloc_csr = [&](DevCsr &d, long long nnz) {
        d.n_rows = d.n_cols = (int)n;
        d.nnz = nnz;
        d.rowptr = (int *)S->keep.alloc(sizeof(int) * (size_t)(n + 1));
        d.colidx = (int *)S->keep.alloc(sizeof(int) * (size_t)std::max<long long>(nnz, 1));
        return d.rowptr && d.colidx;
    };
    if (!alloc_csr(S->L, nnzL)) { delete S; return fail(SF_ERR_OOM, "batched patterns: out of device memory"); }
    cudaError_t e = concat_patterns(dl, S->L.rowptr, S->L.colidx, nnzL, (int)n, s, tmp);
    if (e != cudaSuccess) { delete S; return from_cuda(e, "batched concatenation"); }
    if (pair_has_M(pair)) {
        S->hasM = true;
        if (!alloc_csr(S->M, nnzM)) { delete S; return fail(SF_ERR_OOM, "batched patterns: out of device memory"); }
        e = concat_patterns(dm, S->M.rowptr, S->M.colidx, nnzM, (int)n, s, tmp);
        if (e != cudaSuccess) { delete S; return from_cuda(e, "batched concatenation"); }
    }
    return finish_inspect(S, o, s, out, t0);
}

SF_API sf_status sf_execute(const sf_schedule *S, sf_dtype dt, int32_t k, const void *L_vals, const void *M_vals,
                            const void *x_in, const void *b, void *y, void *x_save, void *stream) {
    if (!S) return fail(SF_ERR_INVALID_ARG, "schedule is NULL");
    if (dt != SF_F64 && dt != SF_F32) return fail(SF_ERR_INVALID_ARG, "unknown dtype %d", (int)dt);
    if (k < 1 || k > 1024) return fail(SF_ERR_INVALID_ARG, "k must be in [1, 1024]");
    if (!L_vals && S->pair != SF_SPMV_TRSV && S->pair != SF_ILU0_TRSV)
        return fail(SF_ERR_INVALID_ARG, "L_vals is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t es = dt == SF_F64 ? 8 : 4;
    ExecArgs a{};
    a.Lv = L_vals;
    a.Mv = M_vals;
    a.xin = x_in;
    a.b = b;
    a.y = y;
    a.xs = x_save;
    int mode = 0;
    switch (S->pair) {
        case SF_TRSV_SPMV:
            if (!M_vals || !b || !y) return fail(SF_ERR_INVALID_ARG, "SF_TRSV_SPMV needs M_vals, b and y");
            if (x_in) return fail(SF_ERR_INVALID_ARG, "x_in must be NULL for SF_TRSV_SPMV");
            mode = M_TRSV_SPMV;
            if (!x_save) {
                sf_status st = get_scratch(S, (size_t)S->n * k * es, s, &a.xs);
                if (st != SF_OK) return st;
            }
            break;
        case SF_SPMV_TRSV:
            if (!M_vals || !x_in || !b || !y) return fail(SF_ERR_INVALID_ARG, "SF_SPMV_TRSV needs M_vals, x_in, b and y");
            if (!L_vals && (!S->tril_ok || S->epoch_flags))
                return fail(SF_ERR_INVALID_ARG, "L_vals may be NULL (L read from A) only when L's pattern is tril(A)'s "
                                                "and rows publish through their values");
            mode = M_SPMV_TRSV;
            break;
        case SF_TRSV_TRSV:
            if (!b || !y) return fail(SF_ERR_INVALID_ARG, "SF_TRSV_TRSV needs b and y");
            if (M_vals || x_in) return fail(SF_ERR_INVALID_ARG, "M_vals and x_in must be NULL for SF_TRSV_TRSV");
            mode = M_TRSV_TRSV;
            if (!x_save) {
                sf_status st = get_scratch(S, (size_t)S->n * k * es, s, &a.xs);
                if (st != SF_OK) return st;
            }
            break;
        case SF_ILU0_TRSV:
            if (!M_vals || !b || !y) return fail(SF_ERR_INVALID_ARG, "SF_ILU0_TRSV needs M_vals (A), b and y");
            if (L_vals || x_in) return fail(SF_ERR_INVALID_ARG, "L_vals and x_in must be NULL for SF_ILU0_TRSV");
            mode = M_ILU0_TRSV;
            if (!x_save) {
                sf_status st = get_scratch(S, (size_t)S->M.nnz * es, s, &a.xs);
                if (st != SF_OK) return st;
            }
            break;
        case SF_IC0_TRSV:
            if (!b || !y) return fail(SF_ERR_INVALID_ARG, "SF_IC0_TRSV needs b and y");
            if (M_vals || x_in) return fail(SF_ERR_INVALID_ARG, "M_vals and x_in must be NULL for SF_IC0_TRSV");
            mode = M_IC0_TRSV;
            if (!x_save) {
                sf_status st = get_scratch(S, (size_t)S->L.nnz * es, s, &a.xs);
                if (st != SF_OK) return st;
            }
            break;
        case SF_TRSV:
            if (!b || !y) return fail(SF_ERR_INVALID_ARG, "SF_TRSV needs b and y");
            if (M_vals || x_in) return fail(SF_ERR_INVALID_ARG, "M_vals and x_in must be NULL for SF_TRSV");
            mode = M_TRSV;
            break;
        case SF_IC0:
            if (!x_save) return fail(SF_ERR_INVALID_ARG, "SF_IC0 needs x_save (the factor values)");
            if (M_vals || x_in || b || y) return fail(SF_ERR_INVALID_ARG, "M_vals, x_in, b and y must be NULL for SF_IC0");
            mode = M_IC0;
            break;
    }
    return launch(S, S->fwd, mode, dt, k, a, s);
}

SF_API sf_status sf_adjoint(const sf_schedule *S, sf_dtype dt, int32_t k, const void *L_vals, const void *M_vals,
                            const void *x_in, const void *saved, const void *gy, void *gb, void *gx_in,
                            void *gL_vals, void *gM_vals, void *stream) {
    if (!S) return fail(SF_ERR_INVALID_ARG, "schedule is NULL");
    if (dt != SF_F64 && dt != SF_F32) return fail(SF_ERR_INVALID_ARG, "unknown dtype %d", (int)dt);
    if (k < 1 || k > 1024) return fail(SF_ERR_INVALID_ARG, "k must be in [1, 1024]");
    if (S->pair != SF_TRSV_SPMV && S->pair != SF_SPMV_TRSV)
        return fail(SF_ERR_UNSUPPORTED, "adjoints exist for SF_TRSV_SPMV and SF_SPMV_TRSV only");
    if (!S->adj.present) return fail(SF_ERR_UNSUPPORTED, "schedule was inspected without SF_WANT_ADJOINT");
    if (!L_vals || !M_vals || !gy || !gb) return fail(SF_ERR_INVALID_ARG, "L_vals, M_vals, gy and gb are required");
    ExecArgs a{};
    a.Lv = L_vals;
    a.Mv = M_vals;
    a.xin = x_in;
    a.saved = saved;
    a.gy = gy;
    a.gb = gb;
    a.gx = gx_in;
    a.gL = gL_vals;
    a.gM = gM_vals;
    int mode;
    if (S->pair == SF_TRSV_SPMV) {
        if (gx_in || x_in) return fail(SF_ERR_INVALID_ARG, "x_in and gx_in must be NULL for SF_TRSV_SPMV");
        if ((gL_vals || gM_vals) && !saved) return fail(SF_ERR_INVALID_ARG, "value gradients need saved = x");
        mode = M_ADJ_TRSV_SPMV;
    } else {
        if (gL_vals && !saved) return fail(SF_ERR_INVALID_ARG, "gL_vals needs saved = z");
        if (gM_vals && !x_in) return fail(SF_ERR_INVALID_ARG, "gM_vals (gradient of A) needs x_in");
        mode = M_ADJ_SPMV_TRSV;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int dtype = dt == SF_F64 ? 0 : 1;
    // 1. values of L^T and M^T (A^T) in transposed order, one coalesced gather each; the
    //    row-block executors of the SpTRSV -> SpMV adjoint read M^T only in their pre-pass
    //    (u = M^T gy), which then reads M's values through the permutation instead
    a.mt_direct = (mode == M_ADJ_TRSV_SPMV && k == 1 && !S->epoch_flags && S->adj.exec_mode >= 2 &&
                   S->adj.exec_mode <= 4) ? 1 : 0;
    SF_CK(launch_gather_vals(dtype, S->L.nnz, S->LT.perm, L_vals, S->LTv, s), "adjoint gather");
    if (!a.mt_direct) SF_CK(launch_gather_vals(dtype, S->M.nnz, S->MT.perm, M_vals, S->MTv, s), "adjoint gather");
    // 2. the fused pass on the transposed schedule
    sf_status st = launch(S, S->adj, mode, dt, k, a, s);
    if (st != SF_OK) return st;
    // 3. value gradients restricted to the patterns, streamed row by row
    if (S->pair == SF_TRSV_SPMV) {
        if (gL_vals)   // gL_ij = -sum_c lam_ic x_jc
            SF_CK(launch_grad_entries(dtype, S->L.nnz, k, S->L_row, S->L.colidx, gb, saved, -1.0, gL_vals, s),
                  "adjoint gradients");
        if (gM_vals)   // gM_ij = sum_c gy_ic x_jc
            SF_CK(launch_grad_entries(dtype, S->M.nnz, k, S->M_row, S->M.colidx, gy, saved, 1.0, gM_vals, s),
                  "adjoint gradients");
    } else {
        if (gL_vals)   // gL_ij = -sum_c lam_ic z_jc
            SF_CK(launch_grad_entries(dtype, S->L.nnz, k, S->L_row, S->L.colidx, gb, saved, -1.0, gL_vals, s),
                  "adjoint gradients");
        if (gM_vals)   // gA_ij = -sum_c lam_ic x_in_jc
            SF_CK(launch_grad_entries(dtype, S->M.nnz, k, S->M_row, S->M.colidx, gb, x_in, -1.0, gM_vals, s),
                  "adjoint gradients");
    }
    return SF_OK;
}

SF_API sf_status sf_spmv(sf_dtype dt, int32_t k, const sf_csr *M, const void *M_vals, const void *x, const void *b,
                         void *y, void *stream) {
    if (dt != SF_F64 && dt != SF_F32) return fail(SF_ERR_INVALID_ARG, "unknown dtype %d", (int)dt);
    if (k < 1 || k > 1024) return fail(SF_ERR_INVALID_ARG, "k must be in [1, 1024]");
    sf_status st = check_csr_args(M, "M", false);
    if (st != SF_OK) return st;
    if (!M_vals || !x || !y) return fail(SF_ERR_INVALID_ARG, "M_vals, x and y are required");
    const long long mean = std::max<long long>(1, (M->nnz + M->n_rows - 1) / M->n_rows);
    const int kt = std::min(pow2_ceil(k), 32);
    const int lpr = std::max(kt, std::min(32, pow2_ceil((mean + 1) / 2)));
    cudaError_t e = launch_spmv(dt == SF_F64 ? 0 : 1, lpr, kt, M->n_rows, k, M->rowptr, M->colidx, M_vals, x, b, y,
                                (cudaStream_t)stream);
    if (e != cudaSuccess) return from_cuda(e, "spmv launch");
    return SF_OK;
}

SF_API sf_status sf_schedule_check(const sf_schedule *S, void *stream, int32_t *row) {
    if (row) *row = -1;
    if (!S) return fail(SF_ERR_INVALID_ARG, "schedule is NULL");
    SF_CK(cudaStreamSynchronize((cudaStream_t)stream), "stream synchronize");
    const Dir *dirs[2] = {&S->fwd, &S->adj};
    sf_status result = SF_OK;
    for (const Dir *d : dirs) {
        if (!d->present) continue;
        ExecState h;
        SF_CK(cudaMemcpy(&h, d->st, sizeof(ExecState), cudaMemcpyDeviceToHost), "state readback");
        if (h.err_code && result == SF_OK) {
            result = (sf_status)h.err_code;
            if (row) *row = h.err_row;
            fail(result, "%s pass: %s at row %d", d == &S->fwd ? "forward" : "adjoint",
                 sf_status_string(result), h.err_row);
        }
        if (h.err_code) {
            const unsigned z[2] = {0u, 0u};
            SF_CK(cudaMemcpy(&d->st->err_code, z, sizeof z, cudaMemcpyHostToDevice), "state reset");
        }
    }
    return result;
}

namespace {
sf_status validate_dir(const sf_schedule *S, const Dir &d, const std::vector<int> &Lrp, const std::vector<int> &Lci,
                       const std::vector<int> &Mrp, const std::vector<int> &Mci) {
    const long long nv = d.nv;
    const int n = S->n;
    std::vector<int> order((size_t)nv), pp((size_t)d.n_parts + 1);
    SF_CK(cudaMemcpy(order.data(), d.order, sizeof(int) * nv, cudaMemcpyDeviceToHost), "validate");
    SF_CK(cudaMemcpy(pp.data(), d.part_ptr, sizeof(int) * (d.n_parts + 1), cudaMemcpyDeviceToHost), "validate");
    std::vector<long long> pos((size_t)nv, -1);
    for (long long q = 0; q < nv; ++q) {
        const unsigned o = (unsigned)order[q];
        const long long v = (long long)(o >> 31) * n + (o & 0x7fffffffu);
        if ((o & 0x7fffffffu) >= (unsigned)n || v >= nv || pos[v] >= 0)
            return fail(SF_ERR_BAD_PATTERN, "order is not a permutation (position %lld)", q);
        pos[v] = q;
    }
    const bool fwd = d.kind == K_SEP || d.kind == K_PAIRED;
    for (int i = 0; i < n; ++i) {
        for (int e = Lrp[i]; e < Lrp[i + 1]; ++e) {
            const int j = Lci[e];
            if (j == i) continue;
            const bool ok = fwd ? pos[j] < pos[i] : pos[i] < pos[j];
            if (!ok) return fail(SF_ERR_BAD_PATTERN, "DAG edge of L(%d,%d) violated", i, j);
        }
        if (d.kind == K_SEP)
            for (int e = Mrp[i]; e < Mrp[i + 1]; ++e)
                if (!(pos[Mci[e]] < pos[(long long)n + i])) return fail(SF_ERR_BAD_PATTERN, "F edge (%d,%d) violated", i, Mci[e]);
        if (d.kind == K_SEP_T)
            for (int e = Mrp[i]; e < Mrp[i + 1]; ++e)
                if (!(pos[i] < pos[(long long)n + Mci[e]]))
                    return fail(SF_ERR_BAD_PATTERN, "adjoint F edge (%d,%d) violated", i, Mci[e]);
    }
    if (pp[0] != 0 || pp[d.n_parts] != nv) return fail(SF_ERR_BAD_PATTERN, "partitions do not cover the order");
    for (int p = 0; p < d.n_parts; ++p)
        if (pp[p + 1] <= pp[p]) return fail(SF_ERR_BAD_PATTERN, "empty or decreasing partition %d", p);
    return SF_OK;
}
}  // namespace

SF_API sf_status sf_validate(const sf_schedule *S) {
    if (!S) return fail(SF_ERR_INVALID_ARG, "schedule is NULL");
    const int n = S->n;
    std::vector<int> Lrp((size_t)n + 1), Lci((size_t)std::max<long long>(S->L.nnz, 1)), Mrp, Mci;
    SF_CK(cudaMemcpy(Lrp.data(), S->L.rowptr, sizeof(int) * (n + 1), cudaMemcpyDeviceToHost), "validate");
    SF_CK(cudaMemcpy(Lci.data(), S->L.colidx, sizeof(int) * S->L.nnz, cudaMemcpyDeviceToHost), "validate");
    if (S->hasM) {
        Mrp.resize((size_t)n + 1);
        Mci.resize((size_t)std::max<long long>(S->M.nnz, 1));
        SF_CK(cudaMemcpy(Mrp.data(), S->M.rowptr, sizeof(int) * (n + 1), cudaMemcpyDeviceToHost), "validate");
        SF_CK(cudaMemcpy(Mci.data(), S->M.colidx, sizeof(int) * S->M.nnz, cudaMemcpyDeviceToHost), "validate");
    }
    sf_status st = validate_dir(S, S->fwd, Lrp, Lci, Mrp, Mci);
    if (st != SF_OK || !S->adj.present) return st;
    return validate_dir(S, S->adj, Lrp, Lci, Mrp, Mci);
}

SF_API sf_status sf_schedule_info(const sf_schedule *S, int32_t *depth, int32_t *n_parts, int64_t *n_items) {
    if (!S) return fail(SF_ERR_INVALID_ARG, "schedule is NULL");
    if (depth) *depth = S->fwd.depth;
    if (n_parts) *n_parts = S->fwd.n_parts;
    if (n_items) *n_items = S->fwd.nv;
    return SF_OK;
}

SF_API sf_status sf_schedule_query(const sf_schedule *S, sf_info *info) {
    if (!S || !info) return fail(SF_ERR_INVALID_ARG, "NULL argument");
    memset(info, 0, sizeof *info);
    info->pair = S->pair;
    info->n = S->n;
    info->instances = S->instances;
    info->depth = S->fwd.depth;
    info->n_parts = S->fwd.n_parts;
    info->n_items = S->fwd.nv;
    if (S->adj.present) {
        info->adj_depth = S->adj.depth;
        info->adj_n_parts = S->adj.n_parts;
        info->adj_n_items = S->adj.nv;
        info->adj_part_cost_target = S->adj.C;
    }
    info->lanes_per_row = S->fwd.lpr;
    info->adj_lanes_per_row = S->adj.lpr;
    info->team_lanes = S->fwd.team;
    info->adj_team_lanes = S->adj.team;
    info->block_rows = S->fwd.B;
    info->n_blocks = S->fwd.nb;
    info->adj_block_rows = S->adj.B;
    info->adj_n_blocks = S->adj.nb;
    info->exec_mode = S->fwd.exec_mode;
    info->adj_exec_mode = S->adj.exec_mode;
    info->block_lanes = S->fwd.blpr;
    info->adj_block_lanes = S->adj.blpr;
    info->parts_class0 = S->fwd.n_parts0;
    info->adj_parts_class0 = S->adj.n_parts0;
    info->split_pct = S->fwd.split_pct;
    info->adj_split_pct = S->adj.split_pct;
    info->g2_placement = S->fwd.g2;
    info->adj_g2_placement = S->adj.g2;
    info->min_blocks = S->fwd.minb;
    info->adj_min_blocks = S->adj.minb;
    info->ic0_pairs = (S->pair == SF_IC0_TRSV || S->pair == SF_IC0) ? (S->ic0_pp ? S->ic0_npairs : -1) : 0;
    info->ic0_use_pairs = (S->ic0_pp && S->ic0_use_pairs) ? 1 : 0;
    info->slice_cost = S->fwd.slice_cost;
    info->adj_slice_cost = S->adj.slice_cost;
    info->slice_units = S->fwd.nx;
    info->adj_slice_units = S->adj.nx;
    info->max_slices = S->fwd.max_m;
    info->adj_max_slices = S->adj.max_m;
    info->fwd_rhs_tile = S->fwd.kt ? S->fwd.kt : S->kt;
    info->adj_rhs_tile = S->adj.kt ? S->adj.kt : S->kt;
    info->block_segments = S->fwd.n_segs;
    info->adj_block_segments = S->adj.n_segs;
    info->block_threads = S->fwd.present ? block_threads(S->fwd) : 0;
    info->adj_block_threads = S->adj.present ? block_threads(S->adj) : 0;
    info->rhs_tile = S->kt;
    info->part_cost_target = S->fwd.C;
    info->packing = S->packing;
    info->blocks_per_sm = S->blocks_per_sm;
    info->wide_cost = S->fwd.W;
    info->adj_wide_cost = S->adj.W;
    info->cost_total = S->fwd.cost_total;
    info->adj_cost_total = S->adj.cost_total;
    info->epoch_flags = S->epoch_flags ? 1 : 0;
    info->dynamic_queue = S->dynamic_queue ? 1 : 0;
    info->reuse_ratio = S->reuse;
    info->inspect_ms = S->inspect_ms;
    return SF_OK;
}

SF_API sf_status sf_schedule_export(const sf_schedule *S, int32_t which, int32_t *level, int32_t *order,
                                    int32_t *part_ptr) {
    if (!S) return fail(SF_ERR_INVALID_ARG, "schedule is NULL");
    if (which != 0 && which != 1) return fail(SF_ERR_INVALID_ARG, "which must be 0 or 1");
    const Dir &d = which ? S->adj : S->fwd;
    if (!d.present) return fail(SF_ERR_UNSUPPORTED, "no adjoint schedule");
    if (level) SF_CK(cudaMemcpy(level, d.level, sizeof(int) * d.nv, cudaMemcpyDeviceToHost), "export");
    if (order) SF_CK(cudaMemcpy(order, d.order, sizeof(int) * d.nv, cudaMemcpyDeviceToHost), "export");
    if (part_ptr) SF_CK(cudaMemcpy(part_ptr, d.part_ptr, sizeof(int) * (d.n_parts + 1), cudaMemcpyDeviceToHost), "export");
    return SF_OK;
}

SF_API sf_status sf_schedule_set_launch(sf_schedule *S, int32_t lanes_per_row, int32_t rhs_tile, int32_t blocks_per_sm,
                                        int32_t epoch_flags) {
    if (!S) return fail(SF_ERR_INVALID_ARG, "schedule is NULL");
    if (lanes_per_row && !is_pow2_upto32(lanes_per_row)) return fail(SF_ERR_INVALID_ARG, "bad lanes_per_row");
    if (rhs_tile && !is_pow2_upto32(rhs_tile)) return fail(SF_ERR_INVALID_ARG, "bad rhs_tile");
    if (blocks_per_sm < 0) return fail(SF_ERR_INVALID_ARG, "bad blocks_per_sm");
    if (epoch_flags < -1 || epoch_flags > 1) return fail(SF_ERR_INVALID_ARG, "epoch_flags must be -1, 0 or 1");
    const int lpr = lanes_per_row ? lanes_per_row : S->lpr;
    const int kt = rhs_tile ? rhs_tile : S->kt;
    if (kt > lpr) return fail(SF_ERR_INVALID_ARG, "rhs_tile must not exceed lanes_per_row");
    S->lpr = lpr;
    S->fwd.lpr = lpr;
    S->adj.lpr = lpr;
    if (S->fwd.team < lpr) S->fwd.team = 32;
    if (S->adj.team < lpr) S->adj.team = 32;
    S->kt = kt;
    if (blocks_per_sm) S->blocks_per_sm = blocks_per_sm;
    if (epoch_flags >= 0) S->epoch_flags = epoch_flags == 1;
    return SF_OK;
}

SF_API sf_status sf_schedule_recut(sf_schedule *S, int32_t which, int64_t part_cost_target, int32_t lanes_per_row,
                                   int32_t team_lanes, void *stream) {
    if (!S) return fail(SF_ERR_INVALID_ARG, "schedule is NULL");
    if (which < -1 || which > 1) return fail(SF_ERR_INVALID_ARG, "which must be -1, 0 or 1");
    if (part_cost_target < 0) return fail(SF_ERR_INVALID_ARG, "part_cost_target must be >= 0");
    if (lanes_per_row && !is_pow2_upto32(lanes_per_row)) return fail(SF_ERR_INVALID_ARG, "bad lanes_per_row");
    if (which == 1 && !S->adj.present) return fail(SF_ERR_UNSUPPORTED, "no adjoint schedule");
    if (team_lanes != 0 && team_lanes != 8 && team_lanes != 32)
        return fail(SF_ERR_INVALID_ARG, "team_lanes must be 0, 8 or 32");
    cudaStream_t s = (cudaStream_t)stream;
    SF_CK(cudaStreamSynchronize(s), "recut");      // no launch of this schedule may be in flight
    Arena tmp(s);
    Dir *dirs[2] = {&S->fwd, &S->adj};
    for (int w = 0; w < 2; ++w) {
        if ((which != -1 && which != w) || !dirs[w]->present) continue;
        if (lanes_per_row) dirs[w]->lpr = std::max(lanes_per_row, S->kt);
        if (team_lanes) dirs[w]->team = std::max(team_lanes, dirs[w]->lpr);
        else if (dirs[w]->team < dirs[w]->lpr) dirs[w]->team = 32;
        sf_status st = cut_dir(S, *dirs[w], part_cost_target, s, tmp);
        if (st != SF_OK) return st;
    }
    SF_CK(cudaStreamSynchronize(s), "recut");
    return SF_OK;
}

SF_API sf_status sf_schedule_replace(sf_schedule *S, int32_t which, int32_t g2_placement, void *stream) {
    if (!S) return fail(SF_ERR_INVALID_ARG, "schedule is NULL");
    if (which < -1 || which > 1) return fail(SF_ERR_INVALID_ARG, "which must be -1, 0 or 1");
    if (which == 1 && !S->adj.present) return fail(SF_ERR_UNSUPPORTED, "no adjoint schedule");
    cudaStream_t s = (cudaStream_t)stream;
    SF_CK(cudaStreamSynchronize(s), "replace");
    Arena tmp(s);
    Dir *dirs[2] = {&S->fwd, &S->adj};
    for (int w = 0; w < 2; ++w) {
        Dir &d = *dirs[w];
        if ((which != -1 && which != w) || !d.present || !d.level_asap || d.g2 == g2_placement) continue;
        SF_CK(cudaMemcpyAsync(d.level, d.level_asap, sizeof(int) * d.nv, cudaMemcpyDeviceToDevice, s), "replace");
        SF_CK(place_g2(S->n, d.depth, g2_placement, d.level, s), "second-kernel placement");
        SF_CK(build_order(d.nv, S->n, d.level, d.depth, d.order, s, tmp), "ordering");
        d.g2 = g2_placement;
        sf_status st = cut_dir(S, d, d.C, s, tmp);
        if (st != SF_OK) return st;
        st = block_dir(S, d, d.per_inst ? -1 : d.B, s, tmp);
        if (st != SF_OK) return st;
        if (d.exec_mode == 4 && (st = pack_dir(S, d, s)) != SF_OK) return st;
    }
    SF_CK(cudaStreamSynchronize(s), "replace");
    return SF_OK;
}

SF_API sf_status sf_schedule_reblock(sf_schedule *S, int32_t which, int32_t block_rows, int32_t exec_mode,
                                     int32_t lanes_per_row, void *stream) {
    if (!S) return fail(SF_ERR_INVALID_ARG, "schedule is NULL");
    if (which < -1 || which > 1) return fail(SF_ERR_INVALID_ARG, "which must be -1, 0 or 1");
    if (block_rows < 0 || block_rows > (1 << 20)) return fail(SF_ERR_INVALID_ARG, "block_rows must be in [0, 2^20]");
    if (exec_mode < -1 || exec_mode > 5) return fail(SF_ERR_INVALID_ARG, "exec_mode must be -1 .. 5");
    if (lanes_per_row != 0 && lanes_per_row != 1 && lanes_per_row != 2 && lanes_per_row != 4 && lanes_per_row != 32)
        return fail(SF_ERR_INVALID_ARG, "row-block lanes per row must be 1, 2, 4 or 32");
    if (exec_mode == 5 && lanes_per_row == 32)
        return fail(SF_ERR_INVALID_ARG, "single-CTA executor: CTAs per SM must be 1, 2 or 4");
    if (exec_mode == 5 && block_rows != 0)
        return fail(SF_ERR_INVALID_ARG, "the single-CTA executor runs whole instances: block_rows must be 0");
    if (which == 1 && !S->adj.present) return fail(SF_ERR_UNSUPPORTED, "no adjoint schedule");
    cudaStream_t s = (cudaStream_t)stream;
    SF_CK(cudaStreamSynchronize(s), "reblock");
    Arena tmp(s);
    Dir *dirs[2] = {&S->fwd, &S->adj};
    for (int w = 0; w < 2; ++w) {
        if ((which != -1 && which != w) || !dirs[w]->present) continue;
        Dir &d = *dirs[w];
        // the single-CTA executor takes one block per instance; the row-block executors
        // blocks of B rows (rebuilt at the automatic size when leaving per-instance blocks)
        const int B = exec_mode == 5 ? -1 : (block_rows ? block_rows : ((exec_mode >= 2 && d.per_inst) ? 0 : -2));
        if (B == -1 ? !d.per_inst : (B == 0 || (B > 0 && (B != d.B || d.per_inst)))) {
            sf_status st = block_dir(S, d, B, s, tmp);
            if (st != SF_OK) return st;
        }
        if (exec_mode >= 0) d.exec_mode = exec_mode;
        if (exec_mode == 5) d.cta_per_sm = lanes_per_row;
        else if (lanes_per_row) d.blpr = lanes_per_row;
        if (d.exec_mode == 4) {
            sf_status st = pack_dir(S, d, s);
            if (st != SF_OK) return st;
        }
    }
    SF_CK(cudaStreamSynchronize(s), "reblock");
    return SF_OK;
}

SF_API sf_status sf_schedule_launches(const sf_schedule *S, int32_t which, int32_t k, int32_t *count) {
    if (!S || !count) return fail(SF_ERR_INVALID_ARG, "schedule or count is NULL");
    if (which != 0 && which != 1) return fail(SF_ERR_INVALID_ARG, "which must be 0 or 1");
    if (k < 1) return fail(SF_ERR_INVALID_ARG, "k must be >= 1");
    const Dir &d = which ? S->adj : S->fwd;
    if (!d.present) return fail(SF_ERR_UNSUPPORTED, "no adjoint schedule");
    const bool vf_pair = S->pair == SF_TRSV_SPMV || S->pair == SF_SPMV_TRSV || S->pair == SF_TRSV ||
                         S->pair == SF_TRSV_TRSV;
    // the same choice as launch(): values publish rows for k = 1, or for any k with 16 or more
    // lanes per row
    const int kt_s = d.kt ? d.kt : S->kt;
    const int kt = kt_s ? std::min(kt_s, 32) : std::min(pow2_ceil(k), 32);
    const int lpr = std::max(d.lpr, kt);
    const bool vf = !S->epoch_flags && vf_pair && (long long)S->n * k <= 0x7fffffffLL && (k == 1 || lpr >= 16);
    int n = 0;
    if (k == 1 && d.exec_mode == 5) n = 1;                                          // single-CTA executor
    else if (vf && k == 1 && d.exec_mode >= 2 && d.nb > 0) n = 2 + (d.exec_mode == 4 ? 1 : 0);   // pre-pass(es) + executor
    else n = (vf ? 1 : 0) + 1;                                                  // value-flag reset + executor
    if (which == 1) {
        const bool mt_direct = S->pair == SF_TRSV_SPMV && vf && k == 1 && d.exec_mode >= 2 && d.exec_mode <= 4;
        n += 1 + (mt_direct ? 0 : 1) + 2;   // value gathers and both gradient passes
    }
    *count = n;
    return SF_OK;
}

SF_API sf_status sf_schedule_set_exec_events(sf_schedule *S, int32_t which, void *ev_start, void *ev_stop) {
    if (!S) return fail(SF_ERR_INVALID_ARG, "schedule is NULL");
    if (which != 0 && which != 1) return fail(SF_ERR_INVALID_ARG, "which must be 0 or 1");
    if ((ev_start == nullptr) != (ev_stop == nullptr)) return fail(SF_ERR_INVALID_ARG, "set both events or neither");
    Dir &d = which ? S->adj : S->fwd;
    if (!d.present) return fail(SF_ERR_UNSUPPORTED, "no adjoint schedule");
    d.ev_start = (cudaEvent_t)ev_start;
    d.ev_stop = (cudaEvent_t)ev_stop;
    return SF_OK;
}

SF_API sf_status sf_schedule_set_occupancy(sf_schedule *S, int32_t which, int32_t min_blocks) {
    if (!S) return fail(SF_ERR_INVALID_ARG, "schedule is NULL");
    if (which < -1 || which > 1) return fail(SF_ERR_INVALID_ARG, "which must be -1, 0 or 1");
    if (min_blocks < 0 || min_blocks > 3) return fail(SF_ERR_INVALID_ARG, "min_blocks must be 0, 1, 2 or 3");
    if (which == 1 && !S->adj.present) return fail(SF_ERR_UNSUPPORTED, "no adjoint schedule");
    Dir *dirs[2] = {&S->fwd, &S->adj};
    for (int w = 0; w < 2; ++w)
        if ((which == -1 || which == w) && dirs[w]->present) dirs[w]->minb = min_blocks ? min_blocks : 1;
    return SF_OK;
}

SF_API sf_status sf_schedule_set_ic0_pairs(sf_schedule *S, int32_t use) {
    if (!S) return fail(SF_ERR_INVALID_ARG, "schedule is NULL");
    if (use != 0 && use != 1) return fail(SF_ERR_INVALID_ARG, "use must be 0 or 1");
    if (S->pair != SF_IC0_TRSV && S->pair != SF_IC0) return fail(SF_ERR_UNSUPPORTED, "not an IC0 schedule");
    if (use && !S->ic0_pp) return fail(SF_ERR_UNSUPPORTED, "no intersection pairs were listed for this schedule");
    S->ic0_use_pairs = use != 0;
    return SF_OK;
}

SF_API sf_status sf_schedule_set_split(sf_schedule *S, int32_t which, int32_t class0_pct) {
    if (!S) return fail(SF_ERR_INVALID_ARG, "schedule is NULL");
    if (which < -1 || which > 1) return fail(SF_ERR_INVALID_ARG, "which must be -1, 0 or 1");
    if (class0_pct < 0 || class0_pct > 99) return fail(SF_ERR_INVALID_ARG, "class0_pct must be in [0, 99]");
    if (which == 1 && !S->adj.present) return fail(SF_ERR_UNSUPPORTED, "no adjoint schedule");
    Dir *dirs[2] = {&S->fwd, &S->adj};
    for (int w = 0; w < 2; ++w)
        if ((which == -1 || which == w) && dirs[w]->present) dirs[w]->split_pct = class0_pct;
    return SF_OK;
}

SF_API sf_status sf_schedule_set_rhs_tile(sf_schedule *S, int32_t which, int32_t rhs_tile) {
    if (!S) return fail(SF_ERR_INVALID_ARG, "schedule is NULL");
    if (which < -1 || which > 1) return fail(SF_ERR_INVALID_ARG, "which must be -1, 0 or 1");
    if (rhs_tile != 0 && !is_pow2_upto32(rhs_tile))
        return fail(SF_ERR_INVALID_ARG, "rhs_tile must be 0 or a power of two in [1, 32]");
    if (which == 1 && !S->adj.present) return fail(SF_ERR_UNSUPPORTED, "no adjoint schedule");
    Dir *dirs[2] = {&S->fwd, &S->adj};
    for (int w = 0; w < 2; ++w)
        if ((which == -1 || which == w) && dirs[w]->present) dirs[w]->kt = rhs_tile;
    return SF_OK;
}

SF_API sf_status sf_schedule_set_packing(sf_schedule *S, int32_t packing) {
    if (!S) return fail(SF_ERR_INVALID_ARG, "schedule is NULL");
    if (packing != 0 && packing != 1) return fail(SF_ERR_INVALID_ARG, "packing must be 0 (separated) or 1 (interleaved)");
    if (S->pair != SF_SPMV_TRSV)
        return fail(SF_ERR_UNSUPPORTED, "the packing of the forward pass can be chosen for SF_SPMV_TRSV only");
    S->packing = packing;
    return SF_OK;
}

SF_API sf_status sf_schedule_set_slices(sf_schedule *S, int32_t which, int64_t cost_per_slice, void *stream) {
    if (!S) return fail(SF_ERR_INVALID_ARG, "schedule is NULL");
    if (which < -1 || which > 1) return fail(SF_ERR_INVALID_ARG, "which must be -1, 0 or 1");
    if (cost_per_slice < 0) return fail(SF_ERR_INVALID_ARG, "cost_per_slice must be >= 0");
    if (which == 1 && !S->adj.present) return fail(SF_ERR_UNSUPPORTED, "no adjoint schedule");
    cudaStream_t s = (cudaStream_t)stream;
    SF_CK(cudaStreamSynchronize(s), "slices");
    Arena tmp(s);
    Dir *dirs[2] = {&S->fwd, &S->adj};
    for (int w = 0; w < 2; ++w) {
        if ((which != -1 && which != w) || !dirs[w]->present) continue;
        if (dirs[w]->slice_cost == cost_per_slice) continue;
        dirs[w]->slice_cost = cost_per_slice;
        // re-cut (same cost target): rows above the slice cost get partitions of their own
        sf_status st = cut_dir(S, *dirs[w], dirs[w]->C, s, tmp);
        if (st != SF_OK) return st;
    }
    SF_CK(cudaStreamSynchronize(s), "slices");
    return SF_OK;
}

SF_API sf_status sf_schedule_export_blocks(const sf_schedule *S, int32_t which, int32_t *order, int32_t *block_ptr,
                                           int32_t *seg_ptr, int32_t *block_seg) {
    if (!S) return fail(SF_ERR_INVALID_ARG, "schedule is NULL");
    if (which != 0 && which != 1) return fail(SF_ERR_INVALID_ARG, "which must be 0 or 1");
    const Dir &d = which ? S->adj : S->fwd;
    if (!d.present) return fail(SF_ERR_UNSUPPORTED, "no adjoint schedule");
    if (order) SF_CK(cudaMemcpy(order, d.border, sizeof(int) * d.nv, cudaMemcpyDeviceToHost), "export");
    if (block_ptr) SF_CK(cudaMemcpy(block_ptr, d.block_ptr, sizeof(int) * (d.nb + 1), cudaMemcpyDeviceToHost), "export");
    if (seg_ptr)
        SF_CK(cudaMemcpy(seg_ptr, d.seg_ptr, sizeof(int) * ((size_t)d.n_segs + 1), cudaMemcpyDeviceToHost), "export");
    if (block_seg) SF_CK(cudaMemcpy(block_seg, d.block_seg, sizeof(int) * (d.nb + 1), cudaMemcpyDeviceToHost), "export");
    return SF_OK;
}

SF_API sf_status sf_schedule_set_timeout(sf_schedule *S, uint64_t timeout_ns) {
    if (!S) return fail(SF_ERR_INVALID_ARG, "schedule is NULL");
    S->timeout_ns = timeout_ns ? timeout_ns : 2000000000ull;
    return SF_OK;
}

SF_API sf_status sf_schedule_debug_swap(sf_schedule *S, int64_t q1, int64_t q2) {
    if (!S) return fail(SF_ERR_INVALID_ARG, "schedule is NULL");
    if (q1 < 0 || q2 < 0 || q1 >= S->fwd.nv || q2 >= S->fwd.nv) return fail(SF_ERR_INVALID_ARG, "position out of range");
    int *orders[2] = {S->fwd.order, S->fwd.border};
    for (int *ord : orders) {
        if (!ord) continue;
        int a = 0, b = 0;
        SF_CK(cudaMemcpy(&a, ord + q1, sizeof(int), cudaMemcpyDeviceToHost), "swap");
        SF_CK(cudaMemcpy(&b, ord + q2, sizeof(int), cudaMemcpyDeviceToHost), "swap");
        SF_CK(cudaMemcpy(ord + q1, &b, sizeof(int), cudaMemcpyHostToDevice), "swap");
        SF_CK(cudaMemcpy(ord + q2, &a, sizeof(int), cudaMemcpyHostToDevice), "swap");
    }
    if (S->fwd.bdesc) {
        int2 a, b;
        SF_CK(cudaMemcpy(&a, S->fwd.bdesc + q1, sizeof(int2), cudaMemcpyDeviceToHost), "swap");
        SF_CK(cudaMemcpy(&b, S->fwd.bdesc + q2, sizeof(int2), cudaMemcpyDeviceToHost), "swap");
        SF_CK(cudaMemcpy(S->fwd.bdesc + q1, &b, sizeof(int2), cudaMemcpyHostToDevice), "swap");
        SF_CK(cudaMemcpy(S->fwd.bdesc + q2, &a, sizeof(int2), cudaMemcpyHostToDevice), "swap");
    }
    if (S->fwd.pmeta) {   // packed records follow the block order
        S->fwd.packed_B = 0;
        if (S->fwd.exec_mode == 4) {
            sf_status st = pack_dir(S, S->fwd, 0);
            if (st != SF_OK) return st;
            SF_CK(cudaDeviceSynchronize(), "swap");
        }
    }
    return SF_OK;
}

SF_API void sf_schedule_destroy(sf_schedule *S) {
    if (!S) return;
    if (S->scratch) cudaFree(S->scratch);
    if (S->scratch2) cudaFree(S->scratch2);
    if (S->fwd.xlist) cudaFree(S->fwd.xlist);
    if (S->adj.xlist) cudaFree(S->adj.xlist);
    delete S;
}

SF_API const char *sf_status_string(sf_status s) {
    switch (s) {
        case SF_OK: return "SF_OK";
        case SF_ERR_INVALID_ARG: return "SF_ERR_INVALID_ARG";
        case SF_ERR_BAD_PATTERN: return "SF_ERR_BAD_PATTERN";
        case SF_ERR_CUDA: return "SF_ERR_CUDA";
        case SF_ERR_OOM: return "SF_ERR_OOM";
        case SF_ERR_TIMEOUT: return "SF_ERR_TIMEOUT";
        case SF_ERR_BREAKDOWN: return "SF_ERR_BREAKDOWN";
        case SF_ERR_NONFINITE: return "SF_ERR_NONFINITE";
        case SF_ERR_UNSUPPORTED: return "SF_ERR_UNSUPPORTED";
    }
    return "unknown sf_status";
}

SF_API sf_status sf_last_error_detail(char *buf, size_t len) {
    if (!buf || len == 0) return SF_ERR_INVALID_ARG;
    snprintf(buf, len, "%s", g_detail);
    return SF_OK;
}
