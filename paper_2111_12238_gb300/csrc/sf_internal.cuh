// Internal declarations shared by the translation units of libsparsefusion.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "sparsefusion.h"

namespace sf {

// Joint-DAG shapes built by the inspector (§2.2: the DAG of SpTRSV is the pattern of L,
// SpMV has no intra-kernel edges, F carries the inter-kernel edges).
//   K_SEP      vertices: kernel-1 rows 0..n-1 (tag 0), kernel-2 rows n..2n-1 (tag 1)
//   K_PAIRED   one vertex per row holding both kernels' iteration i (F = I)
//   K_PAIRED_T the reversed DAG of L (adjoint of SpTRSV->SpMV)
//   K_SEP_T    reversed L solve (tag 0) then A^T rows (tag 1) (adjoint of SpMV->SpTRSV)
enum Kind { K_SEP = 0, K_PAIRED = 1, K_PAIRED_T = 2, K_SEP_T = 3 };

// Executor modes (which item kinds a launch runs).
enum Mode {
    M_TRSV_SPMV = 0,   // separated items: SpTRSV row (tag 0), SpMV row (tag 1)
    M_SPMV_TRSV = 1,   // paired: r_i = b_i - A_i x_in, z_i = (r_i - L_i z) / L_ii
    M_IC0_TRSV = 2,    // paired: up-looking IC0 row i, then solve row i
    M_TRSV = 3,        // single kernel: SpTRSV row
    M_IC0 = 4,         // single kernel: IC0 row
    M_ADJ_TRSV_SPMV = 5,  // paired: u_j = (M^T gy)_j, lam_j = (u_j - (L^T lam)_j) / L_jj
    M_ADJ_SPMV_TRSV = 6,  // separated: lam_j (tag 0), gx_j = -(A^T lam)_j (tag 1)
    M_TRSV_TRSV = 7,   // paired: x_i = (b_i - L_i x) / L_ii, then z_i = (x_i - L_i z) / L_ii
    M_ILU0_TRSV = 8,   // paired: up-looking ILU0 row i of A, then the unit lower solve row i
    M_COUNT = 9
};

// Per-direction launch state, one 32-byte block in device memory. `epoch` numbers the
// launches of the schedule: a ready flag equal to the current epoch means "published in
// this launch", so flags never need clearing. The last warp to leave a launch resets
// the ticket / done counters and advances the epoch (see k_exec).
struct ExecState {
    unsigned ticket;
    unsigned done;
    unsigned epoch;
    unsigned abort;
    unsigned err_code;
    int err_row;
    unsigned pad0;
    unsigned cta_exit;   // single-CTA executor with helper CTAs: CTAs of the launch that have finished
};

// Argument block of the executor. Typed pointers are carried as void* and cast in the
// kernel so that one host-side struct serves both element types.
struct ExecArgs {
    const int *order;
    const int *part_ptr;
    const unsigned char *part_wide;    // 1: the partition is one long item run by the whole warp
    int n_parts;
    int n;
    int k;
    int kt;                 // right-hand-side columns handled side by side (pow2 <= lanes)
    int dynamic;            // 1: partitions from a ticket counter; 0: static round robin
    const int *plist;       // static: class-0 then class-1 partitions (NULL: one class)
    int n_parts0;           // class-0 partitions in plist
    int teams0;             // teams that run class 0; the others run class 1
    const int *block_ptr;   // row-block executor: first position of each block in `order`
    const int2 *bdesc;      // row-block executor: entry range of the row each position waits on
    const int *seg_ptr;     // row-block executor: level segments of `order`
    const int *block_seg;   // row-block executor: first segment of each block
    int block_rows;         // rows per block (B)
    int n_blocks;
    int block_rev;          // blocks run in decreasing row order (transposed schedules)
    unsigned *flags;
    ExecState *st;
    unsigned long long timeout_ns;
    const int *Lrp, *Lci;               // L (lower, diagonal last)
    const int *Mrp, *Mci;               // M or A
    const int *LTrp, *LTci, *LTperm;    // L^T pattern and entry permutation into L
    const int *MTrp, *MTci, *MTperm;    // M^T / A^T
    const void *Lv, *Mv, *xin, *b, *gy, *saved;
    const void *LTv, *MTv;              // values of L^T and M^T / A^T in transposed order (adjoint)
    void *y, *xs, *gb, *gx, *gL, *gM;
    void *aux;                          // row-block executor: (c_i, 1 / L_ii) per row
    const void *rdiag;                  // 1 / L_ii per row (k = 1 value-flag launches), or NULL
    int mt_direct;                      // row-block pre-pass reads M's values through MTperm (no MTv)
    // packed records of the row-block order (exec_mode 4): structures of arrays, stride pack_stride
    const void *pack_meta;              // (order entry, first entry, end) per position
    const int *pack_cols;               // first kTmaU column indices per position
    void *pack_vals;                    // their values (gathered every call)
    void *pack_aux;                     // (c_i, 1 / L_ii) per position (gathered every call)
    int pack_stride;
    // IC0: per L entry t, pairs [ic0_pp[t], ic0_pp[t + 1]) of ic0_pairs are the (p, q) entry
    // positions of the columns that rows i and j share below j (NULL: searched per call)
    const int *ic0_pp;
    const int2 *ic0_pairs;
    void *ic0_rinv;                     // IC0: 1 / L_ii per row, written with the factor row
    // position of the diagonal in every row of M (= A): ILU0 rows, and SpMV -> SpTRSV rows that
    // read L = tril(A) from A's storage (shared storage, Lv == NULL); else NULL
    const int *a_diag;
    // long rows split at execution time: queue units (partition, slice, slices, first partial
    // slot) and the helpers' partial sums (slots x k values, value flags); xlist NULL: none
    const int4 *xlist;
    int nx;
    void *parts;
    // SpMV -> SpTRSV with separated packing (value flags): r = b - A x_in, n x k values, each its
    // own flag; computed by every group of the launch before it takes partitions. NULL: paired.
    void *rsep;
};

// launchers, one translation unit per group of modes (dtype: 0 f64, 1 f32)
// Static assignment needs every block resident: those launches are cooperative.
cudaError_t launch_exec_fwd(int mode, int dtype, int lpr, bool vf, int team, int minb, int blocks, cudaStream_t s,
                            const ExecArgs &a);
cudaError_t launch_exec_pair(int mode, int dtype, int lpr, bool vf, int team, int minb, int blocks, cudaStream_t s,
                            const ExecArgs &a);
cudaError_t launch_exec_adj(int mode, int dtype, int lpr, bool vf, int team, int minb, int blocks, cudaStream_t s,
                            const ExecArgs &a);
// Row-block executor (k = 1): launch and blocks per SM for B rows of shared values and
// `threads` threads per CTA (a multiple of 32, at most kBlockMaxThreads).
constexpr int kBlockMaxThreads = 512;
cudaError_t launch_block_exec(int mode, int dtype, int lpr, int blocks, int threads, cudaStream_t s,
                              const ExecArgs &a, cudaEvent_t ev_start = nullptr, cudaEvent_t ev_stop = nullptr);
int block_exec_occupancy(int mode, int dtype, int lpr, int block_rows, int threads);
size_t block_exec_smem(int mode, int dtype, int block_rows);
// Warp-specialised row-block executor: nc consumer threads (32, 64, 128 or 256) plus
// 512 producer threads; resident CTAs per SM (0: does not fit) and launch.
int block_ws_fits(int mode, int dtype, int rows, int nc);
// Row-block executor with packed records and bulk copies (exec_mode 4): nc consumer threads
// (32, 64, 128 or 256) plus one producer warp. pack_pattern writes the pattern part of the
// packed records (stride nvp = nv rounded up to 4; positions past nv are padding).
cudaError_t pack_pattern(int kind, long long nv, int nvp, const int *border, const int2 *bdesc, const int *Lci,
                         const int *Mci, const int *LTci, const int *MTci, void *meta, int *cols, cudaStream_t s);
int block_tma_fits(int mode, int dtype, int rows, int nc);
cudaError_t launch_block_tma(int mode, int dtype, int blocks, int nc, cudaStream_t s, const ExecArgs &a,
                             cudaEvent_t ev_start, cudaEvent_t ev_stop);
cudaError_t launch_block_ws(int mode, int dtype, int blocks, int nc, cudaStream_t s, const ExecArgs &a,
                            cudaEvent_t ev_start, cudaEvent_t ev_stop);
// Pre-pass of partition launches with value flags: resets vec[0..n*k) to the all-ones pattern
// and writes rdiag[i] = 1 / L_ii (L's diagonal is the last entry of each row).
// The diagonal is Lv[diag_at[i]] instead when diag_at is given (L read from A's storage); vec2,
// when given, is reset too (a second published vector).
cudaError_t launch_rdiag(int dtype, int n, int k, const int *Lrp, const void *Lv, void *vec, void *rdiag,
                         ExecState *st, cudaStream_t s, const int *diag_at = nullptr, void *vec2 = nullptr);
// Table 2 combinations 1 (SpTRSV -> SpTRSV) and 6 (SpILU0 -> SpTRSV); ILU0 launches run whole-warp
// rows with value flags only.
cudaError_t launch_exec_next(int mode, int dtype, int lpr, bool vf, int team, int minb, int blocks, cudaStream_t s,
                             const ExecArgs &a);
int occupancy_next(int mode, int dtype, int lpr, bool vf, int team, int minb);
// Single-CTA executor (exec_mode 5, k = 1): one CTA per block of the per-instance row-block
// order (a.order, a.seg_ptr, a.block_ptr, a.block_seg, a.n_blocks; inst_ptr the instances'
// first rows; bperm the launch order of the blocks), cta_per_sm CTAs per SM (0 automatic).
// vbuf: n values of 8 bytes with every bit set, through which a single SpTRSV -> SpMV system
// hands x to its helper CTAs (left in that state by every launch); NULL runs no helpers.
cudaError_t launch_cta_exec(int mode, int dtype, const int *inst_ptr, const int *bperm, int cta_per_sm, int sms,
                            void *vbuf, cudaStream_t s, const ExecArgs &a, cudaEvent_t ev_start, cudaEvent_t ev_stop);
constexpr int kIluMaxRow = 256;   // longest row of A an ILU0 row keeps on chip
int occupancy_fwd(int mode, int dtype, int lpr, bool vf, int team, int minb);
int occupancy_pair(int mode, int dtype, int lpr, bool vf, int team, int minb);
cudaError_t launch_exec_trsv(int dtype, int lpr, bool vf, int team, int minb, int blocks, cudaStream_t s,
                             const ExecArgs &a);
int occupancy_trsv(int dtype, int lpr, bool vf, int team, int minb);
cudaError_t launch_exec_adj2(int dtype, int lpr, bool vf, int team, int minb, int blocks, cudaStream_t s,
                             const ExecArgs &a);
int occupancy_adj2(int dtype, int lpr, bool vf, int team, int minb);
cudaError_t launch_exec_ic0(int mode, int dtype, int lpr, bool vf, int team, int minb, int blocks, cudaStream_t s,
                            const ExecArgs &a);
int occupancy_ic0(int mode, int dtype, int lpr, bool vf, int team, int minb);
cudaError_t launch_exec_ic0_alone(int dtype, int lpr, bool vf, int team, int minb, int blocks, cudaStream_t s,
                                  const ExecArgs &a);
int occupancy_ic0_alone(int dtype, int lpr, bool vf, int team, int minb);
int occupancy_adj(int mode, int dtype, int lpr, bool vf, int team, int minb);
// Adjoint helpers: dst[t] = src[perm[t]] (values in transposed order), and the value
// gradients out[e] = sign * sum_c coef[row_of[e]*k+c] * vec[ci[e]*k+c] over every entry of a
// pattern (row_of: the row of each entry).
cudaError_t launch_gather_vals(int dtype, long long nnz, const int *perm, const void *src, void *dst, cudaStream_t s);
cudaError_t launch_grad_entries(int dtype, long long nnz, int k, const int *row_of, const int *ci, const void *coef,
                                const void *vec, double sign, void *out, cudaStream_t s);
// Sets the thread-local text returned by sf_last_error_detail.
void set_error_detail(const char *msg);
cudaError_t launch_spmv(int dtype, int lpr, int kt, int nrows, int k, const int *rp, const int *ci,
                        const void *v, const void *x, const void *b, void *y, cudaStream_t s);

// ---------------------------------------------------------------------------------------
// PTX helpers: the memory-model operations the executor and inspector rely on.
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned ld_relaxed_u32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.relaxed.gpu.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u32(unsigned *p, unsigned v) {
    asm volatile("st.release.gpu.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed_u32(unsigned *p, unsigned v) {
    asm volatile("st.relaxed.gpu.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned atom_add_acq_rel_u32(unsigned *p, unsigned v) {
    unsigned old;
    asm volatile("atom.acq_rel.gpu.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}
__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void record_error(ExecState *st, unsigned code, int row) {
    if (atomicCAS(&st->err_code, 0u, code) == 0u) st->err_row = row;
}

}  // namespace sf
