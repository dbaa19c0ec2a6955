// Inspector building blocks (declarations).
#pragma once

#include <vector>

#include "sf_internal.cuh"

namespace sf {

// Device allocations that are released together (temporaries of one inspector call, or
// the arrays a schedule owns).
// Device allocations released together. A temporary arena (constructed with a stream) takes
// stream-ordered memory from the library's pool of the current device, which keeps up to
// 1 GiB of freed memory for the next inspection instead of returning it to the driver; a
// persistent arena (no stream) uses cudaMalloc.
struct Arena {
    std::vector<void *> ptrs;
    bool oom = false;
    bool pooled = false;
    cudaStream_t stream = nullptr;
    Arena() = default;
    explicit Arena(cudaStream_t s) : pooled(true), stream(s) {}
    Arena(const Arena &) = delete;
    Arena &operator=(const Arena &) = delete;
    void *alloc(size_t bytes);
    ~Arena();
};

struct DevCsr {
    int n_rows = 0, n_cols = 0;
    long long nnz = 0;
    int *rowptr = nullptr;
    int *colidx = nullptr;
};

// Transposed pattern plus, per transposed entry, the index of that entry in the source
// CSR (to read the source's values in transposed order).
struct DevCsrT {
    DevCsr t;
    int *perm = nullptr;
};

struct KahnCtl {
    unsigned cnt[3];
    unsigned nsrc;
    unsigned bar_count;
    unsigned bar_gen;
    unsigned err;
    unsigned depth;
    unsigned processed;
};

struct InstDesc {
    const int *rowptr;
    const int *colidx;
    int n;
    int row_off;
    int nnz;
    int nnz_off;
};

// pattern violation codes (high word of the status of k_check_csr)
enum PatCode : unsigned {
    PAT_ROWPTR0 = 1, PAT_NNZ = 2, PAT_ROWPTR = 3, PAT_COL_RANGE = 4, PAT_UNSORTED = 5, PAT_DIAG = 6
};

// Pattern check kernel: minimises (code << 32 | row) of the first violation into *status.
__global__ void k_check_csr(int n_rows, int n_cols, long long nnz, const int *__restrict__ rp,
                            const int *__restrict__ ci, int lower, unsigned long long *status);

int bits_for(unsigned long long maxval);
template <typename T>
cudaError_t scan_excl(const T *in, T *out, long long n, cudaStream_t s, Arena &ar);
cudaError_t radix_sort_pairs(unsigned *keys, unsigned *vals, long long n, int bits, cudaStream_t s, Arena &ar);
cudaError_t check_pattern(const DevCsr &m, int lower, unsigned long long *status_host, cudaStream_t s, Arena &ar);
// a_diag[i] = position of A_ii in row i of A (-1: missing); *bad_host bit 0: a diagonal is
// missing, bit 1: L's pattern is not tril(A)'s. Synchronises s.
cudaError_t tril_map(const DevCsr &A, const DevCsr &L, int *a_diag, unsigned *bad_host, cudaStream_t s, Arena &ar);
// row_of[e] = the row of entry e of m.
cudaError_t row_of_entries(const DevCsr &m, int *row_of, cudaStream_t s);
cudaError_t transpose_csr(const DevCsr &src, DevCsrT &dst, cudaStream_t s, Arena &ar, Arena &keep);
cudaError_t kahn_levels(long long nv, int n1, const int *s1rp, const int *s1ci, const int *s2rp, const int *s2ci,
                        int *level, int *depth_out, cudaStream_t s, Arena &ar, bool *timed_out);
cudaError_t build_order(long long nv, int n1, const int *level, int depth, int *order, cudaStream_t s, Arena &ar);
cudaError_t vertex_costs(int what, int n, const DevCsr &L, const DevCsr *M, const DevCsrT *LT, const DevCsrT *MT,
                         int *cost, cudaStream_t s);
cudaError_t prefix_costs(long long nv, int n1, const int *order, const int *cost, long long *cs, long long *S,
                         long long *total, cudaStream_t s, Arena &ar);
cudaError_t cut_partitions(long long nv, const long long *S, const long long *cs, long long C, long long W,
                           int *part_ptr, unsigned char *part_wide, int *n_parts, cudaStream_t s, Arena &ar);
cudaError_t place_g2(int n, int depth, int mode, int *level, cudaStream_t s);
// IC0 intersection pairs (per L entry: the (p, q) positions of its common columns); nothing is
// built (*pp_out NULL) when the total exceeds max_pairs.
cudaError_t build_ic0_pairs(const DevCsr &L, long long max_pairs, int **pp_out, int2 **pairs_out, long long *np_out,
                            cudaStream_t s, Arena &ar, Arena &keep);
cudaError_t split_partition_classes(int P, const int *part_ptr, const int *order, int *plist, int *n_class0,
                                    cudaStream_t s, Arena &ar);
// Row-block order: blocks of B rows, or (inst_ptr != NULL) one block per instance of a
// block-diagonal system, inst_ptr[0..n_inst] being the instances' first rows.
cudaError_t build_block_order(int kind, int n, long long nv, int B, int depth, const int *level, const DevCsr *M,
                              const DevCsrT *MT, const int *inst_ptr, int n_inst, int *order, int *block_ptr,
                              int *seg_ptr, int *block_seg, int *nb_out, int *n_segs_out, int *max_width_out,
                              cudaStream_t s, Arena &ar);
cudaError_t build_block_desc(int kind, long long nv, const int *order, const DevCsr &L, const DevCsr *M,
                             const DevCsrT &LT, const DevCsrT *MT, int2 *desc, cudaStream_t s);
cudaError_t concat_patterns(const std::vector<InstDesc> &h, int *rp_out, int *ci_out, long long total_nnz,
                            int total_rows, cudaStream_t s, Arena &ar);

}  // namespace sf
