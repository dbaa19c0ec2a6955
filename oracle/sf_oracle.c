/*
 * Sequential FP64 oracle for the sparse-fusion hot path.
 *
 * TEST INFRASTRUCTURE. Only the tests, the smoke check and the benchmark's CPU-baseline
 * leg load this file; the library under paper_2111_12238_gb300/ never does. It shares
 * no code, header, table or helper with the CUDA path.
 *
 * Every routine is the plain definition, run unfused and in program order: sparse
 * fusion (§2, §2.3) only reorders the iterations of the two kernels subject to their
 * dependences, so the fused result must equal the result of running the first kernel to
 * completion and then the second one. Scheduling objects (levels, the linearised order,
 * the partition cut and the validity check) are re-derived here by different algorithms
 * from the ones the GPU inspector uses (a sequential longest-path recurrence instead of
 * Kahn peeling, a counting sort instead of a radix sort).
 *
 * Conventions: CSR with int32 rowptr[n+1] and colidx[nnz] (ascending within a row),
 * double values in CSR order; dense blocks are n x k row-major.
 * Return codes: 0 on success; -(i+1) for a missing or zero diagonal at row i;
 * +(i+1) for an incomplete-Cholesky breakdown (non-positive pivot) at row i, or for a zero
 * incomplete-LU pivot u_ii.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OK 0

/* position of the diagonal entry of row i, or -1 */
static int64_t diag_pos(const int32_t *rp, const int32_t *ci, int32_t i) {
    for (int64_t e = rp[i]; e < rp[i + 1]; ++e)
        if (ci[e] == i) return e;
    return -1;
}

/* ------------------------------------------------------------------ kernels (§2, Table 2) */

/* SpTRSV, forward substitution L x = b (Table 2, "SpTRSV CSR"):
 * x_i = (b_i - sum_{j<i, L_ij != 0} L_ij x_j) / L_ii, rows in order, terms in ascending j. */
int orc_trsv_lower(int32_t n, int32_t k, const int32_t *rp, const int32_t *ci, const double *v,
                   const double *b, double *x) {
    for (int32_t i = 0; i < n; ++i) {
        int64_t d = diag_pos(rp, ci, i);
        if (d < 0 || v[d] == 0.0) return -(i + 1);
        for (int32_t c = 0; c < k; ++c) {
            double s = b[(int64_t)i * k + c];
            for (int64_t e = rp[i]; e < rp[i + 1]; ++e)
                if (ci[e] < i) s -= v[e] * x[(int64_t)ci[e] * k + c];
            x[(int64_t)i * k + c] = s / v[d];
        }
    }
    return OK;
}

/* SpMV y = M x (Table 2, "SpMV CSR"): y_i = sum_j M_ij x_j in ascending j. */
int orc_spmv(int32_t nrows, int32_t k, const int32_t *rp, const int32_t *ci, const double *v,
             const double *x, double *y) {
    for (int32_t i = 0; i < nrows; ++i)
        for (int32_t c = 0; c < k; ++c) {
            double s = 0.0;
            for (int64_t e = rp[i]; e < rp[i + 1]; ++e) s += v[e] * x[(int64_t)ci[e] * k + c];
            y[(int64_t)i * k + c] = s;
        }
    return OK;
}

/* Residual r = b - M x, row by row: r_i = b_i - sum_j M_ij x_j (the SpMV of Table 2,
 * combination 2, with the right-hand side of the following solve folded in). */
int orc_residual(int32_t nrows, int32_t k, const int32_t *rp, const int32_t *ci, const double *v,
                 const double *x, const double *b, double *r) {
    for (int32_t i = 0; i < nrows; ++i)
        for (int32_t c = 0; c < k; ++c) {
            double s = 0.0;
            for (int64_t e = rp[i]; e < rp[i + 1]; ++e) s += v[e] * x[(int64_t)ci[e] * k + c];
            r[(int64_t)i * k + c] = b[(int64_t)i * k + c] - s;
        }
    return OK;
}

/* SpIC0, zero fill-in incomplete Cholesky L L^T ~ A on the pattern of tril(A) (Table 2,
 * "SpIC0"), in its up-looking row form. For each row i and each j < i in the row, in
 * ascending order:
 *   L_ij = (A_ij - sum_{k < j, k in pat(i) and pat(j)} L_ik L_jk) / L_jj,
 * then L_ii = sqrt(A_ii - sum_{k < i} L_ik^2). a holds tril(A) in the same CSR. */
int orc_ic0(int32_t n, const int32_t *rp, const int32_t *ci, const double *a, double *l) {
    for (int32_t i = 0; i < n; ++i) {
        int64_t di = diag_pos(rp, ci, i);
        if (di < 0) return -(i + 1);
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
            int32_t j = ci[e];
            if (j >= i) continue;
            double s = a[e];
            /* intersection of row i (entries before e) with row j (columns < j) */
            int64_t f = rp[i], g = rp[j];
            while (f < e && g < rp[j + 1] && ci[g] < j) {
                if (ci[f] == ci[g]) { s -= l[f] * l[g]; ++f; ++g; }
                else if (ci[f] < ci[g]) ++f;
                else ++g;
            }
            int64_t dj = diag_pos(rp, ci, j);
            if (dj < 0) return -(j + 1);
            l[e] = s / l[dj];
        }
        double s = a[di];
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e)
            if (ci[e] < i) s -= l[e] * l[e];
        if (!(s > 0.0)) return i + 1;
        l[di] = sqrt(s);
    }
    return OK;
}

/* Transposed solve L^T lam = u by backward substitution over the columns of L^T (the rows
 * of L), j = n-1 .. 0: lam_j = w_j / L_jj, then w_i -= L_ji lam_j for the j-row entries
 * i < j. */
int orc_trsv_lower_T(int32_t n, int32_t k, const int32_t *rp, const int32_t *ci, const double *v,
                     const double *u, double *lam) {
    double *w = (double *)malloc(sizeof(double) * (size_t)n * (size_t)(k > 0 ? k : 1));
    if (!w) return -1;
    memcpy(w, u, sizeof(double) * (size_t)n * (size_t)k);
    for (int32_t j = n - 1; j >= 0; --j) {
        int64_t d = diag_pos(rp, ci, j);
        if (d < 0 || v[d] == 0.0) { free(w); return -(j + 1); }
        for (int32_t c = 0; c < k; ++c) lam[(int64_t)j * k + c] = w[(int64_t)j * k + c] / v[d];
        for (int64_t e = rp[j]; e < rp[j + 1]; ++e)
            if (ci[e] < j)
                for (int32_t c = 0; c < k; ++c)
                    w[(int64_t)ci[e] * k + c] -= v[e] * lam[(int64_t)j * k + c];
    }
    free(w);
    return OK;
}

/* u = M^T g for an nrows x ncols CSR M: u_j = sum_i M_ij g_i, accumulated row by row. */
int orc_spmv_T(int32_t nrows, int32_t ncols, int32_t k, const int32_t *rp, const int32_t *ci,
               const double *v, const double *g, double *u) {
    memset(u, 0, sizeof(double) * (size_t)ncols * (size_t)k);
    for (int32_t i = 0; i < nrows; ++i)
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e)
            for (int32_t c = 0; c < k; ++c)
                u[(int64_t)ci[e] * k + c] += v[e] * g[(int64_t)i * k + c];
    return OK;
}

/* ------------------------------------------------------------------ the three pairs (Table 2) */

/* Combination 4 in CSR form: x = L^-1 b, then y = M x. */
int orc_trsv_spmv(int32_t n, int32_t k, const int32_t *lrp, const int32_t *lci, const double *lv,
                  const int32_t *mrp, const int32_t *mci, const double *mv, const double *b,
                  double *x, double *y) {
    int st = orc_trsv_lower(n, k, lrp, lci, lv, b, x);
    if (st) return st;
    return orc_spmv(n, k, mrp, mci, mv, x, y);
}

/* Combination 2: r = b - A x_in, then z = L^-1 r (one Gauss-Seidel half-sweep when
 * L = tril(A)). */
int orc_spmv_trsv(int32_t n, int32_t k, const int32_t *arp, const int32_t *aci, const double *av,
                  const int32_t *lrp, const int32_t *lci, const double *lv, const double *x_in,
                  const double *b, double *z) {
    double *r = (double *)malloc(sizeof(double) * (size_t)n * (size_t)(k > 0 ? k : 1));
    if (!r) return -1;
    orc_residual(n, k, arp, aci, av, x_in, b, r);
    int st = orc_trsv_lower(n, k, lrp, lci, lv, r, z);
    free(r);
    return st;
}

/* Combination 5 in CSR form: L L^T ~ A (zero fill-in), then y = L^-1 b. */
int orc_ic0_trsv(int32_t n, int32_t k, const int32_t *rp, const int32_t *ci, const double *a,
                 const double *b, double *lfac, double *y) {
    int st = orc_ic0(n, rp, ci, a, lfac);
    if (st) return st;
    return orc_trsv_lower(n, k, rp, ci, lfac, b, y);
}

/* Table 2 combination 1: x = L^-1 b, then z = L^-1 x with the same L (two forward
 * substitutions in program order). */
int orc_trsv_trsv(int32_t n, int32_t k, const int32_t *rp, const int32_t *ci, const double *v,
                  const double *b, double *x, double *z) {
    int st = orc_trsv_lower(n, k, rp, ci, v, b, x);
    if (st) return st;
    return orc_trsv_lower(n, k, rp, ci, v, x, z);
}

/* position of column j in row i (ascending columns), or -1 */
static int64_t find_col(const int32_t *rp, const int32_t *ci, int32_t i, int32_t j) {
    int64_t lo = rp[i], hi = rp[i + 1];
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (ci[mid] < j) lo = mid + 1;
        else hi = mid;
    }
    return (lo < rp[i + 1] && ci[lo] == j) ? lo : -1;
}

/* Zero fill-in incomplete LU of a square A with its diagonal present (Table 2 combination 6),
 * in the row-oriented IKJ form (Saad, Iterative Methods for Sparse Linear Systems, Alg. 10.4):
 * for each row i, for each k < i in the row, ascending: a_ik /= u_kk, then every later entry
 * a_ij of row i with (k, j) in the pattern loses a_ik * u_kj. The result lu holds the strictly
 * lower part of the unit lower factor L and the upper factor U (diagonal included) on A's
 * pattern. Returns -(i+1) for a missing diagonal, +(k+1) for a zero pivot u_kk. */
int orc_ilu0(int32_t n, const int32_t *rp, const int32_t *ci, const double *a, double *lu) {
    memcpy(lu, a, sizeof(double) * (size_t)rp[n]);
    for (int32_t i = 0; i < n; ++i)
        if (diag_pos(rp, ci, i) < 0) return -(i + 1);
    for (int32_t i = 0; i < n; ++i) {
        for (int64_t e = rp[i]; e < rp[i + 1] && ci[e] < i; ++e) {
            int32_t kr = ci[e];
            int64_t dk = diag_pos(rp, ci, kr);
            if (lu[dk] == 0.0) return kr + 1;
            lu[e] /= lu[dk];
            for (int64_t f = e + 1; f < rp[i + 1]; ++f) {
                int64_t g = find_col(rp, ci, kr, ci[f]);
                if (g >= 0) lu[f] -= lu[e] * lu[g];
            }
        }
    }
    return OK;
}

/* ILU0, then y = L^-1 b with the unit lower factor L of lu (Table 2 combination 6). */
int orc_ilu0_trsv(int32_t n, int32_t k, const int32_t *rp, const int32_t *ci, const double *a,
                  const double *b, double *lu, double *y) {
    int st = orc_ilu0(n, rp, ci, a, lu);
    if (st) return st;
    for (int32_t i = 0; i < n; ++i)
        for (int32_t c = 0; c < k; ++c) {
            double s = b[(int64_t)i * k + c];
            for (int64_t e = rp[i]; e < rp[i + 1] && ci[e] < i; ++e) s -= lu[e] * y[(int64_t)ci[e] * k + c];
            y[(int64_t)i * k + c] = s;
        }
    return OK;
}

/* Adjoint of y = M L^-1 b with x = L^-1 b (not in the paper; closed forms):
 * u = M^T gy, lam = L^-T u, gb = lam, gL_ij = -sum_c lam_ic x_jc on pattern(L),
 * gM_ij = sum_c gy_ic x_jc on pattern(M). gL, gM may be NULL. */
int orc_adj_trsv_spmv(int32_t n, int32_t k, const int32_t *lrp, const int32_t *lci,
                      const double *lv, const int32_t *mrp, const int32_t *mci, const double *mv,
                      const double *x, const double *gy, double *gb, double *gL, double *gM) {
    double *u = (double *)malloc(sizeof(double) * (size_t)n * (size_t)(k > 0 ? k : 1));
    if (!u) return -1;
    orc_spmv_T(n, n, k, mrp, mci, mv, gy, u);
    int st = orc_trsv_lower_T(n, k, lrp, lci, lv, u, gb);
    free(u);
    if (st) return st;
    for (int32_t i = 0; i < n; ++i) {
        if (gL)
            for (int64_t e = lrp[i]; e < lrp[i + 1]; ++e) {
                double s = 0.0;
                for (int32_t c = 0; c < k; ++c)
                    s += gb[(int64_t)i * k + c] * x[(int64_t)lci[e] * k + c];
                gL[e] = -s;
            }
        if (gM)
            for (int64_t e = mrp[i]; e < mrp[i + 1]; ++e) {
                double s = 0.0;
                for (int32_t c = 0; c < k; ++c)
                    s += gy[(int64_t)i * k + c] * x[(int64_t)mci[e] * k + c];
                gM[e] = s;
            }
    }
    return OK;
}

/* Adjoint of z = L^-1 (b - A x_in) (not in the paper; closed forms):
 * lam = L^-T gz, gb = lam, gx = -A^T lam, gL_ij = -sum_c lam_ic z_jc,
 * gA_ij = -sum_c lam_ic x_in_jc. gx, gL, gA may be NULL. */
int orc_adj_spmv_trsv(int32_t n, int32_t k, const int32_t *arp, const int32_t *aci,
                      const double *av, const int32_t *lrp, const int32_t *lci, const double *lv,
                      const double *x_in, const double *z, const double *gz, double *gb,
                      double *gx, double *gL, double *gA) {
    int st = orc_trsv_lower_T(n, k, lrp, lci, lv, gz, gb);
    if (st) return st;
    if (gx) {
        orc_spmv_T(n, n, k, arp, aci, av, gb, gx);
        for (int64_t t = 0; t < (int64_t)n * k; ++t) gx[t] = -gx[t];
    }
    for (int32_t i = 0; i < n; ++i) {
        if (gL)
            for (int64_t e = lrp[i]; e < lrp[i + 1]; ++e) {
                double s = 0.0;
                for (int32_t c = 0; c < k; ++c)
                    s += gb[(int64_t)i * k + c] * z[(int64_t)lci[e] * k + c];
                gL[e] = -s;
            }
        if (gA)
            for (int64_t e = arp[i]; e < arp[i + 1]; ++e) {
                double s = 0.0;
                for (int32_t c = 0; c < k; ++c)
                    s += gb[(int64_t)i * k + c] * x_in[(int64_t)aci[e] * k + c];
                gA[e] = -s;
            }
    }
    return OK;
}

/* ------------------------------------------------------------------ schedule objects */
/* Schedule kinds (one joint DAG each):
 *   0 SEP     : SpTRSV rows (tag 0, vertices 0..n-1) then SpMV rows (tag 1, n..2n-1),
 *               DAG edges j->i for L_ij != 0, j < i (§2.2: the DAG of SpTRSV is L) and
 *               F edges j->n+i for M_ij != 0 (F = pattern(M), §2.2 "Dependency Matrix F").
 *   1 PAIRED  : one vertex per row i holding both kernels' iteration i (F = I); edges of L.
 *   2 PAIRED_T: transposed DAG for the adjoint of SpTRSV->SpMV: edges i->j for L_ij != 0,
 *               i > j.
 *   3 SEP_T   : adjoint of SpMV->SpTRSV: tag 0 = rows of L^T solve (edges i->j for
 *               L_ij != 0, i > j), tag 1 = rows of A^T (edges i -> n+j for A_ij != 0).
 * The wavefront number of §3.1 / §3.2.2 is the longest-path level, 0-based here:
 * level(v) = 0 without predecessors, else 1 + max over predecessors. */

int orc_levels(int32_t kind, int32_t n, const int32_t *lrp, const int32_t *lci,
               const int32_t *mrp, const int32_t *mci, int32_t *level) {
    if (kind == 0 || kind == 1) {
        for (int32_t i = 0; i < n; ++i) {
            int32_t lv = 0;
            for (int64_t e = lrp[i]; e < lrp[i + 1]; ++e)
                if (lci[e] < i && level[lci[e]] + 1 > lv) lv = level[lci[e]] + 1;
            level[i] = lv;
        }
        if (kind == 0)
            for (int32_t i = 0; i < n; ++i) {
                int32_t lv = 0;
                for (int64_t e = mrp[i]; e < mrp[i + 1]; ++e)
                    if (level[mci[e]] + 1 > lv) lv = level[mci[e]] + 1;
                level[n + i] = lv;
            }
        return OK;
    }
    if (kind == 2 || kind == 3) {
        for (int32_t j = 0; j < n; ++j) level[j] = 0;
        for (int32_t i = n - 1; i >= 0; --i)          /* level[i] is final when row i is reached */
            for (int64_t e = lrp[i]; e < lrp[i + 1]; ++e)
                if (lci[e] < i && level[i] + 1 > level[lci[e]]) level[lci[e]] = level[i] + 1;
        if (kind == 3) {
            for (int32_t j = 0; j < n; ++j) level[n + j] = -1;
            for (int32_t i = 0; i < n; ++i)
                for (int64_t e = mrp[i]; e < mrp[i + 1]; ++e)
                    if (level[i] + 1 > level[n + mci[e]]) level[n + mci[e]] = level[i] + 1;
            for (int32_t j = 0; j < n; ++j)
                if (level[n + j] < 0) level[n + j] = 0;
        }
        return OK;
    }
    return -1;
}

/* Vertex cost c(v) (§3.1: the number of nonzeros the iteration touches), plus one so that
 * every vertex costs something. Per kind and tag:
 *   SEP    tag 0: nnz(L_i) + 1                  tag 1: nnz(M_i) + 1
 *   PAIRED (SpMV->SpTRSV, kernel 3): nnz(A_i) + nnz(L_i) + 1
 *   PAIRED (SpIC0->SpTRSV, kernel 4): 2 nnz(L_i) + sum_{j in L_i, j<i} nnz(L_j) + 1
 *   PAIRED (SpTRSV alone, kernel 5): nnz(L_i) + 1
 *   PAIRED (SpIC0 alone, kernel 6): nnz(L_i) + sum_{j in L_i, j<i} nnz(L_j) + 1
 *   PAIRED (SpTRSV->SpTRSV, kernel 7): 2 nnz(L_i) + 1 (the row is read by both solves)
 *   PAIRED (SpILU0->SpTRSV, kernel 8, M = A, L = tril(A)):
 *          nnz(A_i) + sum_{j in L_i, j<i} nnz(A_j) + nnz(L_i) + 1
 *   PAIRED_T (kernel 2): nnz(M^T_j) + nnz(L^T_j) + 1
 *   SEP_T  tag 0: nnz(L^T_j) + 1      tag 1: nnz(A^T_j) + 1
 * (the adjoint's value gradients are a separate streaming pass, not part of these items)
 * `what` selects the formula: 0 SEP, 1 PAIRED_T, 2 SEP_T, 3 SpMV->SpTRSV,
 * 4 SpIC0->SpTRSV, 5 SpTRSV, 6 SpIC0, 7 SpTRSV->SpTRSV, 8 SpILU0->SpTRSV. Output cost[v]
 * for every vertex. */
int orc_costs(int32_t what, int32_t n, const int32_t *lrp, const int32_t *lci, const int32_t *mrp,
              const int32_t *mci, int64_t *cost) {
    int64_t *colL = NULL, *colM = NULL;
    if (what == 1 || what == 2) {
        colL = (int64_t *)calloc((size_t)n, sizeof(int64_t));
        colM = (int64_t *)calloc((size_t)n, sizeof(int64_t));
        if (!colL || !colM) { free(colL); free(colM); return -1; }
        for (int64_t e = 0; e < lrp[n]; ++e) colL[lci[e]]++;
        for (int64_t e = 0; e < mrp[n]; ++e) colM[mci[e]]++;
    }
    for (int32_t i = 0; i < n; ++i) {
        int64_t nl = lrp[i + 1] - lrp[i];
        int64_t nm = mrp ? (int64_t)(mrp[i + 1] - mrp[i]) : 0;
        int64_t s = 0;
        if (what == 4 || what == 6)
            for (int64_t e = lrp[i]; e < lrp[i + 1]; ++e)
                if (lci[e] < i) s += lrp[lci[e] + 1] - lrp[lci[e]];
        if (what == 8) /* rows k of A that row i of SpILU0 eliminates with */
            for (int64_t e = lrp[i]; e < lrp[i + 1]; ++e)
                if (lci[e] < i) s += mrp[lci[e] + 1] - mrp[lci[e]];
        switch (what) {
            case 0: cost[i] = nl + 1; cost[n + i] = nm + 1; break;
            case 1: cost[i] = colM[i] + colL[i] + 1; break;
            case 2: cost[i] = colL[i] + 1; cost[n + i] = colM[i] + 1; break;
            case 3: cost[i] = nm + nl + 1; break;
            case 4: cost[i] = 2 * nl + s + 1; break;
            case 5: cost[i] = nl + 1; break;
            case 6: cost[i] = nl + s + 1; break;
            case 7: cost[i] = 2 * nl + 1; break;
            case 8: cost[i] = nm + s + nl + 1; break;
            default: free(colL); free(colM); return -1;
        }
    }
    free(colL);
    free(colM);
    return OK;
}

/* Placement of the second kernel's vertices in a separated schedule (kinds 0 and 3), using
 * their slack (§3.2.2): such a vertex (an SpMV row, or an A^T row of the adjoint) is a sink of
 * the joint DAG, so any wavefront from its earliest one (the longest-path level) to the last
 * one, depth - 1, keeps every edge pointing forward. mode 0 keeps the earliest wavefront,
 * mode < 0 moves every such vertex to the last wavefront (as late as possible), mode d > 0
 * delays it by d wavefronts, at most to the last. Levels of the first kernel are unchanged,
 * and so is the depth. Paired kinds are left as they are. */
void orc_place_g2(int32_t kind, int32_t n, int32_t *level, int32_t mode) {
    if ((kind != 0 && kind != 3) || mode == 0) return;
    int32_t depth = 0;
    for (int64_t v = 0; v < 2LL * n; ++v)
        if (level[v] + 1 > depth) depth = level[v] + 1;
    for (int64_t v = n; v < 2LL * n; ++v) {
        int64_t l = mode < 0 ? depth - 1 : (int64_t)level[v] + mode;
        level[v] = (int32_t)(l < depth - 1 ? l : depth - 1);
    }
}

/* Linearised order of the joint DAG: vertices sorted by (level, tag, row), the canonical
 * tie-break among the many valid topological orders. Vertex v = tag*n + row is encoded as
 * row | tag << 31. Counting sort by level over vertices in increasing v. */
int orc_order(int64_t nv, int32_t n, const int32_t *level, int32_t *order) {
    int32_t depth = 0;
    for (int64_t v = 0; v < nv; ++v)
        if (level[v] + 1 > depth) depth = level[v] + 1;
    int64_t *start = (int64_t *)calloc((size_t)depth + 1, sizeof(int64_t));
    if (!start) return -1;
    for (int64_t v = 0; v < nv; ++v) start[level[v] + 1]++;
    for (int32_t l = 0; l < depth; ++l) start[l + 1] += start[l];
    for (int64_t v = 0; v < nv; ++v) {
        uint32_t tag = (uint32_t)(v / n), row = (uint32_t)(v % n);
        order[start[level[v]]++] = (int32_t)(row | (tag << 31));
    }
    free(start);
    return depth;
}

/* Partition cut of the linearised order (coarsening of consecutive wavefronts, §3.1,
 * into contiguous work items): with S_q the exclusive prefix sum of c(order[q]), item q
 * belongs to partition floor(S_q / C); partitions are the maximal runs of equal quotient.
 * An item whose cost exceeds W (W > 0) is "wide" and sits in a partition of its own.
 * Writes part_ptr[0..P] and returns P. */
int64_t orc_partition(int64_t nv, int32_t n, const int32_t *order, const int64_t *cost,
                      int64_t C, int64_t W, int32_t *part_ptr) {
    int64_t S = 0, P = 0, prev = -1;
    int prev_wide = 0;
    for (int64_t q = 0; q < nv; ++q) {
        uint32_t o = (uint32_t)order[q];
        int64_t v = (int64_t)(o >> 31) * n + (o & 0x7fffffffu);
        int64_t p = S / C;
        int wide = W > 0 && cost[v] > W;
        if (q == 0 || p != prev || wide || prev_wide) part_ptr[P++] = (int32_t)q;
        prev = p;
        prev_wide = wide;
        S += cost[v];
    }
    part_ptr[P] = (int32_t)nv;
    return P;
}

/* Row-block order (the schedule of the row-block executor). Rows are cut into blocks of B
 * consecutive rows, taken in increasing row order for the forward kinds and in decreasing
 * row order for the transposed ones (so that every dependence points to the same or an
 * earlier block). A vertex belongs to the block of its own row for the first kernel; a
 * second-kernel vertex belongs to the latest block among the rows it reads (block 0 if it
 * reads none). Vertices are ordered by (block, level, tag, row). Writes order[nv] and
 * block_ptr[nb+1]; returns nb = ceil(n / B). */
int64_t orc_block_order(int32_t kind, int32_t n, const int32_t *lrp, const int32_t *lci,
                        const int32_t *mrp, const int32_t *mci, const int32_t *level, int64_t B,
                        int32_t *order, int32_t *block_ptr) {
    const int64_t nb = (n + B - 1) / B;
    const int64_t nv = (kind == 0 || kind == 3) ? 2LL * n : n;
    const int rev = kind == 2 || kind == 3;
    int64_t *blk = (int64_t *)malloc(sizeof(int64_t) * (size_t)nv);
    if (!blk) return -1;
    for (int32_t i = 0; i < n; ++i) blk[i] = rev ? nb - 1 - i / B : i / B;
    if (kind == 0)                       /* SpMV row i reads x_j for M_ij != 0 */
        for (int32_t i = 0; i < n; ++i) {
            int64_t b = 0;
            for (int64_t e = mrp[i]; e < mrp[i + 1]; ++e)
                if (blk[mci[e]] > b) b = blk[mci[e]];
            blk[n + i] = b;
        }
    if (kind == 3) {                     /* A^T row j reads lam_i for A_ij != 0 */
        for (int32_t j = 0; j < n; ++j) blk[n + j] = 0;
        for (int32_t i = 0; i < n; ++i)
            for (int64_t e = mrp[i]; e < mrp[i + 1]; ++e)
                if (blk[i] > blk[n + mci[e]]) blk[n + mci[e]] = blk[i];
    }
    int32_t depth = 0;
    for (int64_t v = 0; v < nv; ++v)
        if (level[v] + 1 > depth) depth = level[v] + 1;
    const int64_t nkeys = nb * depth;
    int64_t *start = (int64_t *)calloc((size_t)nkeys + 1, sizeof(int64_t));
    if (!start) { free(blk); return -1; }
    for (int64_t v = 0; v < nv; ++v) start[blk[v] * depth + level[v] + 1]++;
    for (int64_t t = 0; t < nkeys; ++t) start[t + 1] += start[t];
    for (int64_t b = 0; b <= nb; ++b) block_ptr[b] = (int32_t)start[b * depth];
    for (int64_t v = 0; v < nv; ++v) {
        uint32_t tag = (uint32_t)(v / n), row = (uint32_t)(v % n);
        order[start[blk[v] * depth + level[v]]++] = (int32_t)(row | (tag << 31));
    }
    free(start);
    free(blk);
    return nb;
}

/* Row-block order with one block per instance of a block-diagonal system (the schedule of
 * the single-CTA executor): instance t holds rows [inst_ptr[t], inst_ptr[t+1]); every vertex,
 * of either kernel, belongs to the instance of its row (the instances share no entry, so no
 * dependence crosses a block). Vertices are ordered by (block, level, tag, row). Writes
 * order[nv] and block_ptr[n_inst+1]; returns n_inst, or -1 on a bad argument. */
int64_t orc_block_order_instances(int32_t kind, int32_t n, const int32_t *level, int32_t n_inst,
                                  const int32_t *inst_ptr, int32_t *order, int32_t *block_ptr) {
    if (n_inst < 1 || inst_ptr[0] != 0 || inst_ptr[n_inst] != n) return -1;
    const int64_t nv = (kind == 0 || kind == 3) ? 2LL * n : n;
    int64_t *blk = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nv > 0 ? nv : 1));
    if (!blk) return -1;
    for (int32_t t = 0; t < n_inst; ++t) {
        if (inst_ptr[t + 1] < inst_ptr[t]) { free(blk); return -1; }
        for (int32_t i = inst_ptr[t]; i < inst_ptr[t + 1]; ++i) {
            blk[i] = t;
            if (nv > n) blk[n + i] = t;
        }
    }
    int32_t depth = 0;
    for (int64_t v = 0; v < nv; ++v)
        if (level[v] + 1 > depth) depth = level[v] + 1;
    const int64_t nkeys = (int64_t)n_inst * depth;
    int64_t *start = (int64_t *)calloc((size_t)nkeys + 1, sizeof(int64_t));
    if (!start) { free(blk); return -1; }
    for (int64_t v = 0; v < nv; ++v) start[blk[v] * depth + level[v] + 1]++;
    for (int64_t t = 0; t < nkeys; ++t) start[t + 1] += start[t];
    for (int64_t b = 0; b <= n_inst; ++b) block_ptr[b] = (int32_t)start[b * depth];
    for (int64_t v = 0; v < nv; ++v) {
        uint32_t tag = (uint32_t)(v / n), row = (uint32_t)(v % n);
        order[start[blk[v] * depth + level[v]]++] = (int32_t)(row | (tag << 31));
    }
    free(start);
    free(blk);
    return n_inst;
}

/* Level segments of a row-block order: a new segment starts at the first position of every
 * block and wherever the level changes from the previous position. The vertices of one
 * segment share a block and a level, so none depends on another (§2.2: every edge of the
 * joint DAG goes from a lower wavefront to a higher one). Writes seg_ptr[nseg+1] (capacity
 * nv+1) and block_seg[nb+1]; returns nseg. */
int64_t orc_block_segments(int32_t kind, int32_t n, int64_t nb, const int32_t *order, const int32_t *block_ptr,
                           const int32_t *level, int32_t *seg_ptr, int32_t *block_seg) {
    const int64_t nv = (kind == 0 || kind == 3) ? 2LL * n : n;
    int64_t ns = 0;
    int32_t prev = -1;
    for (int64_t b = 0; b < nb; ++b) {
        block_seg[b] = (int32_t)ns;
        for (int64_t q = block_ptr[b]; q < block_ptr[b + 1]; ++q) {
            const uint32_t o = (uint32_t)order[q];
            const int64_t v = (int64_t)(o >> 31) * n + (o & 0x7fffffffu);
            if (q == block_ptr[b] || level[v] != prev) seg_ptr[ns++] = (int32_t)q;
            prev = level[v];
        }
    }
    block_seg[nb] = (int32_t)ns;
    seg_ptr[ns] = (int32_t)nv;
    return ns;
}

/* Validity of a schedule (§3.2: a fused schedule must honour every intra- and
 * inter-kernel dependence): order is a permutation of the vertices, every DAG and F edge
 * u -> v has pos(u) < pos(v), partitions are contiguous, non-empty and cover the order.
 * Returns 0 if valid, else a positive code: 1 not a permutation, 2 edge violated,
 * 3 bad partition pointers. */
int orc_validate(int32_t kind, int32_t n, const int32_t *lrp, const int32_t *lci,
                 const int32_t *mrp, const int32_t *mci, const int32_t *order, int64_t nv,
                 const int32_t *part_ptr, int64_t P) {
    int64_t *pos = (int64_t *)malloc(sizeof(int64_t) * (size_t)nv);
    if (!pos) return -1;
    for (int64_t v = 0; v < nv; ++v) pos[v] = -1;
    int rc = 0;
    for (int64_t q = 0; q < nv && !rc; ++q) {
        uint32_t o = (uint32_t)order[q];
        int64_t tag = o >> 31, row = o & 0x7fffffffu;
        int64_t v = tag * n + row;
        if (row >= n || v >= nv || pos[v] >= 0) rc = 1;
        else pos[v] = q;
    }
    for (int32_t i = 0; i < n && !rc; ++i) {
        for (int64_t e = lrp[i]; e < lrp[i + 1] && !rc; ++e) {
            int32_t j = lci[e];
            if (j >= i) continue;
            int ok = (kind == 0 || kind == 1) ? pos[j] < pos[i] : pos[i] < pos[j];
            if (!ok) rc = 2;
        }
        if (kind == 0)
            for (int64_t e = mrp[i]; e < mrp[i + 1] && !rc; ++e)
                if (!(pos[mci[e]] < pos[n + i])) rc = 2;
        if (kind == 3)
            for (int64_t e = mrp[i]; e < mrp[i + 1] && !rc; ++e)
                if (!(pos[i] < pos[n + mci[e]])) rc = 2;
    }
    if (!rc) {
        if (P < 1 || part_ptr[0] != 0 || part_ptr[P] != nv) rc = 3;
        for (int64_t p = 0; p < P && !rc; ++p)
            if (part_ptr[p + 1] <= part_ptr[p]) rc = 3;
    }
    free(pos);
    return rc;
}

/* Reuse ratio of Table 2 / §2.2 "Reuse Ratio": common accesses over the larger of the two
 * kernels' accesses, estimated from variable sizes. pair: 0 SpTRSV->SpMV (combination 4),
 * 1 SpIC0->SpTRSV (combination 5), 2 SpMV->SpTRSV (combination 2). size_L, size_M are
 * nonzero counts. */
double orc_reuse_ratio(int32_t pair, int64_t n, int64_t size_L, int64_t size_M) {
    double a, b;
    switch (pair) {
        case 0: /* x shared: 2n / max(size_L + 2n, size_M + 2n) */
            a = (double)(size_L + 2 * n); b = (double)(size_M + 2 * n);
            return (double)(2 * n) / (a > b ? a : b);
        case 1: /* L shared: 2 size_L / max(size_L, size_L + 2n) */
            a = (double)size_L; b = (double)(size_L + 2 * n);
            return (double)(2 * size_L) / (a > b ? a : b);
        case 2: /* y shared: 2n / max(size_M + 2n, size_L + 2n) */
            a = (double)(size_M + 2 * n); b = (double)(size_L + 2 * n);
            return (double)(2 * n) / (a > b ? a : b);
        case 5: /* combination 1, L and x shared: (2n + 2 size_L) / max(2n + size_L, size_L + 2n) */
            a = (double)(2 * n + size_L); b = (double)(size_L + 2 * n);
            return (double)(2 * n + 2 * size_L) / (a > b ? a : b);
        case 6: /* combination 6, A shared: 2 size_A / max(size_A, size_L + 2n), size_M = size_A */
            a = (double)size_M; b = (double)(size_L + 2 * n);
            return (double)(2 * size_M) / (a > b ? a : b);
        default: return -1.0;
    }
}
