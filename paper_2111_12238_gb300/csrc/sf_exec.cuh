// Fused executor (§2.3, Figure 4) as one persistent kernel.
//
// The inspector linearises the joint DAG by (level, kernel, row) and cuts the order into
// contiguous partitions (§3.1 coarsening of wavefronts into work units). Here every warp
// repeatedly takes the next partition from a ticket counter and runs its items; a warp is
// split into 32/LPR groups of LPR lanes, each group running one item (one row of one
// kernel, or one paired row of both kernels) at a time. Instead of the barrier that
// separates s-partitions in the paper's executor, every produced row publishes a ready
// flag with release semantics and every consumer waits on the flags of exactly the rows
// it reads (its DAG predecessors and F row), so a row starts as soon as its inputs exist.
//
// Deadlock freedom: tickets are handed out in the topological order, so every item a
// warp waits on belongs to an earlier partition, whose warp is already running, or to an
// earlier item of its own partition. Waits are bounded by %globaltimer; on expiry the
// warp records SF_ERR_TIMEOUT, raises `abort`, and every warp drains.
#pragma once

#include "sf_internal.cuh"

namespace sf {

template <typename T> struct VT;
template <> struct VT<double> { static constexpr int id = 0; };
template <> struct VT<float> { static constexpr int id = 1; };

constexpr int kUnroll = 4;   // row entries fetched per lane before waiting on them

// Sum over the lanes of a group that share a right-hand-side column (xor partners at
// distance >= kt).
template <int LPR, typename T>
__device__ __forceinline__ T slice_sum(T v, int kt, unsigned gmask) {
#pragma unroll
    for (int off = LPR / 2; off >= 1; off >>= 1)
        if (off >= kt) v += __shfl_xor_sync(gmask, v, off);
    return v;
}
// Sum over all lanes of a group.
template <int LPR, typename T>
__device__ __forceinline__ T group_sum(T v, unsigned gmask) {
#pragma unroll
    for (int off = LPR / 2; off >= 1; off >>= 1) v += __shfl_xor_sync(gmask, v, off);
    return v;
}
// Sum over the kt lanes of one slice (the right-hand-side columns of one entry).
template <typename T>
__device__ __forceinline__ T col_sum(T v, int kt, unsigned smask) {
    for (int off = kt >> 1; off >= 1; off >>= 1) v += __shfl_xor_sync(smask, v, off);
    return v;
}

// Waits until every listed row (j[u] >= 0) is published in this epoch. Flags are polled
// with relaxed loads so that the polls of one batch are in flight together; one acquire
// fence after the last poll orders the subsequent data loads after every observed
// release (fence-acquire pattern). Returns false on abort or timeout.
template <int U>
__device__ __forceinline__ bool wait_rows(const unsigned *flags, const int (&j)[U], unsigned epoch,
                                          ExecState *st, unsigned long long tmo, int row) {
    unsigned pending = 0;
#pragma unroll
    for (int u = 0; u < U; ++u)
        if (j[u] >= 0 && ld_relaxed_u32(flags + j[u]) != epoch) pending |= 1u << u;
    bool any = false;
#pragma unroll
    for (int u = 0; u < U; ++u) any |= j[u] >= 0;
    if (pending) {
        const unsigned long long t0 = global_ns();
        for (unsigned it = 1; pending; ++it) {
#pragma unroll
            for (int u = 0; u < U; ++u)
                if ((pending >> u) & 1u)
                    if (ld_relaxed_u32(flags + j[u]) == epoch) pending &= ~(1u << u);
            if (pending && (it & 31u) == 0u) {
                if (ld_relaxed_u32(&st->abort)) return false;
                if (global_ns() - t0 > tmo) {
                    record_error(st, SF_ERR_TIMEOUT, row);
                    st_relaxed_u32(&st->abort, 1u);
                    return false;
                }
            }
        }
    }
    if (any) fence_acq_rel_gpu();
    return true;
}

// acc = sum over this lane's slice of entries e in [e0, e1) (stride S) of
// vals[PERM ? perm[e] : e] * vec[cols[e] * k + c]. With WAIT the rows cols[e] are waited
// for first and vec is read through L2 (it is produced by other warps in this launch).
template <typename T, bool WAIT, bool PERM>
__device__ __forceinline__ T row_dot(const int *__restrict__ cols, const int *__restrict__ perm,
                                     const T *__restrict__ vals, int e0, int e1, int S, const T *vec,
                                     int k, int c, bool act, const unsigned *flags, unsigned epoch,
                                     ExecState *st, unsigned long long tmo, int row, bool &ok) {
    T acc = T(0);
    for (int e = e0; e < e1; e += S * kUnroll) {
        int j[kUnroll];
        T v[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const int ee = e + u * S;
            j[u] = -1;
            v[u] = T(0);
            if (ee < e1) {
                j[u] = __ldg(cols + ee);
                v[u] = __ldg(vals + (PERM ? __ldg(perm + ee) : ee));
            }
        }
        if (WAIT && ok) ok = wait_rows<kUnroll>(flags, j, epoch, st, tmo, row);
        if (act) {
#pragma unroll
            for (int u = 0; u < kUnroll; ++u)
                if (j[u] >= 0) {
                    const T xv = WAIT ? __ldcg(vec + (size_t)j[u] * k + c) : __ldg(vec + (size_t)j[u] * k + c);
                    acc += v[u] * xv;
                }
        }
    }
    return acc;
}

// out[e] = sign * sum_c coef[c] * vec[cols[e] * k + c] for e in [e0, e1): the pattern-
// restricted outer product of the adjoint gradients. Lanes: slice s = gl / kt takes
// every S-th entry, its kt lanes split the right-hand-side columns.
template <typename T, int LPR>
__device__ __forceinline__ void grad_row(const int *__restrict__ cols, int e0, int e1, const T *coef,
                                         const T *__restrict__ vec, int k, int kt, int gl, int gbase,
                                         T sign, T *out) {
    const int S = LPR / kt, s = gl / kt, cl = gl % kt;
    const unsigned smask = (kt == 32) ? 0xffffffffu : (((1u << kt) - 1u) << (gbase + s * kt));
    for (int e = e0 + s; e < e1; e += S) {
        const int j = __ldg(cols + e);
        T part = T(0);
        for (int c = cl; c < k; c += kt) part += coef[c] * __ldg(vec + (size_t)j * k + c);
        part = col_sum(part, kt, smask);
        if (cl == 0) out[e] = sign * part;
    }
}

template <int LPR>
__device__ __forceinline__ bool group_ok(bool ok, unsigned gmask) {
    return !__any_sync(gmask, !ok);
}

template <int LPR>
__device__ __forceinline__ void publish(const ExecArgs &a, int row, unsigned epoch, int gl,
                                        unsigned gmask, bool ok) {
    __syncwarp(gmask);
    if (gl == 0 && ok) st_release_u32(a.flags + row, epoch);
}

// ---------------------------------------------------------------- item kinds
// SpTRSV row (Table 2, forward substitution): x_i = (b_i - sum_{j<i} L_ij x_j) / L_ii.
// `x` is both the output and the buffer the dependences are read from.
template <typename T, int LPR>
__device__ bool item_trsv(const ExecArgs &a, int row, unsigned epoch, int gl, unsigned gmask, T *x) {
    const int kt = a.kt, S = LPR / kt, s = gl / kt, cl = gl % kt, k = a.k;
    const int rs = a.Lrp[row], dg = a.Lrp[row + 1] - 1;
    const T *Lv = (const T *)a.Lv, *b = (const T *)a.b;
    const T d = __ldg(Lv + dg);
    if (gl == 0 && d == T(0)) record_error(a.st, SF_ERR_NONFINITE, row);
    bool ok = true;
    for (int c0 = 0; c0 < k; c0 += kt) {
        const int c = c0 + cl;
        const bool act = c < k;
        T acc = row_dot<T, true, false>(a.Lci, nullptr, Lv, rs + s, dg, S, x, k, c, act, a.flags, epoch,
                                        a.st, a.timeout_ns, row, ok);
        acc = slice_sum<LPR>(acc, kt, gmask);
        if (s == 0 && act) x[(size_t)row * k + c] = (__ldg(b + (size_t)row * k + c) - acc) / d;
    }
    ok = group_ok<LPR>(ok, gmask);
    publish<LPR>(a, row, epoch, gl, gmask, ok);
    return ok;
}

// SpMV row of the second kernel with F = pattern(M): y_i = sum_j M_ij x_j, each x_j
// waited for (§2.2 "Dependency Matrix F": row i of F lists the first-kernel iterations
// row i of the second kernel reads).
template <typename T, int LPR>
__device__ bool item_spmv_dep(const ExecArgs &a, int row, unsigned epoch, int gl, unsigned gmask, const T *x) {
    const int kt = a.kt, S = LPR / kt, s = gl / kt, cl = gl % kt, k = a.k;
    const int rs = a.Mrp[row], re = a.Mrp[row + 1];
    T *y = (T *)a.y;
    bool ok = true;
    for (int c0 = 0; c0 < k; c0 += kt) {
        const int c = c0 + cl;
        const bool act = c < k;
        T acc = row_dot<T, true, false>(a.Mci, nullptr, (const T *)a.Mv, rs + s, re, S, x, k, c, act, a.flags,
                                        epoch, a.st, a.timeout_ns, row, ok);
        acc = slice_sum<LPR>(acc, kt, gmask);
        if (s == 0 && act) y[(size_t)row * k + c] = acc;
    }
    return group_ok<LPR>(ok, gmask);
}

// Paired SpMV -> SpTRSV row (combination 2, F = I): r_i = b_i - A_i x_in stays in
// registers, then z_i = (r_i - sum_{j<i} L_ij z_j) / L_ii.
template <typename T, int LPR>
__device__ bool item_spmv_trsv(const ExecArgs &a, int row, unsigned epoch, int gl, unsigned gmask) {
    const int kt = a.kt, S = LPR / kt, s = gl / kt, cl = gl % kt, k = a.k;
    const int ra = a.Mrp[row], re = a.Mrp[row + 1];
    const int rs = a.Lrp[row], dg = a.Lrp[row + 1] - 1;
    const T *Lv = (const T *)a.Lv, *b = (const T *)a.b;
    T *z = (T *)a.y;
    const T d = __ldg(Lv + dg);
    if (gl == 0 && d == T(0)) record_error(a.st, SF_ERR_NONFINITE, row);
    bool ok = true;
    for (int c0 = 0; c0 < k; c0 += kt) {
        const int c = c0 + cl;
        const bool act = c < k;
        T accA = row_dot<T, false, false>(a.Mci, nullptr, (const T *)a.Mv, ra + s, re, S, (const T *)a.xin, k, c,
                                          act, a.flags, epoch, a.st, a.timeout_ns, row, ok);
        T accL = row_dot<T, true, false>(a.Lci, nullptr, Lv, rs + s, dg, S, z, k, c, act, a.flags, epoch, a.st,
                                         a.timeout_ns, row, ok);
        accA = slice_sum<LPR>(accA, kt, gmask);
        accL = slice_sum<LPR>(accL, kt, gmask);
        if (s == 0 && act) {
            const T r = __ldg(b + (size_t)row * k + c) - accA;
            z[(size_t)row * k + c] = (r - accL) / d;
        }
    }
    ok = group_ok<LPR>(ok, gmask);
    publish<LPR>(a, row, epoch, gl, gmask, ok);
    return ok;
}

// Paired SpIC0 -> SpTRSV row (combination 5, F = I), IC0 in its up-looking row form:
// for each j < i in row i, ascending, L_ij = (A_ij - sum_{k<j, k in both rows} L_ik L_jk)
// / L_jj; then L_ii = sqrt(A_ii - sum_{k<i} L_ik^2); then the solve row with the fresh
// L_i stays on chip: y_i = (b_i - sum_j L_ij y_j) / L_ii. Factor values go to a.xs.
template <typename T, int LPR, bool SOLVE>
__device__ bool item_ic0(const ExecArgs &a, int row, unsigned epoch, int gl, unsigned gmask) {
    const int rs = a.Lrp[row], dg = a.Lrp[row + 1] - 1;
    const T *Av = (const T *)a.Lv;
    T *lf = (T *)a.xs;
    bool ok = true;
    // every predecessor row publishes its factor row and its solve row together
    for (int e = rs + gl; e < dg; e += LPR * kUnroll) {
        int j[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const int ee = e + u * LPR;
            j[u] = ee < dg ? __ldg(a.Lci + ee) : -1;
        }
        if (ok) ok = wait_rows<kUnroll>(a.flags, j, epoch, a.st, a.timeout_ns, row);
    }
    ok = group_ok<LPR>(ok, gmask);
    for (int t = rs; t < dg; ++t) {
        const int jr = __ldg(a.Lci + t);
        const int js = __ldg(a.Lrp + jr), jd = __ldg(a.Lrp + jr + 1) - 1;
        T part = T(0);
        for (int g = js + gl; g < jd; g += LPR) {
            const int kc = __ldg(a.Lci + g);
            int lo = rs, hi = t;            // kc among row i's columns before j
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (__ldg(a.Lci + mid) < kc) lo = mid + 1; else hi = mid;
            }
            if (lo < t && __ldg(a.Lci + lo) == kc) part += lf[lo] * __ldcg(lf + g);
        }
        part = group_sum<LPR>(part, gmask);
        if (gl == 0) lf[t] = (__ldg(Av + t) - part) / __ldcg(lf + jd);
        __syncwarp(gmask);
    }
    T sq = T(0);
    for (int t = rs + gl; t < dg; t += LPR) {
        const T v = lf[t];
        sq += v * v;
    }
    sq = group_sum<LPR>(sq, gmask);
    const T dd = __ldg(Av + dg) - sq;
    if (gl == 0 && !(dd > T(0))) record_error(a.st, SF_ERR_BREAKDOWN, row);
    const T lii = sqrt(dd);
    if (gl == 0) lf[dg] = lii;
    if (SOLVE) {
        const int kt = a.kt, S = LPR / kt, s = gl / kt, cl = gl % kt, k = a.k;
        const T *b = (const T *)a.b;
        T *y = (T *)a.y;
        __syncwarp(gmask);
        for (int c0 = 0; c0 < k; c0 += kt) {
            const int c = c0 + cl;
            T acc = T(0);
            if (c < k)
                for (int t = rs + s; t < dg; t += S)
                    acc += lf[t] * __ldcg(y + (size_t)__ldg(a.Lci + t) * k + c);
            acc = slice_sum<LPR>(acc, kt, gmask);
            if (s == 0 && c < k) y[(size_t)row * k + c] = (__ldg(b + (size_t)row * k + c) - acc) / lii;
        }
    }
    publish<LPR>(a, row, epoch, gl, gmask, ok);
    return ok;
}

// Adjoint of SpTRSV -> SpMV as a paired pass on the transposed schedule (item j = column
// j of L): u_j = (M^T gy)_j needs no wait; lam_j = (u_j - sum_{i>j} L_ij lam_i) / L_jj
// waits for lam_i; gb = lam. After publishing, the row's gradients:
// gL_j* = -lam_j x_*, gM_j* = gy_j x_*.
template <typename T, int LPR>
__device__ bool item_adj_trsv_spmv(const ExecArgs &a, int j, unsigned epoch, int gl, int gbase, unsigned gmask) {
    const int kt = a.kt, S = LPR / kt, s = gl / kt, cl = gl % kt, k = a.k;
    const int ms = a.MTrp[j], me = a.MTrp[j + 1];
    const int ls = a.LTrp[j], le = a.LTrp[j + 1];     // first entry of L^T row j is L_jj
    const T *Lv = (const T *)a.Lv, *gy = (const T *)a.gy, *x = (const T *)a.saved;
    T *lam = (T *)a.gb;
    const T d = __ldg(Lv + __ldg(a.LTperm + ls));
    if (gl == 0 && d == T(0)) record_error(a.st, SF_ERR_NONFINITE, j);
    bool ok = true;
    for (int c0 = 0; c0 < k; c0 += kt) {
        const int c = c0 + cl;
        const bool act = c < k;
        T u = row_dot<T, false, true>(a.MTci, a.MTperm, (const T *)a.Mv, ms + s, me, S, gy, k, c, act, a.flags,
                                      epoch, a.st, a.timeout_ns, j, ok);
        T accL = row_dot<T, true, true>(a.LTci, a.LTperm, Lv, ls + 1 + s, le, S, lam, k, c, act, a.flags, epoch,
                                        a.st, a.timeout_ns, j, ok);
        u = slice_sum<LPR>(u, kt, gmask);
        accL = slice_sum<LPR>(accL, kt, gmask);
        if (s == 0 && act) lam[(size_t)j * k + c] = (u - accL) / d;
    }
    ok = group_ok<LPR>(ok, gmask);
    publish<LPR>(a, j, epoch, gl, gmask, ok);
    if (ok && a.gL)
        grad_row<T, LPR>(a.Lci, a.Lrp[j], a.Lrp[j + 1], lam + (size_t)j * k, x, k, kt, gl, gbase, T(-1), (T *)a.gL);
    if (ok && a.gM)
        grad_row<T, LPR>(a.Mci, a.Mrp[j], a.Mrp[j + 1], gy + (size_t)j * k, x, k, kt, gl, gbase, T(1), (T *)a.gM);
    return ok;
}

// Adjoint of SpMV -> SpTRSV, tag 0: lam_j = (gz_j - sum_{i>j} L_ij lam_i) / L_jj, gb = lam,
// then gL_j* = -lam_j z_*, gA_j* = -lam_j x_in_*.
template <typename T, int LPR>
__device__ bool item_adj_lam(const ExecArgs &a, int j, unsigned epoch, int gl, int gbase, unsigned gmask) {
    const int kt = a.kt, S = LPR / kt, s = gl / kt, cl = gl % kt, k = a.k;
    const int ls = a.LTrp[j], le = a.LTrp[j + 1];
    const T *Lv = (const T *)a.Lv, *gz = (const T *)a.gy;
    T *lam = (T *)a.gb;
    const T d = __ldg(Lv + __ldg(a.LTperm + ls));
    if (gl == 0 && d == T(0)) record_error(a.st, SF_ERR_NONFINITE, j);
    bool ok = true;
    for (int c0 = 0; c0 < k; c0 += kt) {
        const int c = c0 + cl;
        const bool act = c < k;
        T accL = row_dot<T, true, true>(a.LTci, a.LTperm, Lv, ls + 1 + s, le, S, lam, k, c, act, a.flags, epoch,
                                        a.st, a.timeout_ns, j, ok);
        accL = slice_sum<LPR>(accL, kt, gmask);
        if (s == 0 && act) lam[(size_t)j * k + c] = (__ldg(gz + (size_t)j * k + c) - accL) / d;
    }
    ok = group_ok<LPR>(ok, gmask);
    publish<LPR>(a, j, epoch, gl, gmask, ok);
    if (ok && a.gL)
        grad_row<T, LPR>(a.Lci, a.Lrp[j], a.Lrp[j + 1], lam + (size_t)j * k, (const T *)a.saved, k, kt, gl, gbase,
                         T(-1), (T *)a.gL);
    if (ok && a.gM)
        grad_row<T, LPR>(a.Mci, a.Mrp[j], a.Mrp[j + 1], lam + (size_t)j * k, (const T *)a.xin, k, kt, gl, gbase,
                         T(-1), (T *)a.gM);
    return ok;
}

// Adjoint of SpMV -> SpTRSV, tag 1: gx_j = -sum_i A_ij lam_i, waiting for each lam_i.
template <typename T, int LPR>
__device__ bool item_adj_gx(const ExecArgs &a, int j, unsigned epoch, int gl, unsigned gmask) {
    const int kt = a.kt, S = LPR / kt, s = gl / kt, cl = gl % kt, k = a.k;
    const int ms = a.MTrp[j], me = a.MTrp[j + 1];
    T *gx = (T *)a.gx;
    bool ok = true;
    for (int c0 = 0; c0 < k; c0 += kt) {
        const int c = c0 + cl;
        const bool act = c < k;
        T acc = row_dot<T, true, true>(a.MTci, a.MTperm, (const T *)a.Mv, ms + s, me, S, (const T *)a.gb, k, c,
                                       act, a.flags, epoch, a.st, a.timeout_ns, j, ok);
        acc = slice_sum<LPR>(acc, kt, gmask);
        if (s == 0 && act) gx[(size_t)j * k + c] = -acc;
    }
    return group_ok<LPR>(ok, gmask);
}

template <int MODE, typename T, int LPR>
__device__ __forceinline__ bool run_item(const ExecArgs &a, int tag, int row, unsigned epoch, int gl, int gbase,
                                         unsigned gmask) {
    if constexpr (MODE == M_TRSV_SPMV) {
        if (tag == 0) return item_trsv<T, LPR>(a, row, epoch, gl, gmask, (T *)a.xs);
        return item_spmv_dep<T, LPR>(a, row, epoch, gl, gmask, (const T *)a.xs);
    } else if constexpr (MODE == M_TRSV) {
        return item_trsv<T, LPR>(a, row, epoch, gl, gmask, (T *)a.y);
    } else if constexpr (MODE == M_SPMV_TRSV) {
        return item_spmv_trsv<T, LPR>(a, row, epoch, gl, gmask);
    } else if constexpr (MODE == M_IC0_TRSV) {
        return item_ic0<T, LPR, true>(a, row, epoch, gl, gmask);
    } else if constexpr (MODE == M_IC0) {
        return item_ic0<T, LPR, false>(a, row, epoch, gl, gmask);
    } else if constexpr (MODE == M_ADJ_TRSV_SPMV) {
        return item_adj_trsv_spmv<T, LPR>(a, row, epoch, gl, gbase, gmask);
    } else {
        if (tag == 0) return item_adj_lam<T, LPR>(a, row, epoch, gl, gbase, gmask);
        if (!a.gx) return true;    // gradient of x_in not requested
        return item_adj_gx<T, LPR>(a, row, epoch, gl, gmask);
    }
}

constexpr int kExecThreads = 256;

template <int MODE, typename T, int LPR>
__global__ void __launch_bounds__(kExecThreads) k_exec(const ExecArgs a) {
    constexpr int G = 32 / LPR;
    const int lane = threadIdx.x & 31;
    const int grp = lane / LPR, gl = lane % LPR, gbase = grp * LPR;
    const unsigned gmask = (LPR == 32) ? 0xffffffffu : (((1u << LPR) - 1u) << gbase);
    const unsigned epoch = ld_relaxed_u32(&a.st->epoch);
    bool ok = true;
    for (;;) {
        int p = 0;
        if (lane == 0) p = ld_relaxed_u32(&a.st->abort) ? a.n_parts : (int)atomicAdd(&a.st->ticket, 1u);
        p = __shfl_sync(0xffffffffu, p, 0);
        if (p >= a.n_parts) break;
        const int q0 = __ldg(a.part_ptr + p), q1 = __ldg(a.part_ptr + p + 1);
        for (int q = q0 + grp; q < q1 && ok; q += G) {
            const unsigned o = (unsigned)__ldg(a.order + q);
            ok = run_item<MODE, T, LPR>(a, (int)(o >> 31), (int)(o & 0x7fffffffu), epoch, gl, gbase, gmask);
        }
        if (!__all_sync(0xffffffffu, ok)) break;
    }
    __syncwarp();
    if (lane == 0) {
        const unsigned total = gridDim.x * (blockDim.x >> 5);
        if (atom_add_acq_rel_u32(&a.st->done, 1u) == total - 1u) {
            st_relaxed_u32(&a.st->ticket, 0u);
            st_relaxed_u32(&a.st->done, 0u);
            st_relaxed_u32(&a.st->abort, 0u);
            st_release_u32(&a.st->epoch, epoch + 1u);
        }
    }
}

// Instantiates and launches k_exec<MODE, T, LPR> for a runtime (dtype, lanes-per-row).
template <int MODE>
cudaError_t launch_mode(int dtype, int lpr, int blocks, cudaStream_t s, const ExecArgs &a) {
#define SF_LAUNCH(T, L) k_exec<MODE, T, L><<<blocks, kExecThreads, 0, s>>>(a); return cudaGetLastError()
    if (dtype == 0) {
        switch (lpr) {
            case 1: SF_LAUNCH(double, 1);
            case 2: SF_LAUNCH(double, 2);
            case 4: SF_LAUNCH(double, 4);
            case 8: SF_LAUNCH(double, 8);
            case 16: SF_LAUNCH(double, 16);
            case 32: SF_LAUNCH(double, 32);
        }
    } else {
        switch (lpr) {
            case 1: SF_LAUNCH(float, 1);
            case 2: SF_LAUNCH(float, 2);
            case 4: SF_LAUNCH(float, 4);
            case 8: SF_LAUNCH(float, 8);
            case 16: SF_LAUNCH(float, 16);
            case 32: SF_LAUNCH(float, 32);
        }
    }
#undef SF_LAUNCH
    return cudaErrorInvalidValue;
}

template <int MODE>
int blocks_per_sm_mode(int dtype, int lpr) {
    int nb = 0;
    const void *f = nullptr;
#define SF_F(T, L) f = (const void *)k_exec<MODE, T, L>; break
    if (dtype == 0) {
        switch (lpr) {
            case 1: SF_F(double, 1); case 2: SF_F(double, 2); case 4: SF_F(double, 4);
            case 8: SF_F(double, 8); case 16: SF_F(double, 16); case 32: SF_F(double, 32);
        }
    } else {
        switch (lpr) {
            case 1: SF_F(float, 1); case 2: SF_F(float, 2); case 4: SF_F(float, 4);
            case 8: SF_F(float, 8); case 16: SF_F(float, 16); case 32: SF_F(float, 32);
        }
    }
#undef SF_F
    if (!f || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, kExecThreads, 0) != cudaSuccess) return 1;
    return nb > 0 ? nb : 1;
}

}  // namespace sf
