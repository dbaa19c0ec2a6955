// Row-block executor: the locality form of the fused executor for one right-hand side.
//
// Rows are cut into blocks of B consecutive rows (in decreasing row order for the
// transposed schedules of the adjoint), every vertex of the joint DAG is assigned to the
// block of its own row (first kernel) or to the latest block among the rows it reads
// (second kernel), and each block's vertices are ordered by (level, kernel, row). A CTA runs
// one block at a time and keeps the block's produced values in shared memory. This is the
// GPU counterpart of the paper's w-partitions that keep dependent iterations together for
// locality (§3.2.1).
//
// Inside a block the vertices of one level form a segment; they are independent of one
// another (every edge of the joint DAG goes from a lower level to a higher one), so the CTA
// runs a segment with all its threads and crosses one barrier before the next. A
// dependence on a row of the same block is then one shared-memory load; only dependences on
// earlier blocks go through global memory, published with value flags (the pre-pass resets
// the global vector to the all-ones pattern and a consumer polls until the value differs
// from it). Shared slots are reset to the same pattern when a block opens and are read
// through the same check, so a schedule that breaks the level order is reported as a
// timeout instead of producing silent garbage.
//
// The per-level step is a short dependent chain, so everything that does not depend on
// values of this launch is moved off it:
//  - a pre-pass (k_block_prep) computes, for every row, the independent part c (b_i,
//    b_i - (A x_in)_i, (M^T gy)_j or gy_j) and the reciprocal of the diagonal, so a
//    first-kernel row finishes as (c - sum) * rinv without a division on the chain;
//  - a three-deep software pipeline over the segments: while segment s runs, the order
//    entries and entry ranges of segment s + 3, the row entries and (c, rinv) of segment
//    s + 2, and the inputs of segment s + 1 that lie in earlier blocks (speculative loads:
//    a value published in time then costs no round trip on the chain) are in flight, in
//    three item buffers used in rotation.
//
// Deadlock freedom: CTAs of a cooperative launch take blocks b, b + gridDim.x, ... in
// increasing order; every dependence points to an earlier block or to a lower level of the
// same block, so the smallest unfinished block always has its inputs finished or in
// progress on a running CTA. Every wait is bounded (timeout_ns) and a CTA leaves only at a
// barrier that all its threads reach (__syncthreads_or of the failure flags).
#pragma once

#include "sf_exec.cuh"

namespace sf {

template <typename T> struct Pair2;
template <> struct Pair2<double> { using type = double2; };
template <> struct Pair2<float> { using type = float2; };

template <typename T> __device__ __forceinline__ T unset_value();
template <> __device__ __forceinline__ double unset_value<double>() { return __longlong_as_double(-1LL); }
template <> __device__ __forceinline__ float unset_value<float>() { return __uint_as_float(0xffffffffu); }

template <typename T>
__device__ __forceinline__ T ld_shared_volatile(const T *p) { return *(const volatile T *)p; }

// Row entries held per lane in registers: 4 per lane for one or two lanes per row, else 8
// per group (three items of a lane are in registers at a time).
template <int LPR>
__host__ __device__ constexpr int block_unroll() { return LPR <= 2 ? 4 : (LPR >= 8 ? 1 : 8 / LPR); }

// The vector a mode's vertices wait on (first-kernel results) and publish into.
template <int MODE, typename T>
__device__ __forceinline__ T *block_vec(const ExecArgs &a) {
    if constexpr (MODE == M_TRSV_SPMV) return (T *)a.xs;
    else if constexpr (MODE == M_TRSV || MODE == M_SPMV_TRSV) return (T *)a.y;
    else return (T *)a.gb;
}

// Entries a vertex waits on: first-kernel rows read the strict part of L (or L^T), second-
// kernel rows read M (SpMV with F = pattern(M)) or A^T (the adjoint's gx rows).
template <int MODE, typename T>
__device__ __forceinline__ void block_entries(const ExecArgs &a, int tag, const int *&ci, const T *&vals) {
    if constexpr (MODE == M_TRSV_SPMV) {
        ci = tag ? a.Mci : a.Lci;
        vals = (const T *)(tag ? a.Mv : a.Lv);
    } else if constexpr (MODE == M_TRSV || MODE == M_SPMV_TRSV) {
        ci = a.Lci;
        vals = (const T *)a.Lv;
    } else if constexpr (MODE == M_ADJ_TRSV_SPMV) {
        ci = a.LTci;
        vals = (const T *)a.LTv;
    } else {
        ci = tag ? a.MTci : a.LTci;
        vals = (const T *)(tag ? a.MTv : a.LTv);
    }
}

// ---------------------------------------------------------------------------- pre-pass
// For every row i: resets the published vector to the all-ones pattern and writes
// aux[i] = (c_i, 1 / L_ii) with c_i the part of the first-kernel row that reads no value
// of this launch:
//   SpTRSV -> SpMV, SpTRSV:      c_i = b_i
//   SpMV -> SpTRSV:              c_i = b_i - (A x_in)_i
//   adjoint of SpTRSV -> SpMV:   c_j = (M^T gy)_j
//   adjoint of SpMV -> SpTRSV:   c_j = gy_j
// (L^T has the same diagonal as L.) A zero diagonal is recorded as SF_ERR_NONFINITE.
template <int MODE, typename T>
__global__ void __launch_bounds__(256) k_block_prep(const ExecArgs a) {
    using V2 = typename Pair2<T>::type;
    T *vec = block_vec<MODE, T>(a);
    V2 *aux = (V2 *)a.aux;
    const T *Lv = (const T *)a.Lv;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < a.n; t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)t;
        vec[i] = unset_value<T>();
        const T d = Lv[__ldg(a.Lrp + i + 1) - 1];
        if (d == T(0)) record_error(a.st, SF_ERR_NONFINITE, i);
        T c;
        if constexpr (MODE == M_TRSV_SPMV || MODE == M_TRSV) {
            c = __ldg((const T *)a.b + i);
        } else if constexpr (MODE == M_ADJ_SPMV_TRSV) {
            c = __ldg((const T *)a.gy + i);
        } else {
            const int *rp = MODE == M_SPMV_TRSV ? a.Mrp : a.MTrp;
            const int *ci = MODE == M_SPMV_TRSV ? a.Mci : a.MTci;
            const T *vals = (const T *)(MODE == M_SPMV_TRSV ? a.Mv : a.MTv);
            const T *src = (const T *)(MODE == M_SPMV_TRSV ? a.xin : a.gy);
            // M^T's values straight from M through the transpose permutation when the
            // adjoint skipped their gather
            const int *perm = (MODE == M_ADJ_TRSV_SPMV && a.mt_direct) ? a.MTperm : nullptr;
            const T *mv = (const T *)a.Mv;
            const int e0 = __ldg(rp + i), e1 = __ldg(rp + i + 1);
            T acc = T(0);
            for (int e = e0; e < e1; e += kUnroll) {
                int j[kUnroll];
                T v[kUnroll];
#pragma unroll
                for (int u = 0; u < kUnroll; ++u) {
                    j[u] = e + u < e1 ? __ldg(ci + e + u) : -1;
                    v[u] = e + u < e1 ? (perm ? __ldg(mv + __ldg(perm + e + u)) : __ldg(vals + e + u)) : T(0);
                }
#pragma unroll
                for (int u = 0; u < kUnroll; ++u)
                    if (j[u] >= 0) acc += v[u] * __ldg(src + j[u]);
            }
            c = MODE == M_SPMV_TRSV ? __ldg((const T *)a.b + i) - acc : acc;
        }
        V2 o;
        o.x = c;
        o.y = T(1) / d;
        aux[i] = o;
    }
}

// ---------------------------------------------------------------------------- executor
// One vertex of a segment with its prefetched data. row < 0: no vertex.
template <typename T, int U>
struct BItem {
    int row, tag, rs, re;
    T c, r;        // first-kernel rows: independent part and 1 / diagonal
    int j[U];      // the lane's first U entries (column, -1 past the row's end)
    T v[U];
    T x[U];        // inputs from earlier blocks, loaded ahead (reset pattern if not yet there)
};

template <int MODE, typename T, int LPR, int U>
__device__ __forceinline__ void block_load(const ExecArgs &a, bool valid, unsigned o, int2 dd, int gl,
                                           BItem<T, U> &it) {
    using V2 = typename Pair2<T>::type;
    it.row = valid ? (int)(o & 0x7fffffffu) : -1;
    it.tag = (int)(o >> 31);
    it.rs = dd.x;
    it.re = dd.y;
    if constexpr (MODE == M_ADJ_SPMV_TRSV) {
        if (it.tag == 1 && !a.gx) it.row = -1;
    }
    const int *ci;
    const T *vals;
    block_entries<MODE, T>(a, it.tag, ci, vals);
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int e = it.rs + gl + u * LPR;
        const bool in = it.row >= 0 && e < it.re;
        it.j[u] = in ? __ldg(ci + e) : -1;
        it.v[u] = in ? __ldg(vals + e) : T(0);
    }
    it.c = T(0);
    it.r = T(0);
    if (it.row >= 0 && it.tag == 0 && gl == 0) {
        const V2 cr = __ldg((const V2 *)a.aux + it.row);
        it.c = cr.x;
        it.r = cr.y;
    }
}

// Speculative loads of the inputs that lie outside the block [row0, row0 + rows).
template <typename T, int U>
__device__ __forceinline__ void block_early(const T *vec, int row0, int rows, BItem<T, U> &it) {
#pragma unroll
    for (int u = 0; u < U; ++u) {
        it.x[u] = unset_value<T>();
        if (it.j[u] >= 0 && (unsigned)(it.j[u] - row0) >= (unsigned)rows) it.x[u] = ld_relaxed_val(vec + it.j[u]);
    }
}

template <typename T>
struct TailSum {
    T acc;
    bool ok;
};

// Entries past the registers' U per lane (rows longer than U * LPR), one at a time.
template <typename T>
__device__ __noinline__ TailSum<T> block_dot_tail(const int *__restrict__ cols, const T *__restrict__ vals, int e0,
                                                  int e1, int S, const T *vec, const T *xs, int row0, int rows,
                                                  ExecState *st, unsigned long long tmo, int row, T acc) {
    bool ok = true;
    for (int e = e0; e < e1 && ok; e += S) {
        const int j = __ldg(cols + e);
        const T v = __ldg(vals + e);
        const unsigned lj = (unsigned)(j - row0);
        T x = lj < (unsigned)rows ? ld_shared_volatile(xs + lj) : ld_relaxed_val(vec + j);
        Waiter w;
        while (is_unset(x)) {
            if (!w.pause(st, tmo, row)) {
                ok = false;
                break;
            }
            x = lj < (unsigned)rows ? ld_shared_volatile(xs + lj) : ld_relaxed_val(vec + j);
        }
        acc += v * x;
    }
    return TailSum<T>{acc, ok};
}

// Bounded wait for the inputs still showing the reset pattern (bit u of `pending`).
template <typename T, int U>
__device__ __noinline__ bool block_wait(const T *vec, const T *xs, int row0, int rows, const int *j, T *xv,
                                        unsigned pending, ExecState *st, unsigned long long tmo, int row) {
    Waiter w;
    while (pending) {
        if (!w.pause(st, tmo, row)) return false;
        for (int u = 0; u < U; ++u)
            if ((pending >> u) & 1u) {
                const unsigned lj = (unsigned)(j[u] - row0);
                xv[u] = lj < (unsigned)rows ? ld_shared_volatile(xs + lj) : ld_relaxed_val(vec + j[u]);
                if (!is_unset(xv[u])) pending &= ~(1u << u);
            }
    }
    return true;
}

// Runs a loaded vertex: gathers its inputs, finishes the dot product and publishes.
//   first-kernel row:  v = (c - sum) * rinv   (SpTRSV row, SpTRSV^T row of the adjoint)
//   SpMV row (F = pattern(M)): y_i = sum;     A^T row of the adjoint: gx_j = -sum
template <int MODE, typename T, int LPR, int U>
__device__ __forceinline__ bool block_run(const ExecArgs &a, T *xs, int row0, int rows, const BItem<T, U> &it,
                                          int gl, unsigned gmask) {
    if (it.row < 0) return true;
    T *vec = block_vec<MODE, T>(a);
    T xv[U];
    unsigned pending = 0;
#pragma unroll
    for (int u = 0; u < U; ++u) {
        xv[u] = T(0);
        if (it.j[u] >= 0) {
            const unsigned lj = (unsigned)(it.j[u] - row0);
            xv[u] = lj < (unsigned)rows ? ld_shared_volatile(xs + lj) : it.x[u];
            if (is_unset(xv[u])) pending |= 1u << u;
        }
    }
    bool ok = true;
    if (pending) {   // slow path, off the registers: copies in and out of local arrays
        int jj[U];
        T xx[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            jj[u] = it.j[u];
            xx[u] = xv[u];
        }
        ok = block_wait<T, U>(vec, xs, row0, rows, jj, xx, pending, a.st, a.timeout_ns, it.row);
#pragma unroll
        for (int u = 0; u < U; ++u) xv[u] = xx[u];
    }
    T acc0 = T(0), acc1 = T(0);
#pragma unroll
    for (int u = 0; u < U; ++u) {
        if (u & 1) acc1 += it.v[u] * xv[u];
        else acc0 += it.v[u] * xv[u];
    }
    T acc = acc0 + acc1;
    const int e0 = it.rs + gl + U * LPR;
    if (e0 < it.re) {
        const int *ci;
        const T *vals;
        block_entries<MODE, T>(a, it.tag, ci, vals);
        const TailSum<T> t = block_dot_tail<T>(ci, vals, e0, it.re, LPR, vec, xs, row0, rows, a.st, a.timeout_ns,
                                               it.row, acc);
        acc = t.acc;
        ok = ok && t.ok;
    }
    acc = group_sum<LPR>(acc, gmask);
    if (gl == 0) {
        if (it.tag == 0) {
            T v = (it.c - acc) * it.r;
            if (is_unset(v)) v = canonical_nan(v);
            // a first-kernel row always lies in its own block; the check keeps a corrupted
            // order (the testing hook that swaps positions) from touching foreign slots
            const unsigned lr = (unsigned)(it.row - row0);
            if (lr < (unsigned)rows) *(volatile T *)(xs + lr) = v;
            st_relaxed_val(vec + it.row, v);
        } else if constexpr (MODE == M_TRSV_SPMV) {
            ((T *)a.y)[it.row] = acc;
        } else if constexpr (MODE == M_ADJ_SPMV_TRSV) {
            ((T *)a.gx)[it.row] = -acc;
        }
    }
    return group_ok<LPR>(ok, gmask);
}

// One level step over segment s: issues the loads of the later segments (see the header),
// runs this segment, crosses the barrier and shifts the pipeline registers. Returns false
// (uniformly over the CTA) when a wait failed anywhere in the CTA.
template <int MODE, typename T, int LPR, int U>
__device__ __forceinline__ bool block_step(const ExecArgs &a, T *xs, int row0, int rows, int grp, int NG, int gl,
                                           unsigned gmask, const BItem<T, U> &cur, BItem<T, U> &nx1,
                                           BItem<T, U> &nx2, bool &v2, unsigned &o2, int2 &d2, int (&p)[5], int s,
                                           int s1, bool &ok) {
    T *vec = block_vec<MODE, T>(a);
    block_load<MODE, T, LPR, U>(a, v2, o2, d2, gl, nx2);
    const int q3 = p[3] + grp;
    const bool v3 = q3 < p[4];
    const unsigned o3 = v3 ? (unsigned)__ldg(a.order + q3) : 0u;
    const int2 d3 = v3 ? __ldg(a.bdesc + q3) : make_int2(0, 0);
    const int p5 = __ldg(a.seg_ptr + min(s + 5, s1));
    block_early<T, U>(vec, row0, rows, nx1);
    if (ok) ok = block_run<MODE, T, LPR, U>(a, xs, row0, rows, cur, gl, gmask);
    // vertices beyond the first per group (segments wider than the CTA)
    for (int q = p[0] + grp + NG; q < p[1]; q += NG) {
        BItem<T, U> extra;
        block_load<MODE, T, LPR, U>(a, true, (unsigned)__ldg(a.order + q), __ldg(a.bdesc + q), gl, extra);
        block_early<T, U>(vec, row0, rows, extra);
        if (ok) ok = block_run<MODE, T, LPR, U>(a, xs, row0, rows, extra, gl, gmask);
    }
    if (__syncthreads_or(!ok)) {
        ok = false;
        return false;
    }
    v2 = v3;
    o2 = o3;
    d2 = d3;
#pragma unroll
    for (int k = 0; k < 4; ++k) p[k] = p[k + 1];
    p[4] = p5;
    return true;
}

template <int MODE, typename T, int LPR>
__global__ void __launch_bounds__(kBlockMaxThreads, 1) k_block_exec(const ExecArgs a) {
    constexpr int U = block_unroll<LPR>();
    extern __shared__ __align__(16) unsigned char sm_raw[];
    __shared__ unsigned s_abort;
    T *xs = reinterpret_cast<T *>(sm_raw);
    constexpr int GPW = 32 / LPR;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int grp = warp * GPW + lane / LPR, gl = lane % LPR, gbase = (lane / LPR) * LPR;
    const unsigned gmask = (LPR == 32) ? 0xffffffffu : (((1u << LPR) - 1u) << gbase);
    const int NG = (blockDim.x >> 5) * GPW;
    const int B = a.block_rows, nb = a.n_blocks;
    const unsigned epoch = ld_relaxed_u32(&a.st->epoch);
    T *vec = block_vec<MODE, T>(a);
    bool ok = true;
    for (int b = blockIdx.x; b < nb; b += gridDim.x) {
        const int row0 = a.block_rev ? (nb - 1 - b) * B : b * B;
        const int rows = min(B, a.n - row0);
        for (int i = threadIdx.x; i < rows; i += blockDim.x) xs[i] = unset_value<T>();
        const int s0 = __ldg(a.block_seg + b), s1 = __ldg(a.block_seg + b + 1);
        // p[k]: first position of segment s + k (clamped to the block's end)
        int p[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) p[k] = __ldg(a.seg_ptr + min(s0 + k, s1));
        // fill the pipeline: entries of segments s0 and s0 + 1, order entries of s0 + 2,
        // out-of-block inputs of s0
        BItem<T, U> A, Bi, C;
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int q = p[k] + grp;
            const bool v = q < p[k + 1];
            block_load<MODE, T, LPR, U>(a, v, v ? (unsigned)__ldg(a.order + q) : 0u,
                                        v ? __ldg(a.bdesc + q) : make_int2(0, 0), gl, k ? Bi : A);
        }
        const int q2 = p[2] + grp;
        bool v2 = q2 < p[3];
        unsigned o2 = v2 ? (unsigned)__ldg(a.order + q2) : 0u;
        int2 d2 = v2 ? __ldg(a.bdesc + q2) : make_int2(0, 0);
        block_early<T, U>(vec, row0, rows, A);
        __syncthreads();
        // three item buffers in rotation: (run, inputs ahead, entries ahead)
        for (int s = s0; s < s1; s += 3) {
            if (!block_step<MODE, T, LPR, U>(a, xs, row0, rows, grp, NG, gl, gmask, A, Bi, C, v2, o2, d2, p, s, s1, ok))
                break;
            if (s + 1 >= s1) break;
            if (!block_step<MODE, T, LPR, U>(a, xs, row0, rows, grp, NG, gl, gmask, Bi, C, A, v2, o2, d2, p, s + 1, s1,
                                             ok))
                break;
            if (s + 2 >= s1) break;
            if (!block_step<MODE, T, LPR, U>(a, xs, row0, rows, grp, NG, gl, gmask, C, A, Bi, v2, o2, d2, p, s + 2, s1,
                                             ok))
                break;
        }
        if (!ok) break;
        if (threadIdx.x == 0) s_abort = ld_relaxed_u32(&a.st->abort);
        __syncthreads();
        if (s_abort) break;
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

}  // namespace sf
