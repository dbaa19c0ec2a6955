// Fused executor (§2.3, Figure 4) as one persistent kernel.
//
// The inspector linearises the joint DAG by (level, kernel, row) and cuts the order into
// contiguous partitions (§3.1 coarsening of wavefronts into work units). Here every warp
// repeatedly takes the next partition from a ticket counter and runs its items; a warp is
// split into 32/LPR groups of LPR lanes, each group running one item (one row of one
// kernel, or one paired row of both kernels) at a time. Instead of the barrier that
// separates s-partitions in the paper's executor, every produced row is published and
// every consumer waits for exactly the rows it reads (its DAG predecessors and its F
// row), so a row starts as soon as its inputs exist.
//
// Two publication mechanisms:
//  * epoch flags (any k): the producer stores its row, then releases flag[row] = epoch;
//    consumers poll flags with relaxed loads and issue one acquire fence per batch.
//  * value flags (VF, k = 1): the dependency vector is reset to an all-ones NaN pattern
//    before the launch; the producer stores the value with one relaxed store and the
//    consumer polls the value itself, so a hop costs one store and one load.
// Waits back off exponentially with __nanosleep so that waiting warps neither flood L2
// with polls nor starve the lanes of their own warp that compute the awaited rows.
//
// Work assignment: by default partitions go round robin to the warps of a cooperative
// (fully co-resident) launch: warp w runs partitions w, w + W, w + 2W, ... in order. With
// `dynamic` a warp instead draws its next partition from a ticket counter.
// Deadlock freedom, both cases: partitions are topologically ordered and every warp runs
// its own partitions in increasing order, so the smallest unfinished partition belongs to
// a running warp that is working on it (any earlier partition of that warp is finished)
// and all its dependences lie in smaller, finished partitions or earlier items of its own.
// Waits are bounded by %globaltimer; on expiry the warp records SF_ERR_TIMEOUT, raises
// `abort`, and every warp drains.
#pragma once

#include "sf_internal.cuh"

namespace sf {

constexpr int kUnroll = 4;   // row entries fetched per lane before waiting on them
constexpr int kExecThreads = 256;   // threads of an executor block
#ifndef SF_BACKOFF_MIN_NS
#define SF_BACKOFF_MIN_NS 20
#endif
#ifndef SF_BACKOFF_MAX_NS
#define SF_BACKOFF_MAX_NS 64
#endif
// Sleep between polls of a dependence: doubles from the minimum to the maximum (build-time
// constants; shorter sleeps see a published value sooner but load L2 with more polls).
constexpr unsigned kBackoffMinNs = SF_BACKOFF_MIN_NS, kBackoffMaxNs = SF_BACKOFF_MAX_NS;

// ------------------------------------------------------------------ value-flag helpers
template <typename T> __device__ __forceinline__ T ld_relaxed_val(const T *p);
template <> __device__ __forceinline__ double ld_relaxed_val<double>(const double *p) {
    double v;
    asm volatile("ld.relaxed.gpu.f64 %0, [%1];" : "=d"(v) : "l"(p) : "memory");
    return v;
}
template <> __device__ __forceinline__ float ld_relaxed_val<float>(const float *p) {
    float v;
    asm volatile("ld.relaxed.gpu.f32 %0, [%1];" : "=f"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_val(double *p, double v) {
    asm volatile("st.relaxed.gpu.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed_val(float *p, float v) {
    asm volatile("st.relaxed.gpu.f32 [%0], %1;" ::"l"(p), "f"(v) : "memory");
}
// "not yet produced": every bit set (a NaN that arithmetic does not produce)
__device__ __forceinline__ bool is_unset(double v) { return __double_as_longlong(v) == -1LL; }
__device__ __forceinline__ bool is_unset(float v) { return __float_as_uint(v) == 0xffffffffu; }
__device__ __forceinline__ double canonical_nan(double) { return __longlong_as_double(0x7ff8000000000000LL); }
__device__ __forceinline__ float canonical_nan(float) { return __uint_as_float(0x7fc00000u); }
template <typename T>
__device__ __forceinline__ void put_value(T *p, T v) {
    if (is_unset(v)) v = canonical_nan(v);   // a NaN either way; keep the reset pattern unique
    st_relaxed_val(p, v);
}

// ------------------------------------------------------------------ reductions
// Sum over the lanes of a group that share a right-hand-side column (xor partners at
// distance >= kt).
template <int LPR, typename T>
__device__ __forceinline__ T slice_sum(T v, int kt, unsigned gmask) {
#pragma unroll
    for (int off = LPR / 2; off >= 1; off >>= 1)
        if (off >= kt) v += __shfl_xor_sync(gmask, v, off);
    return v;
}
template <int LPR, typename T>
__device__ __forceinline__ T group_sum(T v, unsigned gmask) {
#pragma unroll
    for (int off = LPR / 2; off >= 1; off >>= 1) v += __shfl_xor_sync(gmask, v, off);
    return v;
}
template <typename T>
__device__ __forceinline__ T col_sum(T v, int kt, unsigned smask) {
    for (int off = kt >> 1; off >= 1; off >>= 1) v += __shfl_xor_sync(smask, v, off);
    return v;
}

// Bounded wait bookkeeping shared by both mechanisms: sleeps with exponential backoff,
// checks `abort` and the time limit every 16 rounds.
struct Waiter {
    unsigned ns = kBackoffMinNs;
    unsigned it = 0;
    unsigned long long t0 = 0;
    __device__ __forceinline__ bool pause(ExecState *st, unsigned long long tmo, int row) {
        if (it == 0) t0 = global_ns();
        __nanosleep(ns);
        ns = ns < kBackoffMaxNs ? ns * 2 : kBackoffMaxNs;
        if ((++it & 15u) == 0u) {
            if (ld_relaxed_u32(&st->abort)) return false;
            if (global_ns() - t0 > tmo) {
                record_error(st, SF_ERR_TIMEOUT, row);
                st_relaxed_u32(&st->abort, 1u);
                return false;
            }
        }
        return true;
    }
};

// Epoch flags: waits until every listed row (j[u] >= 0) is published in this epoch, then
// one acquire fence orders the data loads after every observed release.
template <int U>
__device__ __forceinline__ bool wait_flags(const unsigned *flags, const int (&j)[U], unsigned epoch,
                                           ExecState *st, unsigned long long tmo, int row) {
    unsigned pending = 0;
    bool any = false;
#pragma unroll
    for (int u = 0; u < U; ++u) {
        any |= j[u] >= 0;
        if (j[u] >= 0 && ld_relaxed_u32(flags + j[u]) != epoch) pending |= 1u << u;
    }
    Waiter w;
    while (pending) {
        if (!w.pause(st, tmo, row)) return false;
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (((pending >> u) & 1u) && ld_relaxed_u32(flags + j[u]) == epoch) pending &= ~(1u << u);
    }
    if (any) fence_acq_rel_gpu();
    return true;
}

// Value flags (k = 1): loads vec[j[u]] until it is no longer the reset pattern.
template <typename T, int U>
__device__ __forceinline__ bool wait_values(const T *vec, const int (&j)[U], T (&xv)[U], ExecState *st,
                                            unsigned long long tmo, int row) {
    unsigned pending = 0;
#pragma unroll
    for (int u = 0; u < U; ++u) {
        xv[u] = T(0);
        if (j[u] >= 0) {
            xv[u] = ld_relaxed_val(vec + j[u]);
            if (is_unset(xv[u])) pending |= 1u << u;
        }
    }
    Waiter w;
    while (pending) {
        if (!w.pause(st, tmo, row)) return false;
#pragma unroll
        for (int u = 0; u < U; ++u)
            if ((pending >> u) & 1u) {
                xv[u] = ld_relaxed_val(vec + j[u]);
                if (!is_unset(xv[u])) pending &= ~(1u << u);
            }
    }
    return true;
}

// One value-flag load: p[0] once it is no longer the reset pattern (ok false on a timeout).
template <typename T>
__device__ __forceinline__ T poll_value(const T *p, ExecState *st, unsigned long long tmo, int row, bool &ok) {
    T v = ld_relaxed_val(p);
    if (!is_unset(v)) return v;
    Waiter w;
    while (ok) {
        if (!w.pause(st, tmo, row)) {
            ok = false;
            break;
        }
        v = ld_relaxed_val(p);
        if (!is_unset(v)) break;
    }
    return v;
}

// Dependency mode of a row dot product.
enum Dep { D_NONE = 0, D_FLAG = 1, D_VALUE = 2 };

// Epoch-flag read for the scans below: relaxed, and free to overlap with the loads around it
// (the acquire fence that follows a scan orders the data loads).
__device__ __forceinline__ unsigned ld_flag_scan(const unsigned *p) {
    unsigned v;
    asm volatile("ld.relaxed.gpu.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}

// Entries of a row whose epoch flag was unset at the scan; flags read per lane per scan round;
// data loads in flight per lane.
constexpr int kPend = 8;
constexpr int kScanU = 16;
constexpr int kDataU = 8;
// Value-flag rows: unset operands noted per lane before the lane waits for them (their flat
// indices row * k + column fit an int: value flags need n * k < 2^31), and loads in flight per
// lane: 8 for groups of 16 or more lanes (long rows, any number of right-hand sides), else 4
// (short rows and one right-hand side; the high-occupancy variants keep to their registers).
constexpr int kVPend = 4;
__host__ __device__ constexpr int value_unroll(int lpr) { return lpr >= 16 ? 8 : 4; }

// row_dot with epoch flags, as a sliding window over the lane's slice of the row: a scan reads
// the flags ahead without fences and notes the first kPend entries whose rows are unpublished,
// stopping at the next one; one acquire fence; the published entries before that point stream
// with kDataU loads in flight; then the noted entries wait together (one fence) and load
// together, and the window moves on. A long row does most of its work before its last input
// arrives, with no fence between the loads of published entries.
template <typename T, bool PERM>
__device__ __forceinline__ T row_dot_flags(const int *__restrict__ cols, const int *__restrict__ perm,
                                           const T *__restrict__ vals, int e0, int e1, int S, const T *vec, int k,
                                           int c, bool act, const unsigned *flags, unsigned epoch, ExecState *st,
                                           unsigned long long tmo, int row, bool &ok) {
    T acc = T(0);
    int e = e0;
    while (e < e1 && ok) {
        int pend[kPend];
#pragma unroll
        for (int q = 0; q < kPend; ++q) pend[q] = -1;
        int np = 0, stop = e1;
        for (int f = e; f < e1 && stop == e1; f += S * kScanU) {
            int j[kScanU];
            unsigned fl[kScanU];
#pragma unroll
            for (int u = 0; u < kScanU; ++u) {
                const int ee = f + u * S;
                j[u] = ee < e1 ? __ldg(cols + ee) : -1;
            }
#pragma unroll
            for (int u = 0; u < kScanU; ++u) fl[u] = j[u] >= 0 ? ld_flag_scan(flags + j[u]) : epoch;
#pragma unroll
            for (int u = 0; u < kScanU; ++u)
                if (fl[u] != epoch && stop == e1) {
                    const int ee = f + u * S;
                    if (np < kPend) {
#pragma unroll
                        for (int q = 0; q < kPend; ++q)
                            if (q == np) pend[q] = ee;
                        ++np;
                    } else {
                        stop = ee;
                    }
                }
        }
        fence_acq_rel_gpu();
        if (act) {
            for (int f = e; f < stop; f += S * kDataU) {
                T vv[kDataU], xv[kDataU];
#pragma unroll
                for (int u = 0; u < kDataU; ++u) {
                    const int ee = f + u * S;
                    bool use = ee < stop;
#pragma unroll
                    for (int q = 0; q < kPend; ++q) use &= pend[q] != ee;
                    vv[u] = T(0);
                    xv[u] = T(0);
                    if (use) {
                        vv[u] = __ldg(vals + (PERM ? __ldg(perm + ee) : ee));
                        xv[u] = __ldcg(vec + (size_t)__ldg(cols + ee) * k + c);
                    }
                }
#pragma unroll
                for (int u = 0; u < kDataU; ++u) acc += vv[u] * xv[u];
            }
        }
        if (np > 0) {
            int jp[kPend];
#pragma unroll
            for (int q = 0; q < kPend; ++q) jp[q] = pend[q] >= 0 ? __ldg(cols + pend[q]) : -1;
            ok = wait_flags<kPend>(flags, jp, epoch, st, tmo, row);
            if (act && ok) {
                T vv[kPend], xv[kPend];
#pragma unroll
                for (int q = 0; q < kPend; ++q) {
                    vv[q] = T(0);
                    xv[q] = T(0);
                    if (jp[q] >= 0) {
                        vv[q] = __ldg(vals + (PERM ? __ldg(perm + pend[q]) : pend[q]));
                        xv[q] = __ldcg(vec + (size_t)jp[q] * k + c);
                    }
                }
#pragma unroll
                for (int q = 0; q < kPend; ++q) acc += vv[q] * xv[q];
            }
        }
        e = stop;
    }
    return acc;
}

// Waits for the noted operands of a value-flag dot product (bit q of `pending`: vec[pj[q]] was
// still the reset pattern) and adds their products; the noted loads are re-issued together.
template <typename T, int N>
__device__ __forceinline__ T drain_values(const T *vec, const int (&pj)[N], const T (&pv)[N], unsigned pending,
                                          ExecState *st, unsigned long long tmo, int row, bool &ok) {
    T acc = T(0);
    Waiter w;
    while (pending) {
        T xv[N];
#pragma unroll
        for (int q = 0; q < N; ++q) xv[q] = ((pending >> q) & 1u) ? ld_relaxed_val(vec + pj[q]) : T(0);
#pragma unroll
        for (int q = 0; q < N; ++q)
            if (((pending >> q) & 1u) && !is_unset(xv[q])) {
                acc += pv[q] * xv[q];
                pending &= ~(1u << q);
            }
        if (pending && !w.pause(st, tmo, row)) {
            ok = false;
            break;
        }
    }
    return acc;
}

// row_dot with value flags: every operand vec[cols[e] * k + c] is its own flag (the reset
// pattern until its producer stores it). A lane streams its slice with VU loads in flight; the
// loaded operand is the test, so a published entry costs nothing extra and no fence is needed
// anywhere. VU = 4 (groups of fewer than 16 lanes, k = 1): the unset operands of a chunk are
// waited for before the next chunk. VU = 8 (groups of 16 or 32 lanes, any k): unset entries are
// noted (up to kVPend) and the lane moves on; when the list is full, and at the end of the
// slice, it waits for them together, so a long row does most of its work before its last input
// exists.
template <typename T, bool PERM, int VU>
__device__ __forceinline__ T row_dot_values(const int *__restrict__ cols, const int *__restrict__ perm,
                                            const T *__restrict__ vals, int e0, int e1, int S, const T *vec, int k,
                                            int c, bool act, ExecState *st, unsigned long long tmo, int row,
                                            bool &ok) {
    T acc = T(0);
    if constexpr (VU <= 4) {
        // one right-hand side (the host publishes through values with fewer than 16 lanes per
        // row only when k = 1), so the operand of entry e is vec[cols[e]]
        for (int f = e0; f < e1; f += S * VU) {
            int j[VU];
            T vv[VU], xv[VU];
#pragma unroll
            for (int u = 0; u < VU; ++u) {
                const int ee = f + u * S;
                j[u] = -1;
                vv[u] = T(0);
                if (ee < e1) {
                    j[u] = __ldg(cols + ee);
                    vv[u] = __ldg(vals + (PERM ? __ldg(perm + ee) : ee));
                }
            }
            if (ok) ok = wait_values<T, VU>(vec, j, xv, st, tmo, row);
#pragma unroll
            for (int u = 0; u < VU; ++u)
                if (j[u] >= 0) acc += vv[u] * xv[u];
        }
        return acc;
    } else {
        if (!act) return acc;
        int pj[kVPend];
        T pv[kVPend];
#pragma unroll
        for (int q = 0; q < kVPend; ++q) {
            pj[q] = 0;
            pv[q] = T(0);
        }
        int np = 0;
        for (int f = e0; f < e1 && ok; f += S * VU) {
            T vv[VU], xv[VU];
            int jx[VU];
#pragma unroll
            for (int u = 0; u < VU; ++u) {
                const int ee = f + u * S;
                vv[u] = T(0);
                jx[u] = 0;
                if (ee < e1) {
                    vv[u] = __ldg(vals + (PERM ? __ldg(perm + ee) : ee));
                    jx[u] = __ldg(cols + ee) * k + c;
                }
            }
#pragma unroll
            for (int u = 0; u < VU; ++u) xv[u] = (f + u * S < e1) ? ld_relaxed_val(vec + jx[u]) : T(0);
#pragma unroll
            for (int u = 0; u < VU; ++u) {
                if (f + u * S >= e1) continue;
                if (!is_unset(xv[u])) {
                    acc += vv[u] * xv[u];
                    continue;
                }
                if (np == kVPend) {
                    acc += drain_values<T, kVPend>(vec, pj, pv, (1u << kVPend) - 1u, st, tmo, row, ok);
                    np = 0;
                }
#pragma unroll
                for (int q = 0; q < kVPend; ++q)
                    if (q == np) {
                        pj[q] = jx[u];
                        pv[q] = vv[u];
                    }
                ++np;
            }
        }
        if (np > 0 && ok) acc += drain_values<T, kVPend>(vec, pj, pv, (1u << np) - 1u, st, tmo, row, ok);
        return acc;
    }
}

// acc = sum over this lane's slice of entries e in [e0, e1) (stride S) of
// vals[PERM ? perm[e] : e] * vec[cols[e] * k + c]. D_FLAG / D_VALUE wait for the rows
// cols[e] first (vec is produced by other warps in this launch).
template <typename T, int DEP, bool PERM, int VU = 4>
__device__ __forceinline__ T row_dot(const int *__restrict__ cols, const int *__restrict__ perm,
                                     const T *__restrict__ vals, int e0, int e1, int S, const T *vec,
                                     int k, int c, bool act, const unsigned *flags, unsigned epoch,
                                     ExecState *st, unsigned long long tmo, int row, bool &ok) {
    if constexpr (DEP == D_FLAG)
        return row_dot_flags<T, PERM>(cols, perm, vals, e0, e1, S, vec, k, c, act, flags, epoch, st, tmo, row, ok);
    if constexpr (DEP == D_VALUE)
        return row_dot_values<T, PERM, VU>(cols, perm, vals, e0, e1, S, vec, k, c, act, st, tmo, row, ok);
    if constexpr (DEP == D_NONE) {
        // nothing to wait for: kDataU loads in flight per lane, issued before their products
        T acc = T(0);
        if (act) {
            for (int e = e0; e < e1; e += S * kDataU) {
                T vv[kDataU], xv[kDataU];
#pragma unroll
                for (int u = 0; u < kDataU; ++u) {
                    const int ee = e + u * S;
                    vv[u] = T(0);
                    xv[u] = T(0);
                    if (ee < e1) {
                        vv[u] = __ldg(vals + (PERM ? __ldg(perm + ee) : ee));
                        xv[u] = __ldg(vec + (size_t)__ldg(cols + ee) * k + c);
                    }
                }
#pragma unroll
                for (int u = 0; u < kDataU; ++u) acc += vv[u] * xv[u];
            }
        }
        return acc;
    }
}

// Gauss-Seidel row with L = tril(A) read from A's own storage (shared storage, value flags):
// one pass over the lane's slice of A's row gives ax = sum_j A_ij x_in_j over every entry and
// az = sum_{j<i} A_ij z_j over the entries before the diagonal position dp, each z_j waited for
// as in row_dot_values (VU = 4: per chunk, one right-hand side; VU = 8: noted when unset and
// drained when the list fills and at the end).
template <typename T, int VU>
__device__ __forceinline__ void gs_row_dot(const int *__restrict__ cols, const T *__restrict__ vals, int e0, int dp,
                                           int e1, int S, const T *__restrict__ xin, const T *z, int k, int c,
                                           bool act, ExecState *st, unsigned long long tmo, int row, bool &ok, T &ax,
                                           T &az) {
    ax = T(0);
    az = T(0);
    if constexpr (VU <= 4) {
        // one right-hand side (groups of fewer than 16 lanes): chunks of VU entries, the unset
        // z operands of a chunk waited for before the next chunk
        for (int f = e0; f < e1; f += S * VU) {
            int j[VU], jz[VU];
            T vv[VU], xv[VU], zv[VU];
#pragma unroll
            for (int u = 0; u < VU; ++u) {
                const int ee = f + u * S;
                j[u] = jz[u] = -1;
                vv[u] = T(0);
                if (ee < e1) {
                    j[u] = __ldg(cols + ee);
                    vv[u] = __ldg(vals + ee);
                    if (ee < dp) jz[u] = j[u];
                }
            }
#pragma unroll
            for (int u = 0; u < VU; ++u) xv[u] = j[u] >= 0 ? __ldg(xin + j[u]) : T(0);
            if (ok) ok = wait_values<T, VU>(z, jz, zv, st, tmo, row);
#pragma unroll
            for (int u = 0; u < VU; ++u) {
                ax += vv[u] * xv[u];
                if (jz[u] >= 0) az += vv[u] * zv[u];
            }
        }
        return;
    }
    if (!act) return;
    int pj[kVPend];
    T pv[kVPend];
#pragma unroll
    for (int q = 0; q < kVPend; ++q) {
        pj[q] = 0;
        pv[q] = T(0);
    }
    int np = 0;
    for (int f = e0; f < e1 && ok; f += S * VU) {
        T vv[VU], xv[VU], zv[VU];
        int jx[VU];
#pragma unroll
        for (int u = 0; u < VU; ++u) {
            const int ee = f + u * S;
            vv[u] = T(0);
            jx[u] = 0;
            if (ee < e1) {
                vv[u] = __ldg(vals + ee);
                jx[u] = __ldg(cols + ee) * k + c;
            }
        }
#pragma unroll
        for (int u = 0; u < VU; ++u) {
            const int ee = f + u * S;
            xv[u] = ee < e1 ? __ldg(xin + jx[u]) : T(0);
            zv[u] = ee < dp ? ld_relaxed_val(z + jx[u]) : T(0);
        }
#pragma unroll
        for (int u = 0; u < VU; ++u) {
            const int ee = f + u * S;
            if (ee >= e1) continue;
            ax += vv[u] * xv[u];
            if (ee >= dp) continue;
            if (!is_unset(zv[u])) {
                az += vv[u] * zv[u];
                continue;
            }
            if (np == kVPend) {
                az += drain_values<T, kVPend>(z, pj, pv, (1u << kVPend) - 1u, st, tmo, row, ok);
                np = 0;
            }
#pragma unroll
            for (int q = 0; q < kVPend; ++q)
                if (q == np) {
                    pj[q] = jx[u];
                    pv[q] = vv[u];
                }
            ++np;
        }
    }
    if (np > 0 && ok) az += drain_values<T, kVPend>(z, pj, pv, (1u << np) - 1u, st, tmo, row, ok);
}

template <int LPR>
__device__ __forceinline__ bool group_ok(bool ok, unsigned gmask) {
    return !__any_sync(gmask, !ok);
}

// Epoch-flag publication of a row written by the lanes of a group.
__device__ __forceinline__ void publish(const ExecArgs &a, int row, unsigned epoch, int gl, unsigned gmask,
                                        bool ok) {
    __syncwarp(gmask);
    if (gl == 0 && ok) st_release_u32(a.flags + row, epoch);
}

// Writes one produced value: with value flags the store itself publishes it.
template <bool VF, typename T>
__device__ __forceinline__ void store_out(T *p, T v) {
    if (VF) put_value(p, v);
    else *p = v;
}

// Diagonal of a solve row. With a reciprocal table (a.rdiag: 1 / L_ii written by the pre-pass
// of k = 1 launches with value flags) the row finishes with a multiply, which takes the
// division off the dependence chain; the table's pre-pass also checks for zero diagonals.
template <typename T>
__device__ __forceinline__ T load_diag(const ExecArgs &a, const T *vals, int e, int row, int gl) {
    if (a.rdiag) return __ldg((const T *)a.rdiag + row);
    const T d = __ldg(vals + e);
    if (gl == 0 && d == T(0)) record_error(a.st, SF_ERR_NONFINITE, row);
    return d;
}
template <typename T>
__device__ __forceinline__ T finish_row(const ExecArgs &a, T num, T d) { return a.rdiag ? num * d : num / d; }

// ---------------------------------------------------------------- item kinds
// SpTRSV row (Table 2, forward substitution): x_i = (b_i - sum_{j<i} L_ij x_j) / L_ii.
// `x` is both the output and the buffer the dependences are read from.
template <typename T, int LPR, bool VF, int VU = value_unroll(LPR)>
__device__ bool item_trsv(const ExecArgs &a, int row, unsigned epoch, int gl, unsigned gmask, T *x) {
    const int kt = a.kt, S = LPR / kt, s = gl / kt, cl = gl % kt, k = a.k;
    const int rs = __ldg(a.Lrp + row), dg = __ldg(a.Lrp + row + 1) - 1;
    const T *Lv = (const T *)a.Lv, *b = (const T *)a.b;
    const T d = load_diag<T>(a, Lv, dg, row, gl);
    bool ok = true;
    for (int c0 = 0; c0 < k; c0 += kt) {
        const int c = c0 + cl;
        const bool act = c < k;
        // operands that need no wait are loaded before it, off the dependence chain
        const T bc = (s == 0 && act) ? __ldg(b + (size_t)row * k + c) : T(0);
        T acc = row_dot<T, VF ? D_VALUE : D_FLAG, false, VU>(a.Lci, nullptr, Lv, rs + s, dg, S, x, k, c, act, a.flags,
                                                         epoch, a.st, a.timeout_ns, row, ok);
        acc = slice_sum<LPR>(acc, kt, gmask);
        if (s == 0 && act) store_out<VF>(x + (size_t)row * k + c, finish_row<T>(a, bc - acc, d));
    }
    ok = group_ok<LPR>(ok, gmask);
    if (!VF) publish(a, row, epoch, gl, gmask, ok);
    return ok;
}

// SpMV row of the second kernel with F = pattern(M): y_i = sum_j M_ij x_j, each x_j
// waited for (§2.2 "Dependency Matrix F": row i of F lists the first-kernel iterations
// row i of the second kernel reads).
template <typename T, int LPR, bool VF, int VU = value_unroll(LPR)>
__device__ bool item_spmv_dep(const ExecArgs &a, int row, unsigned epoch, int gl, unsigned gmask, const T *x) {
    const int kt = a.kt, S = LPR / kt, s = gl / kt, cl = gl % kt, k = a.k;
    const int rs = __ldg(a.Mrp + row), re = __ldg(a.Mrp + row + 1);
    T *y = (T *)a.y;
    bool ok = true;
    for (int c0 = 0; c0 < k; c0 += kt) {
        const int c = c0 + cl;
        const bool act = c < k;
        T acc = row_dot<T, VF ? D_VALUE : D_FLAG, false, VU>(a.Mci, nullptr, (const T *)a.Mv, rs + s, re, S, x, k, c,
                                                         act, a.flags, epoch, a.st, a.timeout_ns, row, ok);
        acc = slice_sum<LPR>(acc, kt, gmask);
        if (s == 0 && act) y[(size_t)row * k + c] = acc;
    }
    return group_ok<LPR>(ok, gmask);
}

// Solve row of a separated SpMV -> SpTRSV (§3.2.3): r_i was computed before the partitions by
// some group of the launch; only the solve row remains, over L's strict part (A's entries
// before the diagonal in shared storage). Kept out of line so that the paired item's register
// budget does not grow.
template <typename T, int LPR, int VU>
__device__ __noinline__ bool item_spmv_trsv_sep(const ExecArgs &a, int row, unsigned epoch, int gl, unsigned gmask,
                                                int ra) {
    const int kt = a.kt, S = LPR / kt, s = gl / kt, cl = gl % kt, k = a.k;
    int lo, hi;
    const int *cols;
    const T *vals;
    T d;
    if (a.Lv == nullptr) {
        const int dp = __ldg(a.a_diag + row);
        lo = ra;
        hi = dp;
        cols = a.Mci;
        vals = (const T *)a.Mv;
        d = load_diag<T>(a, vals, dp, row, gl);
    } else {
        lo = __ldg(a.Lrp + row);
        hi = __ldg(a.Lrp + row + 1) - 1;
        cols = a.Lci;
        vals = (const T *)a.Lv;
        d = load_diag<T>(a, vals, hi, row, gl);
    }
    const T *r = (const T *)a.rsep;
    T *z = (T *)a.y;
    bool ok = true;
    for (int c0 = 0; c0 < k; c0 += kt) {
        const int c = c0 + cl;
        const bool act = c < k;
        T acc = row_dot<T, D_VALUE, false, VU>(cols, nullptr, vals, lo + s, hi, S, z, k, c, act, a.flags, epoch,
                                               a.st, a.timeout_ns, row, ok);
        acc = slice_sum<LPR>(acc, kt, gmask);
        if (s == 0 && act) {
            const T ri = poll_value(r + (size_t)row * k + c, a.st, a.timeout_ns, row, ok);
            put_value(z + (size_t)row * k + c, finish_row<T>(a, ri - acc, d));
        }
    }
    return group_ok<LPR>(ok, gmask);
}

// Paired SpMV -> SpTRSV row (combination 2, F = I): r_i = b_i - A_i x_in stays in
// registers, then z_i = (r_i - sum_{j<i} L_ij z_j) / L_ii.
template <typename T, int LPR, bool VF, int VU = value_unroll(LPR), bool SEP = true>
__device__ bool item_spmv_trsv(const ExecArgs &a, int row, unsigned epoch, int gl, unsigned gmask) {
    const int kt = a.kt, S = LPR / kt, s = gl / kt, cl = gl % kt, k = a.k;
    const int ra = __ldg(a.Mrp + row), re = __ldg(a.Mrp + row + 1);
    if constexpr (VF) {
        if constexpr (SEP)
            if (a.rsep) return item_spmv_trsv_sep<T, LPR, VU>(a, row, epoch, gl, gmask, ra);
        if (a.Lv == nullptr) {
            // shared storage (Table 2 combination 2 as one Gauss-Seidel half-sweep): L = tril(A) is
            // read from A's row, which is streamed once for both r_i and the solve
            const int dp = __ldg(a.a_diag + row);
            const T *Av = (const T *)a.Mv, *b = (const T *)a.b;
            T *z = (T *)a.y;
            const T d = load_diag<T>(a, Av, dp, row, gl);
            bool ok = true;
            for (int c0 = 0; c0 < k; c0 += kt) {
                const int c = c0 + cl;
                const bool act = c < k;
                const T bc = (s == 0 && act) ? __ldg(b + (size_t)row * k + c) : T(0);
                T ax, az;
                gs_row_dot<T, VU>(a.Mci, Av, ra + s, dp, re, S, (const T *)a.xin, z, k, c, act, a.st, a.timeout_ns, row,
                              ok, ax, az);
                ax = slice_sum<LPR>(ax, kt, gmask);
                az = slice_sum<LPR>(az, kt, gmask);
                if (s == 0 && act) put_value(z + (size_t)row * k + c, finish_row<T>(a, (bc - ax) - az, d));
            }
            return group_ok<LPR>(ok, gmask);
        }
    }
    const int rs = __ldg(a.Lrp + row), dg = __ldg(a.Lrp + row + 1) - 1;
    const T *Lv = (const T *)a.Lv, *b = (const T *)a.b;
    T *z = (T *)a.y;
    const T d = load_diag<T>(a, Lv, dg, row, gl);
    bool ok = true;
    for (int c0 = 0; c0 < k; c0 += kt) {
        const int c = c0 + cl;
        const bool act = c < k;
        const T bc = (s == 0 && act) ? __ldg(b + (size_t)row * k + c) : T(0);
        T accA = row_dot<T, D_NONE, false>(a.Mci, nullptr, (const T *)a.Mv, ra + s, re, S, (const T *)a.xin, k, c,
                                           act, a.flags, epoch, a.st, a.timeout_ns, row, ok);
        accA = slice_sum<LPR>(accA, kt, gmask);
        const T r = bc - accA;   // r_i is complete before the wait on z
        T accL = row_dot<T, VF ? D_VALUE : D_FLAG, false, VU>(a.Lci, nullptr, Lv, rs + s, dg, S, z, k, c, act, a.flags,
                                                          epoch, a.st, a.timeout_ns, row, ok);
        accL = slice_sum<LPR>(accL, kt, gmask);
        if (s == 0 && act) store_out<VF>(z + (size_t)row * k + c, finish_row<T>(a, r - accL, d));
    }
    ok = group_ok<LPR>(ok, gmask);
    if (!VF) publish(a, row, epoch, gl, gmask, ok);
    return ok;
}

// Factor entries of IC0 row i (up-looking form, §2.1) with the common columns found by a
// binary search of row i for every column of row j; returns sum_{k<i} L_ik^2 on every lane.
template <typename T, int LPR>
__device__ __forceinline__ T ic0_row_search(const ExecArgs &a, int rs, int dg, int gl, unsigned gmask) {
    const T *Av = (const T *)a.Lv;
    T *lf = (T *)a.xs;
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
    return group_sum<LPR>(sq, gmask);
}

// Factor entries of IC0 row i with the inspector's intersection pairs (a.ic0_pp/ic0_pairs):
// lanes take one entry each. An entry without pairs depends on no other entry of its row
// (L_ij = A_ij / L_jj), so those finish side by side; entries with pairs follow one at a time
// in increasing column order, the group summing their pair products. 1 / L_jj comes from the
// table the rows publish with their factor (a.ic0_rinv), so an entry costs one multiply. The
// first chunk's pattern and A values (j0, q0, q1, av0) were loaded before the wait. Returns
// sum_{k<i} L_ik^2 on every lane; the sum runs over the lanes that hold entries only.
template <typename T, int LPR, bool VF, int VU = value_unroll(LPR)>
__device__ __forceinline__ T ic0_row_pairs(const ExecArgs &a, int row, int rs, int dg, int gl, unsigned gmask, int j0,
                                           int q0, int q1, T av0, bool &ok) {
    const T *Av = (const T *)a.Lv;
    const T *rinv = (const T *)a.ic0_rinv;
    T *lf = (T *)a.xs;
    const int gbase = (int)(threadIdx.x & 31) - gl;
    T sq = T(0);
    for (int c0 = rs; c0 < dg; c0 += LPR) {
        const int t = c0 + gl;
        const bool mine = t < dg;
        int j = j0, p0 = q0, p1 = q1;
        T av = av0;
        if (c0 != rs && mine) {
            j = __ldg(a.Lci + t);
            p0 = __ldg(a.ic0_pp + t);
            p1 = __ldg(a.ic0_pp + t + 1);
            av = __ldg(Av + t);
        }
        T rj = T(0);
        if (mine) rj = VF ? poll_value(rinv + j, a.st, a.timeout_ns, row, ok) : __ldcg(rinv + j);
        T v = T(0);
        if (mine && p0 == p1) {
            v = av * rj;
            store_out<VF>(lf + t, v);
        }
        unsigned serial = __ballot_sync(gmask, mine && p0 < p1);
        if (serial) {
            __syncwarp(gmask);
            while (serial) {
                const int src = __ffs(serial) - 1;
                serial &= serial - 1;
                const int s0 = __shfl_sync(gmask, p0, src), s1 = __shfl_sync(gmask, p1, src);
                T part = T(0);
                for (int g = s0 + gl; g < s1; g += LPR) {
                    const int2 pq = __ldg(a.ic0_pairs + g);
                    const T lq = VF ? poll_value(lf + pq.y, a.st, a.timeout_ns, row, ok) : __ldcg(lf + pq.y);
                    part += lf[pq.x] * lq;
                }
                part = group_sum<LPR>(part, gmask);
                if (gl == src - gbase) {
                    v = (av - part) * rj;
                    store_out<VF>(lf + t, v);
                }
                __syncwarp(gmask);
            }
        }
        sq += v * v;
    }
    const int w = dg - rs;   // lanes at or past w hold no entry
#pragma unroll
    for (int off = LPR / 2; off >= 1; off >>= 1)
        if (off < w) sq += __shfl_xor_sync(gmask, sq, off);
    return __shfl_sync(gmask, sq, gbase);
}

__device__ __forceinline__ double rsqrt_t(double x) { return rsqrt(x); }
__device__ __forceinline__ float rsqrt_t(float x) { return rsqrtf(x); }

// Paired SpIC0 -> SpTRSV row (combination 5, F = I), IC0 in its up-looking row form:
// for each j < i in row i, ascending, L_ij = (A_ij - sum_{k<j, k in both rows} L_ik L_jk)
// / L_jj; then L_ii = sqrt(A_ii - sum_{k<i} L_ik^2); then the solve row with the fresh
// L_i on chip: y_i = (b_i - sum_j L_ij y_j) / L_ii. Factor values go to a.xs; 1 / L_ii goes
// to a.ic0_rinv with them (one reciprocal square root gives both L_ii and 1 / L_ii).
// With value flags (VF; the pair lists are then present) nothing waits on epoch flags: the
// factor polls 1 / L_jj and the factor entries its pairs read, each solve lane polls its
// column of the predecessor rows of y, and every such value is stored as its own flag.
template <typename T, int LPR, bool SOLVE, bool VF>
__device__ bool item_ic0(const ExecArgs &a, int row, unsigned epoch, int gl, unsigned gmask) {
    const int rs = __ldg(a.Lrp + row), dg = __ldg(a.Lrp + row + 1) - 1;
    const T *Av = (const T *)a.Lv;
    T *lf = (T *)a.xs;
    // pattern-only operands of the first chunk, loaded before the wait
    int j0 = 0, q0 = 0, q1 = 0;
    T av0 = T(0);
    if (a.ic0_pp && rs + gl < dg) {
        j0 = __ldg(a.Lci + rs + gl);
        q0 = __ldg(a.ic0_pp + rs + gl);
        q1 = __ldg(a.ic0_pp + rs + gl + 1);
        av0 = __ldg(Av + rs + gl);
    }
    const T aii = __ldg(Av + dg);
    bool ok = true;
    // every predecessor row publishes its factor row and its solve row together
    for (int e = rs + gl; !VF && e < dg; e += LPR * kUnroll) {
        int j[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const int ee = e + u * LPR;
            j[u] = ee < dg ? __ldg(a.Lci + ee) : -1;
        }
        if (ok) ok = wait_flags<kUnroll>(a.flags, j, epoch, a.st, a.timeout_ns, row);
    }
    ok = group_ok<LPR>(ok, gmask);
    // The solve's first column tile of y over the row's first entries does not depend on the
    // factor: it is loaded before the factor row is computed.
    constexpr int kY = 4;
    T yv[kY];
    T bv = T(0);
    if (SOLVE) {
        const int kt = a.kt, S = LPR / kt, s = gl / kt, cl = gl % kt, k = a.k;
        const T *y = (const T *)a.y;
        if constexpr (VF) {
            int jy[kY];
#pragma unroll
            for (int u = 0; u < kY; ++u) {
                const int t = rs + s + u * S;
                jy[u] = (cl < k && t < dg) ? __ldg(a.Lci + t) * k + cl : -1;
            }
            if (!wait_values<T, kY>(y, jy, yv, a.st, a.timeout_ns, row)) ok = false;
        } else {
#pragma unroll
            for (int u = 0; u < kY; ++u) {
                const int t = rs + s + u * S;
                yv[u] = (cl < k && t < dg) ? __ldcg(y + (size_t)__ldg(a.Lci + t) * k + cl) : T(0);
            }
        }
        if (s == 0 && cl < k) bv = __ldg((const T *)a.b + (size_t)row * k + cl);
    }
    T sq;
    if (VF || a.ic0_pp) sq = ic0_row_pairs<T, LPR, VF>(a, row, rs, dg, gl, gmask, j0, q0, q1, av0, ok);
    else sq = ic0_row_search<T, LPR>(a, rs, dg, gl, gmask);
    const T dd = aii - sq;
    if (gl == 0 && !(dd > T(0))) record_error(a.st, SF_ERR_BREAKDOWN, row);
    const T ri = rsqrt_t(dd);
    if (gl == 0) {
        lf[dg] = dd * ri;
        store_out<VF>((T *)a.ic0_rinv + row, ri);
    }
    if (SOLVE) {
        const int kt = a.kt, S = LPR / kt, s = gl / kt, cl = gl % kt, k = a.k;
        const T *b = (const T *)a.b;
        T *y = (T *)a.y;
        __syncwarp(gmask);
        for (int c0 = 0; c0 < k; c0 += kt) {
            const int c = c0 + cl;
            T acc = T(0);
            int t = rs + s;
            if (c0 == 0) {
#pragma unroll
                for (int u = 0; u < kY; ++u)
                    if (t + u * S < dg) acc += lf[t + u * S] * yv[u];
                t += kY * S;
            }
            if (c < k)
                for (; t < dg; t += S) {
                    const T *yp = y + (size_t)__ldg(a.Lci + t) * k + c;
                    acc += lf[t] * (VF ? poll_value(yp, a.st, a.timeout_ns, row, ok) : __ldcg(yp));
                }
            acc = slice_sum<LPR>(acc, kt, gmask);
            if (s == 0 && c < k)
                store_out<VF>(y + (size_t)row * k + c, ((c0 == 0 ? bv : __ldg(b + (size_t)row * k + c)) - acc) * ri);
        }
    }
    if (VF) return group_ok<LPR>(ok, gmask);
    publish(a, row, epoch, gl, gmask, ok);
    return ok;
}

// Adjoint of SpTRSV -> SpMV as a paired pass on the transposed schedule (item j = column
// j of L): u_j = (M^T gy)_j needs no wait; lam_j = (u_j - sum_{i>j} L_ij lam_i) / L_jj
// waits for lam_i; gb = lam. Values of M^T and L^T come in transposed order (a.MTv, a.LTv);
// the value gradients run afterwards as a separate streaming pass.
template <typename T, int LPR, bool VF, int VU = value_unroll(LPR)>
__device__ bool item_adj_trsv_spmv(const ExecArgs &a, int j, unsigned epoch, int gl, int gbase, unsigned gmask) {
    const int kt = a.kt, S = LPR / kt, s = gl / kt, cl = gl % kt, k = a.k;
    const int ms = __ldg(a.MTrp + j), me = __ldg(a.MTrp + j + 1);
    const int ls = __ldg(a.LTrp + j), le = __ldg(a.LTrp + j + 1);   // first entry of L^T row j is L_jj
    const T *LTv = (const T *)a.LTv, *gy = (const T *)a.gy;
    T *lam = (T *)a.gb;
    const T d = load_diag<T>(a, LTv, ls, j, gl);
    bool ok = true;
    for (int c0 = 0; c0 < k; c0 += kt) {
        const int c = c0 + cl;
        const bool act = c < k;
        T u = row_dot<T, D_NONE, false>(a.MTci, nullptr, (const T *)a.MTv, ms + s, me, S, gy, k, c, act, a.flags,
                                        epoch, a.st, a.timeout_ns, j, ok);
        u = slice_sum<LPR>(u, kt, gmask);   // u_j is complete before the wait on lam
        T accL = row_dot<T, VF ? D_VALUE : D_FLAG, false, VU>(a.LTci, nullptr, LTv, ls + 1 + s, le, S, lam, k, c, act,
                                                          a.flags, epoch, a.st, a.timeout_ns, j, ok);
        accL = slice_sum<LPR>(accL, kt, gmask);
        if (s == 0 && act) store_out<VF>(lam + (size_t)j * k + c, finish_row<T>(a, u - accL, d));
    }
    ok = group_ok<LPR>(ok, gmask);
    if (!VF) publish(a, j, epoch, gl, gmask, ok);
    return ok;
}

// Adjoint of SpMV -> SpTRSV, tag 0: lam_j = (gz_j - sum_{i>j} L_ij lam_i) / L_jj, gb = lam.
template <typename T, int LPR, bool VF, int VU = value_unroll(LPR)>
__device__ bool item_adj_lam(const ExecArgs &a, int j, unsigned epoch, int gl, int gbase, unsigned gmask) {
    const int kt = a.kt, S = LPR / kt, s = gl / kt, cl = gl % kt, k = a.k;
    const int ls = __ldg(a.LTrp + j), le = __ldg(a.LTrp + j + 1);
    const T *LTv = (const T *)a.LTv, *gz = (const T *)a.gy;
    T *lam = (T *)a.gb;
    const T d = load_diag<T>(a, LTv, ls, j, gl);
    bool ok = true;
    for (int c0 = 0; c0 < k; c0 += kt) {
        const int c = c0 + cl;
        const bool act = c < k;
        const T gc = (s == 0 && act) ? __ldg(gz + (size_t)j * k + c) : T(0);
        T accL = row_dot<T, VF ? D_VALUE : D_FLAG, false, VU>(a.LTci, nullptr, LTv, ls + 1 + s, le, S, lam, k, c, act,
                                                          a.flags, epoch, a.st, a.timeout_ns, j, ok);
        accL = slice_sum<LPR>(accL, kt, gmask);
        if (s == 0 && act) store_out<VF>(lam + (size_t)j * k + c, finish_row<T>(a, gc - accL, d));
    }
    ok = group_ok<LPR>(ok, gmask);
    if (!VF) publish(a, j, epoch, gl, gmask, ok);
    return ok;
}

// Adjoint of SpMV -> SpTRSV, tag 1: gx_j = -sum_i A_ij lam_i, waiting for each lam_i.
template <typename T, int LPR, bool VF, int VU = value_unroll(LPR)>
__device__ bool item_adj_gx(const ExecArgs &a, int j, unsigned epoch, int gl, unsigned gmask) {
    const int kt = a.kt, S = LPR / kt, s = gl / kt, cl = gl % kt, k = a.k;
    const int ms = __ldg(a.MTrp + j), me = __ldg(a.MTrp + j + 1);
    T *gx = (T *)a.gx;
    bool ok = true;
    for (int c0 = 0; c0 < k; c0 += kt) {
        const int c = c0 + cl;
        const bool act = c < k;
        T acc = row_dot<T, VF ? D_VALUE : D_FLAG, false, VU>(a.MTci, nullptr, (const T *)a.MTv, ms + s, me, S,
                                                         (const T *)a.gb, k, c, act, a.flags, epoch, a.st,
                                                         a.timeout_ns, j, ok);
        acc = slice_sum<LPR>(acc, kt, gmask);
        if (s == 0 && act) gx[(size_t)j * k + c] = -acc;
    }
    return group_ok<LPR>(ok, gmask);
}

// Paired SpTRSV -> SpTRSV row (Table 2 combination 1, F = I, same L): x_i = (b_i - sum_{j<i}
// L_ij x_j) / L_ii, then z_i = (x_i - sum_{j<i} L_ij z_j) / L_ii while x_i is still in registers
// (the row of L is read twice by the same lanes, the second time from L1). x goes to a.xs,
// z to a.y; with value flags each is published by its store.
template <typename T, int LPR, bool VF, int VU = value_unroll(LPR)>
__device__ bool item_trsv_trsv(const ExecArgs &a, int row, unsigned epoch, int gl, unsigned gmask) {
    const int kt = a.kt, S = LPR / kt, s = gl / kt, cl = gl % kt, k = a.k;
    const int rs = __ldg(a.Lrp + row), dg = __ldg(a.Lrp + row + 1) - 1;
    const T *Lv = (const T *)a.Lv, *b = (const T *)a.b;
    T *x = (T *)a.xs, *z = (T *)a.y;
    const T d = load_diag<T>(a, Lv, dg, row, gl);
    bool ok = true;
    for (int c0 = 0; c0 < k; c0 += kt) {
        const int c = c0 + cl;
        const bool act = c < k;
        const T bc = act ? __ldg(b + (size_t)row * k + c) : T(0);
        T acc = row_dot<T, VF ? D_VALUE : D_FLAG, false, VU>(a.Lci, nullptr, Lv, rs + s, dg, S, x, k, c, act, a.flags,
                                                         epoch, a.st, a.timeout_ns, row, ok);
        acc = slice_sum<LPR>(acc, kt, gmask);
        const T xi = finish_row<T>(a, bc - acc, d);
        if (s == 0 && act) store_out<VF>(x + (size_t)row * k + c, xi);
        T acc2 = row_dot<T, VF ? D_VALUE : D_FLAG, false, VU>(a.Lci, nullptr, Lv, rs + s, dg, S, z, k, c, act, a.flags,
                                                          epoch, a.st, a.timeout_ns, row, ok);
        acc2 = slice_sum<LPR>(acc2, kt, gmask);
        if (s == 0 && act) store_out<VF>(z + (size_t)row * k + c, finish_row<T>(a, xi - acc2, d));
    }
    ok = group_ok<LPR>(ok, gmask);
    if (!VF) publish(a, row, epoch, gl, gmask, ok);
    return ok;
}

// Paired SpILU0 -> SpTRSV row (Table 2 combination 6, F = I), whole warp, value flags only.
// Zero fill-in ILU0 in its row-oriented (IKJ) form on A's pattern: row i's working copy w sits
// in shared memory (lane l owns the entries t = l, l + 32, ...); for each k < i in the row,
// ascending: l_ik = w_ik / u_kk, then every later entry w_ij with (k, j) in row k's pattern
// loses l_ik u_kj (the lane owning j finds it by binary search in row k after its diagonal).
// u_kk and u_kj are the values row k stored (each its own flag). The finished row is stored to
// the factor (a.xs, on A's pattern: strictly lower part of the unit lower L, then U), and the
// solve row with the unit lower factor follows from shared memory:
// y_i = b_i - sum_{k<i} l_ik y_k. A zero pivot u_kk records SF_ERR_BREAKDOWN with row k.
template <typename T>
__device__ bool item_ilu0(const ExecArgs &a, int row, int gl) {
    __shared__ T wbuf[kExecThreads / 32][kIluMaxRow];
    T *w = wbuf[threadIdx.x >> 5];
    const unsigned full = 0xffffffffu;
    const int ra = __ldg(a.Mrp + row), re = __ldg(a.Mrp + row + 1), dp = __ldg(a.a_diag + row);
    const int len = re - ra;
    const T *Av = (const T *)a.Mv;
    T *lu = (T *)a.xs;
    bool ok = true;
    for (int t = gl; t < len; t += 32) w[t] = __ldg(Av + ra + t);
    __syncwarp(full);
    for (int e = ra; e < dp; ++e) {
        const int kr = __ldg(a.Mci + e);
        const int dk = __ldg(a.a_diag + kr), kend = __ldg(a.Mrp + kr + 1);
        T ukk = T(0);
        if (gl == 0) ukk = poll_value(lu + dk, a.st, a.timeout_ns, row, ok);
        ukk = __shfl_sync(full, ukk, 0);
        if (__shfl_sync(full, ok ? 1 : 0, 0) == 0) {
            ok = false;
            break;
        }
        if (gl == 0 && ukk == T(0)) record_error(a.st, SF_ERR_BREAKDOWN, kr);
        const T lik = w[e - ra] / ukk;
        __syncwarp(full);
        if (((e - ra) & 31) == gl) w[e - ra] = lik;
        for (int t = gl; t < len; t += 32) {
            const int f = ra + t;
            if (f <= e) continue;
            const int j = __ldg(a.Mci + f);
            int lo = dk + 1, hi = kend;   // column j among row k's entries after its diagonal
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (__ldg(a.Mci + mid) < j) lo = mid + 1; else hi = mid;
            }
            if (lo < kend && __ldg(a.Mci + lo) == j) w[t] -= lik * poll_value(lu + lo, a.st, a.timeout_ns, row, ok);
        }
        __syncwarp(full);
    }
    ok = !__any_sync(full, !ok);
    for (int t = gl; t < len && ok; t += 32) put_value(lu + ra + t, w[t]);
    const int kt = a.kt, S = 32 / kt, s = gl / kt, cl = gl % kt, k = a.k;
    const T *b = (const T *)a.b;
    T *y = (T *)a.y;
    for (int c0 = 0; c0 < k && ok; c0 += kt) {
        const int c = c0 + cl;
        const bool act = c < k;
        T acc = T(0);
        if (act)
            for (int e = ra + s; e < dp && ok; e += S)
                acc += w[e - ra] * poll_value(y + (size_t)__ldg(a.Mci + e) * k + c, a.st, a.timeout_ns, row, ok);
        acc = slice_sum<32>(acc, kt, full);
        if (s == 0 && act && ok) put_value(y + (size_t)row * k + c, __ldg(b + (size_t)row * k + c) - acc);
    }
    return !__any_sync(full, !ok);
}

// Chunk s of m chunks of the entry range [e0, e1): the m - 1 helper chunks are equal and the
// owner's last chunk (the latest columns, whose inputs arrive last) is half as long, so less of
// the row is left to walk after its last input.
__device__ __forceinline__ void slice_range(int e0, int e1, int s, int m, int &lo, int &hi) {
    const int chunk = (2 * (e1 - e0) + 2 * m - 2) / (2 * m - 1);
    lo = min(e1, e0 + s * chunk);
    hi = s == m - 1 ? e1 : min(e1, lo + chunk);
}

// One slice of a separated SpMV -> SpTRSV solve row (r_i computed before the partitions): as
// run_slice, with the slices splitting L's strict part (A's entries before the diagonal in
// shared storage) and the owner's right-hand side r_i waited for by value. Out of line so that
// the other kinds' slices keep their register budget.
template <typename T, int LPR, int VU>
__device__ __noinline__ bool run_slice_sep(const ExecArgs &a, int row, int s, int m, int slot, int gl,
                                           unsigned gmask) {
    const int kt = a.kt, S = LPR / kt, ls = gl / kt, cl = gl % kt, k = a.k;
    const bool owner = s == m - 1;
    T *parts = (T *)a.parts;
    T *z = (T *)a.y;
    const T *r = (const T *)a.rsep;
    bool ok = true;
    int lo, hi;
    const int *cols;
    const T *vals;
    T d = T(0);
    if (a.Lv == nullptr) {
        const int ra = __ldg(a.Mrp + row), dp = __ldg(a.a_diag + row);
        slice_range(ra, dp, s, m, lo, hi);
        cols = a.Mci;
        vals = (const T *)a.Mv;
        if (owner) d = load_diag<T>(a, vals, dp, row, gl);
    } else {
        const int rs = __ldg(a.Lrp + row), dg = __ldg(a.Lrp + row + 1) - 1;
        slice_range(rs, dg, s, m, lo, hi);
        cols = a.Lci;
        vals = (const T *)a.Lv;
        if (owner) d = load_diag<T>(a, vals, dg, row, gl);
    }
    for (int c0 = 0; c0 < k; c0 += kt) {
        const int c = c0 + cl;
        const bool act = c < k;
        T aw = row_dot<T, D_VALUE, false, VU>(cols, nullptr, vals, lo + ls, hi, S, z, k, c, act, nullptr, 0u, a.st,
                                               a.timeout_ns, row, ok);
        const T p = slice_sum<LPR>(aw, kt, gmask);
        if (!owner) {
            if (ls == 0 && act) put_value(parts + (size_t)(slot + s) * k + c, p);
            continue;
        }
        T help = T(0);
        if (m > 1) {
            T hs = T(0);
            if (act)
                for (int h0 = ls; h0 < m - 1 && ok; h0 += 4 * S) {
                    int j[4];
                    T xv[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int h = h0 + u * S;
                        j[u] = h < m - 1 ? (slot + h) * k + c : -1;
                    }
                    ok = wait_values<T, 4>(parts, j, xv, a.st, a.timeout_ns, row);
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        if (j[u] >= 0) hs += xv[u];
                }
            help = slice_sum<LPR>(hs, kt, gmask);
        }
        if (ls == 0 && act) {
            const T ri = poll_value(r + (size_t)row * k + c, a.st, a.timeout_ns, row, ok);
            put_value(z + (size_t)row * k + c, finish_row<T>(a, ri - (help + p), d));
        }
    }
    return group_ok<LPR>(ok, gmask);
}

// One slice of a long row split at execution time (whole team, value flags). The row's dot
// products are cut into m chunks of entries; slices 0 .. m-2 (the helpers, earlier in the
// queue) each add up their chunk and store the partial sums (one per right-hand-side column)
// to a.parts[(slot + s) * k + c], every value its own flag; slice m-1 (the owner, queued after
// its helpers) adds up the last chunk, whose inputs arrive last, gathers the helpers' partials
// (all lanes, several loads in flight) and finishes the row exactly as the item does (the
// partials summed in a fixed order). Several
// teams thus stream one long row as its inputs arrive. Kinds: SpTRSV rows (SpTRSV -> SpMV
// tag 0, SpTRSV alone), SpMV -> SpTRSV rows (A and L parts, or A's row in shared storage) and
// the transposed solve rows of the adjoints.
template <int MODE, typename T, int LPR, int VU, bool SEP = true>
__device__ bool run_slice(const ExecArgs &a, int tag, int row, int s, int m, int slot, int gl, unsigned gmask) {
    if constexpr (MODE == M_SPMV_TRSV && SEP)
        if (a.rsep) return run_slice_sep<T, LPR, VU>(a, row, s, m, slot, gl, gmask);
    const int kt = a.kt, S = LPR / kt, ls = gl / kt, cl = gl % kt, k = a.k;
    const bool owner = s == m - 1;
    T *parts = (T *)a.parts;
    bool ok = true;
    int lo, hi, lo2 = 0, hi2 = 0;
    const T *vals = nullptr, *vals2 = nullptr;
    const int *cols = nullptr, *cols2 = nullptr;
    const T *vec = nullptr;       // the vector the waited-for part reads
    const T *vec2 = nullptr;      // the vector of the part that waits for nothing
    T *out = nullptr;
    T d = T(0);
    int dp = -1;                  // shared storage: diagonal position of A's row
    const T *first = nullptr;     // owner: b, gz (added) or NULL
    T sign2 = T(1);               // sign of the part that waits for nothing in p
    if constexpr (MODE == M_TRSV || MODE == M_TRSV_SPMV) {
        const int rs = __ldg(a.Lrp + row), dg = __ldg(a.Lrp + row + 1) - 1;
        slice_range(rs, dg, s, m, lo, hi);
        cols = a.Lci;
        vals = (const T *)a.Lv;
        out = MODE == M_TRSV ? (T *)a.y : (T *)a.xs;
        vec = out;
        first = (const T *)a.b;
        if (owner) d = load_diag<T>(a, vals, dg, row, gl);
    } else if constexpr (MODE == M_SPMV_TRSV) {
        const int ra = __ldg(a.Mrp + row), re = __ldg(a.Mrp + row + 1);
        out = (T *)a.y;
        vec = out;
        vec2 = (const T *)a.xin;
        first = (const T *)a.b;
        if (a.Lv == nullptr) {
            dp = __ldg(a.a_diag + row);
            slice_range(ra, re, s, m, lo, hi);
            cols = a.Mci;
            vals = (const T *)a.Mv;
            if (owner) d = load_diag<T>(a, vals, dp, row, gl);
        } else {
            const int rs = __ldg(a.Lrp + row), dg = __ldg(a.Lrp + row + 1) - 1;
            slice_range(rs, dg, s, m, lo, hi);
            slice_range(ra, re, s, m, lo2, hi2);
            cols = a.Lci;
            vals = (const T *)a.Lv;
            cols2 = a.Mci;
            vals2 = (const T *)a.Mv;
            if (owner) d = load_diag<T>(a, vals, dg, row, gl);
        }
    } else if constexpr (MODE == M_ADJ_SPMV_TRSV || MODE == M_ADJ_TRSV_SPMV) {
        const int ls0 = __ldg(a.LTrp + row), le = __ldg(a.LTrp + row + 1);   // L^T row: L_jj first
        slice_range(ls0 + 1, le, s, m, lo, hi);
        cols = a.LTci;
        vals = (const T *)a.LTv;
        out = (T *)a.gb;
        vec = out;
        if (owner) d = load_diag<T>(a, vals, ls0, row, gl);
        if constexpr (MODE == M_ADJ_SPMV_TRSV) {
            first = (const T *)a.gy;
        } else {
            const int ms = __ldg(a.MTrp + row), me = __ldg(a.MTrp + row + 1);
            slice_range(ms, me, s, m, lo2, hi2);
            cols2 = a.MTci;
            vals2 = (const T *)a.MTv;
            vec2 = (const T *)a.gy;
            sign2 = T(-1);   // lam_j = (u_j - sum L^T lam) / L_jj with u = M^T gy: p = sum L^T lam - u
        }
    }
    (void)tag;
    for (int c0 = 0; c0 < k; c0 += kt) {
        const int c = c0 + cl;
        const bool act = c < k;
        // the owner's right-hand side, loaded before any wait
        const T f = (owner && ls == 0 && act && first) ? __ldg(first + (size_t)row * k + c) : T(0);
        // this slice's share p of the row's total, which the owner subtracts from `first`:
        // p = (waited-for part) + sign2 * (part that waits for nothing)
        T p;
        if (dp >= 0) {
            T ax, az;
            gs_row_dot<T, VU>(cols, vals, lo + ls, dp, hi, S, vec2, out, k, c, act, a.st, a.timeout_ns, row, ok, ax,
                              az);
            p = slice_sum<LPR>(ax, kt, gmask) + slice_sum<LPR>(az, kt, gmask);
        } else {
            // the part that waits for nothing first, so that only the waited-for part follows
            // the last input
            T pf = T(0);
            if (cols2) {
                T af = row_dot<T, D_NONE, false>(cols2, nullptr, vals2, lo2 + ls, hi2, S, vec2, k, c, act, nullptr, 0u,
                                                 a.st, a.timeout_ns, row, ok);
                pf = sign2 * slice_sum<LPR>(af, kt, gmask);
            }
            T aw = row_dot<T, D_VALUE, false, VU>(cols, nullptr, vals, lo + ls, hi, S, vec, k, c, act, nullptr, 0u, a.st,
                                                   a.timeout_ns, row, ok);
            p = slice_sum<LPR>(aw, kt, gmask) + pf;
        }
        if (!owner) {
            if (ls == 0 && act) put_value(parts + (size_t)(slot + s) * k + c, p);
            continue;
        }
        // the owner adds up its helpers' partial sums: the lane slices take every S-th helper,
        // four loads in flight, then one reduction over the slices (a fixed order)
        T help = T(0);
        if (m > 1) {
            T hs = T(0);
            if (act)
                for (int h0 = ls; h0 < m - 1 && ok; h0 += 4 * S) {
                    int j[4];
                    T xv[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int h = h0 + u * S;
                        j[u] = h < m - 1 ? (slot + h) * k + c : -1;
                    }
                    ok = wait_values<T, 4>(parts, j, xv, a.st, a.timeout_ns, row);
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        if (j[u] >= 0) hs += xv[u];
                }
            help = slice_sum<LPR>(hs, kt, gmask);
        }
        if (ls == 0 && act) put_value(out + (size_t)row * k + c, finish_row<T>(a, f - (help + p), d));
    }
    return group_ok<LPR>(ok, gmask);
}

// Modes with value-flag launches (k = 1; IC0 modes for any k when the pair lists exist).
constexpr bool mode_has_vf(int m) {
    return m == M_TRSV_SPMV || m == M_TRSV || m == M_SPMV_TRSV || m == M_ADJ_TRSV_SPMV || m == M_ADJ_SPMV_TRSV ||
           m == M_IC0_TRSV || m == M_IC0 || m == M_TRSV_TRSV || m == M_ILU0_TRSV;
}

// SEP: the kernel carries the separated SpMV -> SpTRSV rows (not the three-block kernels,
// whose register budget has no room for them).
template <int MODE, typename T, int LPR, bool VF, int VU, bool SEP = true>
__device__ __forceinline__ bool run_item(const ExecArgs &a, int tag, int row, unsigned epoch, int gl, int gbase,
                                         unsigned gmask) {
    if constexpr (MODE == M_TRSV_SPMV) {
        if (tag == 0) return item_trsv<T, LPR, VF, VU>(a, row, epoch, gl, gmask, (T *)a.xs);
        return item_spmv_dep<T, LPR, VF, VU>(a, row, epoch, gl, gmask, (const T *)a.xs);
    } else if constexpr (MODE == M_TRSV) {
        return item_trsv<T, LPR, VF, VU>(a, row, epoch, gl, gmask, (T *)a.y);
    } else if constexpr (MODE == M_SPMV_TRSV) {
        return item_spmv_trsv<T, LPR, VF, VU, SEP>(a, row, epoch, gl, gmask);
    } else if constexpr (MODE == M_IC0_TRSV) {
        return item_ic0<T, LPR, true, VF>(a, row, epoch, gl, gmask);
    } else if constexpr (MODE == M_IC0) {
        return item_ic0<T, LPR, false, VF>(a, row, epoch, gl, gmask);
    } else if constexpr (MODE == M_ADJ_TRSV_SPMV) {
        return item_adj_trsv_spmv<T, LPR, VF, VU>(a, row, epoch, gl, gbase, gmask);
    } else if constexpr (MODE == M_TRSV_TRSV) {
        return item_trsv_trsv<T, LPR, VF, VU>(a, row, epoch, gl, gmask);
    } else if constexpr (MODE == M_ILU0_TRSV) {
        if constexpr (VF && LPR == 32) return item_ilu0<T>(a, row, gl);
        else return false;   // not instantiated: ILU0 launches are whole-warp value-flag launches
    } else {
        if (tag == 0) return item_adj_lam<T, LPR, VF, VU>(a, row, epoch, gl, gbase, gmask);
        if (!a.gx) return true;    // gradient of x_in not requested
        return item_adj_gx<T, LPR, VF, VU>(a, row, epoch, gl, gmask);
    }
}

// Resident blocks per SM the compiler budgets registers for: the default kernels keep all the
// registers they want (latency-bound chains prefer fewer, faster threads); the occupancy
// variants are held to three blocks of 256 threads (85 registers: value-flag kernels with up
// to four lanes per row) or four (64 registers: IC0 kernels with whole-warp rows, which fit
// there without spilling), for schedules bound by the number of rows in flight.
constexpr int kMinBlocksDefault = 1;
constexpr int kMinBlocksWide = 2;   // value-flag kernels with 16 or 32 lanes per row: 128 registers
constexpr int kMinBlocksHigh = 3;
constexpr int kMinBlocksIc0 = 4;

// Next ticket of a team (its first lane draws it; the caller broadcasts it when needed, so
// the atomic's latency overlaps the current partition's work).
__device__ __forceinline__ int draw_ticket(const ExecArgs &a, int tl, int nunits) {
    if (tl != 0) return 0;
    return ld_relaxed_u32(&a.st->abort) ? nunits : (int)atomicAdd(&a.st->ticket, 1u);
}

// A warp is split into 32/TEAM teams of TEAM lanes; a team runs one partition at a time
// with TEAM/LPR groups of LPR lanes (one item per group per round). Teams are the units of
// the partition assignment, so small partitions do not leave lanes of a warp idle.
template <int MODE, typename T, int LPR, bool VF, int TEAM, int MINB>
__global__ void __launch_bounds__(kExecThreads, MINB) k_exec(const ExecArgs a) {
    static_assert(LPR <= TEAM && TEAM <= 32, "groups fit in a team");
    constexpr int G = TEAM / LPR;
    constexpr int NT = 32 / TEAM;
    const int lane = threadIdx.x & 31;
    const int tl = lane % TEAM, tbase = lane - tl;
    const unsigned tmask = (TEAM == 32) ? 0xffffffffu : (((1u << TEAM) - 1u) << tbase);
    const int grp = tl / LPR, gl = tl % LPR, gbase = tbase + grp * LPR;
    const unsigned gmask = (LPR == 32) ? 0xffffffffu : (((1u << LPR) - 1u) << gbase);
    const unsigned epoch = ld_relaxed_u32(&a.st->epoch);
    const int nteams = gridDim.x * (blockDim.x >> 5) * NT;
    const int team = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * NT + lane / TEAM;
    bool ok = true;
    if constexpr (VF && MODE == M_SPMV_TRSV && MINB < 3) {
        if (a.rsep) {
            // separated packing (§3.2.3, the SpMV vertices in the first wavefront): every group
            // computes r_i = b_i - A_i x_in for its share of the rows, in increasing row order,
            // and publishes it by value; nothing here waits
            const int kt = a.kt, S = LPR / kt, s = gl / kt, cl = gl % kt, k = a.k;
            const T *Av = (const T *)a.Mv, *b = (const T *)a.b;
            T *r = (T *)a.rsep;
            const int ngroups = nteams * G;
            for (int i = team * G + grp; i < a.n; i += ngroups) {
                const int ra = __ldg(a.Mrp + i), re = __ldg(a.Mrp + i + 1);
                for (int c0 = 0; c0 < k; c0 += kt) {
                    const int c = c0 + cl;
                    const bool act = c < k;
                    T ax = row_dot<T, D_NONE, false>(a.Mci, nullptr, Av, ra + s, re, S, (const T *)a.xin, k, c, act,
                                                     nullptr, 0u, a.st, a.timeout_ns, i, ok);
                    ax = slice_sum<LPR>(ax, kt, gmask);
                    if (s == 0 && act) put_value(r + (size_t)i * k + c, __ldg(b + (size_t)i * k + c) - ax);
                }
            }
        }
    }
    // A team holds its current partition (and with tickets the ticket of its next one);
    // every team runs its partitions in increasing order (within its class), so the smallest
    // unfinished partition is always being run by a team whose dependences are all finished.
    // With two classes (separated schedules) teams [0, teams0) run the class-0 list and the
    // others the class-1 list, each round robin in increasing order; second-kernel rows then
    // never hold up a team that the dependence chain is waiting for.
    // With split long rows the units are the entries of a.xlist (partition, slice, slices,
    // partial slot), in queue order; otherwise the partitions themselves.
    const int nunits = a.xlist ? a.nx : a.n_parts;
    int idx = team, stride = nteams, base = 0, end = nunits;
    if (!a.dynamic && a.plist) {
        if (team < a.teams0) {
            stride = a.teams0;
            end = a.n_parts0;
        } else {
            idx = team - a.teams0;
            stride = nteams - a.teams0;
            base = a.n_parts0;
            end = a.n_parts - a.n_parts0;
        }
    }
    auto unit_at = [&](int i) { return i < end ? (a.plist ? __ldg(a.plist + base + i) : base + i) : nunits; };
    int u = a.dynamic ? __shfl_sync(tmask, draw_ticket(a, tl, nunits), tbase) : unit_at(idx);
    while (u < nunits) {
        const int un_first = a.dynamic ? draw_ticket(a, tl, nunits) : 0;
        int p = u;
        int4 sl = make_int4(u, 0, 1, 0);
        if (a.xlist) {
            sl = __ldg(a.xlist + u);
            p = sl.x;
        }
        const int q0 = __ldg(a.part_ptr + p), q1 = __ldg(a.part_ptr + p + 1);
        if constexpr (VF && (MODE == M_TRSV || MODE == M_TRSV_SPMV || MODE == M_SPMV_TRSV || MODE == M_ADJ_SPMV_TRSV ||
                             MODE == M_ADJ_TRSV_SPMV)) {
            if (sl.z > 1) {
                // one slice of a long row split over several teams
                const unsigned o = (unsigned)__ldg(a.order + q0);
                if (ok)
                    ok = run_slice<MODE, T, TEAM, value_unroll(LPR), (MINB < 3)>(a, (int)(o >> 31), (int)(o & 0x7fffffffu), sl.y,
                                                                     sl.z, sl.w, tl, tmask);
                if (!__all_sync(tmask, ok)) break;
                if (a.dynamic) u = __shfl_sync(tmask, un_first, tbase);
                else {
                    idx += stride;
                    u = ld_relaxed_u32(&a.st->abort) ? nunits : unit_at(idx);
                }
                continue;
            }
        }
        if (LPR < TEAM && a.part_wide[p]) {
            // a long row: the whole team runs it (the cut gives it a partition of its own)
            const unsigned o = (unsigned)__ldg(a.order + q0);
            if (ok)
                ok = run_item<MODE, T, TEAM, VF, value_unroll(LPR), (MINB < 3)>(a, (int)(o >> 31), (int)(o & 0x7fffffffu), epoch, tl,
                                                                    tbase, tmask);
        } else {
            for (int q = q0 + grp; q < q1 && ok; q += G) {
                const unsigned o = (unsigned)__ldg(a.order + q);
                ok = run_item<MODE, T, LPR, VF, value_unroll(LPR), (MINB < 3)>(a, (int)(o >> 31), (int)(o & 0x7fffffffu), epoch, gl,
                                                                   gbase, gmask);
            }
        }
        if (!__all_sync(tmask, ok)) break;
        if (a.dynamic) u = __shfl_sync(tmask, un_first, tbase);
        else {
            idx += stride;
            u = ld_relaxed_u32(&a.st->abort) ? nunits : unit_at(idx);
        }
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

template <int MODE, bool VF, int TEAM>
const void *kernel_for_team(int dtype, int lpr, int minb) {
    constexpr int D = kMinBlocksDefault;
    if constexpr ((MODE == M_IC0_TRSV || MODE == M_IC0) && TEAM == 32) {
        if (minb >= kMinBlocksHigh && lpr == 32) {
            constexpr int H = kMinBlocksIc0;
            return dtype == 0 ? (const void *)k_exec<MODE, double, 32, VF, 32, H>
                              : (const void *)k_exec<MODE, float, 32, VF, 32, H>;
        }
    }
    if constexpr (VF && TEAM == 32) {
        if (minb == kMinBlocksWide && (lpr == 16 || lpr == 32)) {
            constexpr int H = kMinBlocksWide;
            if (dtype == 0) return lpr == 16 ? (const void *)k_exec<MODE, double, 16, VF, 32, H>
                                             : (const void *)k_exec<MODE, double, 32, VF, 32, H>;
            return lpr == 16 ? (const void *)k_exec<MODE, float, 16, VF, 32, H> : (const void *)k_exec<MODE, float, 32, VF, 32, H>;
        }
        if (minb >= kMinBlocksHigh) {
            constexpr int H = kMinBlocksHigh;
            if (dtype == 0) {
                if (lpr == 1) return (const void *)k_exec<MODE, double, 1, VF, 32, H>;
                if (lpr == 2) return (const void *)k_exec<MODE, double, 2, VF, 32, H>;
                if (lpr == 4) return (const void *)k_exec<MODE, double, 4, VF, 32, H>;
            } else {
                if (lpr == 1) return (const void *)k_exec<MODE, float, 1, VF, 32, H>;
                if (lpr == 2) return (const void *)k_exec<MODE, float, 2, VF, 32, H>;
                if (lpr == 4) return (const void *)k_exec<MODE, float, 4, VF, 32, H>;
            }
        }
    }
    if (dtype == 0) {
        switch (lpr) {
            case 1: return (const void *)k_exec<MODE, double, 1, VF, TEAM, D>;
            case 2: return (const void *)k_exec<MODE, double, 2, VF, TEAM, D>;
            case 4: return (const void *)k_exec<MODE, double, 4, VF, TEAM, D>;
            case 8: return (const void *)k_exec<MODE, double, 8, VF, TEAM, D>;
        }
        if constexpr (TEAM == 32) {
            if (lpr == 16) return (const void *)k_exec<MODE, double, 16, VF, 32, D>;
            if (lpr == 32) return (const void *)k_exec<MODE, double, 32, VF, 32, D>;
        }
    } else {
        switch (lpr) {
            case 1: return (const void *)k_exec<MODE, float, 1, VF, TEAM, D>;
            case 2: return (const void *)k_exec<MODE, float, 2, VF, TEAM, D>;
            case 4: return (const void *)k_exec<MODE, float, 4, VF, TEAM, D>;
            case 8: return (const void *)k_exec<MODE, float, 8, VF, TEAM, D>;
        }
        if constexpr (TEAM == 32) {
            if (lpr == 16) return (const void *)k_exec<MODE, float, 16, VF, 32, D>;
            if (lpr == 32) return (const void *)k_exec<MODE, float, 32, VF, 32, D>;
        }
    }
    return nullptr;
}

// Teams of 8 lanes serve lanes-per-row up to 8; wider rows use whole-warp teams.
template <int MODE, bool VF>
const void *kernel_for(int dtype, int lpr, int team, int minb) {
    if (team == 8 && lpr <= 8) return kernel_for_team<MODE, VF, 8>(dtype, lpr, minb);
    return kernel_for_team<MODE, VF, 32>(dtype, lpr, minb);
}

template <int MODE>
const void *kernel_for_mode(int dtype, int lpr, bool vf, int team, int minb) {
    if constexpr (mode_has_vf(MODE)) {
        if (vf) return kernel_for<MODE, true>(dtype, lpr, team, minb);
    }
    return kernel_for<MODE, false>(dtype, lpr, team, minb);
}

// Launches k_exec for a runtime (dtype, lanes-per-row, value flags, team lanes, occupancy).
template <int MODE>
cudaError_t launch_mode(int dtype, int lpr, bool vf, int team, int minb, int blocks, cudaStream_t s,
                        const ExecArgs &a) {
    const void *f = kernel_for_mode<MODE>(dtype, lpr, vf, team, minb);
    if (!f) return cudaErrorInvalidValue;
    void *args[] = {(void *)&a};
    if (a.dynamic) return cudaLaunchKernel(f, dim3(blocks), dim3(kExecThreads), args, 0, s);
    return cudaLaunchCooperativeKernel(f, dim3(blocks), dim3(kExecThreads), args, 0, s);
}

template <int MODE>
int blocks_per_sm_mode(int dtype, int lpr, bool vf, int team, int minb) {
    int nb = 0;
    const void *f = kernel_for_mode<MODE>(dtype, lpr, vf, team, minb);
    if (!f || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, kExecThreads, 0) != cudaSuccess) return 1;
    return nb > 0 ? nb : 1;
}

}  // namespace sf
