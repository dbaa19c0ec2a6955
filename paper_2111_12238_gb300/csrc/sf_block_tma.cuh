// Row-block executor with packed records and bulk (TMA) staging (one right-hand side,
// exec_mode 4).
//
// Same schedule as the other row-block executors (blocks of B consecutive rows, one CTA per
// block at a time, level segments, the block's values in shared memory). What differs is how
// a segment's pattern data reaches the SM. The schedule keeps, in position order (the
// row-block order), a packed copy of every position's record: order entry, entry range and
// the first U column indices, as structures of arrays with a stride of nvp (the position
// count rounded up to a multiple of 4). A pre-pass of every call gathers the matching values
// and (c_i, 1 / L_ii) into the same layout. The records of a chunk (up to NC consecutive
// positions of one segment) are then a handful of contiguous byte ranges, so one producer
// lane moves a chunk into a shared-memory stage with 2 + 2U bulk copies (cp.async.bulk,
// completing on the stage's mbarrier) instead of per-entry gathers through the load/store
// unit, which the consumers' shared-memory reads would queue behind.
//
// Protocol per chunk c, stage k = c mod K:
//   producer lane: waits EMPTY[k] (named barrier: the consumers are done with chunk c - K),
//     arms FULL[k] (mbarrier) with the chunk's byte count and issues the bulk copies;
//   consumers: cross a consumers-only barrier (every consumer is done with chunk c - 1: the
//     level barrier that makes shared values visible), wait for FULL[k]'s phase, run their
//     position, arrive on EMPTY[k].
// Chunk ranges are widened to multiples of 4 positions so that every copy starts on a
// 16-byte boundary and has a size that is a multiple of 16 bytes; a consumer finds its
// position at offset q - (q0 & ~3). Every wait is bounded; a failure sets a shared flag after
// which both roles walk the rest of the sequence without work. Consumers wait for every
// stage's phase even then (the producer arms it with no copies), so they never run ahead of
// the producer on the EMPTY barriers; the producer also waits (bounded) for a stage's previous
// copies before re-arming it and for all armed stages before the CTA exits, so no bulk copy is
// ever in flight into a stage being re-armed or into the shared memory of an exited CTA.
#pragma once

#include "sf_block_ws.cuh"

namespace sf {

constexpr int kTmaStages = 4;
constexpr int kTmaU = 8;
constexpr int kTmaMaxConsumers = 256;
constexpr int kTmaProducers = 32;          // one warp; its first lane issues the copies

// Packed pattern part of a record: order entry, first entry, end of the entry range.
struct __align__(16) PackMeta {
    int rt, rs, re, pad;
};

template <typename T>
__host__ __device__ constexpr size_t tma_slot_bytes() {
    return sizeof(PackMeta) + kTmaU * (sizeof(int) + sizeof(T)) + 2 * sizeof(T);
}
// Slots per stage: a chunk of nc positions widened to multiples of 4 on both ends.
__host__ __device__ constexpr int tma_slots(int nc) { return nc + 8; }
template <typename T>
__host__ __device__ constexpr size_t tma_stage_bytes(int nc) { return (size_t)tma_slots(nc) * tma_slot_bytes<T>(); }

template <typename T>
struct TmaStage {
    PackMeta *meta;
    int *j;                         // j[u * S + slot]
    T *v;                           // v[u * S + slot]
    typename Pair2<T>::type *cr;    // (c_i, 1 / L_ii)
};

template <typename T>
__device__ __forceinline__ TmaStage<T> tma_stage(unsigned char *base, int S) {
    using V2 = typename Pair2<T>::type;
    TmaStage<T> st;
    st.meta = reinterpret_cast<PackMeta *>(base);
    st.cr = reinterpret_cast<V2 *>(base + (size_t)S * sizeof(PackMeta));
    st.v = reinterpret_cast<T *>(base + (size_t)S * (sizeof(PackMeta) + sizeof(V2)));
    st.j = reinterpret_cast<int *>(base + (size_t)S * (sizeof(PackMeta) + sizeof(V2) + kTmaU * sizeof(T)));
    return st;
}

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0u;
}
// Bulk copy global -> shared of `bytes` (multiple of 16, both addresses 16-byte aligned),
// completing on `bar`.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// Bounded wait for an mbarrier phase. false: the limit ran out (recorded as a timeout).
static __device__ __noinline__ bool mbar_wait_bounded(unsigned long long *bar, unsigned parity, ExecState *st,
                                               unsigned long long tmo, int row) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (unsigned it = 1;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 63u) == 0u && global_ns() - t0 > tmo) {
            record_error(st, SF_ERR_TIMEOUT, row);
            st_relaxed_u32(&st->abort, 1u);
            return false;
        }
    }
}

// Slow path of a staged row whose inputs are not all published yet: the same sum, each
// input waited for in turn (bounded).
template <typename T>
__device__ __noinline__ TailSum<T> tma_dot_slow(const int *j, const T *v, int S, int cnt, const T *vec, const T *xs,
                                                 int row0, int rows, ExecState *st, unsigned long long tmo, int row) {
    T acc0 = T(0), acc1 = T(0);
    bool ok = true;
    for (int u = 0; u < cnt && ok; ++u) {
        const WaitOne<T> w1 = ws_wait_one<T>(vec, xs, row0, rows, j[u * S], st, tmo, row);
        ok = w1.ok;
        const T p = v[u * S] * w1.x;
        if (u & 1) acc1 += p;
        else acc0 += p;
    }
    return TailSum<T>{acc0 + acc1, ok};
}

template <int MODE, typename T>
__global__ void __launch_bounds__(kTmaMaxConsumers + kTmaProducers, 1) k_block_tma(const ExecArgs a) {
    using V2 = typename Pair2<T>::type;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    __shared__ unsigned s_abort;
    __shared__ __align__(8) unsigned long long s_full[kTmaStages];
    const int NC = blockDim.x - kTmaProducers;
    const int S = tma_slots(NC);
    const int ALL = blockDim.x;
    const int B = a.block_rows, nb = a.n_blocks;
    const int rows_max = min(B, a.n);
    const int nvp = a.pack_stride;
    T *xs = reinterpret_cast<T *>(sm_raw);
    unsigned char *stage0 = sm_raw + (((size_t)rows_max * sizeof(T) + 15) & ~(size_t)15);
    const size_t sbytes = tma_stage_bytes<T>(NC);
    const unsigned epoch = ld_relaxed_u32(&a.st->epoch);
    T *vec = block_vec<MODE, T>(a);
    if (threadIdx.x == 0) {
        s_abort = 0u;
        for (int k = 0; k < kTmaStages; ++k) mbar_init(s_full + k, 1u);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    constexpr int EMPTY0 = 1, LVL = 1 + kTmaStages;
    const bool producer = (int)threadIdx.x >= NC;

    if (producer) {
        // ---------------------------------------------------------------- producer warp
        const int lane = threadIdx.x - NC;
        WsChunks ch;
        int c = 0;
        for (bool more = ch.first(a, NC); more; more = ch.next(a, NC), ++c) {
            const int k = c % kTmaStages;
            if (c >= kTmaStages) named_sync(EMPTY0 + k, ALL);
            if (lane == 0) {
                const int qa = ch.q0 & ~3, qe = (ch.q1 + 3) & ~3;
                const unsigned m = (unsigned)(qe - qa);
                const TmaStage<T> st = tma_stage<T>(stage0 + (size_t)k * sbytes, S);
                // a stage is re-armed only once its previous copies have landed: consumers that
                // skipped a chunk after a failure did not wait for them
                bool work = true;
                if (c >= kTmaStages && !mbar_wait_bounded(s_full + k, (unsigned)((c / kTmaStages - 1) & 1), a.st,
                                                         a.timeout_ns, -1))
                    work = false;
                work = work && ld_shared_volatile(&s_abort) == 0u;
                const unsigned bytes = work ? m * (unsigned)tma_slot_bytes<T>() : 0u;
                mbar_arrive_expect_tx(s_full + k, bytes);
                if (work) {
                    bulk_g2s(st.meta, (const PackMeta *)a.pack_meta + qa, m * (unsigned)sizeof(PackMeta), s_full + k);
                    bulk_g2s(st.cr, (const V2 *)a.pack_aux + qa, m * (unsigned)sizeof(V2), s_full + k);
#pragma unroll
                    for (int u = 0; u < kTmaU; ++u) {
                        bulk_g2s(st.v + u * S, (const T *)a.pack_vals + (size_t)u * nvp + qa, m * (unsigned)sizeof(T),
                                 s_full + k);
                        bulk_g2s(st.j + u * S, a.pack_cols + (size_t)u * nvp + qa, m * 4u, s_full + k);
                    }
                }
                // another CTA's failure is seen through the global word, read every 16 chunks
                if ((c & 15) == 15 && ld_relaxed_u32(&a.st->abort)) s_abort = 1u;
            }
            __syncwarp();
        }
        // no copy may be in flight when the CTA exits
        if (lane == 0)
            for (int i = max(0, c - kTmaStages); i < c; ++i)
                mbar_wait_bounded(s_full + i % kTmaStages, (unsigned)((i / kTmaStages) & 1), a.st, a.timeout_ns, -1);
        __syncwarp();
        for (int i = max(0, c - kTmaStages); i < c; ++i) named_sync(EMPTY0 + i % kTmaStages, ALL);
    } else {
        // ---------------------------------------------------------------- consumers
        const int ct = threadIdx.x;
        WsChunks ch;
        int c = 0;
        int row0 = 0, rows = 0;
        for (bool more = ch.first(a, NC); more; more = ch.next(a, NC), ++c) {
            named_sync(LVL, NC);                     // every consumer is done with chunk c - 1
            if (ch.new_block) {
                row0 = a.block_rev ? (nb - 1 - ch.b) * B : ch.b * B;
                rows = min(B, a.n - row0);
                for (int i = ct; i < rows; i += NC) xs[i] = unset_value<T>();
                named_sync(LVL, NC);
            }
            const int k = c % kTmaStages;
            const TmaStage<T> st = tma_stage<T>(stage0 + (size_t)k * sbytes, S);
            // always wait for the stage, after a failure too (the producer then arms it with
            // no copies): a consumer that ran ahead of the producer would arrive on EMPTY for a
            // later chunk before the producer's sync of the earlier one and merge the phases
            bool ok = mbar_wait_bounded(s_full + k, (unsigned)((c / kTmaStages) & 1), a.st, a.timeout_ns, -1);
            ok = ok && ld_shared_volatile(&s_abort) == 0u;
            const int q = ch.q0 + ct;
            if (ok && q < ch.q1) {
                const int slot = q - (ch.q0 & ~3);
                const PackMeta md = st.meta[slot];
                const int row = md.rt & 0x7fffffff, tag = (int)((unsigned)md.rt >> 31);
                bool skip = false;
                if constexpr (MODE == M_ADJ_SPMV_TRSV) skip = tag == 1 && !a.gx;
                if (!skip) {
                    const int len = md.re - md.rs;
                    const int cnt = min(len, kTmaU);
                    // fast path: all staged entries at once, no call on the way; an input still
                    // showing the reset pattern sends the row to the bounded slow path
                    T acc0 = T(0), acc1 = T(0);
                    bool unset = false;
#pragma unroll
                    for (int u = 0; u < kTmaU; ++u) {
                        if (u < cnt) {
                            const int j = st.j[u * S + slot];
                            const unsigned lj = (unsigned)(j - row0);
                            // rows of the block were published before the level barrier:
                            // plain shared loads, which the compiler may batch
                            const T x = lj < (unsigned)rows ? xs[lj] : ld_relaxed_val(vec + j);
                            unset |= is_unset(x);
                            const T p = st.v[u * S + slot] * x;
                            if (u & 1) acc1 += p;
                            else acc0 += p;
                        }
                    }
                    T acc = acc0 + acc1;
                    if (unset) {
                        const TailSum<T> r = tma_dot_slow<T>(st.j + slot, st.v + slot, S, cnt, vec, xs, row0, rows,
                                                              a.st, a.timeout_ns, row);
                        acc = r.acc;
                        ok = ok && r.ok;
                    }
                    if (len > kTmaU && ok) {
                        const int *ci;
                        const T *vals;
                        block_entries<MODE, T>(a, tag, ci, vals);
                        const TailSum<T> ts = block_dot_tail<T>(ci, vals, md.rs + kTmaU, md.re, 1, vec, xs, row0, rows,
                                                                a.st, a.timeout_ns, row, acc);
                        acc = ts.acc;
                        ok = ts.ok;
                    }
                    if (ok) {
                        if (tag == 0) {
                            const V2 cr = st.cr[slot];
                            T v = (cr.x - acc) * cr.y;
                            if (is_unset(v)) v = canonical_nan(v);
                            const unsigned lr = (unsigned)(row - row0);
                            if (lr < (unsigned)rows) *(volatile T *)(xs + lr) = v;
                            st_relaxed_val(vec + row, v);
                        } else if constexpr (MODE == M_TRSV_SPMV) {
                            ((T *)a.y)[row] = acc;
                        } else if constexpr (MODE == M_ADJ_SPMV_TRSV) {
                            ((T *)a.gx)[row] = -acc;
                        }
                    }
                }
            }
            if (!ok) s_abort = 1u;
            __syncwarp();
            named_arrive(EMPTY0 + k, ALL);
        }
    }
    __syncthreads();
    if ((threadIdx.x & 31) == 0) {
        const unsigned total = gridDim.x * (blockDim.x >> 5);
        if (atom_add_acq_rel_u32(&a.st->done, 1u) == total - 1u) {
            st_relaxed_u32(&a.st->ticket, 0u);
            st_relaxed_u32(&a.st->done, 0u);
            st_relaxed_u32(&a.st->abort, 0u);
            st_release_u32(&a.st->epoch, epoch + 1u);
        }
    }
}

// Pre-pass of every exec_mode 4 call (after k_block_prep): values and (c_i, 1 / L_ii) of every
// position into the packed layout; the pattern part was packed at inspection.
template <int MODE, typename T>
__global__ void __launch_bounds__(256) k_pack_vals(const ExecArgs a) {
    using V2 = typename Pair2<T>::type;
    const int nvp = a.pack_stride;
    const PackMeta *meta = (const PackMeta *)a.pack_meta;
    T *pv = (T *)a.pack_vals;
    V2 *pa = (V2 *)a.pack_aux;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < nvp; t += (long long)gridDim.x * blockDim.x) {
        const int q = (int)t;
        const PackMeta md = meta[q];
        V2 cr;
        cr.x = T(0);
        cr.y = T(0);
        int cnt = 0;
        const T *vals = nullptr;
        if (md.rt != -1) {
            const int tag = (int)((unsigned)md.rt >> 31), row = md.rt & 0x7fffffff;
            const int *ci;
            block_entries<MODE, T>(a, tag, ci, vals);
            cnt = min(md.re - md.rs, kTmaU);
            if (tag == 0) cr = ((const V2 *)a.aux)[row];
        }
#pragma unroll
        for (int u = 0; u < kTmaU; ++u) pv[(size_t)u * nvp + q] = u < cnt ? __ldg(vals + md.rs + u) : T(0);
        pa[q] = cr;
    }
}

}  // namespace sf
