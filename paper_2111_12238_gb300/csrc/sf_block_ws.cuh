// Warp-specialised row-block executor (one right-hand side, exec_mode 3).
//
// Same schedule as k_block_exec (blocks of B consecutive rows, one CTA per block at a time,
// level segments inside a block, the block's values in shared memory), but the work of a
// level step is split between two warp roles so that the step's dependent chain holds only
// the arithmetic:
//  - producer warps walk the CTA's chunks (a chunk is up to NC positions of one segment) and
//    fill a ring of K shared-memory stages with each position's record: order entry, entry
//    count, the first U column indices and values, the row's independent part and 1 / L_ii
//    from the pre-pass, and the range of entries beyond U. Every global read is a cp.async
//    (no registers held, several chunks in flight); the order entries and entry ranges the
//    records are built from are themselves copied D chunks ahead into a small ring;
//  - consumer warps (NC threads, one position each) take a stage, gather the inputs (shared
//    slots for rows of the block, relaxed global loads for rows of earlier blocks), finish
//    the row and publish it.
// Hand-off uses named barriers: FULL[k] (producers arrive once stage k holds its chunk,
// consumers sync before reading it) and EMPTY[k] (consumers arrive after the chunk, producers
// sync before refilling). All consumers arrive at FULL of chunk c + 1 only after finishing
// chunk c, so that barrier is also the level barrier that makes shared values visible.
// Producers publish chunk c at the start of their iteration c + D, once its copies have
// landed (D = K - 1 chunks of copies in flight), before they wait for a free stage or touch
// global memory again; at the end they publish the rest and consume the outstanding EMPTY
// arrivals, so every barrier phase is matched.
//
// Waits on values are bounded (timeout_ns); a failure sets a shared flag after which both
// roles keep walking the barrier sequence without work, so the CTA always terminates.
#pragma once

#include "sf_block.cuh"

namespace sf {

#ifndef SF_WS_STAGES
#define SF_WS_STAGES 4
#endif
#ifndef SF_WS_AHEAD
#define SF_WS_AHEAD 3
#endif
// K stages; D <= K - 1 chunks of copies in flight before a chunk is published. A producer
// refills stage k only after chunk c - K is consumed while publishing chunk c - D, so K - D - 1
// chunks of slack separate the two roles. Named barrier ids 1 .. 2K + 1 must stay below 16.
constexpr int kWsStages = SF_WS_STAGES;   // K
constexpr int kWsAhead = SF_WS_AHEAD;     // D
static_assert(kWsAhead >= 1 && kWsAhead < kWsStages && 2 * kWsStages + 1 < 16, "stage ring");
constexpr int kWsProducers = 512;       // producer threads (16 warps), kWsProducers / NC per record
constexpr int kWsU = 8;                 // entries per record
constexpr int kWsMaxConsumers = 256;

__device__ __forceinline__ void named_sync(int id, int count) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void named_arrive(int id, int count) {
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((unsigned)__cvta_generic_to_shared(smem)),
                 "l"(gmem)
                 : "memory");
}
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((unsigned)__cvta_generic_to_shared(smem)),
                 "l"(gmem)
                 : "memory");
}
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(smem)),
                 "l"(gmem)
                 : "memory");
}
template <typename T>
__device__ __forceinline__ void cp_async_val(T *smem, const T *gmem) {
    if constexpr (sizeof(T) == 8) cp_async8(smem, gmem);
    else cp_async4(smem, gmem);
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// One stage of the ring, structure of arrays over the NC consumer slots.
template <typename T>
struct WsStage {
    typename Pair2<T>::type *cr;   // (c_i, 1 / L_ii) of first-kernel rows
    T *v;                          // v[u * NC + t]
    int *j;                        // j[u * NC + t]
    int *rt;                       // order entry (row | kernel << 31)
    int *cnt;                      // entries in the record, -1: empty slot
    int *tail;                     // first entry beyond the record, -1: none
    int *end;                      // end of the row's entry range
};

template <typename T>
__host__ __device__ constexpr size_t ws_stage_bytes(int nc) {
    return (size_t)nc * (2 * sizeof(T) + kWsU * (sizeof(T) + sizeof(int)) + 4 * sizeof(int));
}

// Ring of order entries and entry ranges, D + 1 chunks deep, filled D chunks ahead.
// Every producer thread keeps its own copy of its record's order entry and entry range.
__host__ __device__ constexpr size_t ws_desc_bytes(int nc) { return (size_t)(kWsAhead + 1) * kWsProducers * 12; }

template <typename T>
__device__ __forceinline__ WsStage<T> ws_stage(unsigned char *base, int nc) {
    using V2 = typename Pair2<T>::type;
    WsStage<T> s;
    s.cr = reinterpret_cast<V2 *>(base);
    s.v = reinterpret_cast<T *>(base + (size_t)nc * sizeof(V2));
    s.j = reinterpret_cast<int *>(base + (size_t)nc * (sizeof(V2) + kWsU * sizeof(T)));
    s.rt = s.j + kWsU * nc;
    s.cnt = s.rt + nc;
    s.tail = s.cnt + nc;
    s.end = s.tail + nc;
    return s;
}

template <typename T>
struct WaitOne {
    T x;
    bool ok;
};

// Bounded wait for one input still showing the reset pattern (a shared slot of the block or
// a published row of an earlier block).
template <typename T>
__device__ __noinline__ WaitOne<T> ws_wait_one(const T *vec, const T *xs, int row0, int rows, int j, ExecState *st,
                                              unsigned long long tmo, int row) {
    const unsigned lj = (unsigned)(j - row0);
    Waiter w;
    T x = lj < (unsigned)rows ? ld_shared_volatile(xs + lj) : ld_relaxed_val(vec + j);
    while (is_unset(x)) {
        if (!w.pause(st, tmo, row)) return WaitOne<T>{x, false};
        x = lj < (unsigned)rows ? ld_shared_volatile(xs + lj) : ld_relaxed_val(vec + j);
    }
    return WaitOne<T>{x, true};
}

// Walk over the chunks of the blocks a CTA runs: blocks b = blockIdx.x, + gridDim.x, ...;
// inside a block its segments in order; a segment wider than nc becomes several chunks.
struct WsChunks {
    int b, nb, stride;
    int s, s1;        // current segment and the block's end segment
    int q0, q1;       // current chunk's positions
    int seg_end;      // end position of the current segment
    int next_end;     // end position of the next segment (loaded one segment ahead)
    bool new_block;   // the current chunk opens a block
    __device__ bool first(const ExecArgs &a, int nc) {
        b = blockIdx.x;
        stride = gridDim.x;
        nb = a.n_blocks;
        return open_block(a, nc);
    }
    __device__ bool open_block(const ExecArgs &a, int nc) {
        for (; b < nb; b += stride) {
            s = __ldg(a.block_seg + b);
            s1 = __ldg(a.block_seg + b + 1);
            if (s < s1) {
                q0 = __ldg(a.seg_ptr + s);
                seg_end = __ldg(a.seg_ptr + s + 1);
                next_end = __ldg(a.seg_ptr + min(s + 2, s1));
                q1 = min(seg_end, q0 + nc);
                new_block = true;
                return true;
            }
        }
        return false;
    }
    __device__ bool next(const ExecArgs &a, int nc) {
        new_block = false;
        if (q1 < seg_end) {
            q0 = q1;
            q1 = min(seg_end, q0 + nc);
            return true;
        }
        if (++s < s1) {
            q0 = seg_end;
            seg_end = next_end;
            next_end = __ldg(a.seg_ptr + min(s + 2, s1));   // used one segment later
            q1 = min(seg_end, q0 + nc);
            return true;
        }
        b += stride;
        return open_block(a, nc);
    }
};

template <int MODE, typename T>
__global__ void __launch_bounds__(kWsMaxConsumers + kWsProducers, 1) k_block_ws(const ExecArgs a) {
    using V2 = typename Pair2<T>::type;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    __shared__ unsigned s_abort;
    const int NC = blockDim.x - kWsProducers;     // consumer threads: 32, 64, 128 or 256
    const int ALL = blockDim.x;
    const int B = a.block_rows, nb = a.n_blocks;
    const int rows_max = min(B, a.n);
    T *xs = reinterpret_cast<T *>(sm_raw);
    unsigned char *stage0 = sm_raw + (((size_t)rows_max * sizeof(T) + 15) & ~(size_t)15);
    const size_t sbytes = ws_stage_bytes<T>(NC);
    const unsigned epoch = ld_relaxed_u32(&a.st->epoch);
    T *vec = block_vec<MODE, T>(a);
    if (threadIdx.x == 0) s_abort = 0u;
    __syncthreads();
    constexpr int FULL0 = 1, EMPTY0 = 1 + kWsStages, BLK = 1 + 2 * kWsStages;
    const bool producer = (int)threadIdx.x >= NC;

    if (producer) {
        // ------------------------------------------------------------------ producers
        // PPS = kWsProducers / NC threads build each record: thread `sub` of a slot copies the
        // entries u = sub, sub + PPS, ... and thread 0 also the record's metadata and (c, 1/L_ii).
        // Iteration c: wait until the copies of chunk c - D have landed (and with them the
        // order entries of chunk c, copied D iterations earlier) and publish chunk c - D; wait
        // until chunk c - K has been consumed; issue the copies of chunk c's records and of the
        // order entries and entry ranges of chunk c + D; commit them as one group.
        const int pt = threadIdx.x - NC;
        const int PPS = kWsProducers / NC;
        const int t = pt / PPS, sub = pt % PPS;
        unsigned char *dbase = stage0 + (size_t)kWsStages * sbytes;
        int2 *rdd = reinterpret_cast<int2 *>(dbase);                                      // [(D+1) * P]
        int *ro = reinterpret_cast<int *>(dbase + (size_t)(kWsAhead + 1) * kWsProducers * sizeof(int2));
        auto stage_desc = [&](const WsChunks &w, int chunk) {
            const int sl = (chunk % (kWsAhead + 1)) * kWsProducers + pt;
            const int q = w.q0 + t;
            if (t < NC && q < w.q1) {
                cp_async4(ro + sl, a.order + q);
                cp_async8(rdd + sl, a.bdesc + q);
            } else {
                ro[sl] = -1;
            }
        };
        WsChunks cur, ahead;
        bool more = cur.first(a, NC);
        bool more_a = more;
        ahead = cur;
        // order entries of chunks 0 .. D-1, one group each
        for (int i = 0; i < kWsAhead; ++i) {
            if (more_a) {
                stage_desc(ahead, i);
                more_a = ahead.next(a, NC);
            }
            cp_async_commit();
        }
        int c = 0;
        for (; more; ++c) {
            cp_async_wait<kWsAhead - 1>();
            __syncwarp();
            if (c >= kWsAhead) named_arrive(FULL0 + (c - kWsAhead) % kWsStages, ALL);
            const int k = c % kWsStages;
            if (c >= kWsStages) named_sync(EMPTY0 + k, ALL);
            const WsStage<T> st = ws_stage<T>(stage0 + (size_t)k * sbytes, NC);
            // another CTA's failure is seen through the global word, read every 16 chunks
            if ((c & 15) == 15 && pt == 0 && ld_relaxed_u32(&a.st->abort)) s_abort = 1u;
            const bool work = ld_shared_volatile(&s_abort) == 0u;
            const int sl = (c % (kWsAhead + 1)) * kWsProducers + pt;
            const int oi = t < NC ? ro[sl] : -1;
            int cnt = -1;
            if (work && oi != -1) {
                const unsigned o = (unsigned)oi;
                const int2 dd = rdd[sl];
                const int tag = (int)(o >> 31), row = (int)(o & 0x7fffffffu);
                bool skip = false;
                if constexpr (MODE == M_ADJ_SPMV_TRSV) skip = tag == 1 && !a.gx;
                if (!skip) {
                    const int len = dd.y - dd.x;
                    cnt = min(len, kWsU);
                    const int *ci;
                    const T *vals;
                    block_entries<MODE, T>(a, tag, ci, vals);
                    for (int u = sub; u < cnt; u += PPS) {
                        cp_async4(st.j + u * NC + t, ci + dd.x + u);
                        cp_async_val<T>(st.v + u * NC + t, vals + dd.x + u);
                    }
                    if (sub == 0) {
                        if (tag == 0) {
                            if constexpr (sizeof(V2) == 16) cp_async16(st.cr + t, (const V2 *)a.aux + row);
                            else cp_async8(st.cr + t, (const V2 *)a.aux + row);
                        }
                        st.rt[t] = oi;
                        st.tail[t] = len > kWsU ? dd.x + kWsU : -1;
                        st.end[t] = dd.y;
                    }
                }
            }
            if (sub == 0 && t < NC) st.cnt[t] = cnt;
            if (more_a) {
                stage_desc(ahead, c + kWsAhead);
                more_a = ahead.next(a, NC);
            }
            cp_async_commit();
            more = cur.next(a, NC);
        }
        // publish the last chunks, then match the consumers' outstanding EMPTY arrivals
        cp_async_wait<0>();
        __syncwarp();
        for (int i = max(0, c - kWsAhead); i < c; ++i) named_arrive(FULL0 + i % kWsStages, ALL);
        for (int i = max(0, c - kWsStages); i < c; ++i) named_sync(EMPTY0 + i % kWsStages, ALL);
    } else {
        // ------------------------------------------------------------------ consumers
        const int ct = threadIdx.x;
        WsChunks ch;
        int c = 0;
        int row0 = 0, rows = 0;
        for (bool more = ch.first(a, NC); more; more = ch.next(a, NC), ++c) {
            if (ch.new_block) {
                named_sync(BLK, NC);                 // every consumer is done with the last block
                row0 = a.block_rev ? (nb - 1 - ch.b) * B : ch.b * B;
                rows = min(B, a.n - row0);
                for (int i = ct; i < rows; i += NC) xs[i] = unset_value<T>();
                named_sync(BLK, NC);
            }
            const int k = c % kWsStages;
            named_sync(FULL0 + k, ALL);
            const WsStage<T> st = ws_stage<T>(stage0 + (size_t)k * sbytes, NC);
            const int cnt = st.cnt[ct];
            if (cnt >= 0 && ld_shared_volatile(&s_abort) == 0u) {
                const int rt = st.rt[ct];
                const int row = rt & 0x7fffffff, tag = (int)((unsigned)rt >> 31);
                // the record's entries in order; an input still showing the reset pattern
                // (a row of an earlier block not yet published) is waited for in place
                const int *jr = st.j + ct;
                const T *vr = st.v + ct;
                T acc = T(0);
                bool ok = true;
                for (int u = 0; u < cnt; ++u) {
                    const int j = jr[u * NC];
                    const unsigned lj = (unsigned)(j - row0);
                    T x = lj < (unsigned)rows ? ld_shared_volatile(xs + lj) : ld_relaxed_val(vec + j);
                    if (is_unset(x)) {
                        const WaitOne<T> w1 = ws_wait_one<T>(vec, xs, row0, rows, j, a.st, a.timeout_ns, row);
                        x = w1.x;
                        ok = ok && w1.ok;
                    }
                    acc += vr[u * NC] * x;
                }
                const int tl = st.tail[ct];
                if (tl >= 0 && ok) {
                    const int *ci;
                    const T *vals;
                    block_entries<MODE, T>(a, tag, ci, vals);
                    const TailSum<T> ts = block_dot_tail<T>(ci, vals, tl, st.end[ct], 1, vec, xs, row0, rows, a.st,
                                                            a.timeout_ns, row, acc);
                    acc = ts.acc;
                    ok = ts.ok;
                }
                if (!ok) {
                    s_abort = 1u;
                } else if (tag == 0) {
                    const V2 cr = st.cr[ct];
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

}  // namespace sf
