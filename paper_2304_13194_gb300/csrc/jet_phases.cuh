// The passes of Jet refinement (Sec. 4) as device functions over a "grid" of
// blocks: either the blocks of one kernel launch or the blocks of one thread
// block cluster that runs a whole level.  Each phase touches only the arrays
// of `Level`, carves its shared memory from a caller-provided arena, and is
// bit-exact: every decision is an integer comparison with fixed tie-breaks
// (lowest part id, then lowest vertex id) and only order-independent integer
// atomics are used.
//
// Design (GB300-first, not a translation of the paper's Kokkos kernels):
//  * No persistent vertex-part hash table (Sec. 4.3).  conn(v, .) is
//    recomputed from the CSR row in registers (rows of <= 16 entries, one
//    thread per vertex) or in a per-warp shared-memory table cleared as it
//    is read (longer rows, one warp per vertex).  One list holds both kinds
//    of rows: a block stages the long rows its threads meet and its warps
//    take them afterwards, so a pass is one phase, not two.
//  * ext[v] (neighbours in other parts) is kept exact by the apply phase, so
//    passes list boundary vertices first and never stream interior rows.
//  * The apply phase also commits the moves: nxt[v] packs the source and
//    destination parts, so a neighbour's old part is known while part[] is
//    being overwritten.
//  * Lists are staged in shared memory and reserved with one atomic per
//    block flush.
//  * Serial end-of-phase work (the controller of Alg. 3, the rebalancing
//    plan, the eviction scan of Jetrs) is a "tail" that one block runs once
//    every block of the phase is done: the last block to finish in a kernel
//    launch, block 0 after the barrier in the cluster loop.
//  * Arrays that phases modify (part, prio, nxt, ext, stamps, lists) are read
//    with ordinary loads, never through the non-coherent read-only path, so
//    that the cluster-resident loop sees them after each cluster barrier.
#pragma once

#include "jet_internal.cuh"

#include <cuda/atomic>

namespace jet {

struct Grid {
    int bid;   // rank of this block among the cooperating blocks
    int nb;    // number of cooperating blocks
};

__device__ __forceinline__ Grid launch_grid() { return Grid{(int)blockIdx.x, (int)gridDim.x}; }

// The entries of a list of `len` that block G.bid takes.  Dealt (`spread`):
// the list is cut into chunks of kDealChunk entries (one 32-byte sector of
// int32 ids) dealt round-robin over the blocks, so a run of long rows that
// one producer appended together is spread over many blocks instead of
// landing in one block's share (contiguous shares made single blocks take
// hundreds of long rows while the rest of the grid idled), and every warp
// load of the list still reads whole sectors.  Otherwise each block takes
// one contiguous share (whole warps), which keeps the neighbour gathers of
// consecutive vertices in the block's L1: the work lists of the scans are in
// vertex order and are dealt only on levels with long rows; X and M are in
// append order and are always dealt.  A block walks its entries blockDim at
// a time; all its threads make the same number of passes.
constexpr int kDealChunk = 8;
struct Deal {
    int64_t len, seg;
    int nb, bid;
    bool spread;
    __device__ __forceinline__ Deal(int64_t n, Grid G, bool spread_) : len(n), nb(G.nb), bid(G.bid), spread(spread_) {
        int64_t s = (n + G.nb - 1) / G.nb;
        seg = (s + 31) & ~int64_t(31);
    }
    // list index of block-local position q (increasing in q)
    __device__ __forceinline__ int64_t at(int64_t q) const {
        if (spread) {
            const int64_t c = q / kDealChunk;
            return (c * nb + bid) * kDealChunk + (q % kDealChunk);
        }
        return q < seg ? (int64_t)bid * seg + q : len;
    }
    // pass p has at least one entry for this block
    __device__ __forceinline__ bool live(int64_t p) const { return at(p * (int64_t)blockDim.x) < len; }
    // list index of this thread in pass p (>= len: none)
    __device__ __forceinline__ int64_t entry(int64_t p) const { return at(p * (int64_t)blockDim.x + threadIdx.x); }
};

// A value other blocks of the same kernel changed (atomics, stores before
// their completion ticket): a device-scope load served by L2, never by a
// stale L1 line.
template <class T>
__device__ __forceinline__ T ld_gpu(const T *p) {
    return cuda::atomic_ref<T, cuda::thread_scope_device>(*const_cast<T *>(p)).load(cuda::memory_order_relaxed);
}

// nxt[v] = source part << 16 | destination part (k <= JET_MAX_K < 2^16).
__device__ __forceinline__ int32_t nxt_pack(int32_t from, int32_t to) { return (int32_t)(((uint32_t)from << 16) | (uint32_t)to); }
__device__ __forceinline__ int32_t nxt_to(int32_t x) { return x & 0xFFFF; }
__device__ __forceinline__ int32_t nxt_from(int32_t x) { return (int32_t)((uint32_t)x >> 16); }

struct LpExport {           // optional dense outputs of the single-pass API
    int32_t *pd;            // P_d (P_s where undefined)
    int32_t *gain;          // F (kNoneGain where undefined)
    int32_t *f2;            // F2 for X members
};

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------
template <bool EW>
__device__ __forceinline__ int32_t edge_w(const DGraph &g, int64_t j) {
    if constexpr (EW) return __ldg(g.ew + j);
    else return 1;
}

// An entry of a long row (read once per pass, coalesced over the lanes):
// kept out of L1 so that the neighbours' fields gathered next stay there.
__device__ __forceinline__ int32_t ld_stream(const int32_t *p) {
    int32_t v;
    asm("ld.global.nc.L1::no_allocate.b32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}
template <bool EW>
__device__ __forceinline__ int32_t edge_w_stream(const DGraph &g, int64_t j) {
    if constexpr (EW) return ld_stream(g.ew + j);
    else return 1;
}

__device__ __forceinline__ bool ablate_locks(uint32_t abl) { return (abl & (ABL_NO_LOCKS | ABL_BASELINE_LP)) != 0; }

// First filter, Eq. gainconn_filter: -F < floor(c * conn(v,P_s)) or F >= 0
// (ablations: weak afterburner keeps F >= 0, baseline LP and strict gain keep
// F > 0).
__device__ __forceinline__ bool first_filter(int32_t F, int32_t conn_s, int32_t cq16, uint32_t abl) {
    if (abl & (ABL_BASELINE_LP | ABL_STRICT_GAIN)) return F > 0;
    if (abl & ABL_WEAK_AFTERBURN) return F >= 0;
    if (F >= 0) return true;
    long long lim = ((long long)cq16 * (long long)conn_s) >> 16;
    return -(long long)F < lim;
}

__device__ __forceinline__ unsigned long long part_key(int32_t conn, int32_t p) {
    // larger key: larger connectivity, then smaller part id
    return ((unsigned long long)(uint32_t)conn << 32) | (unsigned long long)(0xFFFFFFFFu - (uint32_t)p);
}
__device__ __forceinline__ int32_t key_part(unsigned long long key) {
    return (int32_t)(0xFFFFFFFFu - (uint32_t)(key & 0xFFFFFFFFull));
}
__device__ __forceinline__ int32_t key_conn(unsigned long long key) { return (int32_t)(key >> 32); }

// Block-level sum of a counter, one atomic per block.
__device__ __forceinline__ void flush_counter(int64_t *dst, long long v, long long *red) {
    v = block_sum_i64(v, red);
    if (threadIdx.x == 0 && v) atomic_add_i64(dst, v);
}

// Graph-loop guard: the first kernel of every iteration branch clears the
// loop condition; only the controller at the end of a completed iteration
// sets it again, so the device loop cannot outlive a missing controller.
__device__ __forceinline__ void disarm_loop(const Level &L, Grid G) {
    if (L.use_graph && G.bid == 0 && threadIdx.x == 0)
        cudaGraphSetConditional((cudaGraphConditionalHandle)L.h_loop, 0u);
}

// In a kernel launch: true in the last block to finish (all blocks call it
// once, after their part of the phase).  The block's threads meet at a
// barrier, then one thread fences (which orders every write the barrier
// made it wait for) and takes the block's ticket, so the last block sees
// the writes of all blocks; the tails read them with device-scope loads.
// No block waits for another.
__device__ __forceinline__ bool last_block(Ctl *ctl) {
    __shared__ int s_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const int t = atomicAdd(&ctl->ticket, 1);
        s_last = t == (int)gridDim.x - 1;
        if (s_last) {
            __threadfence();
            ctl->ticket = 0;   // for the next kernel that counts
        }
    }
    __syncthreads();
    return s_last != 0;
}

// Block-aggregated append into a global list: members are staged in shared
// memory and reserved in the global list with one atomic per flush instead
// of one per warp on a single hot counter.
struct Appender {
    int32_t *buf;
    int cap;
    int *cnt;
    int *base;
    __device__ __forceinline__ void init() {
        if (threadIdx.x == 0) *cnt = 0;
        __syncthreads();
    }
    __device__ __forceinline__ void add(bool pred, int32_t v) {   // all lanes of the warp call it
        unsigned m = __ballot_sync(0xffffffffu, pred);
        if (!m) return;
        int leader = __ffs(m) - 1;
        int b = 0;
        if ((int)lane_id() == leader) b = atomicAdd(cnt, __popc(m));
        b = __shfl_sync(0xffffffffu, b, leader);
        if (pred) buf[b + __popc(m & ((1u << lane_id()) - 1u))] = v;
    }
    // Flushes when another round of up to `adds` members per thread could
    // overflow the buffer, or always with force.  All threads call it.
    __device__ __forceinline__ void flush(int32_t *gcount, int32_t *glist, bool force, int adds = 1) {
        __syncthreads();
        int c = *cnt;
        if (c > 0 && (force || c > cap - adds * (int)blockDim.x)) {
            if (threadIdx.x == 0) *base = atomicAdd(gcount, c);
            __syncthreads();
            int b = *base;
            for (int i = threadIdx.x; i < c; i += blockDim.x) glist[b + i] = buf[i];
            __syncthreads();
            if (threadIdx.x == 0) *cnt = 0;
            __syncthreads();
        }
    }
    // Long rows staged for the block: when another round could overflow the
    // buffer (or with force), the block's warps take the staged rows in turn
    // (`row(v)`, all 32 lanes), except rows longer than `hub`, which are
    // set aside (up to kHugeCap of them; more stay with the warps) and then
    // taken by the whole block one after another (`block_row(v)`, every
    // thread): a hub row no longer serialises one warp for the whole pass.
    // All threads call it.
    template <class Row, class BlockRow>
    __device__ __forceinline__ void drain(bool force, const int64_t *xadj, Row &&row, BlockRow &&block_row,
                                          int64_t hub = kHugeDeg) {
        __shared__ int32_t huge[kHugeCap];
        __shared__ int nhuge;
        __syncthreads();
        int c = *cnt;
        if (c > 0 && (force || c > cap - (int)blockDim.x)) {
            if (threadIdx.x == 0) nhuge = 0;
            __syncthreads();
            const int warps = blockDim.x >> 5;
            for (int s = threadIdx.x >> 5; s < c; s += warps) {
                const int32_t v = buf[s];
                int defer = 0;
                if (lane_id() == 0 && ld_xadj(xadj, (int64_t)v + 1) - ld_xadj(xadj, v) > hub) {
                    const int slot = atomicAdd(&nhuge, 1);
                    if (slot < kHugeCap) {
                        huge[slot] = v;
                        defer = 1;
                    }
                }
                defer = __shfl_sync(0xffffffffu, defer, 0);
                if (!defer) row(v);
            }
            __syncthreads();
            const int nh = nhuge < kHugeCap ? nhuge : kHugeCap;
            for (int s = 0; s < nh; ++s) block_row(huge[s]);
            __syncthreads();
            if (threadIdx.x == 0) *cnt = 0;
            __syncthreads();
        }
    }
};

#define JET_APPENDER(name, bufptr, capacity)                    \
    __shared__ int name##_cnt, name##_base;                      \
    Appender name{(bufptr), (capacity), &name##_cnt, &name##_base}; \
    name.init()

// ---------------------------------------------------------------------------
// shared-memory arena per phase (bytes, for blocks of T threads; `tables`:
// the level has long rows, so the row phases need one k-entry table per warp)
// ---------------------------------------------------------------------------
constexpr int kScanCap = 4096;          // list staging of the scan phases
constexpr int kListCap = 2048;          // X / M staging
constexpr int kBigCap = 1024;           // long-row staging
constexpr int kSmemBuckets = 1024;      // slot buckets aggregated per block when nA * kSlots fits

__host__ __device__ constexpr size_t align16(size_t x) { return (x + 15) & ~size_t(15); }
__host__ __device__ constexpr size_t arena_max(size_t a, size_t b) { return a > b ? a : b; }
__host__ __device__ constexpr size_t arena_tables(int32_t k, int T, bool tables) {
    return tables ? (size_t)(T / 32) * (size_t)k * 4 : 0;
}
__host__ __device__ constexpr size_t sm_lp_scan() { return (size_t)kScanCap * 4; }
__host__ __device__ constexpr size_t sm_lp_select(int32_t k, int T, bool tables) {
    return (size_t)(kListCap + kBigCap) * 4 + arena_tables(k, T, tables);
}
__host__ __device__ constexpr size_t sm_afterburn() { return (size_t)(kListCap + kBigCap) * 4; }
__host__ __device__ constexpr size_t sm_apply(int32_t k) { return align16((size_t)k * 8) + (size_t)kBigCap * 4; }
__host__ __device__ constexpr size_t sm_rb_scan() { return (size_t)kSmemBuckets * 8 + (size_t)kScanCap * 4; }
__host__ __device__ constexpr size_t sm_rb_cand(int32_t k, int T, bool tables) {
    return (size_t)kSmemBuckets * 8 + (size_t)kBigCap * 4 + arena_tables(k, T, tables);
}
__host__ __device__ constexpr size_t sm_rb_tilehist(int32_t k) { return (size_t)k * 4; }
__host__ __device__ constexpr size_t sm_rb_take(int32_t k, int T) { return align16((size_t)k * 8) + (size_t)2 * T * 4; }
__host__ __device__ constexpr size_t sm_rb_cookie(int T) { return (size_t)2 * T * 4; }
// the largest arena any phase needs
__host__ __device__ constexpr size_t arena_bytes(int32_t k, int T) {
    return arena_max(arena_max(arena_max(sm_lp_scan(), sm_lp_select(k, T, true)), arena_max(sm_afterburn(), sm_apply(k))),
                     arena_max(arena_max(sm_rb_scan(), sm_rb_cand(k, T, true)),
                               arena_max(sm_rb_tilehist(k), arena_max(sm_rb_take(k, T), sm_rb_cookie(T)))));
}

// ---------------------------------------------------------------------------
// controller helpers (one block)
// ---------------------------------------------------------------------------
// Max part weight; the weights are left in spw[0..k) for compute_classes.
__device__ inline long long block_max_pw(const int64_t *pw, int32_t k, long long *sh, long long *spw) {
    long long m = 0;
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        long long w = ld_gpu(&pw[i]);
        spw[i] = w;
        m = w > m ? w : m;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        long long t = __shfl_xor_sync(0xffffffffu, m, o);
        m = t > m ? t : m;
    }
    __syncthreads();
    if (lane_id() == 0) sh[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        long long t = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            long long u = __shfl_xor_sync(0xffffffffu, t, o);
            t = u > t ? u : t;
        }
        if (threadIdx.x == 0) sh[0] = t;
    }
    __syncthreads();
    long long r = sh[0];
    __syncthreads();
    return r;
}

// Rebalancing classes (Alg. 5): A = {p : w_p > L} numbered in ascending id,
// B = {p : w_p <= sigma} listed in ascending id, excess of each A part, the
// capacity prefix of B (Jetrs) and zeroed slot buckets.  Any block size;
// spw holds the part weights (block_max_pw).
__device__ inline void compute_classes(const Level &L, long long *sh, const long long *spw, long long Llim,
                                       long long sigma) {
    Ctl *ctl = L.ctl;
    long long ca = 0, cb = 0, cc = 0;
    for (int p0 = 0; p0 < L.k; p0 += blockDim.x) {
        int p = p0 + threadIdx.x;
        bool inA = false, inB = false;
        long long w = 0;
        if (p < L.k) {
            w = spw[p];
            inA = w > Llim;
            inB = w <= sigma;
        }
        long long tA = 0, tB = 0, tC = 0;
        long long ia = ca + block_exscan_i64(inA ? 1 : 0, sh, &tA);
        long long ib = cb + block_exscan_i64(inB ? 1 : 0, sh, &tB);
        long long cap = inB ? (sigma - w) : 0;
        long long ic = cc + block_exscan_i64(cap, sh, &tC);
        if (p < L.k) {
            L.aidx[p] = inA ? (int32_t)ia : -1;
            L.inB[p] = inB ? 1 : 0;
            if (inA) L.excess[ia] = w - Llim;
            if (inB) { L.Bs[ib] = p; L.capC[ib] = ic; }
        }
        ca += tA; cb += tB; cc += tC;
    }
    if (threadIdx.x == 0) {
        ctl->nA = (int32_t)ca;
        ctl->nB = (int32_t)cb;
        L.capC[cb] = cc;
    }
    __syncthreads();
    int32_t nkeys = (int32_t)ca * kSlots;
    for (int i = threadIdx.x; i < nkeys; i += blockDim.x) L.bucketw[i] = 0;
    __syncthreads();
}

// Mode of the next iteration (Alg. 3): balanced -> Jetlp; else Jetrw while the
// weak counter is below b_max, else Jetrs; DONE by the stop rule or the cap.
// Updates the weak counter and the cap flag it is given.
__device__ __forceinline__ int32_t next_mode_of(const Level &L, bool balanced, int32_t noimp, int32_t it,
                                                int32_t &weak, int32_t &hit_cap) {
    if (noimp >= L.max_no_improve) return MODE_DONE;
    if (it >= L.max_iters) { hit_cap = 1; return MODE_DONE; }
    if (balanced) { weak = 0; return MODE_LP; }
    if (weak < L.weak_limit) { weak += 1; return MODE_RW; }
    return MODE_RS;
}

__device__ inline int32_t choose_mode(const Level &L, bool balanced) {
    Ctl *ctl = L.ctl;
    int32_t weak = ctl->weak, cap = ctl->hit_cap;
    int32_t m = next_mode_of(L, balanced, ctl->noimp, ctl->it, weak, cap);
    ctl->weak = weak;
    ctl->hit_cap = cap;
    return m;
}

__device__ __forceinline__ void reset_counters(Ctl *ctl) {
    ctl->nW = ctl->nX = ctl->nM = 0;
    ctl->nXh = ctl->nMh = 0;
    ctl->ncand = 0;
    ctl->degx = ctl->degm = 0;
    ctl->nbnd = ctl->nexam = ctl->degexam = 0;
}

// Algorithmic DRAM bytes of one iteration's refinement kernels, from the
// counters the iteration gathered: every array a kernel streams is counted
// once per launch over the subset it touches; gathers and scatters at
// neighbours (part, prio, nxt, mstamp, ext of u) are taken as cache hits.
// beta = bytes per CSR entry (8 with edge weights, 4 without), n vertices,
// k parts, T rebalancing tiles, nA oversized parts; w = rows the Jetlp select
// reads (unlocked boundary vertices), nb = boundary vertices, c =
// rebalancing candidates, r = listed candidates (rows read), deg(S) = total
// row length over S.
//   lp_scan      4n + 4 nb + 4 w           ext of every vertex, lock stamp of the
//                                          boundary ones, work-list writes
//   lp_select    24 w + beta deg(W) + 12|X| list, xadj pair, part; rows; prio, nxt, X list
//   afterburn    32|X| + beta deg(X) + 8|M|  X list, xadj pair, prio, nxt, part; rows;
//                                          mstamp, M list (4|X| + 8|M| without afterburner)
//   apply        36|M| + beta deg(M) + 16k  M list, nxt, vwgt, xadj pair, ext, part
//                                          (+4|M| lock stamps and 8|X| priority resets
//                                          after Jetlp); rows; part weights
//   rb_scan      8n + 16c + 4r             part, bucket key; vwgt, ext, weighted degree
//                                          and destination of candidates; work list
//   rb_cand      28r (+4r Jetrw) + beta deg(R)  list, xadj pair, part, key (+ destination); rows
//   rb_tilehist  4n + 4c + 4 T nA          key, vwgt of candidates, tile sums
//   rb_tilescan  8 T nA                    tile sums read and written
//   rb_take      4n + 4c + 4 T nA + 8|M|   key, vwgt, tile offsets; mstamp, M list
//                (Jetrs: + 8n + 8T          evicted weight per vertex and per tile,
//                 instead of the M list)
//   rb_cookie    8n + 8T + 16|M|           evicted weight, tile offsets; part, nxt,
//                                          mstamp, M list
// plus 8n (read P_iter, write P_best) in the kernel that copied the best
// partition during this iteration (the afterburner for Jetlp, rb_scan for
// rebalancing) when the previous controller asked for it; the copy after
// the level's last iteration is not a refinement kernel.
struct IterCounts {
    int64_t nx, nm, degx, degm, nbnd, nexam, degexam, ncand, na;
    bool copied;
};
__device__ __forceinline__ void iter_bytes(const Level &L, int32_t kind, const IterCounts &q, int64_t *b /* [JET_K_COUNT] */) {
    const int64_t n = L.g.n, beta = L.g.ew ? 8 : 4, T = L.ntiles, k = L.k;
    const int64_t cp = q.copied ? 8 * n : 0;
    for (int i = 0; i < JET_K_COUNT; ++i) b[i] = 0;
    if (kind == MODE_LP) {
        const bool ab = !(L.abl & (ABL_NO_AFTERBURN | ABL_BASELINE_LP));
        const int64_t w = q.nexam, X = q.nx, M = q.nm;
        b[JET_K_LP_SCAN] = 4 * n + 4 * q.nbnd + 4 * w;
        b[JET_K_LP_SELECT] = 24 * w + beta * q.degexam + 12 * X;
        b[JET_K_AFTERBURN] = cp + (ab ? 32 * X + beta * q.degx : 4 * X) + 8 * M;
        b[JET_K_APPLY] = 40 * M + beta * q.degm + 16 * k + 8 * X;
    } else {
        const bool rs = kind == MODE_RS;
        const int64_t c = q.ncand, r = q.nbnd, M = q.nm, tn = T * q.na;
        b[JET_K_RB_SCAN] = cp + 8 * n + 16 * c + 4 * r;
        b[JET_K_RB_CAND] = (rs ? 28 : 32) * r + beta * q.degexam;
        b[JET_K_RB_TILEHIST] = 4 * n + 4 * c + 4 * tn;
        b[JET_K_RB_TILESCAN] = 8 * tn;
        b[JET_K_RB_TAKE] = 4 * n + 4 * c + 4 * tn + (rs ? 8 * n + 8 * T : 8 * M);
        if (rs) b[JET_K_RB_COOKIE] = 8 * n + 8 * T + 16 * M;
        b[JET_K_APPLY] = 36 * M + beta * q.degm + 16 * k;
    }
}

// End of an iteration (Alg. 3 after updatePartsAndDS), one block, after every
// block of the apply phase: exact cut, max part weight, P_best / counters,
// trace record, next mode, rebalancing classes for the next iteration.
// Thread 0 loads every control value it needs before it uses any (one memory
// round trip), decides in registers, then stores.  Returns the next mode
// (all threads).
__device__ inline int32_t ph_controller(const Level &L) {
    __shared__ long long sh[40];
    __shared__ long long spw[JET_MAX_K];
    __shared__ int32_t next_mode;
    __shared__ long long s_lim[2];
    Ctl *ctl = L.ctl;
    // thread 0 gathers: values of earlier kernels (plain loads) and of this
    // one (ld_gpu), issued together with the mode and before the part-weight
    // reduction so that the round trips overlap
    long long cut0 = 0, Llim = 0, sigma = 0, best_cut0 = 0, best_maxw0 = 0, ncand = 0, degx = 0, nbnd = 0, nexam = 0,
              degexam = 0, dcut = 0, degm = 0;
    int32_t it = 0, noimp0 = 0, best_bal0 = 0, kc = 0, weak = 0, hit_cap = 0, nX = 0, nM = 0, nA = 0, copied = 0;
    int64_t kb0[JET_K_COUNT];
    int32_t kc4[4] = {0, 0, 0, 0};
    const int32_t kind = ctl->mode;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < 4; ++i) kc4[i] = ctl->kcount[i];
        cut0 = ctl->cut; Llim = ctl->L; sigma = ctl->sigma; best_cut0 = ctl->best_cut; best_maxw0 = ctl->best_maxw;
        it = ctl->it; noimp0 = ctl->noimp; best_bal0 = ctl->best_bal;
        weak = ctl->weak; hit_cap = ctl->hit_cap;
        nX = ctl->nX + ctl->nXh; nM = ctl->nM + ctl->nMh; nA = ctl->nA; copied = ctl->copy_best;
        ncand = ctl->ncand; degx = ctl->degx; nbnd = ctl->nbnd; nexam = ctl->nexam; degexam = ctl->degexam;
        dcut = ld_gpu(&ctl->dcut); degm = ld_gpu(&ctl->degm);
#pragma unroll
        for (int i = 0; i < JET_K_COUNT; ++i) kb0[i] = ctl->kbytes[i];
    }
    if (kind == MODE_DONE) {
        if (threadIdx.x == 0) {
            ctl->copy_best = 0;
            if (L.use_graph) {
                cudaGraphSetConditional((cudaGraphConditionalHandle)L.h_loop, 0u);
                cudaGraphSetConditional((cudaGraphConditionalHandle)L.h_next, (unsigned)MODE_DONE);
            }
        }
        return MODE_DONE;
    }
    if (threadIdx.x == 0) kc = kind == 0 ? kc4[0] : kind == 1 ? kc4[1] : kind == 2 ? kc4[2] : kc4[3];
    long long maxw = block_max_pw(L.pw, L.k, sh, spw);
    if (threadIdx.x == 0) {
        // decide
        const long long cut = cut0 + dcut;
        const bool bal = maxw <= Llim;
        int32_t noimp = noimp0 + 1, best_bal = best_bal0, copy = 0;
        long long best_cut = best_cut0, best_maxw = best_maxw0;
        if (bal) {
            if (!best_bal0 || cut < best_cut0) {
                if (!best_bal0 || 1000000LL * cut < L.phi_ppm * best_cut0) noimp = 0;
                best_cut = cut; best_maxw = maxw; best_bal = 1;
                copy = 1;
            }
        } else if (!best_bal0 && maxw < best_maxw0) {
            best_cut = cut; best_maxw = maxw; noimp = 0;
            copy = 1;
        }
        const int32_t m = next_mode_of(L, bal, noimp, it + 1, weak, hit_cap);
        // scatter
        ctl->dcut = 0;
        ctl->cut = cut;
        ctl->maxw = maxw;
        ctl->noimp = noimp;
        ctl->best_cut = best_cut; ctl->best_maxw = best_maxw; ctl->best_bal = best_bal;
        ctl->copy_best = copy;
        if (it < kTrace && L.trace) {
            TraceRec r;
            r.kind = kind; r.flags = copy; r.na = kind == MODE_LP ? 0 : nA; r.pad = 0;
            r.nx = (kind == MODE_LP) ? (int64_t)nX : ncand;
            r.nm = nM;
            r.cut = cut; r.maxw = maxw;
            r.degx = degx; r.degm = degm;
            r.nbnd = nbnd; r.nexam = nexam; r.degexam = degexam;
            L.trace[it] = r;
        }
        {
            const IterCounts q{kind == MODE_LP ? (int64_t)nX : 0, nM, degx, degm, nbnd, nexam, degexam, ncand,
                               kind == MODE_LP ? 0 : nA, copied != 0};
            int64_t kb[JET_K_COUNT];
            iter_bytes(L, kind, q, kb);
#pragma unroll
            for (int i = 0; i < JET_K_COUNT; ++i) ctl->kbytes[i] = kb0[i] + kb[i];
        }
        if (kind == MODE_LP) ctl->lp_epoch = it;
        ctl->kcount[kind] = kc + 1;
        ctl->it = it + 1;
        ctl->weak = weak;
        ctl->hit_cap = hit_cap;
        reset_counters(ctl);
        ctl->mode = m;
        next_mode = m;
        s_lim[0] = Llim;
        s_lim[1] = sigma;
        if (L.use_graph) {
            // the next iteration's switch (DONE: no branch) and the loop flag
            // (the next iteration's first kernel clears it)
            cudaGraphSetConditional((cudaGraphConditionalHandle)L.h_next, (unsigned)m);
            cudaGraphSetConditional((cudaGraphConditionalHandle)L.h_loop, m == MODE_DONE ? 0u : 1u);
        }
    }
    __syncthreads();
    int32_t m = next_mode;
    if (m == MODE_RW || m == MODE_RS) compute_classes(L, sh, spw, s_lim[0], s_lim[1]);
    return m;
}

// Level start, one block: control block from the initial cut and weights.
__device__ inline void ph_ctl_init(const Level &L, const int64_t *cut2) {
    __shared__ long long sh[40];
    __shared__ long long spw[JET_MAX_K];
    Ctl *ctl = L.ctl;
    long long maxw = block_max_pw(L.pw, L.k, sh, spw);
    if (threadIdx.x == 0) {
        ctl->cut = *cut2 / 2;
        ctl->dcut = 0;
        ctl->maxw = maxw;
        ctl->best_cut = ctl->cut;
        ctl->best_maxw = maxw;
        ctl->best_bal = maxw <= ctl->L;
        ctl->it = 0; ctl->noimp = 0; ctl->weak = 0; ctl->lp_epoch = -1;
        ctl->copy_best = 0; ctl->hit_cap = 0; ctl->ticket = 0;
        ctl->bar_count = 0; ctl->bar_gen = 0; ctl->bar_err = 0;
        ctl->kcount[0] = ctl->kcount[1] = ctl->kcount[2] = ctl->kcount[3] = 0;
        for (int i = 0; i < JET_KERNELS; ++i) ctl->kbytes[i] = 0;
        reset_counters(ctl);
        ctl->mode = choose_mode(L, maxw <= ctl->L);
    }
    __syncthreads();
    if (ctl->mode == MODE_RW || ctl->mode == MODE_RS) compute_classes(L, sh, spw, ctl->L, ctl->sigma);
}

// P_best <- P_iter when the controller asked for it (first phase of the next
// iteration, and once after the level's loop).
__device__ inline void copy_best_rows(const Level &L, Grid G) {
    const int64_t stride = (int64_t)G.nb * blockDim.x;
    if (((reinterpret_cast<uintptr_t>(L.part) | reinterpret_cast<uintptr_t>(L.best)) & 15) != 0) {
        for (int64_t i = (int64_t)G.bid * blockDim.x + threadIdx.x; i < L.g.n; i += stride) L.best[i] = L.part[i];
        return;
    }
    const int4 *src = reinterpret_cast<const int4 *>(L.part);
    int4 *dst = reinterpret_cast<int4 *>(L.best);
    int64_t n4 = L.g.n / 4;
    for (int64_t i = (int64_t)G.bid * blockDim.x + threadIdx.x; i < n4; i += stride) dst[i] = src[i];
    if (G.bid == 0 && threadIdx.x < (L.g.n & 3)) {
        int64_t i = n4 * 4 + threadIdx.x;
        L.best[i] = L.part[i];
    }
}
__device__ inline void ph_copy_best(const Level &L, Grid G) {
    if (L.ctl->copy_best) copy_best_rows(L, G);
}

// ---------------------------------------------------------------------------
// Jetlp (Alg. 4)
// ---------------------------------------------------------------------------

// Step 0: the work list.  A vertex with no neighbour in another part (ext ==
// 0) has no destination (Alg. 4: A_v is empty) and a locked vertex is
// skipped (Sec. 4.1.3); the scan reads ext four vertices at a time and lists
// the others.  Interior rows are never read.
__device__ inline void ph_lp_scan(const Level &L, Grid G, char *arena) {
    disarm_loop(L, G);
    __shared__ long long red[40];
    Ctl *ctl = L.ctl;
    const int32_t epoch = ctl->lp_epoch;   // loaded before the appender's barrier
    JET_APPENDER(wapp, reinterpret_cast<int32_t *>(arena), kScanCap);
    const bool use_locks = !ablate_locks(L.abl);
    const int64_t n = L.g.n, nq = (n + 3) / 4;
    const bool vec = (reinterpret_cast<uintptr_t>(L.ext) & 15) == 0;
    long long nb = 0;
    for (int64_t q0 = (int64_t)G.bid * blockDim.x; q0 < nq; q0 += (int64_t)G.nb * blockDim.x) {
        int64_t q = q0 + threadIdx.x;
        int64_t v0 = 4 * q;
        int32_t e[4] = {0, 0, 0, 0};
        if (q < nq) {
            if (vec && v0 + 3 < n) {
                int4 x = *reinterpret_cast<const int4 *>(L.ext + v0);
                e[0] = x.x; e[1] = x.y; e[2] = x.z; e[3] = x.w;
            } else {
#pragma unroll
                for (int i = 0; i < 4; ++i) e[i] = v0 + i < n ? L.ext[v0 + i] : 0;
            }
        }
        int32_t ls[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) ls[i] = (e[i] > 0 && use_locks) ? L.lstamp[v0 + i] : INT32_MIN;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            nb += e[i] > 0;
            wapp.add(e[i] > 0 && ls[i] != epoch, (int32_t)(v0 + i));
        }
        wapp.flush(&ctl->nW, L.listW, false, 4);
    }
    wapp.flush(&ctl->nW, L.listW, true, 4);
    flush_counter(&ctl->nbnd, nb, red);
}

// Block-wide maximum, returned to every thread; sh holds >= 32 values.
__device__ __forceinline__ unsigned long long block_max_u64(unsigned long long v, unsigned long long *sh) {
    v = warp_max_u64(v);
    __syncthreads();
    if (lane_id() == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    const unsigned nw = (blockDim.x + 31) >> 5;
    unsigned long long t = threadIdx.x < nw ? sh[threadIdx.x] : 0ULL;
    if (threadIdx.x < 32) t = warp_max_u64(t);
    if (threadIdx.x == 0) sh[0] = t;
    __syncthreads();
    const unsigned long long r = sh[0];
    __syncthreads();
    return r;
}

// Sum over the block's per-warp tables of part p's connectivity.
__device__ __forceinline__ int32_t tables_sum(const int32_t *tabs, int32_t k, int32_t p) {
    int32_t c = 0;
    const int warps = blockDim.x >> 5;
    for (int w = 0; w < warps; ++w) c += tabs[w * k + p];
    return c;
}

// Clears the block's per-warp tables (all threads).
__device__ __forceinline__ void tables_clear(int32_t *tabs, int32_t k) {
    const int n = (int)(blockDim.x >> 5) * k;
    for (int i = threadIdx.x; i < n; i += blockDim.x) tabs[i] = 0;
}

// Long rows are walked kRowBatch entries per thread at a time: the entries'
// neighbour ids (and weights) are loaded together, then the neighbours'
// fields, then they are used, so a thread keeps kRowBatch dependent gather
// chains in flight instead of one (a hub row of 160k entries otherwise takes
// a block as long as a whole pass).
constexpr int kRowBatch = 4;    // warp rows (17 to hub_degree entries)
constexpr int kHubBatch = 8;    // hub rows (one block each)

// conn(v, .) of the entries first, first + step, ... < end added into tab.
template <bool EW, int U = kRowBatch>
__device__ __forceinline__ void row_to_table(const Level &L, int64_t first, int64_t end, int64_t step, int32_t *tab) {
    const DGraph &g = L.g;
    for (int64_t j0 = first; j0 < end; j0 += U * step) {
        int32_t u[U], w[U], p[U];
#pragma unroll
        for (int q = 0; q < U; ++q) {
            const int64_t j = j0 + q * step;
            u[q] = j < end ? ld_stream(g.adj + j) : -1;
            w[q] = j < end ? edge_w_stream<EW>(g, j) : 0;
        }
#pragma unroll
        for (int q = 0; q < U; ++q) p[q] = u[q] >= 0 ? L.part[u[q]] : -1;
#pragma unroll
        for (int q = 0; q < U; ++q)
            if (p[q] >= 0) atomicAdd(&tab[p[q]], w[q]);
    }
}

// One hub row of step 1 (longer than kHugeDeg) by the whole block: each warp
// adds its share of conn(v, .) into its own k-entry table (tabs, zero
// between rows), the parts then sum the warps' entries; the same result as
// the warp version.
template <bool EW>
__device__ __forceinline__ void lp_select_block_row(const Level &L, LpExport ex, int32_t v, int32_t *tabs, long long *red,
                                                    long long &nexam, long long &degexam, long long &degx) {
    const DGraph &g = L.g;
    const int32_t ps = L.part[v];
    const int64_t beg = ld_xadj(g.xadj, v), end = ld_xadj(g.xadj, (int64_t)v + 1);
    int32_t *tab = tabs + (threadIdx.x >> 5) * L.k;
    row_to_table<EW, kHubBatch>(L, beg + threadIdx.x, end, blockDim.x, tab);
    __syncthreads();
    const int32_t conn_s = tables_sum(tabs, L.k, ps);
    unsigned long long best = 0;
    for (int p = threadIdx.x; p < L.k; p += blockDim.x) {
        const int32_t c = tables_sum(tabs, L.k, p);
        if (c > 0 && p != ps) {
            const unsigned long long key = part_key(c, p);
            best = key > best ? key : best;
        }
    }
    __syncthreads();
    tables_clear(tabs, L.k);
    best = block_max_u64(best, reinterpret_cast<unsigned long long *>(red));
    if (threadIdx.x == 0) {
        int32_t F = kNoneGain, pd = -1;
        bool inX = false;
        if (best) {
            pd = key_part(best);
            F = key_conn(best) - conn_s;
            inX = first_filter(F, conn_s, L.cq16, L.abl);
        }
        nexam += 1;
        degexam += end - beg;
        if (inX) {
            L.prio[v] = F;
            L.nxt[v] = nxt_pack(ps, pd);
            L.listX[L.g.n - 1 - atomicAdd(&L.ctl->nXh, 1)] = v;   // hub region, spread over the next phase's blocks
            degx += end - beg;
        }
        if (ex.pd) { ex.pd[v] = pd >= 0 ? pd : ps; ex.gain[v] = F; }
    }
}

// One long row of step 1, by a whole warp: conn(v, .) in the warp's dense
// table, which is all-zero between rows (the read pass clears every entry it
// finds set, and meets each distinct part once).
template <bool EW>
__device__ __forceinline__ void lp_select_row(const Level &L, LpExport ex, int32_t v, int32_t *tab, Appender &xapp,
                                              long long &nexam, long long &degexam, long long &degx) {
    const DGraph &g = L.g;
    const unsigned lane = lane_id();
    int32_t ps = L.part[v];
    int32_t F = kNoneGain, pd = -1;
    bool inX = false;
    int64_t beg = ld_xadj(g.xadj, v), end = ld_xadj(g.xadj, (int64_t)v + 1);
    row_to_table<EW>(L, beg + lane, end, 32, tab);
    __syncwarp();
    int32_t conn_s = tab[ps];
    __syncwarp();
    unsigned long long best = 0;
    // read (and clear) the k entries of the table: at most k / 32 shared
    // loads a lane, cheaper than gathering the row's parts a second time
    for (int p = lane; p < L.k; p += 32) {
        const int32_t c = tab[p];
        if (c != 0) {
            tab[p] = 0;
            if (p != ps) {
                const unsigned long long key = part_key(c, p);
                best = key > best ? key : best;
            }
        }
    }
    __syncwarp();
    best = warp_max_u64(best);
    if (best) {
        pd = key_part(best);
        F = key_conn(best) - conn_s;
        inX = first_filter(F, conn_s, L.cq16, L.abl);
    }
    if (lane == 0) {
        nexam += 1;
        degexam += end - beg;
        if (inX) {
            L.prio[v] = F;
            L.nxt[v] = nxt_pack(ps, pd);
            degx += end - beg;
        }
        if (ex.pd) { ex.pd[v] = pd >= 0 ? pd : ps; ex.gain[v] = F; }
    }
    xapp.add(lane == 0 && inX, v);   // the block's X staging: no global atomic per row
}

// Step 1 (Alg. 4 first loop, Eq. for P_d, Eq. gainconn_filter) over the work
// list.  Rows of <= 16 entries: one thread per vertex, the row preloaded into
// registers so all its loads are in flight together; longer rows are staged
// for the block's warps.  prio holds F only for members of X; every other
// entry stays kNoneGain (reset after the afterburner).
template <bool EW>
__device__ inline void ph_lp_select(const Level &L, LpExport ex, Grid G, char *arena) {
    __shared__ long long red[40];
    Ctl *ctl = L.ctl;
    const int32_t nbig = ctl->nbig;
    const Deal dl(ctl->nW, G, nbig > 0);
    if (!dl.live(0)) return;
    int32_t *a32 = reinterpret_cast<int32_t *>(arena);
    JET_APPENDER(xapp, a32, kListCap);
    JET_APPENDER(bigs, a32 + kListCap, kBigCap);
    int32_t *tab = a32 + kListCap + kBigCap + (threadIdx.x >> 5) * L.k;
    if (nbig > 0) {
        for (int i = threadIdx.x; i < (int)(blockDim.x >> 5) * L.k; i += blockDim.x) a32[kListCap + kBigCap + i] = 0;
        __syncthreads();
    }
    const DGraph g = L.g;
    long long nexam = 0, degexam = 0, degx = 0;
    auto big_row = [&](int32_t v) { lp_select_row<EW>(L, ex, v, tab, xapp, nexam, degexam, degx); };
    auto hub_row = [&](int32_t v) {
        lp_select_block_row<EW>(L, ex, v, a32 + kListCap + kBigCap, red, nexam, degexam, degx);
    };
    for (int64_t p = 0; dl.live(p); ++p) {
        const int64_t i = dl.entry(p);
        bool inX = false, big = false;
        int32_t v = -1;
        if (i < dl.len) {
            v = L.listW[i];
            int64_t beg = ld_xadj(g.xadj, v), end = ld_xadj(g.xadj, (int64_t)v + 1);
            int d = (int)(end - beg);
            int32_t ps = L.part[v];
            if (d > kSmallDeg) {
                big = true;
            } else {
                nexam += 1;
                degexam += d;
                int32_t F = kNoneGain, pd = -1;
                int32_t pp[kSmallDeg], ww[kSmallDeg];
#pragma unroll
                for (int t = 0; t < kSmallDeg; ++t) {
                    if (t < d) {
                        pp[t] = L.part[__ldg(g.adj + beg + t)];
                        ww[t] = edge_w<EW>(g, beg + t);
                    } else {
                        pp[t] = -1; ww[t] = 0;
                    }
                }
                int32_t conn_s = 0;
#pragma unroll
                for (int t = 0; t < kSmallDeg; ++t) conn_s += (pp[t] == ps) ? ww[t] : 0;
                unsigned long long best = 0;
#pragma unroll
                for (int t = 0; t < kSmallDeg; ++t) {
                    if (t < d && pp[t] != ps) {
                        int32_t c = 0;
#pragma unroll
                        for (int u = 0; u < kSmallDeg; ++u) c += (pp[u] == pp[t]) ? ww[u] : 0;
                        unsigned long long key = part_key(c, pp[t]);
                        best = key > best ? key : best;
                    }
                }
                if (best) {
                    pd = key_part(best);
                    F = key_conn(best) - conn_s;
                    inX = first_filter(F, conn_s, L.cq16, L.abl);
                }
                if (inX) {
                    L.prio[v] = F;
                    L.nxt[v] = nxt_pack(ps, pd);
                    degx += d;
                }
                if (ex.pd) { ex.pd[v] = pd >= 0 ? pd : ps; ex.gain[v] = F; }
            }
        }
        xapp.add(inX, v);
        bigs.add(big, v);
        // room for this pass's adds and a whole drain of warp rows (each of
        // which may add its vertex)
        xapp.flush(&ctl->nX, L.listX, false, 1 + kBigCap / (int)blockDim.x);
        bigs.drain(false, g.xadj, big_row, hub_row, L.hub_deg);
    }
    xapp.flush(&ctl->nX, L.listX, true);
    bigs.drain(true, g.xadj, big_row, hub_row, L.hub_deg);
    xapp.flush(&ctl->nX, L.listX, true);
    flush_counter(&ctl->nexam, nexam, red);
    flush_counter(&ctl->degexam, degexam, red);
    flush_counter(&ctl->degx, degx, red);
}

// Step 2: afterburner (Alg. 4 second loop, ord of Sec. 4.1.1) and the second
// filter M = {v in X : F2 >= 0}.  A neighbour u counts in its destination
// part when it precedes v in ord (higher F, ties to the lower id).
// F2 share of the entries first, first + step, ... < end of v's row (batched
// as row_to_table): a neighbour counts at its destination when it precedes
// v in ord; its move is loaded only for the neighbours that take it.
template <bool EW, int U = kRowBatch>
__device__ __forceinline__ long long afterburn_row(const Level &L, int32_t v, int32_t Fv, int32_t pd, int32_t ps,
                                                   int64_t first, int64_t end, int64_t step) {
    const DGraph &g = L.g;
    long long f2 = 0;
    for (int64_t j0 = first; j0 < end; j0 += U * step) {
        int32_t u[U], w[U], pu[U], fu[U];
#pragma unroll
        for (int q = 0; q < U; ++q) {
            const int64_t j = j0 + q * step;
            u[q] = j < end ? ld_stream(g.adj + j) : -1;
            w[q] = j < end ? edge_w_stream<EW>(g, j) : 0;
        }
#pragma unroll
        for (int q = 0; q < U; ++q) {
            pu[q] = u[q] >= 0 ? L.part[u[q]] : -1;
            fu[q] = u[q] >= 0 ? L.prio[u[q]] : kNoneGain;
        }
#pragma unroll
        for (int q = 0; q < U; ++q)
            if (u[q] >= 0 && (fu[q] > Fv || (fu[q] == Fv && u[q] < v))) pu[q] = nxt_to(L.nxt[u[q]]);
#pragma unroll
        for (int q = 0; q < U; ++q) f2 += pu[q] == pd ? w[q] : (pu[q] == ps ? -w[q] : 0);
    }
    return f2;
}

// One hub row of step 2 by the whole block.
template <bool EW>
__device__ __forceinline__ void afterburn_block_row(const Level &L, LpExport ex, int32_t v, int32_t it, long long *red) {
    const int32_t Fv = L.prio[v], pd = nxt_to(L.nxt[v]), ps = L.part[v];
    const int64_t beg = ld_xadj(L.g.xadj, v), end = ld_xadj(L.g.xadj, (int64_t)v + 1);
    long long f2 = afterburn_row<EW, kHubBatch>(L, v, Fv, pd, ps, beg + threadIdx.x, end, blockDim.x);
    f2 = block_sum_i64(f2, red);
    if (threadIdx.x == 0) {
        if (ex.f2) ex.f2[v] = (int32_t)f2;
        if (f2 >= 0) {
            L.mstamp[v] = it;
            L.listM[L.g.n - 1 - atomicAdd(&L.ctl->nMh, 1)] = v;   // hub region
        }
    }
}

template <bool EW>
__device__ inline void ph_afterburn(const Level &L, LpExport ex, Grid G, char *arena) {
    __shared__ long long red[40];
    Ctl *ctl = L.ctl;
    const int32_t it = ctl->it, nX = ctl->nX, nXh = ctl->nXh;   // one round trip
    const bool full_ab = !(L.abl & (ABL_NO_AFTERBURN | ABL_BASELINE_LP));
    // hub rows of X, one block each, dealt round-robin over the blocks
    for (int32_t h = G.bid; h < nXh; h += G.nb) {
        const int32_t v = L.listX[L.g.n - 1 - h];
        if (full_ab) {
            afterburn_block_row<EW>(L, ex, v, it, red);
        } else if (threadIdx.x == 0) {
            L.mstamp[v] = it;
            L.listM[L.g.n - 1 - atomicAdd(&ctl->nMh, 1)] = v;
        }
    }
    const Deal dl(nX, G, true);
    if (!dl.live(0)) return;
    int32_t *a32 = reinterpret_cast<int32_t *>(arena);
    JET_APPENDER(mapp, a32, kListCap);
    JET_APPENDER(bigs, a32 + kListCap, kBigCap);
    const bool full = !(L.abl & (ABL_NO_AFTERBURN | ABL_BASELINE_LP));
    const unsigned lane = lane_id();
    auto big_row = [&](int32_t v) {
        int32_t Fv = L.prio[v], pd = nxt_to(L.nxt[v]), ps = L.part[v];
        int64_t beg = ld_xadj(L.g.xadj, v), end = ld_xadj(L.g.xadj, (int64_t)v + 1);
        int32_t f2 = (int32_t)afterburn_row<EW>(L, v, Fv, pd, ps, beg + lane, end, 32);
        f2 = warp_sum_i32(f2);
        if (lane == 0) {
            if (ex.f2) ex.f2[v] = f2;
            if (f2 >= 0) L.mstamp[v] = it;
        }
        mapp.add(lane == 0 && f2 >= 0, v);   // the block's M staging: no global atomic per row
    };
    auto hub_row = [&](int32_t v) { afterburn_block_row<EW>(L, ex, v, it, red); };
    for (int64_t p = 0; dl.live(p); ++p) {
        const int64_t i = dl.entry(p);
        bool inM = false, big = false;
        int32_t v = -1;
        if (i < dl.len) {
            v = L.listX[i];
            if (!full) {
                inM = true;
            } else {
                int64_t beg = ld_xadj(L.g.xadj, v);
                int d = (int)(ld_xadj(L.g.xadj, (int64_t)v + 1) - beg);
                if (d > kSmallDeg) {
                    big = true;
                } else {
                    int32_t Fv = L.prio[v], pd = nxt_to(L.nxt[v]), ps = L.part[v];
                    int32_t uu[kSmallDeg], ww[kSmallDeg];
#pragma unroll
                    for (int t = 0; t < kSmallDeg; ++t) {
                        uu[t] = t < d ? __ldg(L.g.adj + beg + t) : -1;
                        ww[t] = t < d ? edge_w<EW>(L.g, beg + t) : 0;
                    }
                    int32_t f2 = 0;
#pragma unroll
                    for (int t = 0; t < kSmallDeg; ++t) {
                        if (t < d) {
                            int32_t u = uu[t];
                            int32_t pu = L.part[u];
                            const int32_t fu = L.prio[u];
                            const int32_t nu = L.nxt[u];
                            if (fu > Fv || (fu == Fv && u < v)) pu = nxt_to(nu);
                            f2 += pu == pd ? ww[t] : (pu == ps ? -ww[t] : 0);
                        }
                    }
                    inM = f2 >= 0;
                    if (ex.f2) ex.f2[v] = f2;
                }
            }
            if (inM) L.mstamp[v] = it;
        }
        mapp.add(inM, v);
        bigs.add(big, v);
        // room for this pass's adds and a whole drain of warp rows
        mapp.flush(&ctl->nM, L.listM, false, 1 + kBigCap / (int)blockDim.x);
        bigs.drain(false, L.g.xadj, big_row, hub_row, L.hub_deg);
    }
    mapp.flush(&ctl->nM, L.listM, true);
    bigs.drain(true, L.g.xadj, big_row, hub_row, L.hub_deg);
    mapp.flush(&ctl->nM, L.listM, true);
}

// ---------------------------------------------------------------------------
// Apply M (Alg. 3 updatePartsAndDS) and commit it: exact cut change, part
// weights, neighbour counts ext, P_s[v] <- P_d[v]; Jetlp movers are locked
// for the next Jetlp (Sec. 4.1.3) and the priorities of X go back to
// kNoneGain.  A neighbour that moves too is recognised by its stamp and its
// old part read from nxt, never from part[] (which the commit overwrites);
// for an edge with both ends moving the smaller id accounts for the cut.
// ---------------------------------------------------------------------------
// Effect of v's move a -> b over the entries first, first + step, ... < end
// of its row, batched as row_to_table: the stamps of a batch are loaded
// together, then the move or the part of each neighbour, whichever it needs.
// A neighbour that stays gets its ext[] updated; c receives the cut change
// (an edge whose ends both move counts once, at the smaller id), ne the
// neighbours in other parts after the move.
template <bool EW, int U = kRowBatch>
__device__ __forceinline__ void apply_row(const Level &L, int32_t v, int32_t a, int32_t b, int32_t it, int64_t first,
                                          int64_t end, int64_t step, long long &c, long long &ne) {
    const DGraph &g = L.g;
    for (int64_t j0 = first; j0 < end; j0 += U * step) {
        int32_t u[U], w[U], x[U];
        bool mu[U];
#pragma unroll
        for (int q = 0; q < U; ++q) {
            const int64_t j = j0 + q * step;
            u[q] = j < end ? ld_stream(g.adj + j) : -1;
            w[q] = j < end ? edge_w_stream<EW>(g, j) : 0;
        }
#pragma unroll
        for (int q = 0; q < U; ++q) mu[q] = u[q] >= 0 && L.mstamp[u[q]] == it;
#pragma unroll
        for (int q = 0; q < U; ++q) x[q] = u[q] < 0 ? 0 : (mu[q] ? L.nxt[u[q]] : L.part[u[q]]);
#pragma unroll
        for (int q = 0; q < U; ++q) {
            if (u[q] < 0) continue;
            const int32_t pu = mu[q] ? nxt_from(x[q]) : x[q];
            const int32_t pn = mu[q] ? nxt_to(x[q]) : x[q];
            const int32_t diff = (int)(pn != b) - (int)(pu != a);
            ne += pn != b;
            if (!mu[q]) {
                if (diff) atomicAdd(&L.ext[u[q]], diff);
                c += (long long)w[q] * diff;
            } else if (u[q] > v) {
                c += (long long)w[q] * diff;   // an edge whose ends both move counts at the smaller id
            }
        }
    }
}

// The same over a short row (at most kSmallDeg entries, one thread), in
// batches of U neighbours whose stamps, packed moves and parts are loaded
// together before any of them is updated: a batch costs one round trip,
// where an update of ext[] between two neighbours would hold the next
// neighbour's loads behind it.
template <bool EW, int U = kSmallDeg / 2>
__device__ __forceinline__ void apply_short_row(const Level &L, int32_t v, int32_t a, int32_t b, int32_t it,
                                                int64_t beg, int d, long long &c, long long &ne) {
    const DGraph &g = L.g;
#pragma unroll
    for (int t0 = 0; t0 < kSmallDeg; t0 += U) {
        if (t0 >= d) break;
        int32_t u[U], w[U], ms[U], x[U], p[U];
#pragma unroll
        for (int q = 0; q < U; ++q) {
            const int t = t0 + q;
            u[q] = t < d ? __ldg(g.adj + beg + t) : -1;
            w[q] = t < d ? edge_w<EW>(g, beg + t) : 0;
        }
#pragma unroll
        for (int q = 0; q < U; ++q) {
            ms[q] = u[q] >= 0 ? L.mstamp[u[q]] : 0;
            x[q] = u[q] >= 0 ? L.nxt[u[q]] : 0;
            p[q] = u[q] >= 0 ? L.part[u[q]] : 0;
        }
#pragma unroll
        for (int q = 0; q < U; ++q) {
            if (u[q] < 0) continue;
            const bool mu = ms[q] == it;
            const int32_t pu = mu ? nxt_from(x[q]) : p[q];
            const int32_t pn = mu ? nxt_to(x[q]) : p[q];
            const int32_t diff = (int)(pn != b) - (int)(pu != a);
            ne += pn != b;
            if (!mu) {
                if (diff) atomicAdd(&L.ext[u[q]], diff);
                c += (long long)w[q] * diff;
            } else if (u[q] > v) {
                c += (long long)w[q] * diff;   // an edge whose ends both move counts at the smaller id
            }
        }
    }
}

// One hub row of the apply phase by the whole block.
template <bool EW>
__device__ __forceinline__ void apply_block_row(const Level &L, int32_t v, int32_t it, bool lp, long long *red,
                                                long long &dc, long long &dm) {
    const int32_t x = L.nxt[v];
    const int32_t a = nxt_from(x), b = nxt_to(x);
    const int64_t beg = ld_xadj(L.g.xadj, v), end = ld_xadj(L.g.xadj, (int64_t)v + 1);
    long long c = 0, ne = 0;
    apply_row<EW, kHubBatch>(L, v, a, b, it, beg + threadIdx.x, end, blockDim.x, c, ne);
    c = block_sum_i64(c, red);
    ne = block_sum_i64(ne, red);
    if (threadIdx.x == 0) {
        dc += c;
        dm += end - beg;
        L.ext[v] = (int32_t)ne;
        L.part[v] = b;
        if (lp) L.lstamp[v] = it;
    }
}

template <bool EW>
__device__ inline void ph_apply(const Level &L, Grid G, char *arena) {
    __shared__ long long red[40];
    Ctl *ctl = L.ctl;
    const int32_t kind = ctl->mode, nM = ctl->nM, nX = ctl->nX, it = ctl->it, nMh = ctl->nMh, nXh = ctl->nXh;
    if (kind == MODE_DONE) return;
    const bool lp = kind == MODE_LP;
    long long *shpw = reinterpret_cast<long long *>(arena);
    int32_t *stage = reinterpret_cast<int32_t *>(arena + align16((size_t)L.k * 8));
    for (int i = threadIdx.x; i < L.k; i += blockDim.x) shpw[i] = 0;
    JET_APPENDER(bigs, stage, kBigCap);
    const unsigned lane = lane_id();
    long long dc = 0, dm = 0;
    auto big_row = [&](int32_t v) {
        int32_t x = L.nxt[v];
        int32_t a = nxt_from(x), b = nxt_to(x);
        int64_t beg = ld_xadj(L.g.xadj, v), end = ld_xadj(L.g.xadj, (int64_t)v + 1);
        long long c = 0, ne = 0;
        apply_row<EW>(L, v, a, b, it, beg + lane, end, 32, c, ne);
        c = warp_sum_i64(c);
        ne = warp_sum_i64(ne);
        if (lane == 0) {
            dc += c;
            dm += end - beg;
            L.ext[v] = (int32_t)ne;
            L.part[v] = b;
            if (lp) L.lstamp[v] = it;
        }
    };
    auto hub_row = [&](int32_t v) { apply_block_row<EW>(L, v, it, lp, red, dc, dm); };
    const Deal dl(nM, G, true);
    for (int64_t p = 0; dl.live(p); ++p) {
        const int64_t i = dl.entry(p);
        bool big = false;
        int32_t v = -1;
        if (i < dl.len) {
            v = L.listM[i];
            int32_t x = L.nxt[v];
            int32_t a = nxt_from(x), b = nxt_to(x);
            long long wv = L.g.vw[v];
            atomicAdd(reinterpret_cast<unsigned long long *>(&shpw[a]), (unsigned long long)(-wv));
            atomicAdd(reinterpret_cast<unsigned long long *>(&shpw[b]), (unsigned long long)wv);
            int64_t beg = ld_xadj(L.g.xadj, v);
            int d = (int)(ld_xadj(L.g.xadj, (int64_t)v + 1) - beg);
            if (d > kSmallDeg) {
                big = true;
            } else {
                long long c = 0, ne = 0;
                apply_short_row<EW>(L, v, a, b, it, beg, d, c, ne);
                dc += c;
                L.ext[v] = (int32_t)ne;
                L.part[v] = b;
                if (lp) L.lstamp[v] = it;
                dm += d;
            }
        }
        bigs.add(big, v);
        bigs.drain(false, L.g.xadj, big_row, hub_row, L.hub_deg);
    }
    bigs.drain(true, L.g.xadj, big_row, hub_row, L.hub_deg);
    // hub rows of M, one block each, dealt round-robin over the blocks
    for (int32_t h = G.bid; h < nMh; h += G.nb) {
        const int32_t v = L.listM[L.g.n - 1 - h];
        if (threadIdx.x == 0) {
            const int32_t x = L.nxt[v];
            const long long wv = L.g.vw[v];
            atomicAdd(reinterpret_cast<unsigned long long *>(&shpw[nxt_from(x)]), (unsigned long long)(-wv));
            atomicAdd(reinterpret_cast<unsigned long long *>(&shpw[nxt_to(x)]), (unsigned long long)wv);
        }
        apply_block_row<EW>(L, v, it, lp, red, dc, dm);
    }
    if (lp) {
        const int64_t stride = (int64_t)G.nb * blockDim.x;
        for (int64_t i = (int64_t)G.bid * blockDim.x + threadIdx.x; i < nX; i += stride) L.prio[L.listX[i]] = kNoneGain;
        for (int64_t i = (int64_t)G.bid * blockDim.x + threadIdx.x; i < nXh; i += stride)
            L.prio[L.listX[L.g.n - 1 - i]] = kNoneGain;
    }
    dc = block_sum_i64(dc, red);
    dm = block_sum_i64(dm, red);
    if (threadIdx.x == 0 && dc) atomic_add_i64(&ctl->dcut, dc);
    if (threadIdx.x == 0 && dm) atomic_add_i64(&ctl->degm, dm);
    __syncthreads();
    for (int i = threadIdx.x; i < L.k; i += blockDim.x)
        if (shpw[i]) atomic_add_i64(&L.pw[i], shpw[i]);
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Rebalancing (Alg. 5 Jetrw, Sec. 4.2.2 Jetrs)
// ---------------------------------------------------------------------------
__device__ __forceinline__ int32_t random_B(const Level &L, int32_t v, int32_t it, int32_t nB) {
    uint64_t h = splitmix64(L.seed ^ (0x9E3779B97F4A7C15ULL * (uint64_t)(it + 1)) ^ (uint64_t)(uint32_t)v);
    return L.Bs[h % (uint64_t)nB];
}

// Adds w (a vertex weight, or 0) into bucketw[key] with one atomic per
// distinct key in the warp: the lanes of one key reduce their weights with
// one warp reduction (their sum is below 2^31: the library refuses graphs
// whose total vertex weight is not).
__device__ __forceinline__ void bucket_add(const Level &L, int32_t key, long long w) {
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    const int s = __reduce_add_sync(peers, (int)w);
    if (key >= 0 && (int)lane_id() == __ffs(peers) - 1) atomic_add_i64(&L.bucketw[key], (long long)s);
}

// Per-block slot buckets in shared memory when nA * kSlots keys fit.
struct SmemBuckets {
    long long *b;
    int32_t nkeys;
    bool on;
    __device__ __forceinline__ void init(const Level &L, long long *buf) {
        b = buf;
        nkeys = L.ctl->nA * kSlots;
        on = nkeys <= kSmemBuckets;
        if (on)
            for (int i = threadIdx.x; i < nkeys; i += blockDim.x) b[i] = 0;
        __syncthreads();
    }
    __device__ __forceinline__ void add(const Level &L, int32_t key, long long w) {   // all lanes call
        if (on) {
            if (key >= 0) atomicAdd(reinterpret_cast<unsigned long long *>(&b[key]), (unsigned long long)w);
        } else {
            bucket_add(L, key, w);
        }
    }
    __device__ __forceinline__ void add_one(const Level &L, int32_t key, long long w) {   // one thread
        if (on) atomicAdd(reinterpret_cast<unsigned long long *>(&b[key]), (unsigned long long)w);
        else atomic_add_i64(&L.bucketw[key], w);
    }
    __device__ __forceinline__ void flush(const Level &L) {
        if (!on) return;
        __syncthreads();
        for (int i = threadIdx.x; i < nkeys; i += blockDim.x)
            if (b[i]) atomic_add_i64(&L.bucketw[i], b[i]);
        __syncthreads();
    }
};

// Step 0 (Alg. 5 first loop): the candidates are the vertices of oversized
// parts allowed to leave (heavy-vertex rule of Sec. 4.2.2: stay if vwgt >
// 1.5 (w_p - opt)).  A candidate with no neighbour in another part (ext == 0)
// touches no part of B (its own part is oversized): conn(v, P_s) is its
// weighted degree, Jetrw sends it to a random part of B and both losses
// equal that degree — it is finished here without reading its row.  The
// others are listed for the row phase.
template <bool STRONG>
__device__ inline void ph_rb_scan(const Level &L, Grid G, char *arena) {
    disarm_loop(L, G);
    __shared__ long long red[40];
    Ctl *ctl = L.ctl;
    const int32_t it = ctl->it, nB = ctl->nB;   // loaded before the barriers of the set-up below
    const int64_t opt = ctl->opt;
    SmemBuckets sb;
    sb.init(L, reinterpret_cast<long long *>(arena));
    JET_APPENDER(wapp, reinterpret_cast<int32_t *>(arena + kSmemBuckets * 8), kScanCap);
    const int64_t n = L.g.n, nq = (n + 3) / 4;
    const bool vec = (reinterpret_cast<uintptr_t>(L.part) & 15) == 0;
    long long ncand = 0, nlist = 0;
    for (int64_t q0 = (int64_t)G.bid * blockDim.x; q0 < nq; q0 += (int64_t)G.nb * blockDim.x) {
        int64_t q = q0 + threadIdx.x;
        int64_t v0 = 4 * q;
        int32_t pp[4] = {-1, -1, -1, -1};
        if (q < nq) {
            if (vec && v0 + 3 < n) {
                int4 x = *reinterpret_cast<const int4 *>(L.part + v0);
                pp[0] = x.x; pp[1] = x.y; pp[2] = x.z; pp[3] = x.w;
            } else {
#pragma unroll
                for (int i = 0; i < 4; ++i) pp[i] = v0 + i < n ? L.part[v0 + i] : -1;
            }
        }
        // all loads of the four vertices are issued before any decision
        int32_t aa[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) aa[i] = (pp[i] >= 0 && nB > 0) ? L.aidx[pp[i]] : -1;
        long long pwv[4];
        int32_t vwv[4], ex[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            bool c = aa[i] >= 0;
            pwv[i] = c ? L.pw[pp[i]] : 0;
            vwv[i] = c ? L.g.vw[v0 + i] : 0;
            ex[i] = c ? L.ext[v0 + i] : 0;
        }
        bool cand[4];
        int32_t wd[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            cand[i] = aa[i] >= 0 && 2LL * vwv[i] <= 3LL * (pwv[i] - opt);
            wd[i] = (cand[i] && ex[i] == 0) ? L.wdeg[v0 + i] : 0;
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            int32_t v = (int32_t)(v0 + i);
            int32_t key = -1;
            long long wv = 0;
            bool listed = cand[i] && ex[i] != 0;
            if (cand[i]) {
                ncand += 1;
                if (!listed) {
                    int32_t loss = wd[i];
                    if constexpr (!STRONG) L.nxt[v] = nxt_pack(pp[i], random_B(L, v, it, nB));
                    key = aa[i] * kSlots + slot_of(loss);
                    wv = vwv[i];
                    if (L.rbloss) L.rbloss[v] = loss;
                }
            }
            if (pp[i] >= 0 && !listed) L.key[v] = key;
            sb.add(L, key, wv);
            wapp.add(listed, v);
            nlist += listed;
        }
        wapp.flush(&ctl->nW, L.listW, false, 4);
    }
    wapp.flush(&ctl->nW, L.listW, true, 4);
    sb.flush(L);
    flush_counter(&ctl->ncand, ncand, red);
    flush_counter(&ctl->nbnd, nlist, red);
}

// One long candidate row of step 1, by a whole warp (dense per-warp table as
// in the Jetlp select).
template <bool EW, bool STRONG>
__device__ __forceinline__ void rb_cand_row(const Level &L, int32_t v, int32_t *tab, int32_t it, int32_t nB,
                                            SmemBuckets &sb, long long &degrows) {
    const DGraph &g = L.g;
    const unsigned lane = lane_id();
    int32_t ps = L.part[v];
    int32_t a = L.aidx[ps];
    int64_t beg = ld_xadj(g.xadj, v), end = ld_xadj(g.xadj, (int64_t)v + 1);
    row_to_table<EW>(L, beg + lane, end, 32, tab);
    __syncwarp();
    int32_t conn_s = tab[ps];
    __syncwarp();
    unsigned long long best = 0;
    long long S = 0;
    int32_t cnt = 0;
    auto take = [&](int32_t c, int32_t p) {   // part p met once with connectivity c > 0
        if (L.inB[p]) {
            if constexpr (!STRONG) {
                unsigned long long k2 = part_key(c, p);
                best = k2 > best ? k2 : best;
            } else {
                S += c; cnt += 1;
            }
        }
    };
    // read (and clear) the k entries of the table, as in lp_select_row
    for (int p = lane; p < L.k; p += 32) {
        const int32_t c = tab[p];
        if (c != 0) {
            tab[p] = 0;
            take(c, p);
        }
    }
    __syncwarp();
    int32_t loss;
    if constexpr (!STRONG) {
        best = warp_max_u64(best);
        int32_t dest, cd;
        if (best) { dest = key_part(best); cd = key_conn(best); }
        else { dest = random_B(L, v, it, nB); cd = 0; }
        if (lane == 0) L.nxt[v] = nxt_pack(ps, dest);
        loss = conn_s - cd;
    } else {
        S = warp_sum_i64(S);
        cnt = warp_sum_i32(cnt);
        loss = conn_s - (cnt > 0 ? (int32_t)(S / cnt) : 0);
    }
    if (lane == 0) {
        int32_t key = a * kSlots + slot_of(loss);
        L.key[v] = key;
        if (L.rbloss) L.rbloss[v] = loss;
        sb.add_one(L, key, (long long)g.vw[v]);
        degrows += end - beg;
    }
}

// One hub row of the rebalancing candidates by the whole block.
template <bool EW, bool STRONG>
__device__ __forceinline__ void rb_cand_block_row(const Level &L, int32_t v, int32_t *tabs, long long *red, int32_t it,
                                                  int32_t nB, SmemBuckets &sb, long long &degrows) {
    const DGraph &g = L.g;
    const int32_t ps = L.part[v];
    const int32_t a = L.aidx[ps];
    const int64_t beg = ld_xadj(g.xadj, v), end = ld_xadj(g.xadj, (int64_t)v + 1);
    int32_t *tab = tabs + (threadIdx.x >> 5) * L.k;
    row_to_table<EW, kHubBatch>(L, beg + threadIdx.x, end, blockDim.x, tab);
    __syncthreads();
    const int32_t conn_s = tables_sum(tabs, L.k, ps);
    unsigned long long best = 0;
    long long S = 0, cnt = 0;
    for (int p = threadIdx.x; p < L.k; p += blockDim.x) {
        const int32_t c = tables_sum(tabs, L.k, p);
        if (c > 0 && L.inB[p]) {
            if constexpr (!STRONG) {
                const unsigned long long k2 = part_key(c, p);
                best = k2 > best ? k2 : best;
            } else {
                S += c;
                cnt += 1;
            }
        }
    }
    __syncthreads();
    tables_clear(tabs, L.k);
    int32_t loss = 0;
    if constexpr (!STRONG) {
        best = block_max_u64(best, reinterpret_cast<unsigned long long *>(red));
        if (threadIdx.x == 0) {
            int32_t dest, cd;
            if (best) { dest = key_part(best); cd = key_conn(best); }
            else { dest = random_B(L, v, it, nB); cd = 0; }
            L.nxt[v] = nxt_pack(ps, dest);
            loss = conn_s - cd;
        }
    } else {
        S = block_sum_i64(S, red);
        cnt = block_sum_i64(cnt, red);
        loss = conn_s - (cnt > 0 ? (int32_t)(S / cnt) : 0);
    }
    if (threadIdx.x == 0) {
        const int32_t key = a * kSlots + slot_of(loss);
        L.key[v] = key;
        if (L.rbloss) L.rbloss[v] = loss;
        sb.add_one(L, key, (long long)g.vw[v]);
        degrows += end - beg;
    }
}

// Step 1 for the listed candidates: Jetrw destination (best-connected part of
// B, lowest id on ties, else a random one) and loss, or the Jetrs loss
// (Sec. 4.2.2), then the slot bucket.  Short rows one thread each, long rows
// staged for the block's warps.
template <bool EW, bool STRONG>
__device__ inline void ph_rb_cand(const Level &L, Grid G, char *arena) {
    __shared__ long long red[40];
    Ctl *ctl = L.ctl;
    const int32_t nB = ctl->nB, nbig = ctl->nbig, it = ctl->it;   // one round trip
    const Deal dl(ctl->nW, G, nbig > 0);
    if (!dl.live(0)) return;
    SmemBuckets sb;
    sb.init(L, reinterpret_cast<long long *>(arena));
    int32_t *a32 = reinterpret_cast<int32_t *>(arena + kSmemBuckets * 8);
    JET_APPENDER(bigs, a32, kBigCap);
    int32_t *tab = a32 + kBigCap + (threadIdx.x >> 5) * L.k;
    if (nbig > 0) {
        for (int i = threadIdx.x; i < (int)(blockDim.x >> 5) * L.k; i += blockDim.x) a32[kBigCap + i] = 0;
        __syncthreads();
    }
    const DGraph g = L.g;
    long long degrows = 0;
    auto big_row = [&](int32_t v) { rb_cand_row<EW, STRONG>(L, v, tab, it, nB, sb, degrows); };
    auto hub_row = [&](int32_t v) { rb_cand_block_row<EW, STRONG>(L, v, a32 + kBigCap, red, it, nB, sb, degrows); };
    for (int64_t p = 0; dl.live(p); ++p) {
        const int64_t i = dl.entry(p);
        int32_t key = -1;
        long long wv = 0;
        bool big = false;
        int32_t v = -1;
        if (i < dl.len) {
            v = L.listW[i];
            int32_t ps = L.part[v];
            int32_t a = L.aidx[ps];
            int64_t beg = ld_xadj(g.xadj, v), end = ld_xadj(g.xadj, (int64_t)v + 1);
            int d = (int)(end - beg);
            if (d > kSmallDeg) {
                big = true;
            } else {
                degrows += d;
                int32_t pp[kSmallDeg], ww[kSmallDeg];
#pragma unroll
                for (int t = 0; t < kSmallDeg; ++t) {
                    if (t < d) {
                        pp[t] = L.part[__ldg(g.adj + beg + t)];
                        ww[t] = edge_w<EW>(g, beg + t);
                    } else {
                        pp[t] = -1; ww[t] = 0;
                    }
                }
                int32_t conn_s = 0;
#pragma unroll
                for (int t = 0; t < kSmallDeg; ++t) conn_s += (pp[t] == ps) ? ww[t] : 0;
                int32_t loss;
                if constexpr (!STRONG) {
                    unsigned long long best = 0;
#pragma unroll
                    for (int t = 0; t < kSmallDeg; ++t) {
                        if (t < d && L.inB[pp[t]]) {
                            int32_t c = 0;
#pragma unroll
                            for (int u = 0; u < kSmallDeg; ++u) c += (pp[u] == pp[t]) ? ww[u] : 0;
                            unsigned long long k2 = part_key(c, pp[t]);
                            best = k2 > best ? k2 : best;
                        }
                    }
                    int32_t dest, cd;
                    if (best) { dest = key_part(best); cd = key_conn(best); }
                    else { dest = random_B(L, v, it, nB); cd = 0; }
                    L.nxt[v] = nxt_pack(ps, dest);
                    loss = conn_s - cd;
                } else {
                    long long S = 0;
                    int32_t c = 0;
#pragma unroll
                    for (int t = 0; t < kSmallDeg; ++t) {
                        if (t < d && L.inB[pp[t]]) {
                            S += ww[t];
                            bool first = true;
#pragma unroll
                            for (int u = 0; u < kSmallDeg; ++u)
                                if (u < t && pp[u] == pp[t]) first = false;
                            c += first ? 1 : 0;
                        }
                    }
                    loss = conn_s - (c > 0 ? (int32_t)(S / c) : 0);
                }
                key = a * kSlots + slot_of(loss);
                wv = g.vw[v];
                if (L.rbloss) L.rbloss[v] = loss;
                L.key[v] = key;
            }
        }
        sb.add(L, key, wv);
        bigs.add(big, v);
        bigs.drain(false, g.xadj, big_row, hub_row, L.hub_deg);
    }
    bigs.drain(true, g.xadj, big_row, hub_row, L.hub_deg);
    sb.flush(L);
    flush_counter(&ctl->degexam, degrows, red);
}

// Step 2 (tail of step 1, one block): per oversized part (one warp each), the
// boundary slot s* where the weight taken so far reaches the excess (Alg. 5
// scan: a candidate is taken while the weight before it is below w_p - L) and
// the weight still to take inside s*.  s* = kSlots means every candidate is
// taken.
__device__ inline void ph_rb_plan(const Level &L) {
    const Ctl *ctl = L.ctl;
    const int32_t nA = ctl->nA;
    const int warps = blockDim.x >> 5;
    const unsigned lane = lane_id();
    constexpr int kBatch = 4;                      // parts per warp whose loads are in flight together
    for (int a0 = threadIdx.x >> 5; a0 < nA; a0 += warps * kBatch) {
        long long tb[kBatch], t32b[kBatch], exb[kBatch];
#pragma unroll
        for (int b = 0; b < kBatch; ++b) {
            const int a = a0 + b * warps;
            tb[b] = a < nA ? ld_gpu(&L.bucketw[a * kSlots + lane]) : 0;    // slots 0..31 on the lanes
            t32b[b] = a < nA ? ld_gpu(&L.bucketw[a * kSlots + 32]) : 0;
            exb[b] = a < nA ? L.excess[a] : 0;
        }
#pragma unroll
        for (int b = 0; b < kBatch; ++b) {
        const int a = a0 + b * warps;
        if (a >= nA) break;
        const long long t = tb[b], t32 = t32b[b];
        long long x = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            long long y = __shfl_up_sync(0xffffffffu, x, o);
            if ((int)lane >= o) x += y;
        }
        const long long ex = exb[b];
        unsigned m = __ballot_sync(0xffffffffu, x >= ex);
        long long tot31 = __shfl_sync(0xffffffffu, x, 31);
        int32_t ss;
        long long need;
        if (m) {
            int s0 = __ffs(m) - 1;
            long long before = __shfl_sync(0xffffffffu, x - t, s0);
            ss = s0;
            need = ex - before;
        } else if (tot31 + t32 >= ex) {
            ss = 32;
            need = ex - tot31;
        } else {
            ss = kSlots;
            need = 0;
        }
        if (lane == 0) { L.sstar[a] = ss; L.need[a] = need; }
        }
    }
}

// Step 3: per tile of blockDim vertices, the weight of each part's
// boundary-slot members (they are taken in vertex order).
__device__ inline void ph_rb_tilehist(const Level &L, Grid G, char *arena) {
    int32_t *h = reinterpret_cast<int32_t *>(arena);
    const int32_t nA = L.ctl->nA;
    for (int64_t t = G.bid; t < L.ntiles; t += G.nb) {
        const int64_t v = t * blockDim.x + threadIdx.x;
        const int32_t kv = v < L.g.n ? L.key[v] : -1;   // in flight with nA and the clearing below
        for (int i = threadIdx.x; i < nA; i += blockDim.x) h[i] = 0;
        __syncthreads();
        if (kv >= 0) {
            int32_t a = kv / kSlots, s = kv - a * kSlots;
            if (s == L.sstar[a]) atomicAdd(&h[a], L.g.vw[v]);
        }
        __syncthreads();
        for (int i = threadIdx.x; i < nA; i += blockDim.x) L.tilehist[t * nA + i] = h[i];
        __syncthreads();
    }
}

// Exclusive scan of each part's tile sums over the tiles (one block per part,
// eight consecutive tiles per thread).
__device__ inline void ph_rb_tilescan(const Level &L, Grid G) {
    __shared__ long long sh[40];
    const int32_t nA = L.ctl->nA;
    const int64_t nt = L.ntiles;
    constexpr int kItems = 8;
    for (int a = G.bid; a < nA; a += G.nb) {
        long long carry = 0;
        for (int64_t t0 = 0; t0 < nt; t0 += (int64_t)blockDim.x * kItems) {
            int64_t tb = t0 + (int64_t)threadIdx.x * kItems;
            long long x[kItems];
            long long s = 0;
#pragma unroll
            for (int i = 0; i < kItems; ++i) {
                x[i] = tb + i < nt ? L.tilehist[(tb + i) * nA + a] : 0;
                s += x[i];
            }
            long long tot = 0;
            long long pre = carry + block_exscan_i64(s, sh, &tot);
#pragma unroll
            for (int i = 0; i < kItems; ++i) {
                if (tb + i < nt) L.tilehist[(tb + i) * nA + a] = (int32_t)pre;
                pre += x[i];
            }
            carry += tot;
        }
    }
}

// Step 4: take the candidates (slot < s*, or slot == s* with the member weight
// before them, in vertex order, below `need`).  Jetrw moves the taken
// vertices to P_d; Jetrs records their weight for the cookie cutter.
template <bool STRONG>
__device__ inline void ph_rb_take(const Level &L, Grid G, char *arena) {
    long long *run = reinterpret_cast<long long *>(arena);
    int32_t *mbuf = reinterpret_cast<int32_t *>(arena + align16((size_t)L.k * 8));
    JET_APPENDER(mapp, mbuf, 2 * (int)blockDim.x);
    __shared__ long long red[40];
    Ctl *ctl = L.ctl;
    const int32_t nA = ctl->nA, it = ctl->it;
    const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
    const unsigned lt_mask = (1u << lane) - 1u;
    for (int64_t tile = G.bid; tile < L.ntiles; tile += G.nb) {
        int64_t vv = tile * blockDim.x + threadIdx.x;
        int32_t kv = -1, a = 0, s = 0;
        if (vv < L.g.n) kv = L.key[vv];
        if (!__syncthreads_or(kv >= 0)) {          // no candidate in this tile
            if constexpr (STRONG) {
                if (vv < L.g.n) L.etaken[vv] = 0;
                if (threadIdx.x == 0) L.tiletaken[tile] = 0;
            }
            continue;
        }
        for (int i = threadIdx.x; i < nA; i += blockDim.x) run[i] = L.tilehist[tile * nA + i];
        __syncthreads();
        if (kv >= 0) { a = kv / kSlots; s = kv - a * kSlots; }
        int32_t ss = kv >= 0 ? L.sstar[a] : 0;
        bool member = kv >= 0 && s == ss;
        long long w = (kv >= 0) ? (long long)L.g.vw[vv] : 0;
        long long mine = 0;
        // ordered prefix over the boundary-slot members, warp after warp
        const unsigned nphase = __syncthreads_or(member) ? (blockDim.x >> 5) : 0u;
        for (unsigned wi = 0; wi < nphase; ++wi) {
            if (warp == wi) {
                int32_t grp = member ? a : -(int32_t)lane - 1;
                unsigned peers = __match_any_sync(0xffffffffu, grp);
                long long pre = 0;
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    long long x = __shfl_sync(0xffffffffu, member ? w : 0LL, j);
                    if ((peers & lt_mask) >> j & 1u) pre += x;
                }
                long long base = member ? run[a] : 0;
                mine = base + pre;
                __syncwarp();
                if (member && (peers >> lane) == 1u) run[a] = mine + w;
            }
            __syncthreads();
        }
        bool taken = kv >= 0 && (s < ss || (member && mine < L.need[a]));
        if constexpr (!STRONG) {
            if (taken) L.mstamp[vv] = it;
            mapp.add(taken, (int32_t)vv);
            mapp.flush(&ctl->nM, L.listM, true);
        } else {
            if (vv < L.g.n) L.etaken[vv] = taken ? w : 0;
            long long tt = block_sum_i64(taken ? w : 0, red);
            if (threadIdx.x == 0) L.tiletaken[tile] = tt;
        }
        __syncthreads();
    }
}

// Jetrs (tail of step 4, one block): exclusive scan of the evicted weight
// over the tiles.
__device__ inline void ph_rb_tiletaken_scan(const Level &L) {
    __shared__ long long sh[40];
    long long carry = 0;
    for (int64_t t0 = 0; t0 < L.ntiles; t0 += blockDim.x) {
        int64_t t = t0 + threadIdx.x;
        long long x = t < L.ntiles ? ld_gpu(&L.tiletaken[t]) : 0;
        long long tot = 0;
        long long ex = block_exscan_i64(x, sh, &tot);
        if (t < L.ntiles) L.tiletaken[t] = carry + ex;
        carry += tot;
    }
}

// Jetrs cookie cutter: evicted vertices in vertex order, destinations B in
// ascending id with capacities sigma - w_b laid end to end; a vertex goes to
// the capacity interval that holds the middle of its weight span.
__device__ inline void ph_rb_cookie(const Level &L, Grid G, char *arena) {
    __shared__ long long sh[40];
    JET_APPENDER(mapp, reinterpret_cast<int32_t *>(arena), 2 * (int)blockDim.x);
    Ctl *ctl = L.ctl;
    const int32_t it = ctl->it, nB = ctl->nB;
    const long long total2 = 2 * L.capC[nB];
    for (int64_t tile = G.bid; tile < L.ntiles; tile += G.nb) {
        int64_t v = tile * blockDim.x + threadIdx.x;
        long long wv = v < L.g.n ? L.etaken[v] : 0;
        if (!__syncthreads_or(wv > 0)) continue;
        long long pre = block_exscan_i64(wv, sh, nullptr) + L.tiletaken[tile];
        int32_t dest = -1;
        if (wv > 0) {
            long long mid2 = 2 * pre + wv;
            if (mid2 < total2) {
                int lo = 0, hi = nB - 1;  // largest b with 2 C_b <= mid2
                while (lo < hi) {
                    int mid = (lo + hi + 1) >> 1;
                    if (2 * L.capC[mid] <= mid2) lo = mid; else hi = mid - 1;
                }
                if (mid2 < 2 * L.capC[lo + 1]) dest = L.Bs[lo];
            }
        }
        bool mv = dest >= 0;
        if (mv) { L.nxt[v] = nxt_pack(L.part[v], dest); L.mstamp[v] = it; }
        mapp.add(mv, (int32_t)v);
        mapp.flush(&ctl->nM, L.listM, true);
    }
}

}  // namespace jet
