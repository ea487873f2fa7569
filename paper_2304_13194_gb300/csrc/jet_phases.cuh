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
//    is read (longer rows, one warp per vertex).
//  * ext[v] (neighbours in other parts) is kept exact by the apply phase, so
//    passes list boundary vertices first and never stream interior rows.
//  * Lists are staged in shared memory and reserved with one atomic per
//    block flush.
//  * Arrays that phases modify (part, prio, nxt, ext, stamps, lists) are read
//    with ordinary loads, never through the non-coherent read-only path, so
//    that the cluster-resident loop sees them after each cluster barrier.
#pragma once

#include "jet_internal.cuh"

namespace jet {

struct Grid {
    int bid;   // rank of this block among the cooperating blocks
    int nb;    // number of cooperating blocks
};

// Control values (counters, mode, part weights) written by other blocks
// before the last kernel boundary or cluster barrier.  Plain loads: the
// barrier's release/acquire order makes the writes visible, while volatile
// (system-scope) loads cost about a microsecond each on a memory system that
// is coherent with the host CPU.
template <class T>
__device__ __forceinline__ T vread(const T *p) { return *p; }

__device__ __forceinline__ Grid launch_grid() { return Grid{(int)blockIdx.x, (int)gridDim.x}; }

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

__device__ __forceinline__ bool ablate_locks(uint32_t abl) { return (abl & (ABL_NO_LOCKS | ABL_BASELINE_LP)) != 0; }

// First filter, Eq. gainconn_filter: -F < floor(c * conn(v,P_s)) or F >= 0
// (ablations: weak afterburner keeps F >= 0, baseline LP keeps F > 0).
__device__ __forceinline__ bool first_filter(int32_t F, int32_t conn_s, int32_t cq16, uint32_t abl) {
    if (abl & ABL_BASELINE_LP) return F > 0;
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

__device__ __forceinline__ bool is_big_row(const DGraph &g, int32_t v) {
    return ld_xadj(g.xadj, (int64_t)v + 1) - ld_xadj(g.xadj, v) > kSmallDeg;
}

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
};

#define JET_APPENDER(name, bufptr, capacity)                    \
    __shared__ int name##_cnt, name##_base;                      \
    Appender name{(bufptr), (capacity), &name##_cnt, &name##_base}; \
    name.init()

// ---------------------------------------------------------------------------
// shared-memory arena per phase (bytes, for blocks of T threads)
// ---------------------------------------------------------------------------
constexpr int kScanCap = 4096;          // list staging of the scan phases
constexpr int kListCap = 2048;          // X / M staging
constexpr int kBigCap = 1024;           // long-row list staging
constexpr int kSmemBuckets = 1024;      // slot buckets aggregated per block when nA * kSlots fits

__host__ __device__ constexpr size_t arena_table(int32_t k, int T) { return (size_t)(T / 32) * (size_t)k * 4; }
__host__ __device__ constexpr size_t arena_max(size_t a, size_t b) { return a > b ? a : b; }
// the largest arena any phase needs
__host__ __device__ constexpr size_t arena_bytes(int32_t k, int T) {
    return arena_max(arena_max(arena_max((size_t)kScanCap * 4, (size_t)(kListCap + kBigCap) * 4),
                               arena_max((size_t)kSmemBuckets * 8 + (size_t)kScanCap * 4, arena_table(k, T))),
                     arena_max((((size_t)k * 8 + 15) & ~size_t(15)) + (size_t)2 * T * 4, (size_t)k * 8));
}

// ---------------------------------------------------------------------------
// controller helpers (one block)
// ---------------------------------------------------------------------------
__device__ inline long long block_max_pw(const int64_t *pw, int32_t k, long long *sh) {
    long long m = 0;
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        long long w = vread(&pw[i]);
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
// capacity prefix of B (Jetrs) and zeroed slot buckets.  Any block size.
__device__ inline void compute_classes(const Level &L, long long *sh) {
    Ctl *ctl = L.ctl;
    long long ca = 0, cb = 0, cc = 0;
    for (int p0 = 0; p0 < L.k; p0 += blockDim.x) {
        int p = p0 + threadIdx.x;
        bool inA = false, inB = false;
        long long w = 0;
        if (p < L.k) {
            w = vread(&L.pw[p]);
            inA = w > ctl->L;
            inB = w <= ctl->sigma;
        }
        long long tA = 0, tB = 0, tC = 0;
        long long ia = ca + block_exscan_i64(inA ? 1 : 0, sh, &tA);
        long long ib = cb + block_exscan_i64(inB ? 1 : 0, sh, &tB);
        long long cap = inB ? (ctl->sigma - w) : 0;
        long long ic = cc + block_exscan_i64(cap, sh, &tC);
        if (p < L.k) {
            L.aidx[p] = inA ? (int32_t)ia : -1;
            L.inB[p] = inB ? 1 : 0;
            if (inA) L.excess[ia] = w - ctl->L;
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
__device__ inline int32_t choose_mode(const Level &L, bool balanced) {
    Ctl *ctl = L.ctl;
    if (ctl->noimp >= L.max_no_improve) return MODE_DONE;
    if (ctl->it >= L.max_iters) { ctl->hit_cap = 1; return MODE_DONE; }
    if (balanced) { ctl->weak = 0; return MODE_LP; }
    if (ctl->weak < L.weak_limit) { ctl->weak += 1; return MODE_RW; }
    return MODE_RS;
}

// End of an iteration (Alg. 3 after updatePartsAndDS), one block: exact cut,
// max part weight, P_best / counters, trace record, next mode, rebalancing
// classes for the next iteration.  Returns the next mode (all threads).
__device__ inline int32_t ph_controller(const Level &L) {
    __shared__ long long sh[40];
    __shared__ int32_t next_mode;
    Ctl *ctl = L.ctl;
    int32_t kind = vread(&ctl->mode);
    if (kind == MODE_DONE) {
        if (threadIdx.x == 0) {
            ctl->copy_best = 0;
            if (L.use_graph) {
                cudaGraphSetConditional((cudaGraphConditionalHandle)L.h_loop, 0u);
                cudaGraphSetConditional((cudaGraphConditionalHandle)L.h_mode, (unsigned)MODE_DONE);
            }
        }
        return MODE_DONE;
    }
    long long maxw = block_max_pw(L.pw, L.k, sh);
    if (threadIdx.x == 0) {
        long long cut = ctl->cut + vread(&ctl->dcut);
        ctl->dcut = 0;
        ctl->cut = cut;
        ctl->maxw = maxw;
        int32_t it = ctl->it;              // index of the iteration just run
        bool bal = maxw <= ctl->L;
        ctl->noimp += 1;
        int32_t copy = 0;
        if (bal) {
            if (!ctl->best_bal || cut < ctl->best_cut) {
                if (!ctl->best_bal || 1000000LL * cut < L.phi_ppm * ctl->best_cut) ctl->noimp = 0;
                ctl->best_cut = cut; ctl->best_maxw = maxw; ctl->best_bal = 1;
                copy = 1;
            }
        } else if (!ctl->best_bal && maxw < ctl->best_maxw) {
            ctl->best_cut = cut; ctl->best_maxw = maxw; ctl->noimp = 0;
            copy = 1;
        }
        ctl->copy_best = copy;
        if (it < kTrace && L.trace) {
            TraceRec r;
            r.kind = kind; r.pad = 0;
            r.nx = (kind == MODE_LP) ? (int64_t)(vread(&ctl->nX) + vread(&ctl->nXb)) : vread(&ctl->ncand);
            r.nm = (int64_t)(vread(&ctl->nM) + vread(&ctl->nMb));
            r.cut = cut; r.maxw = maxw;
            r.degx = vread(&ctl->degx); r.degm = vread(&ctl->degm);
            r.nbnd = vread(&ctl->nbnd); r.nexam = vread(&ctl->nexam); r.degexam = vread(&ctl->degexam);
            L.trace[it] = r;
        }
        if (kind == MODE_LP) ctl->lp_epoch = it;
        ctl->kcount[kind] += 1;
        ctl->it = it + 1;
        ctl->nX = ctl->nXb = ctl->nM = ctl->nMb = 0;
        ctl->nW = ctl->nWb = 0;
        ctl->ncand = 0;
        ctl->degx = ctl->degm = 0;
        ctl->nbnd = ctl->nexam = ctl->degexam = 0;
        int32_t m = choose_mode(L, bal);
        ctl->mode = m;
        next_mode = m;
        if (L.use_graph) {
            cudaGraphSetConditional((cudaGraphConditionalHandle)L.h_mode, (unsigned)m);
            cudaGraphSetConditional((cudaGraphConditionalHandle)L.h_loop, m == MODE_DONE ? 0u : 1u);
        }
    }
    __syncthreads();
    int32_t m = next_mode;
    if (m == MODE_RW || m == MODE_RS) compute_classes(L, sh);
    return m;
}

// Level start, one block: control block from the initial cut and weights.
__device__ inline void ph_ctl_init(const Level &L, const int64_t *cut2) {
    __shared__ long long sh[40];
    Ctl *ctl = L.ctl;
    long long maxw = block_max_pw(L.pw, L.k, sh);
    if (threadIdx.x == 0) {
        ctl->cut = *cut2 / 2;
        ctl->dcut = 0;
        ctl->maxw = maxw;
        ctl->best_cut = ctl->cut;
        ctl->best_maxw = maxw;
        ctl->best_bal = maxw <= ctl->L;
        ctl->it = 0; ctl->noimp = 0; ctl->weak = 0; ctl->lp_epoch = -1;
        ctl->copy_best = 0; ctl->hit_cap = 0;
        ctl->kcount[0] = ctl->kcount[1] = ctl->kcount[2] = ctl->kcount[3] = 0;
        ctl->nX = ctl->nXb = ctl->nM = ctl->nMb = 0;
        ctl->nW = ctl->nWb = 0;
        ctl->ncand = 0;
        ctl->degx = ctl->degm = 0;
        ctl->nbnd = ctl->nexam = ctl->degexam = 0;
        ctl->mode = choose_mode(L, maxw <= ctl->L);
    }
    __syncthreads();
    if (ctl->mode == MODE_RW || ctl->mode == MODE_RS) compute_classes(L, sh);
}

// P_best <- P_iter when the controller asked for it.
__device__ inline void ph_copy_best(const Level &L, Grid G) {
    if (!vread(&L.ctl->copy_best)) return;
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
    JET_APPENDER(wapp, reinterpret_cast<int32_t *>(arena), kScanCap);
    Ctl *ctl = L.ctl;
    const int32_t epoch = vread(&ctl->lp_epoch);
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

// Step 1 (Alg. 4 first loop, Eq. for P_d, Eq. gainconn_filter) for the listed
// vertices with rows of <= 16 entries: one thread per vertex, the row
// preloaded into registers so all its loads are in flight together.  Longer
// rows are passed on to the warp phase.  prio holds F only for members of X;
// every other entry stays kNoneGain (reset after the afterburner).
template <bool EW>
__device__ inline void ph_lp_select_list(const Level &L, LpExport ex, Grid G, char *arena) {
    __shared__ long long red[40];
    Ctl *ctl = L.ctl;
    const int32_t nW = vread(&ctl->nW);
    if ((int64_t)G.bid * blockDim.x >= nW) return;
    JET_APPENDER(xapp, reinterpret_cast<int32_t *>(arena), kListCap);
    JET_APPENDER(bapp, reinterpret_cast<int32_t *>(arena) + kListCap, kBigCap);
    const DGraph g = L.g;
    long long nexam = 0, degexam = 0, degx = 0;
    for (int64_t i0 = (int64_t)G.bid * blockDim.x; i0 < nW; i0 += (int64_t)G.nb * blockDim.x) {
        int64_t i = i0 + threadIdx.x;
        bool inX = false, big = false;
        int32_t v = -1;
        if (i < nW) {
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
                    L.nxt[v] = pd;
                    degx += d;
                }
                if (ex.pd) { ex.pd[v] = pd >= 0 ? pd : ps; ex.gain[v] = F; }
            }
        }
        xapp.add(inX, v);
        bapp.add(big, v);
        xapp.flush(&ctl->nX, L.listX, false);
        bapp.flush(&ctl->nWb, L.listWb, false);
    }
    xapp.flush(&ctl->nX, L.listX, true);
    bapp.flush(&ctl->nWb, L.listWb, true);
    flush_counter(&ctl->nexam, nexam, red);
    flush_counter(&ctl->degexam, degexam, red);
    flush_counter(&ctl->degx, degx, red);
}

// Long rows: one warp per vertex, dense per-warp table in shared memory.
// The table is all-zero between vertices: the read pass takes every touched
// entry with atomicExch(.., 0), which also detects each distinct part once.
template <bool EW>
__device__ inline void ph_lp_select_big(const Level &L, LpExport ex, Grid G, char *arena) {
    __shared__ long long red[40];
    Ctl *ctl = L.ctl;
    const int32_t nWb = vread(&ctl->nWb);
    const int warps = blockDim.x >> 5;
    if ((int64_t)G.bid * warps >= nWb) return;
    int32_t *tab = reinterpret_cast<int32_t *>(arena) + (threadIdx.x >> 5) * L.k;
    for (int i = threadIdx.x; i < warps * L.k; i += blockDim.x) reinterpret_cast<int32_t *>(arena)[i] = 0;
    __syncthreads();
    const DGraph g = L.g;
    const unsigned lane = lane_id();
    long long nexam = 0, degexam = 0, degx = 0;
    for (int64_t w = (int64_t)G.bid * warps + (threadIdx.x >> 5); w < nWb; w += (int64_t)G.nb * warps) {
        int32_t v = L.listWb[w];
        int32_t ps = L.part[v];
        int32_t F = kNoneGain, pd = -1;
        bool inX = false;
        int64_t beg = ld_xadj(g.xadj, v), end = ld_xadj(g.xadj, (int64_t)v + 1);
        for (int64_t j = beg + lane; j < end; j += 32) atomicAdd(&tab[L.part[__ldg(g.adj + j)]], edge_w<EW>(g, j));
        __syncwarp();
        int32_t conn_s = tab[ps];
        __syncwarp();
        unsigned long long best = 0;
        for (int64_t j = beg + lane; j < end; j += 32) {
            int32_t p = L.part[__ldg(g.adj + j)];
            int32_t c = atomicExch(&tab[p], 0);
            if (c > 0 && p != ps) {
                unsigned long long key = part_key(c, p);
                best = key > best ? key : best;
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
                L.nxt[v] = pd;
                L.listXb[atomicAdd(&ctl->nXb, 1)] = v;
                degx += end - beg;
            }
            if (ex.pd) { ex.pd[v] = pd >= 0 ? pd : ps; ex.gain[v] = F; }
        }
    }
    __syncthreads();
    flush_counter(&ctl->nexam, nexam, red);
    flush_counter(&ctl->degexam, degexam, red);
    flush_counter(&ctl->degx, degx, red);
}

// Step 2: afterburner (Alg. 4 second loop, ord of Sec. 4.1.1) and the second
// filter M = {v in X : F2 >= 0}.  Short rows: one thread per vertex, the row
// preloaded so that the neighbours' gathers are all in flight together.
template <bool EW>
__device__ inline void ph_afterburn_small(const Level &L, LpExport ex, Grid G, char *arena) {
    Ctl *ctl = L.ctl;
    const int32_t nX = vread(&ctl->nX), it = vread(&ctl->it);
    if ((int64_t)G.bid * blockDim.x >= nX) return;
    JET_APPENDER(mapp, reinterpret_cast<int32_t *>(arena), kListCap);
    const bool full = !(L.abl & (ABL_NO_AFTERBURN | ABL_BASELINE_LP));
    for (int64_t i0 = (int64_t)G.bid * blockDim.x; i0 < nX; i0 += (int64_t)G.nb * blockDim.x) {
        int64_t i = i0 + threadIdx.x;
        bool inM = false;
        int32_t v = -1;
        if (i < nX) {
            v = L.listX[i];
            if (!full) {
                inM = true;
            } else {
                int32_t Fv = L.prio[v], pd = L.nxt[v], ps = L.part[v];
                int64_t beg = ld_xadj(L.g.xadj, v);
                int d = (int)(ld_xadj(L.g.xadj, (int64_t)v + 1) - beg);
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
                        int32_t fu = L.prio[u];
                        if (fu > Fv || (fu == Fv && u < v)) pu = L.nxt[u];
                        f2 += pu == pd ? ww[t] : (pu == ps ? -ww[t] : 0);
                    }
                }
                inM = f2 >= 0;
                if (ex.f2) ex.f2[v] = f2;
            }
            if (inM) L.mstamp[v] = it;
        }
        mapp.add(inM, v);
        mapp.flush(&ctl->nM, L.listM, false);
    }
    mapp.flush(&ctl->nM, L.listM, true);
}

template <bool EW>
__device__ __forceinline__ int32_t afterburn_term(const Level &L, int32_t v, int32_t Fv, int32_t pd, int32_t ps,
                                                  int64_t j) {
    int32_t u = __ldg(L.g.adj + j);
    int32_t pu = L.part[u];
    int32_t fu = L.prio[u];
    if (fu > Fv || (fu == Fv && u < v)) pu = L.nxt[u];
    int32_t w = edge_w<EW>(L.g, j);
    return pu == pd ? w : (pu == ps ? -w : 0);
}

template <bool EW>
__device__ inline void ph_afterburn_big(const Level &L, LpExport ex, Grid G) {
    Ctl *ctl = L.ctl;
    const int32_t nXb = vread(&ctl->nXb), it = vread(&ctl->it);
    const int warps = blockDim.x >> 5;
    const unsigned lane = lane_id();
    for (int64_t w = (int64_t)G.bid * warps + (threadIdx.x >> 5); w < nXb; w += (int64_t)G.nb * warps) {
        int32_t v = L.listXb[w];
        bool inM;
        int32_t f2 = 0;
        if (L.abl & (ABL_NO_AFTERBURN | ABL_BASELINE_LP)) {
            inM = true;
        } else {
            int32_t Fv = L.prio[v], pd = L.nxt[v], ps = L.part[v];
            int64_t beg = ld_xadj(L.g.xadj, v), end = ld_xadj(L.g.xadj, (int64_t)v + 1);
            for (int64_t j = beg + lane; j < end; j += 32) f2 += afterburn_term<EW>(L, v, Fv, pd, ps, j);
            f2 = warp_sum_i32(f2);
            inM = f2 >= 0;
        }
        if (lane == 0) {
            if (ex.f2 && !(L.abl & (ABL_NO_AFTERBURN | ABL_BASELINE_LP))) ex.f2[v] = f2;
            if (inM) {
                L.mstamp[v] = it;
                L.listMb[atomicAdd(&ctl->nMb, 1)] = v;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Apply M (Alg. 3 updatePartsAndDS): exact cut change, part weights, and the
// neighbour counts ext.  For an edge with both ends moving, the smaller id
// accounts for the cut.
// ---------------------------------------------------------------------------
template <bool EW>
__device__ inline void ph_apply_small(const Level &L, Grid G, char *arena) {
    __shared__ long long red[40];
    Ctl *ctl = L.ctl;
    if (vread(&ctl->mode) == MODE_DONE) return;
    const int32_t nM = vread(&ctl->nM), it = vread(&ctl->it);
    if ((int64_t)G.bid * blockDim.x >= nM) return;
    long long *shpw = reinterpret_cast<long long *>(arena);
    for (int i = threadIdx.x; i < L.k; i += blockDim.x) shpw[i] = 0;
    __syncthreads();
    long long dc = 0, dm = 0;
    for (int64_t i = (int64_t)G.bid * blockDim.x + threadIdx.x; i < nM; i += (int64_t)G.nb * blockDim.x) {
        int32_t v = L.listM[i];
        int32_t a = L.part[v], b = L.nxt[v];
        long long wv = L.g.vw[v];
        atomicAdd(reinterpret_cast<unsigned long long *>(&shpw[a]), (unsigned long long)(-wv));
        atomicAdd(reinterpret_cast<unsigned long long *>(&shpw[b]), (unsigned long long)wv);
        int64_t beg = ld_xadj(L.g.xadj, v);
        int d = (int)(ld_xadj(L.g.xadj, (int64_t)v + 1) - beg);
        // rows in listM are short (long ones are in listMb): preload them
        int32_t uu[kSmallDeg];
#pragma unroll
        for (int t = 0; t < kSmallDeg; ++t) uu[t] = t < d ? __ldg(L.g.adj + beg + t) : -1;
        int32_t ne = 0;
#pragma unroll
        for (int t = 0; t < kSmallDeg; ++t) {
            if (t < d) {
                int32_t u = uu[t];
                int32_t pu = L.part[u];
                bool mu = L.mstamp[u] == it;
                int32_t pn = mu ? L.nxt[u] : pu;
                int32_t diff = (int)(pn != b) - (int)(pu != a);
                ne += pn != b;
                if (!mu) {
                    if (diff) atomicAdd(&L.ext[u], diff);
                    dc += (long long)edge_w<EW>(L.g, beg + t) * diff;
                } else if (u > v) {
                    dc += (long long)edge_w<EW>(L.g, beg + t) * diff;
                }
            }
        }
        L.ext[v] = ne;
        dm += d;
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

template <bool EW>
__device__ __forceinline__ int64_t apply_edge(const Level &L, int32_t v, int32_t a, int32_t b, int32_t it, int64_t j,
                                              int32_t *other) {
    int32_t u = __ldg(L.g.adj + j);
    int32_t pu = L.part[u];
    bool mu = L.mstamp[u] == it;
    int32_t pn = mu ? L.nxt[u] : pu;
    *other = pn != b;
    if (!mu) {
        int32_t dx = (int)(pn != b) - (int)(pu != a);
        if (dx) atomicAdd(&L.ext[u], dx);
    } else if (u < v) {
        return 0;
    }
    int32_t w = edge_w<EW>(L.g, j);
    return (int64_t)w * ((int)(pn != b) - (int)(pu != a));
}

template <bool EW>
__device__ inline void ph_apply_big(const Level &L, Grid G) {
    Ctl *ctl = L.ctl;
    if (vread(&ctl->mode) == MODE_DONE) return;
    const int32_t nMb = vread(&ctl->nMb), it = vread(&ctl->it);
    const int warps = blockDim.x >> 5;
    const unsigned lane = lane_id();
    for (int64_t w = (int64_t)G.bid * warps + (threadIdx.x >> 5); w < nMb; w += (int64_t)G.nb * warps) {
        int32_t v = L.listMb[w];
        int32_t a = L.part[v], b = L.nxt[v];
        int64_t beg = ld_xadj(L.g.xadj, v), end = ld_xadj(L.g.xadj, (int64_t)v + 1);
        long long dc = 0;
        int32_t ne = 0;
        for (int64_t j = beg + lane; j < end; j += 32) {
            int32_t o;
            dc += apply_edge<EW>(L, v, a, b, it, j, &o);
            ne += o;
        }
        dc = warp_sum_i64(dc);
        ne = warp_sum_i32(ne);
        if (lane == 0) {
            long long wv = L.g.vw[v];
            atomic_add_i64(&L.pw[a], -wv);
            atomic_add_i64(&L.pw[b], wv);
            if (dc) atomic_add_i64(&ctl->dcut, dc);
            atomic_add_i64(&ctl->degm, end - beg);
            L.ext[v] = ne;
        }
    }
}

// Commit: P_s[v] <- P_d[v]; Jetlp movers are locked for the next Jetlp
// (Sec. 4.1.3); rebalancing leaves the locks alone.  After a Jetlp the
// priorities of X go back to kNoneGain.
// The counters a commit needs, read once the move lists are final (before the
// apply step): in the cluster loop the controller of block 0 resets them
// while other blocks may still be committing.
struct CommitSnap {
    int32_t kind, nM, nMb, nX, nXb, it;
};
__device__ __forceinline__ CommitSnap commit_snapshot(const Level &L) {
    const Ctl *ctl = L.ctl;
    return CommitSnap{vread(&ctl->mode), vread(&ctl->nM), vread(&ctl->nMb),
                      vread(&ctl->nX),   vread(&ctl->nXb), vread(&ctl->it)};
}

__device__ __forceinline__ void ph_commit_snap(const Level &L, Grid G, const CommitSnap &cs) {
    if (cs.kind == MODE_DONE) return;
    const int64_t stride = (int64_t)G.nb * blockDim.x;
    int64_t total = (int64_t)cs.nM + cs.nMb;
    for (int64_t i = (int64_t)G.bid * blockDim.x + threadIdx.x; i < total; i += stride) {
        int32_t v = i < cs.nM ? L.listM[i] : L.listMb[i - cs.nM];
        L.part[v] = L.nxt[v];
        if (cs.kind == MODE_LP) L.lstamp[v] = cs.it;
    }
    if (cs.kind == MODE_LP) {
        int64_t tx = (int64_t)cs.nX + cs.nXb;
        for (int64_t i = (int64_t)G.bid * blockDim.x + threadIdx.x; i < tx; i += stride)
            L.prio[i < cs.nX ? L.listX[i] : L.listXb[i - cs.nX]] = kNoneGain;
    }
}

__device__ inline void ph_commit(const Level &L, Grid G) { ph_commit_snap(L, G, commit_snapshot(L)); }

// ---------------------------------------------------------------------------
// Rebalancing (Alg. 5 Jetrw, Sec. 4.2.2 Jetrs)
// ---------------------------------------------------------------------------
__device__ __forceinline__ int32_t random_B(const Level &L, int32_t v, int32_t it, int32_t nB) {
    uint64_t h = splitmix64(L.seed ^ (0x9E3779B97F4A7C15ULL * (uint64_t)(it + 1)) ^ (uint64_t)(uint32_t)v);
    return L.Bs[h % (uint64_t)nB];
}

// Adds w into bucketw[key] with one atomic per distinct key in the warp.
__device__ __forceinline__ void bucket_add(const Level &L, int32_t key, long long w) {
    unsigned peers = __match_any_sync(0xffffffffu, key);
    long long s = 0;
#pragma unroll
    for (int j = 0; j < 32; ++j) {
        long long x = __shfl_sync(0xffffffffu, w, j);
        if ((peers >> j) & 1u) s += x;
    }
    if (key >= 0 && (int)lane_id() == __ffs(peers) - 1) atomic_add_i64(&L.bucketw[key], s);
}

// Per-block slot buckets in shared memory when nA * kSlots keys fit.
struct SmemBuckets {
    long long *b;
    int32_t nkeys;
    bool on;
    __device__ __forceinline__ void init(const Level &L, long long *buf) {
        b = buf;
        nkeys = vread(&L.ctl->nA) * kSlots;
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
// others are listed for the row phases.
template <bool STRONG>
__device__ inline void ph_rb_scan(const Level &L, Grid G, char *arena) {
    disarm_loop(L, G);
    __shared__ long long red[40];
    SmemBuckets sb;
    sb.init(L, reinterpret_cast<long long *>(arena));
    JET_APPENDER(wapp, reinterpret_cast<int32_t *>(arena + kSmemBuckets * 8), kScanCap);
    Ctl *ctl = L.ctl;
    const int32_t it = vread(&ctl->it);
    const int32_t nB = vread(&ctl->nB);
    const int64_t opt = vread(&ctl->opt);
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
                    if constexpr (!STRONG) L.nxt[v] = random_B(L, v, it, nB);
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

// Step 1 for listed candidates with rows of <= 16 entries: Jetrw destination
// (best-connected part of B, lowest id on ties, else a random one) and loss,
// or the Jetrs loss (Sec. 4.2.2), then the slot bucket.
template <bool EW, bool STRONG>
__device__ inline void ph_rb_cand_list(const Level &L, Grid G, char *arena) {
    __shared__ long long red[40];
    Ctl *ctl = L.ctl;
    const int32_t nW = vread(&ctl->nW), nB = vread(&ctl->nB);
    if ((int64_t)G.bid * blockDim.x >= nW) return;
    SmemBuckets sb;
    sb.init(L, reinterpret_cast<long long *>(arena));
    JET_APPENDER(bapp, reinterpret_cast<int32_t *>(arena + kSmemBuckets * 8), kBigCap);
    const int32_t it = vread(&ctl->it);
    const DGraph g = L.g;
    long long degrows = 0;
    for (int64_t i0 = (int64_t)G.bid * blockDim.x; i0 < nW; i0 += (int64_t)G.nb * blockDim.x) {
        int64_t i = i0 + threadIdx.x;
        int32_t key = -1;
        long long wv = 0;
        bool big = false;
        int32_t v = -1;
        if (i < nW) {
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
                    L.nxt[v] = dest;
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
        bapp.add(big, v);
        bapp.flush(&ctl->nWb, L.listWb, false);
    }
    bapp.flush(&ctl->nWb, L.listWb, true);
    sb.flush(L);
    flush_counter(&ctl->degexam, degrows, red);
}

// Listed candidates with long rows: one warp per vertex.
template <bool EW, bool STRONG>
__device__ inline void ph_rb_cand_big(const Level &L, Grid G, char *arena) {
    Ctl *ctl = L.ctl;
    const int32_t nWb = vread(&ctl->nWb);
    const int warps = blockDim.x >> 5;
    if ((int64_t)G.bid * warps >= nWb) return;
    int32_t *tab = reinterpret_cast<int32_t *>(arena) + (threadIdx.x >> 5) * L.k;
    for (int i = threadIdx.x; i < warps * L.k; i += blockDim.x) reinterpret_cast<int32_t *>(arena)[i] = 0;
    __syncthreads();
    const int32_t it = vread(&ctl->it), nB = vread(&ctl->nB);
    const DGraph g = L.g;
    const unsigned lane = lane_id();
    for (int64_t w = (int64_t)G.bid * warps + (threadIdx.x >> 5); w < nWb; w += (int64_t)G.nb * warps) {
        int32_t v = L.listWb[w];
        int32_t ps = L.part[v];
        int32_t a = L.aidx[ps];
        int64_t beg = ld_xadj(g.xadj, v), end = ld_xadj(g.xadj, (int64_t)v + 1);
        for (int64_t j = beg + lane; j < end; j += 32) atomicAdd(&tab[L.part[__ldg(g.adj + j)]], edge_w<EW>(g, j));
        __syncwarp();
        int32_t conn_s = tab[ps];
        __syncwarp();
        unsigned long long best = 0;
        long long S = 0;
        int32_t cnt = 0;
        for (int64_t j = beg + lane; j < end; j += 32) {
            int32_t p = L.part[__ldg(g.adj + j)];
            int32_t c = atomicExch(&tab[p], 0);
            if (c > 0 && L.inB[p]) {
                if constexpr (!STRONG) {
                    unsigned long long k2 = part_key(c, p);
                    best = k2 > best ? k2 : best;
                } else {
                    S += c; cnt += 1;
                }
            }
        }
        __syncwarp();
        int32_t loss;
        if constexpr (!STRONG) {
            best = warp_max_u64(best);
            int32_t dest, cd;
            if (best) { dest = key_part(best); cd = key_conn(best); }
            else { dest = random_B(L, v, it, nB); cd = 0; }
            if (lane == 0) L.nxt[v] = dest;
            loss = conn_s - cd;
        } else {
            S = warp_sum_i64(S);
            cnt = warp_sum_i32(cnt);
            loss = conn_s - (cnt > 0 ? (int32_t)(S / cnt) : 0);
        }
        int32_t key = a * kSlots + slot_of(loss);
        if (lane == 0) {
            L.key[v] = key;
            if (L.rbloss) L.rbloss[v] = loss;
            atomic_add_i64(&L.bucketw[key], (long long)g.vw[v]);
            atomic_add_i64(&ctl->degexam, end - beg);
        }
    }
    __syncthreads();
}

// Step 2: per oversized part (one warp each), the boundary slot s* where the
// weight taken so far reaches the excess (Alg. 5 scan: a candidate is taken
// while the weight before it is below w_p - L) and the weight still to take
// inside s*.  s* = kSlots means every candidate is taken.
__device__ inline void ph_rb_plan(const Level &L, Grid G) {
    const Ctl *ctl = L.ctl;
    const int32_t nA = vread(&ctl->nA);
    const int warps = blockDim.x >> 5;
    const unsigned lane = lane_id();
    for (int a = G.bid * warps + (threadIdx.x >> 5); a < nA; a += G.nb * warps) {
        long long t = L.bucketw[a * kSlots + lane];          // slots 0..31 on the lanes
        long long t32 = L.bucketw[a * kSlots + 32];
        long long x = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            long long y = __shfl_up_sync(0xffffffffu, x, o);
            if ((int)lane >= o) x += y;
        }
        long long ex = L.excess[a];
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

// Step 3: per tile of blockDim vertices, the weight of each part's
// boundary-slot members (they are taken in vertex order).
__device__ inline void ph_rb_tilehist(const Level &L, Grid G, char *arena) {
    int32_t *h = reinterpret_cast<int32_t *>(arena);
    const int32_t nA = vread(&L.ctl->nA);
    for (int64_t t = G.bid; t < L.ntiles; t += G.nb) {
        for (int i = threadIdx.x; i < nA; i += blockDim.x) h[i] = 0;
        __syncthreads();
        int64_t v = t * blockDim.x + threadIdx.x;
        if (v < L.g.n) {
            int32_t kv = L.key[v];
            if (kv >= 0) {
                int32_t a = kv / kSlots, s = kv - a * kSlots;
                if (s == L.sstar[a]) atomicAdd(&h[a], L.g.vw[v]);
            }
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
    const int32_t nA = vread(&L.ctl->nA);
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
    int32_t *mbuf = reinterpret_cast<int32_t *>(arena + (((size_t)L.k * 8 + 15) & ~size_t(15)));
    JET_APPENDER(mapp, mbuf, 2 * (int)blockDim.x);
    Ctl *ctl = L.ctl;
    const int32_t nA = vread(&ctl->nA), it = vread(&ctl->it);
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
            bool big = taken && is_big_row(L.g, (int32_t)vv);
            mapp.add(taken && !big, (int32_t)vv);
            if (big) L.listMb[atomicAdd(&ctl->nMb, 1)] = (int32_t)vv;
            mapp.flush(&ctl->nM, L.listM, true);
        } else {
            __shared__ long long red[40];
            if (vv < L.g.n) L.etaken[vv] = taken ? w : 0;
            long long tt = block_sum_i64(taken ? w : 0, red);
            if (threadIdx.x == 0) L.tiletaken[tile] = tt;
        }
        __syncthreads();
    }
}

// Jetrs: exclusive scan of the evicted weight over tiles (one block).
__device__ inline void ph_rb_tiletaken_scan(const Level &L) {
    __shared__ long long sh[40];
    long long carry = 0;
    for (int64_t t0 = 0; t0 < L.ntiles; t0 += blockDim.x) {
        int64_t t = t0 + threadIdx.x;
        long long x = t < L.ntiles ? L.tiletaken[t] : 0;
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
    const int32_t it = vread(&ctl->it), nB = vread(&ctl->nB);
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
        if (mv) { L.nxt[v] = dest; L.mstamp[v] = it; }
        bool big = mv && is_big_row(L.g, (int32_t)v);
        mapp.add(mv && !big, (int32_t)v);
        if (big) L.listMb[atomicAdd(&ctl->nMb, 1)] = (int32_t)v;
        mapp.flush(&ctl->nM, L.listM, true);
    }
}

}  // namespace jet
