// Jet refinement on one level (Sec. 4): Jetlp (Alg. 4), Jetrw (Alg. 5),
// Jetrs (Sec. 4.2.2) and the driver of Alg. 3, for sm_103a.
//
// Design (GB300-first, not a translation of the paper's Kokkos kernels):
//  * No persistent vertex-part hash table (Sec. 4.3).  Every pass recomputes
//    conn(v, .) from the CSR row: rows of <= 16 entries are handled one thread
//    per vertex in registers; longer rows one warp per vertex with a dense
//    per-warp connectivity table in shared memory that is cleared as it is read
//    (atomicExch), so only touched entries are written.
//  * Every decision is an integer comparison with fixed tie-breaks (lowest
//    part id, then lowest vertex id), so the result does not depend on thread
//    order and equals the CPU oracle bit for bit.  Only order-independent
//    integer atomics are used.
//  * Iteration control (mode choice, best tracking, stop rule) lives on the
//    device in a one-block controller kernel; the whole level loop is a CUDA
//    graph with a WHILE node around a SWITCH over {Jetlp, Jetrw, Jetrs}, so no
//    host round trip happens per iteration (the paper blames that round trip
//    for its weaker coarse-level speedup, Sec. 6.2).
#include "jet_internal.cuh"

#include <algorithm>
#include <cstdio>

namespace jet {

// ---------------------------------------------------------------------------
// edge helpers
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

// ---------------------------------------------------------------------------
// cut and part weights of a partition (Sec. 2.1), used at level start
// ---------------------------------------------------------------------------
template <bool EW>
__global__ void __launch_bounds__(kTB) k_cut_pw(DGraph g, int32_t k, const int32_t *__restrict__ part,
                                                 int64_t *__restrict__ pw, int64_t *__restrict__ cut2,
                                                 int32_t *__restrict__ ext, int32_t *__restrict__ wdeg) {
    extern __shared__ long long shpw[];
    __shared__ long long red[40];
    for (int i = threadIdx.x; i < k; i += blockDim.x) shpw[i] = 0;
    __syncthreads();
    long long c = 0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < g.n; v += (int64_t)gridDim.x * blockDim.x) {
        int32_t p = part[v];
        atomicAdd(reinterpret_cast<unsigned long long *>(&shpw[p]), (unsigned long long)(long long)(g.vw ? g.vw[v] : 1));
        int64_t e = ld_xadj(g.xadj, v + 1);
        int32_t nx = 0, wd = 0, cv = 0;
        for (int64_t j = ld_xadj(g.xadj, v); j < e; ++j) {
            int32_t w = edge_w<EW>(g, j);
            bool other = part[g.adj[j]] != p;
            cv += other ? w : 0;
            nx += other ? 1 : 0;
            wd += w;
        }
        c += cv;
        if (ext) ext[v] = nx;
        if (wdeg) wdeg[v] = wd;
    }
    c = block_sum_i64(c, red);
    if (threadIdx.x == 0 && c) atomic_add_i64(cut2, c);
    __syncthreads();
    for (int i = threadIdx.x; i < k; i += blockDim.x)
        if (shpw[i]) atomic_add_i64(&pw[i], shpw[i]);
}

// ---------------------------------------------------------------------------
// controller helpers (one block of 1024 threads)
// ---------------------------------------------------------------------------
__device__ long long block_max_pw(const int64_t *pw, int32_t k, long long *sh) {
    long long m = 0;
    for (int i = threadIdx.x; i < k; i += blockDim.x) m = pw[i] > m ? pw[i] : m;
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
// capacity prefix of B (Jetrs) and zeroed slot buckets.  blockDim.x >= k.
__device__ void compute_classes(const Level &L, long long *sh) {
    Ctl *ctl = L.ctl;
    int p = threadIdx.x;
    bool inA = false, inB = false;
    long long w = 0;
    if (p < L.k) {
        w = L.pw[p];
        inA = w > ctl->L;
        inB = w <= ctl->sigma;
    }
    long long tA = 0, tB = 0, tC = 0;
    long long ia = block_exscan_i64(inA ? 1 : 0, sh, &tA);
    long long ib = block_exscan_i64(inB ? 1 : 0, sh, &tB);
    long long cap = inB ? (ctl->sigma - w) : 0;
    long long cb = block_exscan_i64(cap, sh, &tC);
    if (p < L.k) {
        L.aidx[p] = inA ? (int32_t)ia : -1;
        L.inB[p] = inB ? 1 : 0;
        if (inA) L.excess[ia] = w - ctl->L;
        if (inB) { L.Bs[ib] = p; L.capC[ib] = cb; }
    }
    if (threadIdx.x == 0) {
        ctl->nA = (int32_t)tA;
        ctl->nB = (int32_t)tB;
        L.capC[tB] = tC;
    }
    __syncthreads();
    int32_t nkeys = (int32_t)tA * kSlots;
    for (int i = threadIdx.x; i < nkeys; i += blockDim.x) L.bucketw[i] = 0;
}

// Mode of the next iteration (Alg. 3): balanced -> Jetlp; else Jetrw while the
// weak counter is below b_max, else Jetrs; DONE by the stop rule or the cap.
__device__ int32_t choose_mode(const Level &L, bool balanced) {
    Ctl *ctl = L.ctl;
    if (ctl->noimp >= L.max_no_improve) return MODE_DONE;
    if (ctl->it >= L.max_iters) { ctl->hit_cap = 1; return MODE_DONE; }
    if (balanced) { ctl->weak = 0; return MODE_LP; }
    if (ctl->weak < L.weak_limit) { ctl->weak += 1; return MODE_RW; }
    return MODE_RS;
}

__global__ void __launch_bounds__(1024) k_ctl_init(Level L, const int64_t *cut2) {
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

// Sets the CUDA-graph conditionals for the first iteration.
__global__ void k_graph_start(Level L) {
    if (threadIdx.x == 0) {
        int32_t m = L.ctl->mode;
        cudaGraphSetConditional((cudaGraphConditionalHandle)L.h_mode, (unsigned)m);
        cudaGraphSetConditional((cudaGraphConditionalHandle)L.h_loop, m == MODE_DONE ? 0u : 1u);
    }
}

// End of an iteration (Alg. 3 after updatePartsAndDS): exact cut, max part
// weight, P_best / counters, trace record, next mode.
__global__ void __launch_bounds__(1024) k_controller(Level L) {
    __shared__ long long sh[40];
    __shared__ int32_t next_mode;
    Ctl *ctl = L.ctl;
    int32_t kind = ctl->mode;
    if (kind == MODE_DONE) {
        if (threadIdx.x == 0) {
            ctl->copy_best = 0;
            if (L.use_graph) {
                cudaGraphSetConditional((cudaGraphConditionalHandle)L.h_loop, 0u);
                cudaGraphSetConditional((cudaGraphConditionalHandle)L.h_mode, (unsigned)MODE_DONE);
            }
        }
        return;
    }
    long long maxw = block_max_pw(L.pw, L.k, sh);
    if (threadIdx.x == 0) {
        long long cut = ctl->cut + ctl->dcut;
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
            r.nx = (kind == MODE_LP) ? (int64_t)(ctl->nX + ctl->nXb) : ctl->ncand;
            r.nm = (int64_t)(ctl->nM + ctl->nMb);
            r.cut = cut; r.maxw = maxw;
            r.degx = ctl->degx; r.degm = ctl->degm;
            r.nbnd = ctl->nbnd; r.nexam = ctl->nexam; r.degexam = ctl->degexam;
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
    if (next_mode == MODE_RW || next_mode == MODE_RS) compute_classes(L, sh);
}

// P_best <- P_iter when the controller asked for it.
__global__ void __launch_bounds__(kTB) k_copy_best(Level L) {
    if (!L.ctl->copy_best) return;
    if (((reinterpret_cast<uintptr_t>(L.part) | reinterpret_cast<uintptr_t>(L.best)) & 15) != 0) {
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < L.g.n; i += (int64_t)gridDim.x * blockDim.x)
            L.best[i] = L.part[i];
        return;
    }
    const int4 *src = reinterpret_cast<const int4 *>(L.part);
    int4 *dst = reinterpret_cast<int4 *>(L.best);
    int64_t n4 = L.g.n / 4;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
    if (blockIdx.x == 0 && threadIdx.x < (L.g.n & 3)) {
        int64_t i = n4 * 4 + threadIdx.x;
        L.best[i] = L.part[i];
    }
}

// ---------------------------------------------------------------------------
// Jetlp step 1: destination, gain and first filter (Alg. 4 first loop, Eq.
// for P_d, Eq. gainconn_filter).  Short rows: one thread per vertex.
// ---------------------------------------------------------------------------
struct LpExport {           // optional dense outputs of the single-pass API
    int32_t *pd;            // P_d (P_s where undefined)
    int32_t *gain;          // F (kNoneGain where undefined)
    int32_t *f2;            // F2 for X members
};

// Graph-loop guard: the first kernel of every iteration branch clears the
// loop condition; only the controller at the end of a completed iteration
// sets it again, so the device loop cannot outlive a missing controller.
__device__ __forceinline__ void disarm_loop(const Level &L) {
    if (L.use_graph && blockIdx.x == 0 && threadIdx.x == 0)
        cudaGraphSetConditional((cudaGraphConditionalHandle)L.h_loop, 0u);
}

// Block-level sums of the select counters, one atomic per block.
__device__ __forceinline__ void flush_counter(int64_t *dst, long long v, long long *red) {
    v = block_sum_i64(v, red);
    if (threadIdx.x == 0 && v) atomic_add_i64(dst, v);
}

// Jetlp step 0: the work list.  A vertex with no neighbour in another part
// (ext == 0) has no destination (Alg. 4: A_v is empty) and a locked vertex is
// skipped (Sec. 4.1.3); the scan reads ext four vertices at a time and lists
// the others.  Interior rows are never read.
__global__ void __launch_bounds__(kTB) k_lp_scan(Level L) {
    disarm_loop(L);
    __shared__ long long red[40];
    JET_BLOCK_APPENDER(wapp, 4096);
    Ctl *ctl = L.ctl;
    const int32_t epoch = ctl->lp_epoch;
    const bool use_locks = !ablate_locks(L.abl);
    const int64_t n = L.g.n, nq = (n + 3) / 4;
    const bool vec = (reinterpret_cast<uintptr_t>(L.ext) & 15) == 0;
    long long nb = 0;
    for (int64_t q0 = (int64_t)blockIdx.x * blockDim.x; q0 < nq; q0 += (int64_t)gridDim.x * blockDim.x) {
        int64_t q = q0 + threadIdx.x;
        int64_t v0 = 4 * q;
        int32_t e[4] = {0, 0, 0, 0};
        if (q < nq) {
            if (vec && v0 + 3 < n) {
                int4 x = __ldg(reinterpret_cast<const int4 *>(L.ext + v0));
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

// Jetlp step 1 (Alg. 4 first loop, Eq. for P_d, Eq. gainconn_filter) for the
// listed vertices with rows of <= 16 entries: one thread per vertex, the row
// preloaded into registers so all its loads are in flight together.  Longer
// rows are passed on to the warp kernel.  prio holds F only for members of X;
// every other entry stays kNoneGain (reset after the afterburner).
template <bool EW>
__global__ void __launch_bounds__(kTB, 4) k_lp_select_list(Level L, LpExport ex) {
    __shared__ long long red[40];
    Ctl *ctl = L.ctl;
    const int32_t nW = ctl->nW;
    if ((int64_t)blockIdx.x * blockDim.x >= nW) return;
    JET_BLOCK_APPENDER(xapp, 2048);
    JET_BLOCK_APPENDER(bapp, 1024);
    const DGraph g = L.g;
    long long nexam = 0, degexam = 0, degx = 0;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x; i0 < nW; i0 += (int64_t)gridDim.x * blockDim.x) {
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
                        pp[t] = __ldg(L.part + __ldg(g.adj + beg + t));
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
__global__ void __launch_bounds__(kTB) k_lp_select_big(Level L, LpExport ex) {
    extern __shared__ int32_t tabs[];
    __shared__ long long red[40];
    Ctl *ctl = L.ctl;
    const int32_t nWb = ctl->nWb;
    const int warps = blockDim.x >> 5;
    if ((int64_t)blockIdx.x * warps >= nWb) return;
    int32_t *tab = tabs + (threadIdx.x >> 5) * L.k;
    for (int i = threadIdx.x; i < warps * L.k; i += blockDim.x) tabs[i] = 0;
    __syncthreads();
    const DGraph g = L.g;
    const unsigned lane = lane_id();
    long long nexam = 0, degexam = 0, degx = 0;
    for (int64_t w = (int64_t)blockIdx.x * warps + (threadIdx.x >> 5); w < nWb; w += (int64_t)gridDim.x * warps) {
        int32_t v = L.listWb[w];
        int32_t ps = L.part[v];
        int32_t F = kNoneGain, pd = -1;
        bool inX = false;
        int64_t beg = ld_xadj(g.xadj, v), end = ld_xadj(g.xadj, (int64_t)v + 1);
        for (int64_t j = beg + lane; j < end; j += 32)
            atomicAdd(&tab[__ldg(L.part + __ldg(g.adj + j))], edge_w<EW>(g, j));
        __syncwarp();
        int32_t conn_s = tab[ps];
        __syncwarp();
        unsigned long long best = 0;
        for (int64_t j = beg + lane; j < end; j += 32) {
            int32_t p = __ldg(L.part + __ldg(g.adj + j));
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
    flush_counter(&ctl->nexam, nexam, red);
    flush_counter(&ctl->degexam, degexam, red);
    flush_counter(&ctl->degx, degx, red);
}

// ---------------------------------------------------------------------------
// Jetlp step 2: afterburner (Alg. 4 second loop, ord of Sec. 4.1.1) and the
// second filter M = {v in X : F2 >= 0}.
// ---------------------------------------------------------------------------
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

__device__ __forceinline__ bool is_big_row(const DGraph &g, int32_t v) {
    return ld_xadj(g.xadj, (int64_t)v + 1) - ld_xadj(g.xadj, v) > kSmallDeg;
}

// Short rows (X members are listed by row length): one thread per vertex, the
// row preloaded so that the neighbours' gathers are all in flight together.
template <bool EW>
__global__ void __launch_bounds__(kTB, 4) k_afterburn_small(Level L, LpExport ex) {
    Ctl *ctl = L.ctl;
    const int32_t nX = ctl->nX, it = ctl->it;
    if ((int64_t)blockIdx.x * blockDim.x >= nX) return;
    JET_BLOCK_APPENDER(mapp, 2048);
    const bool full = !(L.abl & (ABL_NO_AFTERBURN | ABL_BASELINE_LP));
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x; i0 < nX; i0 += (int64_t)gridDim.x * blockDim.x) {
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
__global__ void __launch_bounds__(kTB) k_afterburn_big(Level L, LpExport ex) {
    Ctl *ctl = L.ctl;
    const int32_t nXb = ctl->nXb, it = ctl->it;
    const int warps = blockDim.x >> 5;
    const unsigned lane = lane_id();
    for (int64_t w = (int64_t)blockIdx.x * warps + (threadIdx.x >> 5); w < nXb; w += (int64_t)gridDim.x * warps) {
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
// Apply M (Alg. 3 updatePartsAndDS): exact cut change and part weights.
// For an edge with both ends moving, the smaller id accounts for it.
// ---------------------------------------------------------------------------
// One edge of a moving vertex v (a -> b): cut change and, for a neighbour
// that stays, its count of neighbours in other parts (ext).  For an edge with
// both ends moving, the smaller id accounts for the cut.  Returns 1 in *other
// when the edge joins different parts afterwards.
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
__global__ void __launch_bounds__(kTB, 4) k_apply_small(Level L) {
    extern __shared__ long long shpw[];
    __shared__ long long red[40];
    Ctl *ctl = L.ctl;
    if (ctl->mode == MODE_DONE) return;
    const int32_t nM = ctl->nM, it = ctl->it;
    if ((int64_t)blockIdx.x * blockDim.x >= nM) return;
    for (int i = threadIdx.x; i < L.k; i += blockDim.x) shpw[i] = 0;
    __syncthreads();
    long long dc = 0, dm = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nM; i += (int64_t)gridDim.x * blockDim.x) {
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
}

template <bool EW>
__global__ void __launch_bounds__(kTB) k_apply_big(Level L) {
    Ctl *ctl = L.ctl;
    if (ctl->mode == MODE_DONE) return;
    const int32_t nMb = ctl->nMb, it = ctl->it;
    const int warps = blockDim.x >> 5;
    const unsigned lane = lane_id();
    for (int64_t w = (int64_t)blockIdx.x * warps + (threadIdx.x >> 5); w < nMb; w += (int64_t)gridDim.x * warps) {
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
// (Sec. 4.1.3); rebalancing leaves the locks alone.
__global__ void __launch_bounds__(kTB) k_commit(Level L) {
    const Ctl *ctl = L.ctl;
    int32_t kind = ctl->mode;
    if (kind == MODE_DONE) return;
    const int32_t nM = ctl->nM, nMb = ctl->nMb, it = ctl->it;
    int64_t total = (int64_t)nM + nMb;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        int32_t v = i < nM ? L.listM[i] : L.listMb[i - nM];
        L.part[v] = L.nxt[v];
        if (kind == MODE_LP) L.lstamp[v] = it;
    }
    if (kind == MODE_LP) {
        // back to "no priority" for every member of X (the afterburner is done)
        const int32_t nX = ctl->nX, nXb = ctl->nXb;
        int64_t tx = (int64_t)nX + nXb;
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < tx; i += (int64_t)gridDim.x * blockDim.x)
            L.prio[i < nX ? L.listX[i] : L.listXb[i - nX]] = kNoneGain;
    }
}

// ---------------------------------------------------------------------------
// Rebalancing step 1: candidates, destination (Jetrw) and loss (Alg. 5 first
// loop; Jetrs loss of Sec. 4.2.2), slot buckets.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool rb_eligible(const Level &L, int32_t v, int32_t p, int32_t &a) {
    a = L.aidx[p];
    if (a < 0 || L.ctl->nB == 0) return false;
    // heavy-vertex restriction (Sec. 4.2.2): stay if vwgt > 1.5 (w_p - opt)
    return 2LL * (long long)L.g.vw[v] <= 3LL * (L.pw[p] - L.ctl->opt);
}

__device__ __forceinline__ int32_t random_B(const Level &L, int32_t v, int32_t it) {
    uint64_t h = splitmix64(L.seed ^ (0x9E3779B97F4A7C15ULL * (uint64_t)(it + 1)) ^ (uint64_t)(uint32_t)v);
    int32_t nB = L.ctl->nB;
    return L.Bs[h % (uint64_t)nB];
}

constexpr int kSmemBuckets = 1024;   // slot buckets aggregated per block when nA * kSlots fits

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
        nkeys = L.ctl->nA * kSlots;
        on = nkeys <= kSmemBuckets;
        if (on)
            for (int i = threadIdx.x; i < nkeys; i += blockDim.x) b[i] = 0;
        __syncthreads();
    }
    // all threads of the warp call add (key may be -1)
    __device__ __forceinline__ void add(const Level &L, int32_t key, long long w) {
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
    }
};

// Rebalancing step 0 (Alg. 5 first loop): the candidates are the vertices of
// oversized parts allowed to leave (heavy-vertex rule).  A candidate with no
// neighbour in another part (ext == 0) touches no part of B (its own part is
// oversized): conn(v, P_s) is its weighted degree, Jetrw sends it to a random
// part of B and both losses equal that degree — it is finished here without
// reading its row.  The others are listed for the row kernels.
template <bool STRONG>
__global__ void __launch_bounds__(kTB) k_rb_scan(Level L) {
    disarm_loop(L);
    __shared__ long long red[40];
    __shared__ long long sbuf[kSmemBuckets];
    SmemBuckets sb;
    sb.init(L, sbuf);
    JET_BLOCK_APPENDER(wapp, 4096);
    Ctl *ctl = L.ctl;
    const int32_t it = ctl->it;
    const int32_t nB = ctl->nB;
    const int64_t opt = ctl->opt;
    const int64_t n = L.g.n, nq = (n + 3) / 4;
    const bool vec = (reinterpret_cast<uintptr_t>(L.part) & 15) == 0;
    long long ncand = 0, nlist = 0;
    for (int64_t q0 = (int64_t)blockIdx.x * blockDim.x; q0 < nq; q0 += (int64_t)gridDim.x * blockDim.x) {
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
            // heavy-vertex restriction (Sec. 4.2.2): stay if vwgt > 1.5 (w_p - opt)
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
                    if constexpr (!STRONG) L.nxt[v] = random_B(L, v, it);
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

// Rebalancing step 1 for listed candidates with rows of <= 16 entries: Jetrw
// destination (best-connected part of B, lowest id on ties, else a random one)
// and loss, or the Jetrs loss (Sec. 4.2.2), then the slot bucket.
template <bool EW, bool STRONG>
__global__ void __launch_bounds__(kTB, 4) k_rb_cand_list(Level L) {
    __shared__ long long red[40];
    __shared__ long long sbuf[kSmemBuckets];
    Ctl *ctl = L.ctl;
    const int32_t nW = ctl->nW;
    if ((int64_t)blockIdx.x * blockDim.x >= nW) return;
    SmemBuckets sb;
    sb.init(L, sbuf);
    JET_BLOCK_APPENDER(bapp, 1024);
    const int32_t it = ctl->it;
    const DGraph g = L.g;
    long long degrows = 0;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x; i0 < nW; i0 += (int64_t)gridDim.x * blockDim.x) {
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
                        pp[t] = __ldg(L.part + __ldg(g.adj + beg + t));
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
                    else { dest = random_B(L, v, it); cd = 0; }
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
__global__ void __launch_bounds__(kTB) k_rb_cand_big(Level L) {
    extern __shared__ int32_t tabs[];
    Ctl *ctl = L.ctl;
    const int32_t nWb = ctl->nWb;
    const int warps = blockDim.x >> 5;
    if ((int64_t)blockIdx.x * warps >= nWb) return;
    int32_t *tab = tabs + (threadIdx.x >> 5) * L.k;
    for (int i = threadIdx.x; i < warps * L.k; i += blockDim.x) tabs[i] = 0;
    __syncthreads();
    const int32_t it = ctl->it;
    const DGraph g = L.g;
    const unsigned lane = lane_id();
    for (int64_t w = (int64_t)blockIdx.x * warps + (threadIdx.x >> 5); w < nWb; w += (int64_t)gridDim.x * warps) {
        int32_t v = L.listWb[w];
        int32_t ps = L.part[v];
        int32_t a = L.aidx[ps];
        int64_t beg = ld_xadj(g.xadj, v), end = ld_xadj(g.xadj, (int64_t)v + 1);
        for (int64_t j = beg + lane; j < end; j += 32)
            atomicAdd(&tab[__ldg(L.part + __ldg(g.adj + j))], edge_w<EW>(g, j));
        __syncwarp();
        int32_t conn_s = tab[ps];
        __syncwarp();
        unsigned long long best = 0;
        long long S = 0;
        int32_t cnt = 0;
        for (int64_t j = beg + lane; j < end; j += 32) {
            int32_t p = __ldg(L.part + __ldg(g.adj + j));
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
            else { dest = random_B(L, v, it); cd = 0; }
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
}

// Rebalancing step 2 (one block): per oversized part, the boundary slot s*
// where the weight taken so far reaches the excess (Alg. 5 scan: a candidate
// is taken while the weight before it is below w_p - L), and the weight still
// to take inside s*.  s* = kSlots means every candidate is taken.
__global__ void __launch_bounds__(kTB) k_rb_plan(Level L) {
    const Ctl *ctl = L.ctl;
    const int32_t nA = ctl->nA;
    const int warps = blockDim.x >> 5;
    const unsigned lane = lane_id();
    for (int a = blockIdx.x * warps + (threadIdx.x >> 5); a < nA; a += gridDim.x * warps) {
        // slots 0..31 on the lanes, slot 32 separately
        long long t = L.bucketw[a * kSlots + lane];
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

// Rebalancing step 3: per tile of kRbTile vertices, the weight of each part's
// boundary-slot members (they are taken in vertex order).
__global__ void __launch_bounds__(kTB) k_rb_tilehist(Level L) {
    extern __shared__ int32_t h[];
    const int32_t nA = L.ctl->nA;
    for (int i = threadIdx.x; i < nA; i += blockDim.x) h[i] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * kRbTile;
    for (int r = 0; r < kRbTile / kTB; ++r) {
        int64_t v = base + r * kTB + threadIdx.x;
        if (v < L.g.n) {
            int32_t kv = L.key[v];
            if (kv >= 0) {
                int32_t a = kv / kSlots, s = kv - a * kSlots;
                if (s == L.sstar[a]) atomicAdd(&h[a], L.g.vw[v]);
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nA; i += blockDim.x) L.tilehist[(int64_t)blockIdx.x * nA + i] = h[i];
}

// Exclusive scan of each part's tile sums over the tiles (one block per part,
// eight consecutive tiles per thread).
__global__ void __launch_bounds__(1024) k_rb_tilescan(Level L) {
    __shared__ long long sh[40];
    const int32_t nA = L.ctl->nA;
    const int64_t nt = L.ntiles;
    constexpr int kItems = 8;
    for (int a = blockIdx.x; a < nA; a += gridDim.x) {
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

// Rebalancing step 4: take the candidates (slot < s*, or slot == s* with the
// member weight before them, in vertex order, below `need`).  Jetrw moves the
// taken vertices to P_d; Jetrs records their weight for the cookie cutter.
template <bool STRONG>
__global__ void __launch_bounds__(kTB) k_rb_take(Level L) {
    extern __shared__ long long run[];
    Ctl *ctl = L.ctl;
    const int32_t nA = ctl->nA, it = ctl->it;
    const int64_t tile = blockIdx.x;
    for (int i = threadIdx.x; i < nA; i += blockDim.x) run[i] = L.tilehist[tile * nA + i];
    __syncthreads();
    const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
    const unsigned lt_mask = (1u << lane) - 1u;
    long long tile_taken = 0;
    JET_BLOCK_APPENDER(mapp, kRbTile + kTB);
    for (int r = 0; r < kRbTile / kTB; ++r) {
        int64_t vv = tile * kRbTile + r * kTB + threadIdx.x;
        int32_t kv = -1, a = 0, s = 0;
        if (vv < L.g.n) kv = L.key[vv];
        if (!__syncthreads_or(kv >= 0)) {          // no candidate in this slice
            if constexpr (STRONG) { if (vv < L.g.n) L.etaken[vv] = 0; }
            continue;
        }
        if (kv >= 0) { a = kv / kSlots; s = kv - a * kSlots; }
        int32_t ss = kv >= 0 ? L.sstar[a] : 0;
        bool member = kv >= 0 && s == ss;
        long long w = (kv >= 0) ? (long long)L.g.vw[vv] : 0;
        long long mine = 0;
        // ordered prefix over the boundary-slot members only where there are some
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
        } else {
            if (vv < L.g.n) L.etaken[vv] = taken ? w : 0;
            tile_taken += taken ? w : 0;
        }
    }
    if constexpr (STRONG) {
        __shared__ long long red[40];
        tile_taken = block_sum_i64(tile_taken, red);
        if (threadIdx.x == 0) L.tiletaken[tile] = tile_taken;
    } else {
        mapp.flush(&ctl->nM, L.listM, true);
    }
}

// Jetrs: exclusive scan of the evicted weight over tiles (one block).
__global__ void __launch_bounds__(1024) k_rb_tiletaken_scan(Level L) {
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
__global__ void __launch_bounds__(kTB) k_rb_cookie(Level L) {
    __shared__ long long sh[40];
    Ctl *ctl = L.ctl;
    const int32_t it = ctl->it, nB = ctl->nB;
    const int64_t tile = blockIdx.x;
    constexpr int kItems = kRbTile / kTB;
    int64_t v0 = tile * kRbTile + (int64_t)threadIdx.x * kItems;
    long long wv[kItems];
    long long s = 0;
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        int64_t v = v0 + i;
        wv[i] = v < L.g.n ? L.etaken[v] : 0;
        s += wv[i];
    }
    long long pre = block_exscan_i64(s, sh, nullptr) + L.tiletaken[tile];
    const long long total2 = 2 * L.capC[nB];
    JET_BLOCK_APPENDER(mapp, kRbTile + kTB);
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        int64_t v = v0 + i;
        int32_t dest = -1;
        if (wv[i] > 0) {
            long long mid2 = 2 * pre + wv[i];
            if (mid2 < total2) {
                int lo = 0, hi = nB - 1;  // largest b with 2 C_b <= mid2
                while (lo < hi) {
                    int mid = (lo + hi + 1) >> 1;
                    if (2 * L.capC[mid] <= mid2) lo = mid; else hi = mid - 1;
                }
                if (mid2 < 2 * L.capC[lo + 1]) dest = L.Bs[lo];
            }
        }
        pre += wv[i];
        bool mv = dest >= 0;
        if (mv) { L.nxt[v] = dest; L.mstamp[v] = it; }
        bool big = mv && is_big_row(L.g, (int32_t)v);
        mapp.add(mv && !big, (int32_t)v);
        if (big) L.listMb[atomicAdd(&ctl->nMb, 1)] = (int32_t)v;
    }
    mapp.flush(&ctl->nM, L.listM, true);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
__global__ void k_collect_big(DGraph g, int32_t *bigv, int32_t *count) {
    int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    bool big = v < g.n && ld_xadj(g.xadj, (int64_t)v + 1) - ld_xadj(g.xadj, v) > kSmallDeg;
    int slot = warp_append(count, big);
    if (big) bigv[slot] = v;
}

__global__ void k_fill_i32(int32_t *p, int64_t n, int32_t val) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = val;
}

__global__ void k_sum_vw(DGraph g, int64_t *out) {
    __shared__ long long red[40];
    long long s = 0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < g.n; v += (int64_t)gridDim.x * blockDim.x)
        s += g.vw[v];
    s = block_sum_i64(s, red);
    if (threadIdx.x == 0 && s) atomic_add_i64(out, s);
}

namespace {

struct LevelBufs {
    DevBuf vert, part_, misc;
    Level L{};
    int32_t nbig = 0;
    int64_t *cut2 = nullptr;
    int32_t *nbig_dev = nullptr;
};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Carves all per-level buffers out of two allocations.
int setup_level(Ctx &c, const DGraph &g, int32_t k, LevelBufs &B) {
    cudaStream_t s = c.stream;
    int64_t n = g.n;
    size_t nn = (size_t)std::max<int64_t>(n, 1);
    int32_t ntiles = (int32_t)std::max<int64_t>((n + kRbTile - 1) / kRbTile, 1);
    // per-vertex int32 arrays: best, nxt, prio, mstamp, lstamp, key, listX, listXb, listM, listMb, bigv,
    // ext, wdeg, listW, listWb
    const int nv32 = 15;
    size_t vbytes = nv32 * align256(nn * 4) + align256(nn * 8) /* etaken */;
    JET_TRY(dev_alloc(B.vert, vbytes, s));
    char *p = B.vert.as<char>();
    auto take32 = [&](void) { int32_t *r = reinterpret_cast<int32_t *>(p); p += align256(nn * 4); return r; };
    Level &L = B.L;
    L.best = take32(); L.nxt = take32(); L.prio = take32(); L.mstamp = take32(); L.lstamp = take32();
    L.key = take32(); L.listX = take32(); L.listXb = take32(); L.listM = take32(); L.listMb = take32();
    int32_t *bigv = take32();
    L.ext = take32();
    L.wdeg = take32();
    L.listW = take32();
    L.listWb = take32();
    L.rbloss = nullptr;
    L.etaken = reinterpret_cast<int64_t *>(p);
    p += align256(nn * 8);
    // per-part and control
    size_t kk = (size_t)k;
    size_t mbytes = align256(sizeof(Ctl)) + align256(kk * 8) /*pw*/ + align256(kk * 4) /*aidx*/ + align256(kk * 4) /*Bs*/ +
                    align256(kk) /*inB*/ + align256((kk + 1) * 8) /*capC*/ + align256(kk * 8) /*excess*/ +
                    align256(kk * kSlots * 8) /*bucketw*/ + align256(kk * 4) /*sstar*/ + align256(kk * 8) /*need*/ +
                    align256((size_t)ntiles * kk * 4) /*tilehist*/ + align256((size_t)ntiles * 8) /*tiletaken*/ +
                    align256(sizeof(TraceRec) * kTrace) + align256(16) /*cut2*/ + align256(16) /*nbig*/;
    JET_TRY(dev_alloc(B.misc, mbytes, s));
    char *q = B.misc.as<char>();
    auto take = [&](size_t bytes) { char *r = q; q += align256(bytes); return r; };
    L.ctl = reinterpret_cast<Ctl *>(take(sizeof(Ctl)));
    L.pw = reinterpret_cast<int64_t *>(take(kk * 8));
    L.aidx = reinterpret_cast<int32_t *>(take(kk * 4));
    L.Bs = reinterpret_cast<int32_t *>(take(kk * 4));
    L.inB = reinterpret_cast<uint8_t *>(take(kk));
    L.capC = reinterpret_cast<int64_t *>(take((kk + 1) * 8));
    L.excess = reinterpret_cast<int64_t *>(take(kk * 8));
    L.bucketw = reinterpret_cast<int64_t *>(take(kk * kSlots * 8));
    L.sstar = reinterpret_cast<int32_t *>(take(kk * 4));
    L.need = reinterpret_cast<int64_t *>(take(kk * 8));
    L.tilehist = reinterpret_cast<int32_t *>(take((size_t)ntiles * kk * 4));
    L.tiletaken = reinterpret_cast<int64_t *>(take((size_t)ntiles * 8));
    L.trace = reinterpret_cast<TraceRec *>(take(sizeof(TraceRec) * kTrace));
    B.cut2 = reinterpret_cast<int64_t *>(take(16));
    B.nbig_dev = reinterpret_cast<int32_t *>(take(16));
    L.ntiles = ntiles;
    L.g = g;
    L.k = k;
    L.bigv = bigv;
    JET_CUDA_TRY(cudaMemsetAsync(L.ctl, 0, sizeof(Ctl), s));
    JET_CUDA_TRY(cudaMemsetAsync(L.pw, 0, kk * 8, s));
    JET_CUDA_TRY(cudaMemsetAsync(B.cut2, 0, 16, s));
    JET_CUDA_TRY(cudaMemsetAsync(B.nbig_dev, 0, 16, s));
    if (n > 0) {
        k_collect_big<<<grid_for(n, kTB), kTB, 0, s>>>(g, bigv, B.nbig_dev);
        k_fill_i32<<<grid_for(n, kTB, 4096), kTB, 0, s>>>(L.lstamp, n, -2);
        k_fill_i32<<<grid_for(n, kTB, 4096), kTB, 0, s>>>(L.mstamp, n, -2);
        k_fill_i32<<<grid_for(n, kTB, 4096), kTB, 0, s>>>(L.prio, n, kNoneGain);
    }
    JET_CUDA_TRY(cudaGetLastError());
    JET_CUDA_TRY(cudaMemcpyAsync(&B.nbig, B.nbig_dev, 4, cudaMemcpyDeviceToHost, s));
    JET_CUDA_TRY(cudaStreamSynchronize(s));
    L.nbig = B.nbig;
    return JET_OK;
}

int list_grid() { return num_sms() * 4; }

size_t table_smem(int32_t k) { return (size_t)(kTB / 32) * (size_t)k * sizeof(int32_t); }

// Kernel sequences of one iteration, by kind.  Each returns, through *nk,
// the number of kernels it enqueued.
int enqueue_lp_select(const Level &L, cudaStream_t s, LpExport ex, int *nk) {
    int n = L.g.n;
    bool ew = L.g.ew != nullptr;
    int lg = list_grid();
    k_lp_scan<<<std::min(lg, grid_for((n + 3) / 4, kTB)), kTB, 0, s>>>(L);
    if (ew) k_lp_select_list<true><<<lg, kTB, 0, s>>>(L, ex);
    else k_lp_select_list<false><<<lg, kTB, 0, s>>>(L, ex);
    *nk = 2;
    if (L.nbig > 0) {
        int gb = std::min(lg, grid_for(L.nbig, kTB / 32));
        if (ew) k_lp_select_big<true><<<gb, kTB, table_smem(L.k), s>>>(L, ex);
        else k_lp_select_big<false><<<gb, kTB, table_smem(L.k), s>>>(L, ex);
        *nk += 1;
    }
    JET_CUDA_TRY(cudaGetLastError());
    return JET_OK;
}

int enqueue_lp_after(const Level &L, cudaStream_t s, LpExport ex, int *nk) {
    int n = L.g.n;
    int lg = list_grid();
    bool ew = L.g.ew != nullptr;
    int ga = std::min(lg, grid_for(n, kTB));
    if (ew) k_afterburn_small<true><<<ga, kTB, 0, s>>>(L, ex);
    else k_afterburn_small<false><<<ga, kTB, 0, s>>>(L, ex);
    *nk = 1;
    if (L.nbig > 0) {
        int gb = std::min(lg, grid_for(L.nbig, kTB / 32));
        if (ew) k_afterburn_big<true><<<gb, kTB, 0, s>>>(L, ex);
        else k_afterburn_big<false><<<gb, kTB, 0, s>>>(L, ex);
        *nk += 1;
    }
    JET_CUDA_TRY(cudaGetLastError());
    return JET_OK;
}

int enqueue_lp(const Level &L, cudaStream_t s, int *nk, LpExport ex = {nullptr, nullptr, nullptr}) {
    int a = 0, b = 0;
    JET_TRY(enqueue_lp_select(L, s, ex, &a));
    JET_TRY(enqueue_lp_after(L, s, ex, &b));
    *nk = a + b;
    return JET_OK;
}

template <bool STRONG>
int enqueue_rb_t(const Level &L, cudaStream_t s, int *nk) {
    int n = L.g.n;
    int lg = list_grid();
    bool ew = L.g.ew != nullptr;
    k_rb_scan<STRONG><<<std::min(lg, grid_for((n + 3) / 4, kTB)), kTB, 0, s>>>(L);
    if (ew) k_rb_cand_list<true, STRONG><<<lg, kTB, 0, s>>>(L);
    else k_rb_cand_list<false, STRONG><<<lg, kTB, 0, s>>>(L);
    *nk = 2;
    if (L.nbig > 0) {
        int gb = std::min(lg, grid_for(L.nbig, kTB / 32));
        if (ew) k_rb_cand_big<true, STRONG><<<gb, kTB, table_smem(L.k), s>>>(L);
        else k_rb_cand_big<false, STRONG><<<gb, kTB, table_smem(L.k), s>>>(L);
        *nk += 1;
    }
    k_rb_plan<<<std::max(1, (L.k + 7) / 8), kTB, 0, s>>>(L);
    k_rb_tilehist<<<L.ntiles, kTB, (size_t)L.k * 4, s>>>(L);
    k_rb_tilescan<<<L.k, 1024, 0, s>>>(L);
    k_rb_take<STRONG><<<L.ntiles, kTB, (size_t)L.k * 8, s>>>(L);
    *nk += 4;
    if (STRONG) {
        k_rb_tiletaken_scan<<<1, 1024, 0, s>>>(L);
        k_rb_cookie<<<L.ntiles, kTB, 0, s>>>(L);
        *nk += 2;
    }
    JET_CUDA_TRY(cudaGetLastError());
    return JET_OK;
}

int enqueue_rb(const Level &L, cudaStream_t s, bool strong, int *nk) {
    return strong ? enqueue_rb_t<true>(L, s, nk) : enqueue_rb_t<false>(L, s, nk);
}

// apply + commit + controller + best copy
int enqueue_tail(const Level &L, cudaStream_t s, int *nk) {
    int lg = list_grid();
    int n = L.g.n;
    bool ew = L.g.ew != nullptr;
    int ga = std::min(lg, grid_for(n, kTB));
    if (ew) k_apply_small<true><<<ga, kTB, (size_t)L.k * 8, s>>>(L);
    else k_apply_small<false><<<ga, kTB, (size_t)L.k * 8, s>>>(L);
    *nk = 1;
    if (L.nbig > 0) {
        int gb = std::min(lg, grid_for(L.nbig, kTB / 32));
        if (ew) k_apply_big<true><<<gb, kTB, 0, s>>>(L);
        else k_apply_big<false><<<gb, kTB, 0, s>>>(L);
        *nk += 1;
    }
    k_commit<<<ga, kTB, 0, s>>>(L);
    k_controller<<<1, 1024, 0, s>>>(L);
    k_copy_best<<<std::min(lg, grid_for(n / 4 + 1, kTB)), kTB, 0, s>>>(L);
    *nk += 3;
    JET_CUDA_TRY(cudaGetLastError());
    return JET_OK;
}

// Level start: part weights, cut, control block, P_best = P_0.
int enqueue_init(Ctx &c, LevelBufs &B, int64_t L_lim, int64_t opt, int64_t sigma) {
    cudaStream_t s = c.stream;
    Level &L = B.L;
    int64_t n = L.g.n;
    // host-known constants go straight into the control block
    int64_t consts[3] = {L_lim, opt, sigma};
    static_assert(offsetof(Ctl, opt) == offsetof(Ctl, L) + 8 && offsetof(Ctl, sigma) == offsetof(Ctl, L) + 16, "layout");
    JET_CUDA_TRY(cudaMemcpyAsync(&L.ctl->L, consts, sizeof(consts), cudaMemcpyHostToDevice, s));
    if (n > 0) {
        int gcut = std::min(list_grid(), grid_for(n, kTB));
        if (L.g.ew) k_cut_pw<true><<<gcut, kTB, (size_t)L.k * 8, s>>>(L.g, L.k, L.part, L.pw, B.cut2, L.ext, L.wdeg);
        else k_cut_pw<false><<<gcut, kTB, (size_t)L.k * 8, s>>>(L.g, L.k, L.part, L.pw, B.cut2, L.ext, L.wdeg);
        c.launches += 1;
    }
    k_ctl_init<<<1, 1024, 0, s>>>(L, B.cut2);
    c.launches += 1;
    if (n > 0) JET_CUDA_TRY(cudaMemcpyAsync(L.best, L.part, (size_t)n * 4, cudaMemcpyDeviceToDevice, s));
    JET_CUDA_TRY(cudaGetLastError());
    // the consts memcpy source lives on this stack frame: make it complete
    JET_CUDA_TRY(cudaStreamSynchronize(s));
    return JET_OK;
}

int read_ctl(Ctx &c, const Level &L, Ctl &h) {
    JET_CUDA_TRY(cudaMemcpyAsync(&h, L.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, c.stream));
    JET_CUDA_TRY(cudaStreamSynchronize(c.stream));
    return JET_OK;
}

struct EventPool {
    std::vector<cudaEvent_t> ev;
    ~EventPool() {
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
    }
    int get(cudaEvent_t &e) {
        cudaError_t r = cudaEventCreate(&e);
        if (r != cudaSuccess) { record_cuda_error(r, "cudaEventCreate", __FILE__, __LINE__); return JET_ECUDA; }
        ev.push_back(e);
        return JET_OK;
    }
};

// Host-driven loop (JET_FLAG_HOSTLOOP / JET_FLAG_PROFILE): the mode is read
// back after every iteration, as in the paper's implementation.  With
// profiling, CUDA events bracket each Jetlp select step on the level's stream.
int run_hostloop(Ctx &c, const Level &L, bool profile, float *sel_ms) {
    EventPool pool;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> marks;
    for (;;) {
        int32_t mode = 0;
        JET_CUDA_TRY(cudaMemcpyAsync(c.pinned, &L.ctl->mode, 4, cudaMemcpyDeviceToHost, c.stream));
        JET_CUDA_TRY(cudaStreamSynchronize(c.stream));
        memcpy(&mode, c.pinned, 4);
        if (mode == MODE_DONE) break;
        int nk = 0;
        if (mode == MODE_LP) {
            LpExport none{nullptr, nullptr, nullptr};
            cudaEvent_t e0 = nullptr, e1 = nullptr;
            if (profile) {
                JET_TRY(pool.get(e0));
                JET_TRY(pool.get(e1));
                JET_CUDA_TRY(cudaEventRecord(e0, c.stream));
            }
            JET_TRY(enqueue_lp_select(L, c.stream, none, &nk));
            c.launches += nk;
            if (profile) {
                JET_CUDA_TRY(cudaEventRecord(e1, c.stream));
                marks.emplace_back(e0, e1);
            }
            JET_TRY(enqueue_lp_after(L, c.stream, none, &nk));
        } else {
            JET_TRY(enqueue_rb(L, c.stream, mode == MODE_RS, &nk));
        }
        c.launches += nk;
        JET_TRY(enqueue_tail(L, c.stream, &nk));
        c.launches += nk;
    }
    float tot = 0.f;
    for (auto &m : marks) {
        float t = 0.f;
        JET_CUDA_TRY(cudaEventElapsedTime(&t, m.first, m.second));
        tot += t;
    }
    if (sel_ms) *sel_ms = tot;
    return JET_OK;
}

// Device-resident loop: graph = start kernel -> WHILE(h_loop) { SWITCH(h_mode)
// {Jetlp | Jetrw | Jetrs} -> apply, commit, controller, best copy }.
// nk_branch[3] / *nk_tail receive the kernel counts of the captured pieces.
int run_graph(Ctx &c, Level L, int *nk_branch, int *nk_tail) {
    cudaStream_t s = c.stream;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    int rc = JET_OK;
    cudaStream_t cap = nullptr;
    auto fail = [&](cudaError_t e, const char *what) {
        record_cuda_error(e, what, __FILE__, __LINE__);
        rc = e == cudaErrorMemoryAllocation ? JET_ENOMEM : JET_ECUDA;
    };
    do {
        cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
        if (e != cudaSuccess) { fail(e, "cudaStreamCreate"); break; }
        if ((e = cudaGraphCreate(&g, 0)) != cudaSuccess) { fail(e, "cudaGraphCreate"); break; }
        cudaGraphConditionalHandle h_loop, h_mode;
        if ((e = cudaGraphConditionalHandleCreate(&h_loop, g, 1, cudaGraphCondAssignDefault)) != cudaSuccess) { fail(e, "handle loop"); break; }
        if ((e = cudaGraphConditionalHandleCreate(&h_mode, g, 0, cudaGraphCondAssignDefault)) != cudaSuccess) { fail(e, "handle mode"); break; }
        L.h_loop = h_loop; L.h_mode = h_mode; L.use_graph = 1;
        // start kernel
        cudaGraphNode_t start;
        {
            cudaKernelNodeParams kp{};
            void *args[] = {&L};
            kp.func = (void *)k_graph_start;
            kp.gridDim = dim3(1); kp.blockDim = dim3(32);
            kp.kernelParams = args;
            if ((e = cudaGraphAddKernelNode(&start, g, nullptr, 0, &kp)) != cudaSuccess) { fail(e, "start node"); break; }
        }
        cudaGraphNodeParams wp{};
        wp.type = cudaGraphNodeTypeConditional;
        wp.conditional.handle = h_loop;
        wp.conditional.type = cudaGraphCondTypeWhile;
        wp.conditional.size = 1;
        cudaGraphNode_t wnode;
        if ((e = cudaGraphAddNode(&wnode, g, &start, nullptr, 1, &wp)) != cudaSuccess) { fail(e, "while node"); break; }
        cudaGraph_t body = wp.conditional.phGraph_out[0];
        cudaGraphNodeParams sp{};
        sp.type = cudaGraphNodeTypeConditional;
        sp.conditional.handle = h_mode;
        sp.conditional.type = cudaGraphCondTypeSwitch;
        sp.conditional.size = 3;
        cudaGraphNode_t snode;
        if ((e = cudaGraphAddNode(&snode, body, nullptr, nullptr, 0, &sp)) != cudaSuccess) { fail(e, "switch node"); break; }
        bool ok = true;
        for (int b = 0; b < 3 && ok; ++b) {
            cudaGraph_t bg = sp.conditional.phGraph_out[b];
            if ((e = cudaStreamBeginCaptureToGraph(cap, bg, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed)) != cudaSuccess) { fail(e, "capture branch"); ok = false; break; }
            int r = b == 0 ? enqueue_lp(L, cap, &nk_branch[0]) : enqueue_rb(L, cap, b == 2, &nk_branch[b]);
            cudaGraph_t outg = nullptr;
            e = cudaStreamEndCapture(cap, &outg);
            if (r != JET_OK) { rc = r; ok = false; break; }
            if (e != cudaSuccess) { fail(e, "end capture branch"); ok = false; break; }
        }
        if (!ok) break;
        if ((e = cudaStreamBeginCaptureToGraph(cap, body, &snode, nullptr, 1, cudaStreamCaptureModeRelaxed)) != cudaSuccess) { fail(e, "capture tail"); break; }
        int r = enqueue_tail(L, cap, nk_tail);
        cudaGraph_t outg = nullptr;
        e = cudaStreamEndCapture(cap, &outg);
        if (r != JET_OK) { rc = r; break; }
        if (e != cudaSuccess) { fail(e, "end capture tail"); break; }
        if ((e = cudaGraphInstantiate(&ge, g, 0)) != cudaSuccess) { fail(e, "cudaGraphInstantiate"); break; }
        if ((e = cudaGraphLaunch(ge, s)) != cudaSuccess) { fail(e, "cudaGraphLaunch"); break; }
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) { fail(e, "sync graph"); break; }
    } while (0);
    if (ge) cudaGraphExecDestroy(ge);
    if (g) cudaGraphDestroy(g);
    if (cap) cudaStreamDestroy(cap);
    return rc;
}

}  // namespace

// Weight of the whole graph (needed for the balance limit).
static int total_vweight(Ctx &c, const DGraph &g, int64_t &W) {
    DevBuf t;
    JET_TRY(dev_alloc(t, 16, c.stream));
    JET_CUDA_TRY(cudaMemsetAsync(t.p, 0, 16, c.stream));
    if (g.n > 0) {
        k_sum_vw<<<std::min(list_grid(), grid_for(g.n, kTB)), kTB, 0, c.stream>>>(g, t.as<int64_t>());
        c.launches += 1;
    }
    JET_CUDA_TRY(cudaGetLastError());
    JET_CUDA_TRY(cudaMemcpyAsync(c.pinned, t.p, 8, cudaMemcpyDeviceToHost, c.stream));
    JET_CUDA_TRY(cudaStreamSynchronize(c.stream));
    W = c.pinned[0];
    return JET_OK;
}

static void fill_level_params(Ctx &c, Level &L, int32_t is_finest, uint64_t seed) {
    const jet_options &o = c.opt;
    L.cq16 = (int32_t)llround((is_finest ? o.c_fine : o.c_coarse) * 65536.0);
    L.phi_ppm = llround(o.phi * 1e6);
    L.max_no_improve = o.max_no_improve;
    L.weak_limit = o.weak_limit;
    L.max_iters = o.max_iters_per_level;
    L.abl = o.flags & (ABL_NO_LOCKS | ABL_NO_AFTERBURN | ABL_WEAK_AFTERBURN | ABL_BASELINE_LP);
    L.seed = seed;
    L.use_graph = 0;
    L.h_loop = L.h_mode = 0;
}

// Algorithmic DRAM bytes of each pass, from the per-iteration trace (neighbour
// gathers and scatters of part/prio/nxt/ext are taken as cache hits; beta =
// bytes per CSR entry: 8 with edge weights, 4 without; "boundary" = ext > 0):
//   Jetlp select   4 n + 4 nb + 28 w + beta deg(W) + 12 |X|
//                  (ext of every vertex, lock stamp of the nb boundary
//                   vertices; for the w listed ones: list write and read,
//                   xadj pair, part, row; priority, P_d and list entry of X)
//   afterburner    20 |X| + beta deg X + 8 |M|, plus 8 |X| to clear priorities
//   rebalance      24 n + 16 c + 32 r + beta deg(R) (+ 16 n for Jetrs)
//                  (part and key of every vertex, tile passes; ext, vwgt,
//                   weighted degree or destination of the c candidates; list,
//                   xadj pair, part, key, destination and row of the r listed)
//   apply+commit   36 |M| + beta deg M + 16 k
static void byte_model(const std::vector<TraceRec> &tr, const DGraph &g, int32_t k, uint32_t abl, LevelReport &rep) {
    int64_t n = g.n, beta = g.ew ? 8 : 4;
    bool ab = !(abl & (ABL_NO_AFTERBURN | ABL_BASELINE_LP));
    for (const TraceRec &r : tr) {
        int64_t b = 36 * r.nm + beta * r.degm + 16 * (int64_t)k;
        if (r.kind == MODE_LP) {
            int64_t sel = 4 * n + 4 * r.nbnd + 28 * r.nexam + beta * r.degexam + 12 * r.nx;
            rep.sel_bytes += sel;
            rep.sel_launches += 1;
            b += sel + (ab ? 20 * r.nx + beta * r.degx : 0) + 8 * r.nm + 8 * r.nx;
        } else {
            b += 24 * n + 16 * r.nx + 32 * r.nbnd + beta * r.degexam + (r.kind == MODE_RS ? 16 * n : 0);
        }
        rep.bytes_model += b;
    }
}

int refine_level(Ctx &c, const DGraph &g, int32_t k, double eps, int32_t is_finest, uint64_t seed,
                 int32_t *part_inout, int64_t *cut_out, int64_t *maxw_out, LevelReport *rep_out) {
    LevelReport rep;
    int64_t W = 0;
    JET_TRY(total_vweight(c, g, W));
    int64_t opt = 0;
    int64_t L_lim = balance_limit(W, k, eps, &opt);
    int64_t sigma = opt + (L_lim - opt) / 2;
    LevelBufs B;
    JET_TRY(setup_level(c, g, k, B));
    c.launches += g.n > 0 ? 4 : 0;
    Level &L = B.L;
    L.part = part_inout;
    fill_level_params(c, L, is_finest, seed);
    JET_TRY(enqueue_init(c, B, L_lim, opt, sigma));
    bool hostloop = (c.opt.flags & (JET_FLAG_HOSTLOOP | JET_FLAG_PROFILE)) != 0;
    int nk_branch[3] = {0, 0, 0}, nk_tail = 0;
    if (g.n > 0) {
        if (hostloop) JET_TRY(run_hostloop(c, L, (c.opt.flags & JET_FLAG_PROFILE) != 0, &rep.sel_ms));
        else JET_TRY(run_graph(c, L, nk_branch, &nk_tail));
        JET_CUDA_TRY(cudaMemcpyAsync(part_inout, L.best, (size_t)g.n * 4, cudaMemcpyDeviceToDevice, c.stream));
    }
    Ctl h;
    JET_TRY(read_ctl(c, L, h));
    int32_t iters = h.it;
    if (!hostloop && g.n > 0) {
        c.launches += 1;  // start kernel
        for (int kd = 0; kd < 3; ++kd) c.launches += (int64_t)h.kcount[kd] * (nk_branch[kd] + nk_tail);
    }
    c.last_trace.iters = iters;
    int32_t nrec = std::min<int32_t>(iters, kTrace);
    c.last_trace.rec.resize((size_t)nrec);
    if (nrec > 0) {
        JET_CUDA_TRY(cudaMemcpyAsync(c.last_trace.rec.data(), L.trace, sizeof(TraceRec) * (size_t)nrec,
                                     cudaMemcpyDeviceToHost, c.stream));
        JET_CUDA_TRY(cudaStreamSynchronize(c.stream));
    }
    rep.iters = iters;
    for (int kd = 0; kd < 3; ++kd) rep.kinds[kd] = h.kcount[kd];
    byte_model(c.last_trace.rec, g, k, L.abl, rep);
    if (rep_out) *rep_out = rep;
    if (cut_out) *cut_out = h.best_cut;
    if (maxw_out) *maxw_out = h.best_maxw;
    if (!h.best_bal) return JET_WUNBALANCED;
    if (h.hit_cap) return JET_WITERLIMIT;
    return JET_OK;
}

// ---- single passes --------------------------------------------------------

__global__ void k_locks_from_mask(const uint8_t *locked, int32_t *lstamp, int64_t n) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        lstamp[v] = (locked && locked[v]) ? 0 : -2;
}

__global__ void k_set_epoch(Ctl *ctl, int32_t epoch, int32_t mode) {
    ctl->lp_epoch = epoch;
    ctl->mode = mode;
    ctl->it = 0;
    ctl->nW = ctl->nWb = 0;
    ctl->nX = ctl->nXb = ctl->nM = ctl->nMb = 0;
    ctl->ncand = 0;
}

__global__ void k_export_lp(Level L, uint8_t *inx, uint8_t *inm) {
    const int32_t it = L.ctl->it;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < L.g.n; v += (int64_t)gridDim.x * blockDim.x) {
        if (inx) inx[v] = L.prio[v] != kNoneGain;
        if (inm) inm[v] = L.mstamp[v] == it;
    }
}

int lp_pass(Ctx &c, const DGraph &g, int32_t k, const int32_t *part, const uint8_t *locked, double cval, uint32_t flags,
            int32_t *pd_out, int32_t *gain_out, uint8_t *inx_out, int32_t *f2_out, uint8_t *inm_out) {
    cudaStream_t s = c.stream;
    if (g.n == 0) return JET_OK;
    LevelBufs B;
    JET_TRY(setup_level(c, g, k, B));
    Level &L = B.L;
    L.part = const_cast<int32_t *>(part);   // read only in this pass
    fill_level_params(c, L, 1, 0);
    L.cq16 = (int32_t)llround(cval * 65536.0);
    L.abl = flags & (ABL_NO_LOCKS | ABL_NO_AFTERBURN | ABL_WEAK_AFTERBURN | ABL_BASELINE_LP);
    {
        int gcut = std::min(list_grid(), grid_for(g.n, kTB));
        if (g.ew) k_cut_pw<true><<<gcut, kTB, (size_t)k * 8, s>>>(g, k, L.part, L.pw, B.cut2, L.ext, nullptr);
        else k_cut_pw<false><<<gcut, kTB, (size_t)k * 8, s>>>(g, k, L.part, L.pw, B.cut2, L.ext, nullptr);
    }
    k_locks_from_mask<<<grid_for(g.n, kTB, 4096), kTB, 0, s>>>(locked, L.lstamp, g.n);
    k_set_epoch<<<1, 1, 0, s>>>(L.ctl, 0, MODE_LP);
    DevBuf tmp_pd, tmp_gain;
    LpExport ex{pd_out, gain_out, f2_out};
    if (!ex.pd || !ex.gain) {
        JET_TRY(dev_alloc(tmp_pd, (size_t)g.n * 4, s));
        JET_TRY(dev_alloc(tmp_gain, (size_t)g.n * 4, s));
        if (!ex.pd) ex.pd = tmp_pd.as<int32_t>();
        if (!ex.gain) ex.gain = tmp_gain.as<int32_t>();
    }
    if (f2_out) JET_CUDA_TRY(cudaMemsetAsync(f2_out, 0, (size_t)g.n * 4, s));
    // the select writes P_d and F only for the vertices it examines
    JET_CUDA_TRY(cudaMemcpyAsync(ex.pd, part, (size_t)g.n * 4, cudaMemcpyDeviceToDevice, s));
    k_fill_i32<<<grid_for(g.n, kTB, 4096), kTB, 0, s>>>(ex.gain, g.n, kNoneGain);
    int nk = 0;
    JET_TRY(enqueue_lp(L, s, &nk, ex));
    k_export_lp<<<grid_for(g.n, kTB, 4096), kTB, 0, s>>>(L, inx_out, inm_out);
    JET_CUDA_TRY(cudaGetLastError());
    JET_CUDA_TRY(cudaStreamSynchronize(s));
    return JET_OK;
}

__global__ void k_export_rb(Level L, int32_t *dest, int32_t *loss) {
    const int32_t it = L.ctl->it;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < L.g.n; v += (int64_t)gridDim.x * blockDim.x) {
        if (dest) dest[v] = L.mstamp[v] == it ? L.nxt[v] : -1;
        if (loss && L.key[v] < 0) loss[v] = kNoneGain;
    }
}

__global__ void __launch_bounds__(1024) k_rb_pass_init(Level L, const int64_t *cut2, int32_t mode) {
    __shared__ long long sh[40];
    Ctl *ctl = L.ctl;
    if (threadIdx.x == 0) {
        ctl->cut = *cut2 / 2;
        ctl->it = 0; ctl->mode = mode;
        ctl->nW = ctl->nWb = 0;
        ctl->nX = ctl->nXb = ctl->nM = ctl->nMb = 0;
        ctl->ncand = 0;
    }
    __syncthreads();
    compute_classes(L, sh);
}

__global__ void k_clear_keys(Level L) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < L.g.n; v += (int64_t)gridDim.x * blockDim.x)
        L.key[v] = -1;
}

int rebalance_pass(Ctx &c, const DGraph &g, int32_t k, double eps, int32_t strong, uint64_t seed, int32_t iter,
                   const int32_t *part, int32_t *dest_out, int32_t *loss_out, int64_t *nmoves, int64_t *ncand) {
    cudaStream_t s = c.stream;
    if (nmoves) *nmoves = 0;
    if (ncand) *ncand = 0;
    if (g.n == 0) return JET_OK;
    int64_t W = 0;
    JET_TRY(total_vweight(c, g, W));
    int64_t opt = 0;
    int64_t L_lim = balance_limit(W, k, eps, &opt);
    int64_t sigma = opt + (L_lim - opt) / 2;
    LevelBufs B;
    JET_TRY(setup_level(c, g, k, B));
    Level &L = B.L;
    L.part = const_cast<int32_t *>(part);   // read only in this pass
    fill_level_params(c, L, 1, seed);
    int64_t consts[3] = {L_lim, opt, sigma};
    JET_CUDA_TRY(cudaMemcpyAsync(&L.ctl->L, consts, sizeof(consts), cudaMemcpyHostToDevice, s));
    int gcut = std::min(list_grid(), grid_for(g.n, kTB));
    if (g.ew) k_cut_pw<true><<<gcut, kTB, (size_t)k * 8, s>>>(g, k, L.part, L.pw, B.cut2, L.ext, L.wdeg);
    else k_cut_pw<false><<<gcut, kTB, (size_t)k * 8, s>>>(g, k, L.part, L.pw, B.cut2, L.ext, L.wdeg);
    L.rbloss = loss_out;
    k_rb_pass_init<<<1, 1024, 0, s>>>(L, B.cut2, strong ? MODE_RS : MODE_RW);
    // the pass API takes the iteration index as a parameter: set ctl->it
    JET_CUDA_TRY(cudaMemcpyAsync(&L.ctl->it, &iter, 4, cudaMemcpyHostToDevice, s));
    k_clear_keys<<<grid_for(g.n, kTB, 4096), kTB, 0, s>>>(L);
    int nk = 0;
    JET_TRY(enqueue_rb(L, s, strong != 0, &nk));
    Ctl h;
    JET_TRY(read_ctl(c, L, h));
    if (nmoves) *nmoves = (int64_t)h.nM + h.nMb;
    if (ncand) *ncand = h.ncand;
    k_export_rb<<<grid_for(g.n, kTB, 4096), kTB, 0, s>>>(L, dest_out, loss_out);
    JET_CUDA_TRY(cudaGetLastError());
    JET_CUDA_TRY(cudaStreamSynchronize(s));
    return JET_OK;
}

int cut_and_weights(Ctx &c, const DGraph &g, int32_t k, const int32_t *part, int64_t *cut_out, int64_t *pw_dev) {
    cudaStream_t s = c.stream;
    DevBuf t;
    JET_TRY(dev_alloc(t, 16 + (size_t)k * 8, s));
    int64_t *cut2 = t.as<int64_t>();
    int64_t *pw = pw_dev ? pw_dev : cut2 + 2;
    JET_CUDA_TRY(cudaMemsetAsync(cut2, 0, 16, s));
    JET_CUDA_TRY(cudaMemsetAsync(pw, 0, (size_t)k * 8, s));
    if (g.n > 0) {
        int gcut = std::min(list_grid(), grid_for(g.n, kTB));
        if (g.ew) k_cut_pw<true><<<gcut, kTB, (size_t)k * 8, s>>>(g, k, part, pw, cut2, nullptr, nullptr);
        else k_cut_pw<false><<<gcut, kTB, (size_t)k * 8, s>>>(g, k, part, pw, cut2, nullptr, nullptr);
    }
    JET_CUDA_TRY(cudaGetLastError());
    JET_CUDA_TRY(cudaMemcpyAsync(c.pinned, cut2, 8, cudaMemcpyDeviceToHost, s));
    JET_CUDA_TRY(cudaStreamSynchronize(s));
    if (cut_out) *cut_out = c.pinned[0] / 2;
    return JET_OK;
}

// ---- a single Jetlp pass in caller-provided scratch ------------------------
// Same kernels and launch configuration as lp_pass; the level arrays, the
// control block and the row-class counter live in `scratch` instead of
// stream-ordered allocations.
int lp_pass_in_scratch(Ctx &c, const DGraph &g, int32_t k, const int32_t *part, const uint8_t *locked, double cval,
                       uint32_t flags, int32_t *pd_out, int32_t *gain_out, uint8_t *inx_out, int32_t *f2_out,
                       uint8_t *inm_out, char *scratch) {
    cudaStream_t s = c.stream;
    if (g.n == 0) return JET_OK;
    size_t nn = (size_t)g.n;
    char *p = scratch;
    auto take32 = [&]() { int32_t *r = reinterpret_cast<int32_t *>(p); p += align256c(nn * 4); return r; };
    Level L{};
    L.g = g;
    L.k = k;
    L.part = const_cast<int32_t *>(part);   // read only in this pass
    L.nxt = take32(); L.prio = take32(); L.mstamp = take32(); L.lstamp = take32();
    L.listX = take32(); L.listXb = take32(); L.listM = take32(); L.listMb = take32();
    int32_t *bigv = take32();
    int32_t *tmp_pd = take32(), *tmp_gain = take32();
    L.ext = take32();
    L.listW = take32();
    L.listWb = take32();
    L.ctl = reinterpret_cast<Ctl *>(p);
    p += align256c(sizeof(Ctl));
    int32_t *nbig_dev = reinterpret_cast<int32_t *>(p);
    p += 256;
    L.pw = reinterpret_cast<int64_t *>(p);
    p += align256c((size_t)JET_MAX_K * 8);
    int64_t *cut2 = reinterpret_cast<int64_t *>(p);
    L.bigv = bigv;
    fill_level_params(c, L, 1, 0);
    L.cq16 = (int32_t)llround(cval * 65536.0);
    L.abl = flags & (ABL_NO_LOCKS | ABL_NO_AFTERBURN | ABL_WEAK_AFTERBURN | ABL_BASELINE_LP);
    // the array keeps the previous call's contents: clear what must start at zero
    JET_CUDA_TRY(cudaMemsetAsync(L.ctl, 0, sizeof(Ctl), s));
    JET_CUDA_TRY(cudaMemsetAsync(nbig_dev, 0, 16, s));
    JET_CUDA_TRY(cudaMemsetAsync(L.pw, 0, (size_t)k * 8, s));
    JET_CUDA_TRY(cudaMemsetAsync(cut2, 0, 16, s));
    {
        int gcut = std::min(list_grid(), grid_for(g.n, kTB));
        if (g.ew) k_cut_pw<true><<<gcut, kTB, (size_t)k * 8, s>>>(g, k, L.part, L.pw, cut2, L.ext, nullptr);
        else k_cut_pw<false><<<gcut, kTB, (size_t)k * 8, s>>>(g, k, L.part, L.pw, cut2, L.ext, nullptr);
    }
    k_collect_big<<<grid_for(g.n, kTB), kTB, 0, s>>>(g, bigv, nbig_dev);
    k_fill_i32<<<grid_for(g.n, kTB, 4096), kTB, 0, s>>>(L.mstamp, g.n, -2);
    k_fill_i32<<<grid_for(g.n, kTB, 4096), kTB, 0, s>>>(L.prio, g.n, kNoneGain);
    k_locks_from_mask<<<grid_for(g.n, kTB, 4096), kTB, 0, s>>>(locked, L.lstamp, g.n);
    k_set_epoch<<<1, 1, 0, s>>>(L.ctl, 0, MODE_LP);
    JET_CUDA_TRY(cudaGetLastError());
    JET_CUDA_TRY(cudaMemcpyAsync(c.pinned, nbig_dev, 4, cudaMemcpyDeviceToHost, s));
    JET_CUDA_TRY(cudaStreamSynchronize(s));
    L.nbig = (int32_t)(c.pinned[0] & 0xFFFFFFFF);
    LpExport ex{pd_out ? pd_out : tmp_pd, gain_out ? gain_out : tmp_gain, f2_out};
    if (f2_out) JET_CUDA_TRY(cudaMemsetAsync(f2_out, 0, nn * 4, s));
    JET_CUDA_TRY(cudaMemcpyAsync(ex.pd, part, nn * 4, cudaMemcpyDeviceToDevice, s));
    k_fill_i32<<<grid_for(g.n, kTB, 4096), kTB, 0, s>>>(ex.gain, g.n, kNoneGain);
    int nk = 0;
    JET_TRY(enqueue_lp(L, s, &nk, ex));
    k_export_lp<<<grid_for(g.n, kTB, 4096), kTB, 0, s>>>(L, inx_out, inm_out);
    JET_CUDA_TRY(cudaGetLastError());
    JET_CUDA_TRY(cudaStreamSynchronize(s));
    return JET_OK;
}

}  // namespace jet
