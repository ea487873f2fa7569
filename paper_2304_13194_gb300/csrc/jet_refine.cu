// Jet refinement on one level (Sec. 4): Jetlp (Alg. 4), Jetrw (Alg. 5),
// Jetrs (Sec. 4.2.2) and the driver of Alg. 3, for sm_103a.
//
// The passes themselves are device functions in jet_phases.cuh.  They run in
// one of two ways:
//  * large levels: one kernel per phase, and the whole level loop is a CUDA
//    graph with a WHILE node around SWITCH nodes over {Jetlp, Jetrw, Jetrs}
//    (two iterations per loop body); the controller, in the last block of
//    the apply kernel, sets the conditionals, so no host round trip happens
//    per iteration (the paper blames that round trip for its weaker
//    coarse-level speedup, Sec. 6.2);
//  * small levels: one thread block cluster (up to 16 SMs) runs every
//    iteration of the level in a single launch, the phases separated by the
//    hardware cluster barrier — no launch or graph node per phase.
#include "jet_phases.cuh"

#include <cooperative_groups.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>

namespace jet {

namespace cg = cooperative_groups;

extern __shared__ __align__(16) unsigned char jet_arena[];

// ---------------------------------------------------------------------------
// cut and part weights of a partition (Sec. 2.1), used at level start; also
// the neighbour counts in other parts (ext) and the weighted degrees
// ---------------------------------------------------------------------------
// Short rows (up to 2 kSmallDeg entries) one thread each; longer rows staged
// for the block's warps, hub rows (over kHugeDeg) for the whole block.
// (A phase over the blocks of a Grid: one kernel launch, or one cluster.)
template <bool EW>
__device__ inline void ph_cut_pw(const DGraph &g, int32_t k, const int32_t *__restrict__ part,
                                 int64_t *__restrict__ pw, int64_t *__restrict__ cut2, int32_t *__restrict__ ext,
                                 int32_t *__restrict__ wdeg, Grid G, char *arena) {
    long long *shpw = reinterpret_cast<long long *>(arena);
    int32_t *stage = reinterpret_cast<int32_t *>(arena + align16((size_t)k * 8));
    __shared__ long long red[40];
    for (int i = threadIdx.x; i < k; i += blockDim.x) shpw[i] = 0;
    JET_APPENDER(bigs, stage, kBigCap);
    long long c = 0;
    const unsigned lane = lane_id();
    // one row's cut share, ext and weighted degree over the entries first,
    // first + step, ... (four entries per thread at a time: their ids, then
    // their parts, in flight together)
    auto row_share = [&](int64_t first, int64_t e, int64_t step, int32_t p, long long &cv, long long &nx,
                         long long &wd) {
        constexpr int U = 4;
        for (int64_t j0 = first; j0 < e; j0 += U * step) {
            int32_t u[U], w[U];
#pragma unroll
            for (int q = 0; q < U; ++q) {
                const int64_t j = j0 + q * step;
                u[q] = j < e ? g.adj[j] : -1;
                w[q] = j < e ? edge_w<EW>(g, j) : 0;
            }
#pragma unroll
            for (int q = 0; q < U; ++q) {
                const bool other = u[q] >= 0 && part[u[q]] != p;
                cv += other ? w[q] : 0;
                nx += other ? 1 : 0;
                wd += w[q];
            }
        }
    };
    auto warp_row = [&](int32_t v) {
        const int32_t p = part[v];
        const int64_t b = ld_xadj(g.xadj, v), e = ld_xadj(g.xadj, (int64_t)v + 1);
        long long cv = 0, nx = 0, wd = 0;
        row_share(b + lane, e, 32, p, cv, nx, wd);
        cv = warp_sum_i64(cv);
        nx = warp_sum_i64(nx);
        wd = warp_sum_i64(wd);
        if (lane == 0) {
            c += cv;
            if (ext) ext[v] = (int32_t)nx;
            if (wdeg) wdeg[v] = (int32_t)wd;
        }
    };
    auto block_row = [&](int32_t v) {
        const int32_t p = part[v];
        const int64_t b = ld_xadj(g.xadj, v), e = ld_xadj(g.xadj, (int64_t)v + 1);
        long long cv = 0, nx = 0, wd = 0;
        row_share(b + threadIdx.x, e, blockDim.x, p, cv, nx, wd);
        cv = block_sum_i64(cv, red);
        nx = block_sum_i64(nx, red);
        wd = block_sum_i64(wd, red);
        if (threadIdx.x == 0) {
            c += cv;
            if (ext) ext[v] = (int32_t)nx;
            if (wdeg) wdeg[v] = (int32_t)wd;
        }
    };
    for (int64_t v0 = (int64_t)G.bid * blockDim.x; v0 < g.n; v0 += (int64_t)G.nb * blockDim.x) {
        const int64_t v = v0 + threadIdx.x;
        bool big = false;
        if (v < g.n) {
            const int32_t p = part[v];
            atomicAdd(reinterpret_cast<unsigned long long *>(&shpw[p]), (unsigned long long)(long long)(g.vw ? g.vw[v] : 1));
            const int64_t b = ld_xadj(g.xadj, v), e = ld_xadj(g.xadj, v + 1);
            if (e - b > 2 * kSmallDeg) {
                big = true;
            } else {
                int32_t nx = 0, wd = 0, cv = 0;
                for (int64_t j = b; j < e; ++j) {
                    const int32_t w = edge_w<EW>(g, j);
                    const bool other = part[g.adj[j]] != p;
                    cv += other ? w : 0;
                    nx += other ? 1 : 0;
                    wd += w;
                }
                c += cv;
                if (ext) ext[v] = nx;
                if (wdeg) wdeg[v] = wd;
            }
        }
        bigs.add(big, (int32_t)v);
        bigs.drain(false, g.xadj, warp_row, block_row);
    }
    bigs.drain(true, g.xadj, warp_row, block_row);
    c = block_sum_i64(c, red);
    if (threadIdx.x == 0 && c) atomic_add_i64(cut2, c);
    __syncthreads();
    for (int i = threadIdx.x; i < k; i += blockDim.x)
        if (shpw[i]) atomic_add_i64(&pw[i], shpw[i]);
    __syncthreads();
}

template <bool EW>
__global__ void __launch_bounds__(kTB) k_cut_pw(DGraph g, int32_t k, const int32_t *__restrict__ part,
                                                 int64_t *__restrict__ pw, int64_t *__restrict__ cut2,
                                                 int32_t *__restrict__ ext, int32_t *__restrict__ wdeg) {
    ph_cut_pw<EW>(g, k, part, pw, cut2, ext, wdeg, launch_grid(), reinterpret_cast<char *>(jet_arena));
}

// dynamic shared memory of k_cut_pw
size_t sm_cut_pw(int32_t k) { return align16((size_t)k * 8) + (size_t)kBigCap * 4; }

// ---------------------------------------------------------------------------
// one kernel per phase (large levels and the single-pass entry points)
// ---------------------------------------------------------------------------
#define JET_ARENA reinterpret_cast<char *>(jet_arena)

// Resident blocks of 256 threads per SM that the row kernels are compiled for
// (register budget 65536 / (256 x blocks)).
#ifndef JET_ROW_MINB
#define JET_ROW_MINB 4
#endif

// Level start: the host-known limits into the control block, then its state
// from the initial cut and part weights.
__global__ void __launch_bounds__(1024) k_ctl_init(Level L, const int64_t *cut2, int64_t Llim, int64_t opt,
                                                   int64_t sigma) {
    if (threadIdx.x == 0) {
        L.ctl->L = Llim;
        L.ctl->opt = opt;
        L.ctl->sigma = sigma;
    }
    __syncthreads();
    ph_ctl_init(L, cut2);
}

// Sets the CUDA-graph conditionals for the first iteration.
__global__ void k_graph_start(Level L) {
    if (threadIdx.x == 0) {
        int32_t m = L.ctl->mode;
        cudaGraphSetConditional((cudaGraphConditionalHandle)L.h_mode, (unsigned)m);
        cudaGraphSetConditional((cudaGraphConditionalHandle)L.h_loop, m == MODE_DONE ? 0u : 1u);
    }
}

__global__ void __launch_bounds__(kTB) k_copy_best(Level L) { ph_copy_best(L, launch_grid()); }
// Jetlp: work list, select, afterburner (+ the P_best copy at its end: the
// copy only reads part, which the afterburner does not change, and stays
// out of the select step)
__global__ void __launch_bounds__(kTB) k_lp_scan(Level L) {
    pdl_enter();
    ph_lp_scan(L, launch_grid(), JET_ARENA);
}
template <bool EW>
__global__ void __launch_bounds__(kTB, JET_ROW_MINB) k_lp_select(Level L, LpExport ex) {
    pdl_enter();
    ph_lp_select<EW>(L, ex, launch_grid(), JET_ARENA);
}
template <bool EW>
__global__ void __launch_bounds__(kTB, JET_ROW_MINB) k_afterburn(Level L, LpExport ex) {
    pdl_enter();
    // the P_best copy only reads part, which this phase leaves alone: its
    // flag is loaded with the phase's first loads, the copy runs last
    const int32_t copy = L.ctl->copy_best;
    ph_afterburn<EW>(L, ex, launch_grid(), JET_ARENA);
    if (copy) copy_best_rows(L, launch_grid());
}
// apply + commit; the last block runs the controller
template <bool EW>
__global__ void __launch_bounds__(kTB, JET_ROW_MINB) k_apply(Level L) {
    pdl_enter();
    ph_apply<EW>(L, launch_grid(), JET_ARENA);
    if (last_block(L.ctl)) ph_controller(L);
}
// rebalancing: candidates (+ the P_best copy at the end), rows (+ plan), tile
// sums, tile scan, take (+ Jetrs eviction scan), cookie cutter
template <bool STRONG>
__global__ void __launch_bounds__(kTB) k_rb_scan(Level L) {
    pdl_enter();
    const int32_t copy = L.ctl->copy_best;   // as in k_afterburn
    ph_rb_scan<STRONG>(L, launch_grid(), JET_ARENA);
    if (copy) copy_best_rows(L, launch_grid());
}
template <bool EW, bool STRONG>
__global__ void __launch_bounds__(kTB, JET_ROW_MINB) k_rb_cand(Level L) {
    pdl_enter();
    ph_rb_cand<EW, STRONG>(L, launch_grid(), JET_ARENA);
    if (last_block(L.ctl)) ph_rb_plan(L);
}
__global__ void __launch_bounds__(kRbTile) k_rb_tilehist(Level L) {
    pdl_enter();
    ph_rb_tilehist(L, launch_grid(), JET_ARENA);
}
__global__ void __launch_bounds__(1024) k_rb_tilescan(Level L) {
    pdl_enter();
    ph_rb_tilescan(L, launch_grid());
}
template <bool STRONG>
__global__ void __launch_bounds__(kRbTile) k_rb_take(Level L) {
    pdl_enter();
    ph_rb_take<STRONG>(L, launch_grid(), JET_ARENA);
    if constexpr (STRONG) {
        if (last_block(L.ctl)) ph_rb_tiletaken_scan(L);
    }
}
__global__ void __launch_bounds__(kRbTile) k_rb_cookie(Level L) {
    pdl_enter();
    ph_rb_cookie(L, launch_grid(), JET_ARENA);
}

// ---------------------------------------------------------------------------
// one cluster per level: every iteration in a single launch
// ---------------------------------------------------------------------------
constexpr int kClusterThreads = 1024;

template <bool EW, bool STRONG>
__device__ __forceinline__ void cluster_rebalance(const Level &L, Grid G, char *arena, cg::cluster_group &cl) {
    ph_rb_scan<STRONG>(L, G, arena);
    cl.sync();
    ph_rb_cand<EW, STRONG>(L, G, arena);
    cl.sync();
    if (G.bid == 0) ph_rb_plan(L);
    cl.sync();
    ph_rb_tilehist(L, G, arena);
    cl.sync();
    ph_rb_tilescan(L, G);
    cl.sync();
    ph_rb_take<STRONG>(L, G, arena);
    cl.sync();
    if constexpr (STRONG) {
        if (G.bid == 0) ph_rb_tiletaken_scan(L);
        cl.sync();
        ph_rb_cookie(L, G, arena);
        cl.sync();
    }
}

// The whole loop of Alg. 3 on one level.  The blocks of the cluster take the
// phases in lockstep (cluster barrier between phases; block 0 runs the
// tails); the loop ends when the controller chooses DONE, which the stop
// rule or the iteration cap guarantees.  Every block reads the same mode
// after the same barrier, so all of them meet every barrier.
template <bool EW>
__device__ inline void cluster_level_loop(const Level &L, Grid G, char *arena, cg::cluster_group &cl) {
    const LpExport none{nullptr, nullptr, nullptr};
    for (;;) {
        const int32_t mode = L.ctl->mode;
        if (mode == MODE_DONE) break;
        ph_copy_best(L, G);   // P_best <- P_iter asked for by the previous controller
        if (mode == MODE_LP) {
            ph_lp_scan(L, G, arena);
            cl.sync();
            ph_lp_select<EW>(L, none, G, arena);
            cl.sync();
            ph_afterburn<EW>(L, none, G, arena);
            cl.sync();
        } else if (mode == MODE_RW) {
            cluster_rebalance<EW, false>(L, G, arena, cl);
        } else {
            cluster_rebalance<EW, true>(L, G, arena, cl);
        }
        ph_apply<EW>(L, G, arena);
        cl.sync();
        if (G.bid == 0) ph_controller(L);
        cl.sync();
    }
    ph_copy_best(L, G);
}

template <bool EW>
__global__ void __launch_bounds__(kClusterThreads, 1) k_refine_cluster(Level L) {
    cg::cluster_group cl = cg::this_cluster();
    const Grid G{(int)cl.block_rank(), (int)cl.num_blocks()};
    cluster_level_loop<EW>(L, G, JET_ARENA, cl);
}

// ---------------------------------------------------------------------------
// one cooperative launch per level: every iteration in a single grid
// ---------------------------------------------------------------------------
// Polls of a block waiting at a grid barrier before it gives up, unless the
// context's options set another limit (with a sleep of ~64 ns between polls
// after the first few: about a second or more, orders of magnitude above the
// longest phase).
constexpr long long kBarPollLimit = 1LL << 22;

__device__ __forceinline__ uint32_t ld_volatile_u32(const uint32_t *p) { return *(const volatile uint32_t *)p; }

// Grid barrier of the persistent loop (cooperative launch: every block is
// resident).  A block reads the generation, fences its writes and arrives;
// the last of the gridDim.x arrivals runs `tail` (every thread of that
// block, with all the other blocks' writes visible), clears the count and
// publishes the next generation; the others wait for it.  Each wait is
// bounded: a block that runs out of polls sets ctl->bar_err and leaves, and
// every block that passes a barrier after that sees the flag and leaves too,
// so the launch always ends; the host then reports JET_ETIMEOUT.  Returns
// false when the loop must stop (all threads of the block agree).
template <class Tail>
__device__ __forceinline__ bool grid_sync(const Level &L, Tail &&tail) {
    __shared__ int s_last, s_ok;
    __shared__ uint32_t s_gen;
    Ctl *ctl = L.ctl;
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t gen = ld_volatile_u32(&ctl->bar_gen);
        __threadfence();
        const uint32_t a = atomicAdd(&ctl->bar_count, 1u);
        const bool last = a == gridDim.x - 1;
        if (last) __threadfence();
        s_gen = gen;
        s_last = last ? 1 : 0;
    }
    __syncthreads();
    if (s_last) {
        tail();
        __syncthreads();
        if (threadIdx.x == 0) {
            atomicExch(&ctl->bar_count, 0u);
            __threadfence();
            atomicExch(&ctl->bar_gen, s_gen + 1u);
        }
    } else if (threadIdx.x == 0) {
        long long polls = 0;
        while (ld_volatile_u32(&ctl->bar_gen) == s_gen) {
            if (++polls > L.poll_limit) {
                atomicExch(&ctl->bar_err, 1);
                break;
            }
            if (polls > 16) __nanosleep(64);
        }
        __threadfence();
    }
    if (threadIdx.x == 0) s_ok = *(volatile int32_t *)&ctl->bar_err == 0;
    __syncthreads();
    return s_ok != 0;
}

struct NoTail {
    __device__ __forceinline__ void operator()() const {}
};

template <bool EW, bool STRONG>
__device__ __forceinline__ bool grid_rebalance(const Level &L, Grid G, char *arena) {
    ph_rb_scan<STRONG>(L, G, arena);
    if (!grid_sync(L, NoTail{})) return false;
    ph_rb_cand<EW, STRONG>(L, G, arena);
    if (!grid_sync(L, [&] { ph_rb_plan(L); })) return false;
    ph_rb_tilehist(L, G, arena);
    if (!grid_sync(L, NoTail{})) return false;
    ph_rb_tilescan(L, G);
    if (!grid_sync(L, NoTail{})) return false;
    ph_rb_take<STRONG>(L, G, arena);
    if constexpr (STRONG) {
        if (!grid_sync(L, [&] { ph_rb_tiletaken_scan(L); })) return false;
        ph_rb_cookie(L, G, arena);
    }
    return grid_sync(L, NoTail{});
}

// The whole loop of Alg. 3 on one level in one cooperative launch: the same
// phases as the per-phase kernels, in the same order, separated by grid
// barriers instead of kernel boundaries; the last block to reach a barrier
// runs the serial tails (rebalancing plan, Jetrs eviction scan, controller).
// Tiles of the rebalancing passes are one block of kRbTile threads, as in
// the per-phase kernels.
template <bool EW>
__global__ void __launch_bounds__(kTB, JET_ROW_MINB) k_refine_grid(Level L) {
    const Grid G = launch_grid();
    char *arena = JET_ARENA;
    const LpExport none{nullptr, nullptr, nullptr};
    for (;;) {
        const int32_t mode = ld_gpu(&L.ctl->mode);
        if (mode == MODE_DONE) break;
        ph_copy_best(L, G);   // P_best <- P_iter asked for by the previous controller
        if (mode == MODE_LP) {
            ph_lp_scan(L, G, arena);
            if (!grid_sync(L, NoTail{})) return;
            ph_lp_select<EW>(L, none, G, arena);
            if (!grid_sync(L, NoTail{})) return;
            ph_afterburn<EW>(L, none, G, arena);
            if (!grid_sync(L, NoTail{})) return;
        } else if (mode == MODE_RW) {
            if (!grid_rebalance<EW, false>(L, G, arena)) return;
        } else {
            if (!grid_rebalance<EW, true>(L, G, arena)) return;
        }
        ph_apply<EW>(L, G, arena);
        if (!grid_sync(L, [&] { ph_controller(L); })) return;
    }
    ph_copy_best(L, G);
}

// ---------------------------------------------------------------------------
// batched form: the small levels of many graphs in one persistent launch
// ---------------------------------------------------------------------------
// A job is one graph's chain of small levels, coarsest first (the levels of
// at most cluster_max_n vertices form the coarse end of its hierarchy).  The
// clusters of one launch take jobs from a counter; a cluster runs the whole
// chain of its job: per level the projection of the coarser level's
// partition, the level's start state (the work of setup_level and
// enqueue_init, as cluster phases), the whole Alg. 3 loop, and the P_best
// copy; then it takes the next job.  Every decision is the one the
// per-level launches take, so results are bit-identical.
struct BatchLevel {
    DGraph g;
    const int32_t *cmap;     // this level -> the next coarser one (unused on the job's coarsest level)
    uint64_t seed;           // Jetrw seed of the level
    int32_t cq16;            // first-filter ratio c of the level (c_fine on level 0)
    int32_t pad;
};
struct BatchStat {           // the control block's outcome of one level
    int64_t best_cut, best_maxw;
    int64_t kbytes[JET_K_COUNT];
    int32_t it, best_bal, hit_cap, pad;
    int32_t kcount[4];
};
struct BatchJob {
    Level L;                 // buffers sized for the chain's largest level; the level fields are set per level
    const BatchLevel *lv;    // [nlv], coarsest first
    BatchStat *stat;         // [nlv]
    const int32_t *init;     // start partition of the coarsest level
    int32_t *part[2];        // level partitions, alternating (level i in part[i & 1])
    int32_t *out;            // receives the finest level's partition (may be null)
    int64_t *cut2;           // scratch: twice the start cut of a level
    int64_t Llim, opt, sigma;
    int32_t nlv, pad;
};

// Start of one level inside a job (all blocks of the cluster): projection,
// per-vertex start values, cut / part weights / ext / weighted degree, the
// long-row count, then the control block (block 0) and P_best = P_0.
__device__ inline void batch_level_start(const BatchJob &job, const Level &L, int32_t i, Grid G, char *arena,
                                         cg::cluster_group &cl) {
    const int64_t n = L.g.n;
    const int64_t t0 = (int64_t)G.bid * blockDim.x + threadIdx.x, stride = (int64_t)G.nb * blockDim.x;
    int32_t *cur = L.part;
    if (i == 0) {
        for (int64_t v = t0; v < n; v += stride) cur[v] = job.init[v];
    } else {
        const int32_t *prev = job.part[(i - 1) & 1];
        const int32_t *cmap = job.lv[i].cmap;
        for (int64_t v = t0; v < n; v += stride) cur[v] = prev[cmap[v]];
    }
    for (int64_t v = t0; v < n; v += stride) {
        L.lstamp[v] = -2;
        L.mstamp[v] = -2;
        L.prio[v] = kNoneGain;
    }
    if (G.bid == 0) {
        int64_t *w = reinterpret_cast<int64_t *>(L.ctl);
        for (int q = threadIdx.x; q < (int)(sizeof(Ctl) / 8); q += blockDim.x) w[q] = 0;
        for (int p = threadIdx.x; p < L.k; p += blockDim.x) L.pw[p] = 0;
        if (threadIdx.x == 0) job.cut2[0] = 0;
    }
    cl.sync();
    for (int64_t v0 = (int64_t)G.bid * blockDim.x; v0 < n; v0 += stride) {
        const int64_t v = v0 + threadIdx.x;
        const bool big = v < n && ld_xadj(L.g.xadj, v + 1) - ld_xadj(L.g.xadj, v) > kSmallDeg;
        const unsigned m = __ballot_sync(0xffffffffu, big);
        if (lane_id() == 0 && m) atomicAdd(&L.ctl->nbig, __popc(m));
    }
    if (L.g.ew) ph_cut_pw<true>(L.g, L.k, cur, L.pw, job.cut2, L.ext, L.wdeg, G, arena);
    else ph_cut_pw<false>(L.g, L.k, cur, L.pw, job.cut2, L.ext, L.wdeg, G, arena);
    cl.sync();
    if (G.bid == 0) {
        if (threadIdx.x == 0) {
            L.ctl->L = job.Llim;
            L.ctl->opt = job.opt;
            L.ctl->sigma = job.sigma;
        }
        __syncthreads();
        ph_ctl_init(L, job.cut2);
    }
    for (int64_t v = t0; v < n; v += stride) L.best[v] = cur[v];
    cl.sync();
}

__global__ void __launch_bounds__(kClusterThreads, 1) k_refine_batch(const BatchJob *jobs, int32_t njobs,
                                                                     int32_t *queue) {
    cg::cluster_group cl = cg::this_cluster();
    const Grid G{(int)cl.block_rank(), (int)cl.num_blocks()};
    char *arena = JET_ARENA;
    __shared__ int s_job;
    __shared__ Level L;   // the level's parameters, in shared memory rather than on each thread's stack
    for (;;) {
        if (G.bid == 0 && threadIdx.x == 0) s_job = atomicAdd(queue, 1);
        cl.sync();
        const int j = *cl.map_shared_rank(&s_job, 0);
        cl.sync();   // every block has read the job before block 0 takes the next
        if (j >= njobs) break;
        const BatchJob &job = jobs[j];
        for (int32_t i = 0; i < job.nlv; ++i) {
            if (threadIdx.x == 0) {
                const BatchLevel &bl = job.lv[i];
                L = job.L;
                L.g = bl.g;
                L.seed = bl.seed;
                L.cq16 = bl.cq16;
                L.ntiles = (int32_t)(((int64_t)bl.g.n + kClusterThreads - 1) / kClusterThreads);
                if (L.ntiles < 1) L.ntiles = 1;
                L.part = job.part[i & 1];
            }
            __syncthreads();
            batch_level_start(job, L, i, G, arena, cl);
            if (L.g.ew) cluster_level_loop<true>(L, G, arena, cl);
            else cluster_level_loop<false>(L, G, arena, cl);
            cl.sync();
            // P_best is the level's result
            const int64_t n = L.g.n, t0 = (int64_t)G.bid * blockDim.x + threadIdx.x, stride = (int64_t)G.nb * blockDim.x;
            int32_t *dst = (i + 1 == job.nlv && job.out) ? job.out : L.part;
            for (int64_t v = t0; v < n; v += stride) dst[v] = L.best[v];
            if (G.bid == 0 && threadIdx.x == 0) {
                const Ctl *c = L.ctl;
                BatchStat &st = job.stat[i];
                st.best_cut = c->best_cut;
                st.best_maxw = c->best_maxw;
                for (int q = 0; q < JET_K_COUNT; ++q) st.kbytes[q] = c->kbytes[q];
                st.it = c->it;
                st.best_bal = c->best_bal;
                st.hit_cap = c->hit_cap;
                for (int q = 0; q < 4; ++q) st.kcount[q] = c->kcount[q];
            }
            cl.sync();
        }
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
// Vertices with rows longer than kSmallDeg (only whether there are any
// matters), counted into the level's control block.
__global__ void k_count_big(DGraph g, int32_t *count) {
    int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    bool big = v < g.n && ld_xadj(g.xadj, (int64_t)v + 1) - ld_xadj(g.xadj, v) > kSmallDeg;
    unsigned m = __ballot_sync(0xffffffffu, big);
    if (lane_id() == 0 && m) atomicAdd(count, __popc(m));
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
    int64_t *cut2 = nullptr;
};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Carves all per-level buffers out of two allocations.
int allow_large_arenas(int device);

// Per-level buffers: 11 int32 arrays per vertex (best, nxt, prio, mstamp,
// lstamp, key, listX, listM, ext, wdeg, listW), then the control block,
// per-part state, rebalancing tiles, the trace (optional) and the cut
// accumulator, in two allocations.
void level_bytes(int64_t nmax, int32_t k, bool with_trace, size_t *vbytes, size_t *mbytes) {
    const size_t nn = (size_t)std::max<int64_t>(nmax, 1), kk = (size_t)k;
    const size_t ntiles = (size_t)std::max<int64_t>((nmax + kRbTile - 1) / kRbTile, 1);
    *vbytes = 11 * align256(nn * 4) + align256(nn * 8) /* etaken */;
    *mbytes = align256(sizeof(Ctl)) + align256(kk * 8) /*pw*/ + align256(kk * 4) /*aidx*/ + align256(kk * 4) /*Bs*/ +
              align256(kk) /*inB*/ + align256((kk + 1) * 8) /*capC*/ + align256(kk * 8) /*excess*/ +
              align256(kk * kSlots * 8) /*bucketw*/ + align256(kk * 4) /*sstar*/ + align256(kk * 8) /*need*/ +
              align256(ntiles * kk * 4) /*tilehist*/ + align256(ntiles * 8) /*tiletaken*/ +
              (with_trace ? align256(sizeof(TraceRec) * kTrace) : 0) + align256(16) /*cut2*/;
}

void carve_level(Level &L, char *vert, char *misc, int64_t nmax, int32_t k, bool with_trace, int64_t **cut2) {
    const size_t nn = (size_t)std::max<int64_t>(nmax, 1), kk = (size_t)k;
    const int32_t ntiles = (int32_t)std::max<int64_t>((nmax + kRbTile - 1) / kRbTile, 1);
    char *p = vert;
    auto take32 = [&](void) { int32_t *r = reinterpret_cast<int32_t *>(p); p += align256(nn * 4); return r; };
    L.best = take32(); L.nxt = take32(); L.prio = take32(); L.mstamp = take32(); L.lstamp = take32();
    L.key = take32(); L.listX = take32(); L.listM = take32();
    L.ext = take32();
    L.wdeg = take32();
    L.listW = take32();
    L.rbloss = nullptr;
    L.etaken = reinterpret_cast<int64_t *>(p);
    char *q = misc;
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
    L.trace = with_trace ? reinterpret_cast<TraceRec *>(take(sizeof(TraceRec) * kTrace)) : nullptr;
    *cut2 = reinterpret_cast<int64_t *>(take(16));
    L.ntiles = ntiles;
    L.k = k;
}

// Buffers and start state of one level, enqueued on the context's stream (no
// host wait): the control block gets the level's long-row count.
int setup_level(Ctx &c, const DGraph &g, int32_t k, LevelBufs &B) {
    JET_TRY(allow_large_arenas(c.device));
    cudaStream_t s = c.stream;
    int64_t n = g.n;
    size_t vbytes = 0, mbytes = 0;
    level_bytes(n, k, true, &vbytes, &mbytes);
    JET_TRY(dev_alloc(B.vert, vbytes, s));
    JET_TRY(dev_alloc(B.misc, mbytes, s));
    Level &L = B.L;
    carve_level(L, B.vert.as<char>(), B.misc.as<char>(), n, k, true, &B.cut2);
    L.g = g;
    JET_CUDA_TRY(cudaMemsetAsync(L.ctl, 0, sizeof(Ctl), s));
    JET_CUDA_TRY(cudaMemsetAsync(L.pw, 0, (size_t)k * 8, s));
    JET_CUDA_TRY(cudaMemsetAsync(B.cut2, 0, 16, s));
    if (n > 0) {
        k_count_big<<<grid_for(n, kTB), kTB, 0, s>>>(g, &L.ctl->nbig);
        k_fill_i32<<<grid_for(n, kTB, 4096), kTB, 0, s>>>(L.lstamp, n, -2);
        k_fill_i32<<<grid_for(n, kTB, 4096), kTB, 0, s>>>(L.mstamp, n, -2);
        k_fill_i32<<<grid_for(n, kTB, 4096), kTB, 0, s>>>(L.prio, n, kNoneGain);
    }
    JET_CUDA_TRY(cudaGetLastError());
    return JET_OK;
}

int list_grid() { return num_sms() * 4; }

// Launch shapes of the refinement kernels (execution choices: results do not
// depend on them), from the context's options:
//   scan kernels   grid-stride over vertices in groups of four, at most
//                  scan_cap blocks (scan_blocks_per_sm per SM, default 8);
//   list kernels   one block per items_per_block list entries (default 64),
//                  at most list_cap blocks (list_blocks_per_sm, default 4);
//   apply          the same, at most apply_cap blocks (apply_blocks_per_sm,
//                  default: the list kernels' value).
int scan_grid(const Level &L, int64_t n) { return std::min(L.scan_cap, grid_for((n + 3) / 4, kTB)); }
int list_blocks(const Level &L, int64_t items) { return std::min(L.list_cap, grid_for(items, L.items_per_block)); }
int apply_blocks(const Level &L, int64_t items) { return std::min(L.apply_cap, grid_for(items, L.items_per_block)); }

// Launch of a kernel that follows another one of the same pass: with
// L.pdl it may be scheduled early and waits on the device (pdl_enter).
template <class... Args>
cudaError_t launch_dep(const Level &L, void (*kern)(Args...), int grid, int block, size_t smem, cudaStream_t s,
                       Args... args) {
    return launch_pdl(kern, grid, block, smem, s, L.pdl != 0, args...);
}

// Per-kernel timing of the host-driven loop (JET_FLAG_PROFILE): a CUDA event
// on the level's stream before every refinement kernel and one after the
// iteration's last kernel; after the host's per-iteration synchronisation the
// intervals are added to the kernels that ran in them.
struct KernProf {
    static constexpr int kMax = 16;
    cudaEvent_t ev[kMax + 1] = {};
    int kid[kMax] = {};
    int cnt = 0;
    float ms[JET_KERNELS] = {};
    ~KernProf() {
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
    }
    int init() {
        for (cudaEvent_t &e : ev) JET_CUDA_TRY(cudaEventCreate(&e));
        return JET_OK;
    }
    int mark(cudaStream_t s, int k) {
        if (cnt >= kMax) return JET_EINVAL;
        kid[cnt] = k;
        JET_CUDA_TRY(cudaEventRecord(ev[cnt++], s));
        return JET_OK;
    }
    int end(cudaStream_t s) {
        JET_CUDA_TRY(cudaEventRecord(ev[cnt], s));
        return JET_OK;
    }
    // after the stream has been synchronised
    int collect() {
        for (int i = 0; i < cnt; ++i) {
            float t = 0.f;
            JET_CUDA_TRY(cudaEventElapsedTime(&t, ev[i], ev[i + 1]));
            ms[kid[i]] += t;
        }
        cnt = 0;
        return JET_OK;
    }
};

static inline int prof_mark(KernProf *pr, cudaStream_t s, int k) { return pr ? pr->mark(s, k) : JET_OK; }

// Kernel sequences of one iteration, by kind.  Each returns, through *nk,
// the number of kernels it enqueued; pr (host loop only) times each launch.
int enqueue_lp_select(const Level &L, cudaStream_t s, LpExport ex, int *nk, KernProf *pr = nullptr) {
    int n = L.g.n;
    bool ew = L.g.ew != nullptr;
    JET_TRY(prof_mark(pr, s, JET_K_LP_SCAN));
    k_lp_scan<<<scan_grid(L, n), kTB, sm_lp_scan(), s>>>(L);
    const size_t sm = sm_lp_select(L.k, kTB, true);
    JET_TRY(prof_mark(pr, s, JET_K_LP_SELECT));
    JET_CUDA_TRY(launch_dep(L, ew ? k_lp_select<true> : k_lp_select<false>, list_blocks(L, n), kTB, sm, s, L, ex));
    *nk = 2;
    JET_CUDA_TRY(cudaGetLastError());
    return JET_OK;
}

int enqueue_lp_after(const Level &L, cudaStream_t s, LpExport ex, int *nk, KernProf *pr = nullptr) {
    int n = L.g.n;
    JET_TRY(prof_mark(pr, s, JET_K_AFTERBURN));
    JET_CUDA_TRY(launch_dep(L, L.g.ew ? k_afterburn<true> : k_afterburn<false>, list_blocks(L, n), kTB, sm_afterburn(), s,
                            L, ex));
    *nk = 1;
    JET_CUDA_TRY(cudaGetLastError());
    return JET_OK;
}

int enqueue_lp(const Level &L, cudaStream_t s, int *nk, LpExport ex = {nullptr, nullptr, nullptr},
               KernProf *pr = nullptr) {
    int a = 0, b = 0;
    JET_TRY(enqueue_lp_select(L, s, ex, &a, pr));
    JET_TRY(enqueue_lp_after(L, s, ex, &b, pr));
    *nk = a + b;
    return JET_OK;
}

template <bool STRONG>
int enqueue_rb_t(const Level &L, cudaStream_t s, int *nk, KernProf *pr) {
    int n = L.g.n;
    bool ew = L.g.ew != nullptr;
    JET_TRY(prof_mark(pr, s, JET_K_RB_SCAN));
    k_rb_scan<STRONG><<<std::min(L.rb_scan_cap, scan_grid(L, n)), kTB, sm_rb_scan(), s>>>(L);
    const size_t sm = sm_rb_cand(L.k, kTB, true);
    JET_TRY(prof_mark(pr, s, JET_K_RB_CAND));
    JET_CUDA_TRY(launch_dep(L, ew ? k_rb_cand<true, STRONG> : k_rb_cand<false, STRONG>, list_blocks(L, n), kTB, sm, s, L));
    JET_TRY(prof_mark(pr, s, JET_K_RB_TILEHIST));
    JET_CUDA_TRY(launch_dep(L, k_rb_tilehist, L.ntiles, kRbTile, sm_rb_tilehist(L.k), s, L));
    JET_TRY(prof_mark(pr, s, JET_K_RB_TILESCAN));
    JET_CUDA_TRY(launch_dep(L, k_rb_tilescan, L.k, 1024, 0, s, L));
    JET_TRY(prof_mark(pr, s, JET_K_RB_TAKE));
    JET_CUDA_TRY(launch_dep(L, k_rb_take<STRONG>, L.ntiles, kRbTile, sm_rb_take(L.k, kRbTile), s, L));
    *nk = 5;
    if (STRONG) {
        JET_TRY(prof_mark(pr, s, JET_K_RB_COOKIE));
        JET_CUDA_TRY(launch_dep(L, k_rb_cookie, L.ntiles, kRbTile, sm_rb_cookie(kRbTile), s, L));
        *nk += 1;
    }
    JET_CUDA_TRY(cudaGetLastError());
    return JET_OK;
}

int enqueue_rb(const Level &L, cudaStream_t s, bool strong, int *nk, KernProf *pr = nullptr) {
    return strong ? enqueue_rb_t<true>(L, s, nk, pr) : enqueue_rb_t<false>(L, s, nk, pr);
}

// apply + commit + controller
int enqueue_tail(const Level &L, cudaStream_t s, int *nk, KernProf *pr = nullptr) {
    int ga = apply_blocks(L, L.g.n);
    JET_TRY(prof_mark(pr, s, JET_K_APPLY));
    JET_CUDA_TRY(launch_dep(L, L.g.ew ? k_apply<true> : k_apply<false>, ga, kTB, sm_apply(L.k), s, L));
    *nk = 1;
    JET_CUDA_TRY(cudaGetLastError());
    return JET_OK;
}

// P_best <- P_iter after the level's last iteration
int enqueue_final_copy(const Level &L, cudaStream_t s) {
    k_copy_best<<<std::min(list_grid(), grid_for(L.g.n / 4 + 1, kTB)), kTB, 0, s>>>(L);
    JET_CUDA_TRY(cudaGetLastError());
    return JET_OK;
}

// Level start: part weights, cut, control block, P_best = P_0 (no host wait).
int enqueue_init(Ctx &c, LevelBufs &B, int64_t L_lim, int64_t opt, int64_t sigma) {
    cudaStream_t s = c.stream;
    Level &L = B.L;
    int64_t n = L.g.n;
    if (n > 0) {
        int gcut = std::min(list_grid(), grid_for(n, kTB));
        if (L.g.ew) k_cut_pw<true><<<gcut, kTB, sm_cut_pw(L.k), s>>>(L.g, L.k, L.part, L.pw, B.cut2, L.ext, L.wdeg);
        else k_cut_pw<false><<<gcut, kTB, sm_cut_pw(L.k), s>>>(L.g, L.k, L.part, L.pw, B.cut2, L.ext, L.wdeg);
        c.launches += 1;
    }
    k_ctl_init<<<1, 1024, 0, s>>>(L, B.cut2, L_lim, opt, sigma);
    c.launches += 1;
    if (n > 0) JET_CUDA_TRY(cudaMemcpyAsync(L.best, L.part, (size_t)n * 4, cudaMemcpyDeviceToDevice, s));
    JET_CUDA_TRY(cudaGetLastError());
    return JET_OK;
}

int read_ctl(Ctx &c, const Level &L, Ctl &h) {
    JET_CUDA_TRY(cudaMemcpyAsync(&h, L.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, c.stream));
    JET_CUDA_TRY(cudaStreamSynchronize(c.stream));
    return JET_OK;
}

// Host-driven loop (JET_FLAG_HOSTLOOP / JET_FLAG_PROFILE): the mode is read
// back after every iteration, as in the paper's implementation.  With
// profiling, CUDA events on the level's stream time every kernel launch;
// kern_ms receives the sums per kernel.
int run_hostloop(Ctx &c, const Level &L, bool profile, float *kern_ms) {
    KernProf prof;
    KernProf *pr = nullptr;
    if (profile) {
        JET_TRY(prof.init());
        pr = &prof;
    }
    for (;;) {
        int32_t mode = 0;
        JET_CUDA_TRY(cudaMemcpyAsync(c.pinned, &L.ctl->mode, 4, cudaMemcpyDeviceToHost, c.stream));
        JET_CUDA_TRY(cudaStreamSynchronize(c.stream));
        if (pr) JET_TRY(pr->collect());
        memcpy(&mode, c.pinned, 4);
        if (mode == MODE_DONE) break;
        int nk = 0;
        if (mode == MODE_LP) {
            LpExport none{nullptr, nullptr, nullptr};
            JET_TRY(enqueue_lp(L, c.stream, &nk, none, pr));
        } else {
            JET_TRY(enqueue_rb(L, c.stream, mode == MODE_RS, &nk, pr));
        }
        c.launches += nk;
        JET_TRY(enqueue_tail(L, c.stream, &nk, pr));
        c.launches += nk;
        if (pr) JET_TRY(pr->end(c.stream));
    }
    JET_TRY(enqueue_final_copy(L, c.stream));
    c.launches += 1;
    if (kern_ms)
        for (int i = 0; i < JET_KERNELS; ++i) kern_ms[i] = prof.ms[i];
    return JET_OK;
}

// Device-resident loop: graph = start kernel -> WHILE(h_loop) { SWITCH(hA)
// {...} -> SWITCH(hB) {...} } -> final best copy, each SWITCH holding one
// iteration {Jetlp | Jetrw | Jetrs, each followed by apply + commit +
// controller}.  Two iterations per loop body: the step from one SWITCH to
// the next costs less than a restart of the loop body.  The controller of
// an iteration sets the other SWITCH's value (DONE: no branch runs) and the
// loop flag.  The apply kernel sits inside every branch so that it follows
// the branch's last kernel by programmatic dependent launch instead of
// waiting for the conditional node to complete.
// nk_branch[3] / *nk_tail receive the kernel counts of the captured pieces.
// The graph is launched on the context's stream and not waited for; *exec_out
// receives the executable graph, which the caller destroys once the stream
// has passed it.
int run_graph(Ctx &c, Level L, int *nk_branch, int *nk_tail, cudaGraphExec_t *exec_out) {
    cudaStream_t s = c.stream;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    *exec_out = nullptr;
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
        cudaGraphConditionalHandle h_loop, h_a, h_b;
        if ((e = cudaGraphConditionalHandleCreate(&h_loop, g, 1, cudaGraphCondAssignDefault)) != cudaSuccess) { fail(e, "handle loop"); break; }
        if ((e = cudaGraphConditionalHandleCreate(&h_a, g, 0, cudaGraphCondAssignDefault)) != cudaSuccess) { fail(e, "handle mode"); break; }
        if ((e = cudaGraphConditionalHandleCreate(&h_b, g, 0, cudaGraphCondAssignDefault)) != cudaSuccess) { fail(e, "handle mode"); break; }
        L.h_loop = h_loop; L.h_mode = h_a; L.h_next = h_b; L.use_graph = 1;
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
        {
            cudaKernelNodeParams kp{};
            void *args[] = {&L};
            kp.func = (void *)k_copy_best;
            kp.gridDim = dim3(std::min(list_grid(), grid_for(L.g.n / 4 + 1, kTB)));
            kp.blockDim = dim3(kTB);
            kp.kernelParams = args;
            cudaGraphNode_t fin;
            if ((e = cudaGraphAddKernelNode(&fin, g, &wnode, 1, &kp)) != cudaSuccess) { fail(e, "final copy node"); break; }
        }
        cudaGraph_t body = wp.conditional.phGraph_out[0];
        bool ok = true;
        cudaGraphNode_t prev{};
        for (int u = 0; u < 2 && ok; ++u) {
            // iteration u of the body: its switch reads hA (u = 0) or hB, its
            // controller sets the other one
            Level Lu = L;
            Lu.h_mode = u == 0 ? h_a : h_b;
            Lu.h_next = u == 0 ? h_b : h_a;
            cudaGraphNodeParams sp{};
            sp.type = cudaGraphNodeTypeConditional;
            sp.conditional.handle = u == 0 ? h_a : h_b;
            sp.conditional.type = cudaGraphCondTypeSwitch;
            sp.conditional.size = 3;
            cudaGraphNode_t snode;
            if ((e = cudaGraphAddNode(&snode, body, u ? &prev : nullptr, nullptr, u ? 1 : 0, &sp)) != cudaSuccess) { fail(e, "switch node"); ok = false; break; }
            prev = snode;
            for (int b = 0; b < 3 && ok; ++b) {
                cudaGraph_t bg = sp.conditional.phGraph_out[b];
                if ((e = cudaStreamBeginCaptureToGraph(cap, bg, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed)) != cudaSuccess) { fail(e, "capture branch"); ok = false; break; }
                int r = b == 0 ? enqueue_lp(Lu, cap, &nk_branch[0]) : enqueue_rb(Lu, cap, b == 2, &nk_branch[b]);
                if (r == JET_OK) r = enqueue_tail(Lu, cap, nk_tail);
                cudaGraph_t outg = nullptr;
                e = cudaStreamEndCapture(cap, &outg);
                if (r != JET_OK) { rc = r; ok = false; break; }
                if (e != cudaSuccess) { fail(e, "end capture branch"); ok = false; break; }
            }
        }
        if (!ok) break;
        if ((e = cudaGraphInstantiate(&ge, g, 0)) != cudaSuccess) { fail(e, "cudaGraphInstantiate"); break; }
        if ((e = cudaGraphLaunch(ge, s)) != cudaSuccess) { fail(e, "cudaGraphLaunch"); break; }
    } while (0);
    if (rc == JET_OK) {
        *exec_out = ge;
    } else if (ge) {
        cudaStreamSynchronize(s);
        cudaGraphExecDestroy(ge);
    }
    if (g) cudaGraphDestroy(g);
    if (cap) cudaStreamDestroy(cap);
    return rc;
}

// The row kernels whose arena can pass 48 KB (per-warp tables for k up to
// JET_MAX_K) are allowed the larger dynamic shared memory once per device.
int allow_large_arenas(int device) {
    static std::mutex mu;
    static bool done[256];
    if (device < 0 || device >= 256) return JET_EINVAL;
    std::lock_guard<std::mutex> lock(mu);
    if (done[device]) return JET_OK;
    const int sel = (int)sm_lp_select(JET_MAX_K, kTB, true), cand = (int)sm_rb_cand(JET_MAX_K, kTB, true);
    JET_CUDA_TRY(cudaFuncSetAttribute(k_lp_select<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sel));
    JET_CUDA_TRY(cudaFuncSetAttribute(k_lp_select<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sel));
    JET_CUDA_TRY(cudaFuncSetAttribute(k_rb_cand<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, cand));
    JET_CUDA_TRY(cudaFuncSetAttribute(k_rb_cand<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, cand));
    JET_CUDA_TRY(cudaFuncSetAttribute(k_rb_cand<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, cand));
    JET_CUDA_TRY(cudaFuncSetAttribute(k_rb_cand<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, cand));
    done[device] = true;
    return JET_OK;
}

// Cluster loop: the largest cluster (at most kMaxCluster blocks of
// kClusterThreads) that the device can co-schedule, cached per device.
constexpr int kMaxCluster = 16;

template <bool EW>
int cluster_size(int device, size_t smem, int *out) {
    static std::mutex mu;
    static int cache[2][256];
    static size_t cache_smem[2][256];
    const int e_idx = EW ? 1 : 0;
    if (device < 0 || device >= 256) { *out = 0; return JET_OK; }
    std::lock_guard<std::mutex> lock(mu);
    if (cache[e_idx][device] != 0 && cache_smem[e_idx][device] >= smem) {
        *out = std::max(cache[e_idx][device], 0);
        return JET_OK;
    }
    JET_CUDA_TRY(cudaFuncSetAttribute(k_refine_cluster<EW>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    JET_CUDA_TRY(cudaFuncSetAttribute(k_refine_cluster<EW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int best = -1;
    for (int cs = kMaxCluster; cs >= 2; cs /= 2) {
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3(cs);
        cfg.blockDim = dim3(kClusterThreads);
        cfg.dynamicSmemBytes = smem;
        cudaLaunchAttribute at{};
        at.id = cudaLaunchAttributeClusterDimension;
        at.val.clusterDim.x = cs;
        at.val.clusterDim.y = 1;
        at.val.clusterDim.z = 1;
        cfg.attrs = &at;
        cfg.numAttrs = 1;
        int nclusters = 0;
        cudaError_t e = cudaOccupancyMaxActiveClusters(&nclusters, k_refine_cluster<EW>, &cfg);
        if (e != cudaSuccess) { cudaGetLastError(); continue; }
        if (nclusters >= 1) { best = cs; break; }
    }
    cache[e_idx][device] = best;
    cache_smem[e_idx][device] = smem;
    *out = best > 0 ? best : 0;
    return JET_OK;
}

// Whole level loop in one cluster launch (tiles of the rebalancing passes are
// one block, kClusterThreads vertices).
template <bool EW>
int run_cluster_t(Ctx &c, Level L, int cs, size_t smem) {
    L.use_graph = 0;
    L.ntiles = (int32_t)std::max<int64_t>(((int64_t)L.g.n + kClusterThreads - 1) / kClusterThreads, 1);
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(cs);
    cfg.blockDim = dim3(kClusterThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = c.stream;
    cudaLaunchAttribute at{};
    at.id = cudaLaunchAttributeClusterDimension;
    at.val.clusterDim.x = cs;
    at.val.clusterDim.y = 1;
    at.val.clusterDim.z = 1;
    cfg.attrs = &at;
    cfg.numAttrs = 1;
    JET_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_refine_cluster<EW>, L));
    return JET_OK;
}

// Persistent loop: blocks of the cooperative launch (at most JET_ROW_MINB per
// SM, as many as the device keeps resident with this arena, and no more than
// the level's list kernels would use), cached per device and edge-weight
// variant; 0 when the device cannot run it.
template <bool EW>
int grid_loop_blocks(int device, size_t smem, int64_t n, int *out) {
    static std::mutex mu;
    static int cache[2][256];
    static size_t cache_smem[2][256];
    const int e_idx = EW ? 1 : 0;
    *out = 0;
    if (device < 0 || device >= 256) return JET_OK;
    int per_sm = 0;
    {
        std::lock_guard<std::mutex> lock(mu);
        if (cache_smem[e_idx][device] < smem || cache[e_idx][device] == 0) {
            JET_CUDA_TRY(cudaFuncSetAttribute(k_refine_grid<EW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            int nb = 0;
            JET_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_refine_grid<EW>, kTB, smem));
            cache[e_idx][device] = nb > 0 ? nb : -1;
            cache_smem[e_idx][device] = smem;
        }
        per_sm = cache[e_idx][device];
    }
    if (per_sm <= 0) return JET_OK;
    int cap = num_sms() * std::min(per_sm, JET_ROW_MINB);
    *out = std::min(cap, grid_for(n, 64));
    return JET_OK;
}

size_t grid_loop_smem(int32_t k) { return (arena_bytes(k, kTB) + 255) & ~size_t(255); }

// Whole level loop in one cooperative launch; *ran = 0 when the device
// cannot run it (the caller takes the CUDA-graph loop instead).
template <bool EW>
int run_grid_t(Ctx &c, Level L, int *ran) {
    *ran = 0;
    if (kRbTile != kTB) return JET_OK;        // tiles must be one block
    const size_t smem = grid_loop_smem(L.k);
    int nb = 0;
    JET_TRY(grid_loop_blocks<EW>(c.device, smem, L.g.n, &nb));
    if (nb <= 0) return JET_OK;
    L.use_graph = 0;
    void *args[] = {&L};
    JET_CUDA_TRY(cudaLaunchCooperativeKernel((void *)k_refine_grid<EW>, dim3(nb), dim3(kTB), args, smem, c.stream));
    *ran = 1;
    return JET_OK;
}

int run_grid(Ctx &c, const Level &L, int *ran) {
    if (L.g.ew) return run_grid_t<true>(c, L, ran);
    return run_grid_t<false>(c, L, ran);
}

size_t cluster_smem(int32_t k) { return (arena_bytes(k, kClusterThreads) + 255) & ~size_t(255); }

// Cluster size usable for this level (0: use the graph loop).
int pick_cluster(Ctx &c, const Level &L, int *cs) {
    *cs = 0;
    if (L.g.n <= 0 || L.g.n > c.opt.cluster_max_n) return JET_OK;
    if (L.g.ew) JET_TRY(cluster_size<true>(c.device, cluster_smem(L.k), cs));
    else JET_TRY(cluster_size<false>(c.device, cluster_smem(L.k), cs));
    if (c.opt.cluster_blocks > 0 && *cs > c.opt.cluster_blocks) *cs = c.opt.cluster_blocks;
    return JET_OK;
}

int run_cluster(Ctx &c, const Level &L, int cs) {
    if (L.g.ew) return run_cluster_t<true>(c, L, cs, cluster_smem(L.k));
    return run_cluster_t<false>(c, L, cs, cluster_smem(L.k));
}

}  // namespace

// Weight of the whole graph (needed for the balance limit).
int total_vweight(Ctx &c, const DGraph &g, int64_t &W) {
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

// Blocks of the rebalancing scan resident on one SM (per device, once).
static int rb_scan_resident() {
    static std::mutex mu;
    static int cached[256];
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 256) return 1;
    std::lock_guard<std::mutex> lock(mu);
    if (cached[dev] == 0) {
        int a = 0, b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_rb_scan<false>, kTB, sm_rb_scan()) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_rb_scan<true>, kTB, sm_rb_scan()) != cudaSuccess) {
            cudaGetLastError();
            return 4;
        }
        cached[dev] = std::max(1, std::min(a, b));
    }
    return cached[dev];
}

static void fill_level_params(Ctx &c, Level &L, int32_t is_finest, uint64_t seed) {
    const jet_options &o = c.opt;
    L.cq16 = (int32_t)llround((is_finest ? o.c_fine : o.c_coarse) * 65536.0);
    L.phi_ppm = llround(o.phi * 1e6);
    L.max_no_improve = o.max_no_improve;
    L.weak_limit = o.weak_limit;
    L.max_iters = o.max_iters_per_level;
    L.abl = o.flags & ABL_ALL;
    L.seed = seed;
    L.use_graph = 0;
    L.h_loop = L.h_mode = L.h_next = 0;
    L.pdl = (o.flags & JET_FLAG_NO_PDL) ? 0 : 1;
    const int sms = num_sms();
    L.hub_deg = o.hub_degree > 0 ? o.hub_degree : kHugeDeg;
    L.list_cap = sms * (o.list_blocks_per_sm > 0 ? o.list_blocks_per_sm : 4);
    L.apply_cap = o.apply_blocks_per_sm > 0 ? sms * o.apply_blocks_per_sm : L.list_cap;
    L.scan_cap = sms * (o.scan_blocks_per_sm > 0 ? o.scan_blocks_per_sm : 8);
    // the rebalancing scan holds more registers than the other scans: a
    // second wave of its blocks would start only as the first one leaves
    L.rb_scan_cap = std::min(L.scan_cap, sms * rb_scan_resident());
    L.items_per_block = o.list_items_per_block > 0 ? o.list_items_per_block : 64;
    L.poll_limit = o.barrier_polls > 0 ? o.barrier_polls : kBarPollLimit;
}

int refine_level_enqueue(Ctx &c, const DGraph &g, int32_t k, double eps, int32_t is_finest, uint64_t seed,
                         int32_t *part_inout, int64_t W, LevelRun &run) {
    run.g = g;
    run.k = k;
    if (run.slot < 0 || run.slot >= JET_MAX_LEVELS) return JET_EINVAL;
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
    run.hostloop = (c.opt.flags & (JET_FLAG_HOSTLOOP | JET_FLAG_PROFILE)) != 0;
    if (!run.hostloop) JET_TRY(pick_cluster(c, L, &run.cluster));
    if (g.n > 0) {
        if (run.hostloop) {
            JET_TRY(run_hostloop(c, L, (c.opt.flags & JET_FLAG_PROFILE) != 0, run.rep.kern_ms));
            run.rep.sel_ms = run.rep.kern_ms[JET_K_LP_SCAN] + run.rep.kern_ms[JET_K_LP_SELECT];
        } else if (run.cluster > 0) {
            JET_TRY(run_cluster(c, L, run.cluster));
        } else {
            if (c.opt.flags & JET_FLAG_GRID_LOOP) JET_TRY(run_grid(c, L, &run.grid));
            if (!run.grid) JET_TRY(run_graph(c, L, run.nk_branch, &run.nk_tail, &run.exec));
        }
        JET_CUDA_TRY(cudaMemcpyAsync(part_inout, L.best, (size_t)g.n * 4, cudaMemcpyDeviceToDevice, c.stream));
    }
    // the control block (and the trace) come back when the stream gets here;
    // the level's buffers are released in stream order after these copies
    char *pin = reinterpret_cast<char *>(c.pinned);
    JET_CUDA_TRY(cudaMemcpyAsync(pin + kPinnedCtlOff + kPinnedCtlStride * (size_t)run.slot, L.ctl, sizeof(Ctl),
                                 cudaMemcpyDeviceToHost, c.stream));
    if (run.want_trace)
        JET_CUDA_TRY(cudaMemcpyAsync(pin + kPinnedTraceOff, L.trace, sizeof(TraceRec) * (size_t)kTrace,
                                     cudaMemcpyDeviceToHost, c.stream));
    return JET_OK;
}

void refine_level_abandon(LevelRun &run) {
    if (run.exec) {
        cudaGraphExecDestroy(run.exec);   // an executable graph still in flight is released on completion
        run.exec = nullptr;
    }
}

int refine_level_finish(Ctx &c, LevelRun &run, int64_t *cut_out, int64_t *maxw_out, LevelReport *rep_out) {
    refine_level_abandon(run);
    const char *pin = reinterpret_cast<const char *>(c.pinned);
    Ctl h;
    memcpy(&h, pin + kPinnedCtlOff + kPinnedCtlStride * (size_t)run.slot, sizeof(Ctl));
    if (h.bar_err) {
        record_error("refinement: a grid barrier wait of the persistent level loop ran out");
        return JET_ETIMEOUT;
    }
    LevelReport rep = run.rep;
    const int32_t iters = h.it;
    const bool kernels = run.cluster == 0 && !run.grid;
    if (!run.hostloop && run.g.n > 0) {
        if (!kernels) {
            c.launches += 1;  // the cluster or cooperative kernel
        } else {
            c.launches += 2;  // start kernel, final copy
            for (int kd = 0; kd < 3; ++kd) c.launches += (int64_t)h.kcount[kd] * (run.nk_branch[kd] + run.nk_tail);
        }
    }
    rep.cluster = run.cluster;
    rep.iters = iters;
    for (int kd = 0; kd < 3; ++kd) rep.kinds[kd] = h.kcount[kd];
    // launches per refinement kernel (one per iteration of its kind) and the
    // byte model the controllers accumulated
    if (kernels && run.g.n > 0) {
        const int32_t lp = h.kcount[MODE_LP], rw = h.kcount[MODE_RW], rs = h.kcount[MODE_RS];
        for (int kk : {JET_K_LP_SCAN, JET_K_LP_SELECT, JET_K_AFTERBURN}) rep.kern_launches[kk] = lp;
        for (int kk : {JET_K_RB_SCAN, JET_K_RB_CAND, JET_K_RB_TILEHIST, JET_K_RB_TILESCAN, JET_K_RB_TAKE})
            rep.kern_launches[kk] = rw + rs;
        rep.kern_launches[JET_K_RB_COOKIE] = rs;
        rep.kern_launches[JET_K_APPLY] = lp + rw + rs;
    }
    rep.bytes_model = 0;
    for (int i = 0; i < JET_K_COUNT; ++i) {
        rep.kern_bytes[i] = h.kbytes[i];
        rep.bytes_model += h.kbytes[i];
    }
    rep.sel_bytes = h.kbytes[JET_K_LP_SCAN] + h.kbytes[JET_K_LP_SELECT];
    rep.sel_launches = h.kcount[MODE_LP];
    if (run.want_trace) {
        c.last_trace.iters = iters;
        const int32_t nrec = std::min<int32_t>(iters, kTrace);
        const TraceRec *ht = reinterpret_cast<const TraceRec *>(pin + kPinnedTraceOff);
        c.last_trace.rec.assign(ht, ht + std::max<int32_t>(nrec, 0));
    }
    if (rep_out) *rep_out = rep;
    if (cut_out) *cut_out = h.best_cut;
    if (maxw_out) *maxw_out = h.best_maxw;
    if (!h.best_bal) return JET_WUNBALANCED;
    if (h.hit_cap) return JET_WITERLIMIT;
    return JET_OK;
}

int refine_level(Ctx &c, const DGraph &g, int32_t k, double eps, int32_t is_finest, uint64_t seed,
                 int32_t *part_inout, int64_t *cut_out, int64_t *maxw_out, LevelReport *rep_out, int64_t W_known) {
    int64_t W = W_known;
    if (W < 0) JET_TRY(total_vweight(c, g, W));
    LevelRun run;
    run.slot = 0;
    run.want_trace = true;
    int r = refine_level_enqueue(c, g, k, eps, is_finest, seed, part_inout, W, run);
    if (r < 0) {
        refine_level_abandon(run);
        return r;
    }
    cudaError_t e = cudaStreamSynchronize(c.stream);
    if (e != cudaSuccess) {
        record_cuda_error(e, "refine: synchronise", __FILE__, __LINE__);
        refine_level_abandon(run);
        return JET_ECUDA;
    }
    return refine_level_finish(c, run, cut_out, maxw_out, rep_out);
}

// ---- batched form: small levels of many graphs ----------------------------

int refine_small_chains(Ctx &c, SmallChain *chains, int32_t nchains, int32_t cluster_blocks, int *ran) {
    *ran = 0;
    if (nchains <= 0) {
        *ran = 1;
        return JET_OK;
    }
    cudaStream_t s = c.stream;
    JET_TRY(allow_large_arenas(c.device));
    int32_t kmax = 1;
    int64_t nlv_total = 0;
    size_t total = 0;
    std::vector<size_t> off((size_t)nchains);
    for (int32_t j = 0; j < nchains; ++j) {
        const SmallChain &ch = chains[j];
        int64_t nmax = 1;
        for (int32_t lv = ch.bottom; lv <= ch.top; ++lv) nmax = std::max<int64_t>(nmax, ch.h->n[lv]);
        size_t vb = 0, mb = 0;
        level_bytes(nmax, ch.k, false, &vb, &mb);
        off[(size_t)j] = total;
        total += align256(vb) + align256(mb) + 2 * align256((size_t)nmax * 4);
        nlv_total += ch.top - ch.bottom + 1;
        kmax = std::max(kmax, ch.k);
    }
    const size_t jobs_off = total;
    const size_t lv_off = jobs_off + align256(sizeof(BatchJob) * (size_t)nchains);
    const size_t st_off = lv_off + align256(sizeof(BatchLevel) * (size_t)nlv_total);
    const size_t q_off = st_off + align256(sizeof(BatchStat) * (size_t)nlv_total);
    DevBuf buf;
    JET_TRY(dev_alloc(buf, q_off + 256, s));
    char *base = buf.as<char>();
    BatchJob *d_jobs = reinterpret_cast<BatchJob *>(base + jobs_off);
    BatchLevel *d_lv = reinterpret_cast<BatchLevel *>(base + lv_off);
    BatchStat *d_st = reinterpret_cast<BatchStat *>(base + st_off);
    int32_t *d_queue = reinterpret_cast<int32_t *>(base + q_off);
    std::vector<BatchJob> jobs((size_t)nchains);
    std::vector<BatchLevel> lvs((size_t)nlv_total);
    int64_t li = 0;
    for (int32_t j = 0; j < nchains; ++j) {
        const SmallChain &ch = chains[j];
        int64_t nmax = 1;
        for (int32_t lv = ch.bottom; lv <= ch.top; ++lv) nmax = std::max<int64_t>(nmax, ch.h->n[lv]);
        size_t vb = 0, mb = 0;
        level_bytes(nmax, ch.k, false, &vb, &mb);
        char *p = base + off[(size_t)j];
        BatchJob &jb = jobs[(size_t)j];
        memset(&jb, 0, sizeof(jb));
        Level &L = jb.L;
        carve_level(L, p, p + align256(vb), nmax, ch.k, false, &jb.cut2);
        fill_level_params(c, L, 0, 0);   // per-level fields (c, seed, graph) are set in the kernel
        jb.part[0] = reinterpret_cast<int32_t *>(p + align256(vb) + align256(mb));
        jb.part[1] = jb.part[0] + align256((size_t)nmax * 4) / 4;
        jb.init = ch.init;
        jb.out = ch.out;
        jb.lv = d_lv + li;
        jb.stat = d_st + li;
        jb.nlv = ch.top - ch.bottom + 1;
        jb.Llim = balance_limit(ch.W, ch.k, ch.eps, &jb.opt);
        jb.sigma = jb.opt + (jb.Llim - jb.opt) / 2;
        for (int32_t lv = ch.top; lv >= ch.bottom; --lv, ++li) {
            BatchLevel &bl = lvs[(size_t)li];
            memset(&bl, 0, sizeof(bl));
            bl.g.n = ch.h->n[lv]; bl.g.nnz = ch.h->nnz[lv]; bl.g.xadj = ch.h->xadj[lv]; bl.g.adj = ch.h->adj[lv];
            bl.g.vw = ch.h->vw[lv]; bl.g.ew = ch.h->ew[lv];
            bl.cmap = ch.h->cmap[lv];
            bl.seed = level_seed(ch.seed, lv);
            bl.cq16 = (int32_t)llround((lv == 0 ? c.opt.c_fine : c.opt.c_coarse) * 65536.0);
        }
    }
    // launch shape: clusters of cluster_blocks blocks, as many as are co-resident
    const size_t smem = cluster_smem(kmax);
    JET_CUDA_TRY(cudaFuncSetAttribute(k_refine_batch, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    JET_CUDA_TRY(cudaFuncSetAttribute(k_refine_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int cs = cluster_blocks > 0 ? cluster_blocks : 4;
    int nclusters = 0;
    for (; cs >= 2; cs /= 2) {
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3(cs);
        cfg.blockDim = dim3(kClusterThreads);
        cfg.dynamicSmemBytes = smem;
        cudaLaunchAttribute at{};
        at.id = cudaLaunchAttributeClusterDimension;
        at.val.clusterDim.x = cs;
        at.val.clusterDim.y = 1;
        at.val.clusterDim.z = 1;
        cfg.attrs = &at;
        cfg.numAttrs = 1;
        cudaError_t e = cudaOccupancyMaxActiveClusters(&nclusters, k_refine_batch, &cfg);
        if (e != cudaSuccess) { cudaGetLastError(); nclusters = 0; }
        if (nclusters >= 1) break;
    }
    if (nclusters < 1) return JET_OK;   // *ran = 0: the caller takes the levels one by one
    nclusters = std::min(nclusters, nchains);
    JET_CUDA_TRY(cudaMemcpyAsync(d_jobs, jobs.data(), sizeof(BatchJob) * (size_t)nchains, cudaMemcpyHostToDevice, s));
    JET_CUDA_TRY(cudaMemcpyAsync(d_lv, lvs.data(), sizeof(BatchLevel) * (size_t)nlv_total, cudaMemcpyHostToDevice, s));
    JET_CUDA_TRY(cudaMemsetAsync(d_queue, 0, 4, s));
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)(nclusters * cs));
    cfg.blockDim = dim3(kClusterThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at{};
    at.id = cudaLaunchAttributeClusterDimension;
    at.val.clusterDim.x = cs;
    at.val.clusterDim.y = 1;
    at.val.clusterDim.z = 1;
    cfg.attrs = &at;
    cfg.numAttrs = 1;
    JET_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_refine_batch, (const BatchJob *)d_jobs, nchains, d_queue));
    c.launches += 1;
    std::vector<BatchStat> st((size_t)nlv_total);
    JET_CUDA_TRY(cudaMemcpyAsync(st.data(), d_st, sizeof(BatchStat) * (size_t)nlv_total, cudaMemcpyDeviceToHost, s));
    JET_CUDA_TRY(cudaStreamSynchronize(s));   // also keeps the host arrays of the copies alive until done
    li = 0;
    for (int32_t j = 0; j < nchains; ++j) {
        SmallChain &ch = chains[j];
        li += ch.top - ch.bottom + 1;
        const BatchStat &b = st[(size_t)li - 1];   // the chain's finest level
        ch.cut = b.best_cut;
        ch.maxw = b.best_maxw;
        ch.status = !b.best_bal ? JET_WUNBALANCED : (b.hit_cap ? JET_WITERLIMIT : JET_OK);
    }
    *ran = 1;
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
    ctl->ticket = 0;
    reset_counters(ctl);
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
    L.abl = flags & ABL_ALL;
    {
        int gcut = std::min(list_grid(), grid_for(g.n, kTB));
        if (g.ew) k_cut_pw<true><<<gcut, kTB, sm_cut_pw(k), s>>>(g, k, L.part, L.pw, B.cut2, L.ext, nullptr);
        else k_cut_pw<false><<<gcut, kTB, sm_cut_pw(k), s>>>(g, k, L.part, L.pw, B.cut2, L.ext, nullptr);
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
        if (dest) dest[v] = L.mstamp[v] == it ? nxt_to(L.nxt[v]) : -1;
        if (loss && L.key[v] < 0) loss[v] = kNoneGain;
    }
}

__global__ void __launch_bounds__(1024) k_rb_pass_init(Level L, const int64_t *cut2, int32_t mode) {
    __shared__ long long sh[40];
    __shared__ long long spw[JET_MAX_K];
    Ctl *ctl = L.ctl;
    if (threadIdx.x == 0) {
        ctl->cut = *cut2 / 2;
        ctl->it = 0; ctl->mode = mode;
        ctl->ticket = 0;
        reset_counters(ctl);
    }
    block_max_pw(L.pw, L.k, sh, spw);   // part weights into shared memory
    compute_classes(L, sh, spw, ctl->L, ctl->sigma);
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
    if (g.ew) k_cut_pw<true><<<gcut, kTB, sm_cut_pw(k), s>>>(g, k, L.part, L.pw, B.cut2, L.ext, L.wdeg);
    else k_cut_pw<false><<<gcut, kTB, sm_cut_pw(k), s>>>(g, k, L.part, L.pw, B.cut2, L.ext, L.wdeg);
    L.rbloss = loss_out;
    k_rb_pass_init<<<1, 1024, 0, s>>>(L, B.cut2, strong ? MODE_RS : MODE_RW);
    // the pass API takes the iteration index as a parameter: set ctl->it
    JET_CUDA_TRY(cudaMemcpyAsync(&L.ctl->it, &iter, 4, cudaMemcpyHostToDevice, s));
    k_clear_keys<<<grid_for(g.n, kTB, 4096), kTB, 0, s>>>(L);
    int nk = 0;
    JET_TRY(enqueue_rb(L, s, strong != 0, &nk));
    Ctl h;
    JET_TRY(read_ctl(c, L, h));
    if (nmoves) *nmoves = (int64_t)h.nM + h.nMh;
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
        if (g.ew) k_cut_pw<true><<<gcut, kTB, sm_cut_pw(k), s>>>(g, k, part, pw, cut2, nullptr, nullptr);
        else k_cut_pw<false><<<gcut, kTB, sm_cut_pw(k), s>>>(g, k, part, pw, cut2, nullptr, nullptr);
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
    JET_TRY(allow_large_arenas(c.device));
    size_t nn = (size_t)g.n;
    char *p = scratch;
    auto take32 = [&]() { int32_t *r = reinterpret_cast<int32_t *>(p); p += align256c(nn * 4); return r; };
    Level L{};
    L.g = g;
    L.k = k;
    L.part = const_cast<int32_t *>(part);   // read only in this pass
    L.nxt = take32(); L.prio = take32(); L.mstamp = take32(); L.lstamp = take32();
    L.listX = take32(); L.listM = take32();
    int32_t *tmp_pd = take32(), *tmp_gain = take32();
    L.ext = take32();
    L.listW = take32();
    L.ctl = reinterpret_cast<Ctl *>(p);
    p += align256c(sizeof(Ctl));
    p += 256;   // spare
    L.pw = reinterpret_cast<int64_t *>(p);
    p += align256c((size_t)JET_MAX_K * 8);
    int64_t *cut2 = reinterpret_cast<int64_t *>(p);
    fill_level_params(c, L, 1, 0);
    L.cq16 = (int32_t)llround(cval * 65536.0);
    L.abl = flags & ABL_ALL;
    // the array keeps the previous call's contents: clear what must start at zero
    JET_CUDA_TRY(cudaMemsetAsync(L.ctl, 0, sizeof(Ctl), s));
    JET_CUDA_TRY(cudaMemsetAsync(L.pw, 0, (size_t)k * 8, s));
    JET_CUDA_TRY(cudaMemsetAsync(cut2, 0, 16, s));
    {
        int gcut = std::min(list_grid(), grid_for(g.n, kTB));
        if (g.ew) k_cut_pw<true><<<gcut, kTB, sm_cut_pw(k), s>>>(g, k, L.part, L.pw, cut2, L.ext, nullptr);
        else k_cut_pw<false><<<gcut, kTB, sm_cut_pw(k), s>>>(g, k, L.part, L.pw, cut2, L.ext, nullptr);
    }
    k_count_big<<<grid_for(g.n, kTB), kTB, 0, s>>>(g, &L.ctl->nbig);
    k_fill_i32<<<grid_for(g.n, kTB, 4096), kTB, 0, s>>>(L.mstamp, g.n, -2);
    k_fill_i32<<<grid_for(g.n, kTB, 4096), kTB, 0, s>>>(L.prio, g.n, kNoneGain);
    k_locks_from_mask<<<grid_for(g.n, kTB, 4096), kTB, 0, s>>>(locked, L.lstamp, g.n);
    k_set_epoch<<<1, 1, 0, s>>>(L.ctl, 0, MODE_LP);
    JET_CUDA_TRY(cudaGetLastError());
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
