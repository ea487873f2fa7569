// Internal definitions shared by the CUDA translation units of libjet.
// Nothing here is part of the C ABI (include/jet.h).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>
#include <cstring>
#include <vector>

#include "jet.h"

namespace jet {

// ---------------------------------------------------------------------------
// constants
// ---------------------------------------------------------------------------
constexpr int32_t kNoneGain = INT32_MIN;   // "negative infinity" gain (Alg. 4)
constexpr int kSlots = 33;                 // slot() values 0..32 for 32-bit losses (Sec. 4.2.1)
constexpr int kSmallDeg = 16;              // rows up to this length: one thread per vertex
constexpr int kHugeDeg = 1024;             // rows longer than this: one whole block per row
constexpr int kHugeCap = 128;              // block-schedule rows set aside per drain of a block
constexpr int kTB = 256;                   // default block size
#ifndef JET_RB_TILE
#define JET_RB_TILE 256
#endif
constexpr int kRbTile = JET_RB_TILE;       // vertices per rebalancing tile (ordered prefixes; one block each)
constexpr int kTrace = 4096;               // per-level trace records kept on the device

enum Mode : int32_t { MODE_LP = 0, MODE_RW = 1, MODE_RS = 2, MODE_DONE = 3 };

// Internal ablation bits (match the JET_FLAG_* values)
constexpr uint32_t ABL_NO_LOCKS = JET_FLAG_NO_LOCKS;
constexpr uint32_t ABL_NO_AFTERBURN = JET_FLAG_NO_AFTERBURN;
constexpr uint32_t ABL_WEAK_AFTERBURN = JET_FLAG_WEAK_AFTERBURN;
constexpr uint32_t ABL_BASELINE_LP = JET_FLAG_BASELINE_LP;
constexpr uint32_t ABL_STRICT_GAIN = JET_FLAG_STRICT_GAIN;
constexpr uint32_t ABL_ALL = ABL_NO_LOCKS | ABL_NO_AFTERBURN | ABL_WEAK_AFTERBURN | ABL_BASELINE_LP | ABL_STRICT_GAIN;

// ---------------------------------------------------------------------------
// error handling
// ---------------------------------------------------------------------------
#define JET_CUDA_TRY(expr)                                                          \
    do {                                                                            \
        cudaError_t e__ = (expr);                                                   \
        if (e__ != cudaSuccess) {                                                   \
            ::jet::record_cuda_error(e__, #expr, __FILE__, __LINE__);               \
            return e__ == cudaErrorMemoryAllocation ? JET_ENOMEM : JET_ECUDA;       \
        }                                                                           \
    } while (0)

#define JET_TRY(expr)                                                               \
    do {                                                                            \
        int s__ = (expr);                                                           \
        if (s__ < 0) return s__;                                                    \
    } while (0)

void record_cuda_error(cudaError_t e, const char *what, const char *file, int line);
void record_error(const char *msg);
const char *last_error_text();

// ---------------------------------------------------------------------------
// device memory owned by the library: stream-ordered allocations
// ---------------------------------------------------------------------------
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    cudaStream_t s = nullptr;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    DevBuf(DevBuf &&o) noexcept : p(o.p), bytes(o.bytes), s(o.s) { o.p = nullptr; o.bytes = 0; }
    DevBuf &operator=(DevBuf &&o) noexcept {
        if (this != &o) { release(); p = o.p; bytes = o.bytes; s = o.s; o.p = nullptr; o.bytes = 0; }
        return *this;
    }
    ~DevBuf() { release(); }
    void release() {
        if (p) { cudaFreeAsync(p, s); p = nullptr; bytes = 0; }
    }
    template <class T> T *as() const { return static_cast<T *>(p); }
};

// Allocate `bytes` (rounded up to 256) on stream s; returns JET_OK/JET_ENOMEM.
int dev_alloc(DevBuf &b, size_t bytes, cudaStream_t s);

// ---------------------------------------------------------------------------
// graph view
// ---------------------------------------------------------------------------
struct DGraph {
    int32_t n = 0;
    int64_t nnz = 0;
    const int64_t *xadj = nullptr;
    const int32_t *adj = nullptr;
    const int32_t *vw = nullptr;   // never null inside the library (materialised)
    const int32_t *ew = nullptr;   // null: unit edge weights
};

// ---------------------------------------------------------------------------
// device control block of one refinement level (Alg. 3 state)
// ---------------------------------------------------------------------------
struct TraceRec {
    int32_t kind;
    int32_t flags;    // bit 0: the controller ordered P_best <- P_iter (copied by the next iteration)
    int32_t na;       // rebalancing: oversized parts (|A|) of this iteration
    int32_t pad;
    int64_t nx, nm, cut, maxw;
    int64_t degx;     // sum of row lengths over X (Jetlp) or over the rebalancing candidates
    int64_t degm;     // sum of row lengths over M
    int64_t nbnd;     // Jetlp: boundary vertices; rebalancing: candidates whose rows were read
    int64_t nexam;    // Jetlp: unlocked boundary vertices whose rows were read
    int64_t degexam;  // total row length over those rows
};

struct Ctl {
    int32_t mode;        // kind of the iteration about to run (Mode)
    int32_t it;          // iterations completed on this level
    int32_t noimp;       // iterations since the last reset (Alg. 3 "iteration counter")
    int32_t weak;        // Jetrw iterations since the last Jetlp
    int32_t lp_epoch;    // iteration index of the last Jetlp (its movers are locked)
    int32_t copy_best;   // set by the controller: P_best <- P_iter this iteration
    int32_t best_bal;
    int32_t nA, nB;      // rebalancing classes for the current iteration
    int32_t nW;          // work list of the current pass (unlocked boundary vertices / listed candidates)
    int32_t nX;          // X list length
    int32_t nM;          // M list length
    int32_t ticket;      // blocks of the current kernel that finished (last-block tails)
    int32_t hit_cap;     // stopped by max_iters
    int32_t nXh, nMh;    // hub rows of X / M, stored from the end of listX / listM downwards
    int32_t kcount[4];   // iterations run per kind (Jetlp, Jetrw, Jetrs)
    int64_t ncand;       // rebalancing candidates (trace)
    int64_t degx, degm;  // row-length sums over X / candidates and over M (byte model)
    int64_t nbnd;        // Jetlp select: boundary vertices (ext > 0) seen
    int64_t nexam;       // ... of which unlocked (rows streamed)
    int64_t degexam;     // ... their total row length
    int64_t cut;         // cost of P_iter
    int64_t dcut;        // cut change accumulated by the apply kernel
    int64_t maxw;        // max part weight of P_iter
    int64_t best_cut, best_maxw;
    int64_t L, opt, sigma;
    // persistent level loop: grid barrier (arrivals, generation) and the
    // flag a block sets when its bounded wait at a barrier ran out
    uint32_t bar_count, bar_gen;
    int32_t bar_err;
    int32_t nbig;        // vertices with rows longer than kSmallDeg (0: no per-warp tables needed)
    int64_t kbytes[JET_KERNELS];   // algorithmic DRAM bytes per refinement kernel (byte model)
    // coarsening
    int32_t hem_stop;
    int32_t pad1;
    int64_t hem_added[64];
    int64_t scratch[8];
};

// Parameters of one refinement level, passed by value to every kernel.
struct Level {
    DGraph g;
    int32_t k;
    int32_t cq16;            // c * 65536
    int64_t phi_ppm;         // phi * 1e6
    int32_t max_no_improve, weak_limit, max_iters;
    uint32_t abl;
    uint64_t seed;
    // per-vertex state
    int32_t *part, *best, *nxt, *prio, *mstamp, *lstamp, *key;
    int32_t *ext;            // neighbours in other parts (exact, kept by the apply kernel)
    int32_t *wdeg;           // weighted degree (rebalancing of interior vertices)
    int32_t *rbloss;         // rebalancing loss export (single-pass API only; may be null)
    int32_t *listX, *listM;
    int32_t *listW;          // work list: vertices whose rows a pass must read
    // per-part state
    int64_t *pw;
    int32_t *aidx, *Bs;
    uint8_t *inB;
    int64_t *capC;           // nB+1 capacity prefix (Jetrs)
    int64_t *excess;         // [nA]
    int64_t *bucketw;        // [nA * kSlots]
    int32_t *sstar;          // [nA] boundary slot
    int64_t *need;           // [nA] weight still to take inside the boundary slot
    int32_t *tilehist;       // [ntiles * k]
    int32_t ntiles;
    int64_t *tiletaken;      // [ntiles]
    int64_t *etaken;         // [n] Jetrs: weight of v in the evicted list (0 if not evicted)
    TraceRec *trace;
    Ctl *ctl;
    // CUDA-graph loop control (0 when driven from the host)
    unsigned long long h_loop, h_mode;
    unsigned long long h_next;   // switch of the next iteration (the loop body holds two iterations)
    int32_t use_graph;
    int32_t pdl;             // launch the row and tile kernels with programmatic dependent launch
    int64_t poll_limit;      // persistent loop: polls at a grid barrier before a block gives up
    int32_t hub_deg;         // rows longer than this are taken by a whole block in the row phases
    // launch shapes (host side; execution choices, results do not depend on them)
    int32_t list_cap;        // most blocks of a list kernel (select, afterburner, rebalancing rows)
    int32_t apply_cap;       // most blocks of the apply kernel
    int32_t scan_cap;        // most blocks of a scan kernel
    int32_t rb_scan_cap;     // the same for the rebalancing scan, at most one wave of resident blocks
    int32_t items_per_block; // list entries per block below those caps
};

// ---------------------------------------------------------------------------
// small device helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

__device__ __forceinline__ int slot_of(int64_t x) {
    if (x < 0) return 0;
    if (x == 0) return 1;
    return 2 + (63 - __clzll((unsigned long long)x));
}

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long t = __shfl_xor_sync(0xffffffffu, v, o);
        v = t > v ? t : v;
    }
    return v;
}

__device__ __forceinline__ long long warp_sum_i64(long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ int warp_sum_i32(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Programmatic dependent launch: a kernel lets the next one in the stream be
// scheduled as soon as all its own blocks have started, and waits for the
// previous kernel to complete (memory visible) before it touches any data.
// Both are no-ops for a kernel launched without the attribute.
__device__ __forceinline__ void pdl_enter() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// A launch that, with pdl, may be scheduled before the previous kernel in
// the stream completes; the kernel must begin with pdl_enter().
template <class... KArgs, class... Args>
cudaError_t launch_pdl(void (*kern)(KArgs...), int grid, int block, size_t smem, cudaStream_t s, bool pdl,
                       Args... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at{};
    at.id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at.val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = &at;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

// Append from any subset of a warp's lanes: one atomic per warp; returns the
// slot for the calling lane.  All lanes of the warp must call it (pred may be
// false).
__device__ __forceinline__ int warp_append(int32_t *counter, bool pred) {
    unsigned m = __ballot_sync(0xffffffffu, pred);
    if (!m) return -1;
    int leader = __ffs(m) - 1;
    int base = 0;
    if ((int)lane_id() == leader) base = atomicAdd(counter, __popc(m));
    base = __shfl_sync(0xffffffffu, base, leader);
    return pred ? base + __popc(m & ((1u << lane_id()) - 1u)) : -1;
}

// Block-aggregated append into a global list.  Members are staged in shared
// memory (CAP entries) and reserved in the global list with one atomic per
// flush, instead of one atomic per warp on a single hot counter.  Between two
// flush() calls every thread may add() at most `adds` times (see flush).
template <int CAP>
struct BlockAppender {
    int32_t *sbuf;
    int *scount;
    int *gbase;
    __device__ __forceinline__ void init() {
        if (threadIdx.x == 0) *scount = 0;
        __syncthreads();
    }
    __device__ __forceinline__ void add(bool pred, int32_t v) {   // called by all threads of a warp
        unsigned m = __ballot_sync(0xffffffffu, pred);
        if (!m) return;
        int leader = __ffs(m) - 1;
        int base = 0;
        if ((int)(threadIdx.x & 31u) == leader) base = atomicAdd(scount, __popc(m));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (pred) sbuf[base + __popc(m & ((1u << (threadIdx.x & 31u)) - 1u))] = v;
    }
    // Flushes when the buffer could overflow on the next round (each thread
    // adding up to `adds` members), or always when force is set.  Called by
    // all threads of the block.
    __device__ __forceinline__ void flush(int32_t *gcount, int32_t *glist, bool force, int adds = 1) {
        __syncthreads();
        int c = *scount;
        if (c > 0 && (force || c > CAP - adds * (int)blockDim.x)) {
            if (threadIdx.x == 0) *gbase = atomicAdd(gcount, c);
            __syncthreads();
            int b = *gbase;
            for (int i = threadIdx.x; i < c; i += blockDim.x) glist[b + i] = sbuf[i];
            __syncthreads();
            if (threadIdx.x == 0) *scount = 0;
            __syncthreads();
        }
    }
};

#define JET_BLOCK_APPENDER(name, CAP)                                                \
    __shared__ int32_t name##_buf[CAP];                                              \
    __shared__ int name##_cnt, name##_base;                                          \
    BlockAppender<CAP> name{name##_buf, &name##_cnt, &name##_base};                  \
    name.init()

__device__ __forceinline__ void atomic_add_i64(int64_t *p, int64_t v) {
    atomicAdd(reinterpret_cast<unsigned long long *>(p), (unsigned long long)v);
}

__device__ __forceinline__ int64_t ld_xadj(const int64_t *x, int64_t i) { return __ldg(x + i); }

// block-wide sum (blockDim.x multiple of 32, <= 1024); result valid in all threads
__device__ __forceinline__ long long block_sum_i64(long long v, long long *sh /* >= 32 */) {
    v = warp_sum_i64(v);
    unsigned w = threadIdx.x >> 5;
    __syncthreads();
    if (lane_id() == 0) sh[w] = v;
    __syncthreads();
    unsigned nw = (blockDim.x + 31) >> 5;
    long long t = (threadIdx.x < nw) ? sh[threadIdx.x] : 0;
    if (threadIdx.x < 32) t = warp_sum_i64(t);
    if (threadIdx.x == 0) sh[0] = t;
    __syncthreads();
    long long r = sh[0];
    __syncthreads();
    return r;
}

// block-wide exclusive scan of one int64 per thread; *total gets the sum
__device__ __forceinline__ long long block_exscan_i64(long long v, long long *sh /* >= 33 */, long long *total) {
    unsigned lane = lane_id(), w = threadIdx.x >> 5;
    long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        long long t = __shfl_up_sync(0xffffffffu, x, o);
        if ((int)lane >= o) x += t;
    }
    __syncthreads();
    if (lane == 31) sh[w] = x;
    __syncthreads();
    unsigned nw = (blockDim.x + 31) >> 5;
    if (threadIdx.x < 32) {
        long long s = (threadIdx.x < nw) ? sh[threadIdx.x] : 0;
        long long y = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            long long t = __shfl_up_sync(0xffffffffu, y, o);
            if ((int)lane >= o) y += t;
        }
        if (threadIdx.x < nw) sh[threadIdx.x] = y - s;  // exclusive warp offsets
        if (threadIdx.x == nw - 1) sh[32] = y;
    }
    __syncthreads();
    long long r = sh[w] + x - v;
    if (total) *total = sh[32];
    __syncthreads();
    return r;
}

inline int grid_for(int64_t items, int per_block, int cap = 1 << 30) {
    int64_t g = (items + per_block - 1) / per_block;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

int num_sms();

// ---------------------------------------------------------------------------
// device-wide exclusive scan (3 phases: tile sums, scan of tile sums, tiles)
// ---------------------------------------------------------------------------
// out[i] = sum_{j<i} f(j) for i in [0, n); *total_dev = sum (device int64).
// Functor F: __device__ int64_t operator()(int64_t i) const.
template <class F> __global__ void k_scan_tiles(F f, int64_t n, int64_t *tile_sums);
template <class F> __global__ void k_scan_apply(F f, int64_t n, const int64_t *tile_off, int64_t *out);
__global__ void k_scan_sums(int64_t *tile_sums, int64_t ntiles, int64_t *total_dev);

constexpr int kScanItems = 8;
constexpr int kScanTile = kTB * kScanItems;

template <class F>
__global__ void __launch_bounds__(kTB) k_scan_tiles(F f, int64_t n, int64_t *tile_sums) {
    __shared__ long long sh[40];
    pdl_enter();
    int64_t base = (int64_t)blockIdx.x * kScanTile;
    long long s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        int64_t idx = base + (int64_t)threadIdx.x * kScanItems + i;
        if (idx < n) s += f(idx);
    }
    s = block_sum_i64(s, sh);
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = s;
}

template <class F>
__global__ void __launch_bounds__(kTB) k_scan_apply(F f, int64_t n, const int64_t *tile_off, int64_t *out) {
    __shared__ long long sh[40];
    pdl_enter();
    int64_t base = (int64_t)blockIdx.x * kScanTile;
    long long vals[kScanItems];
    long long s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        int64_t idx = base + (int64_t)threadIdx.x * kScanItems + i;
        vals[i] = idx < n ? f(idx) : 0;
        s += vals[i];
    }
    long long off = block_exscan_i64(s, sh, nullptr) + tile_off[blockIdx.x];
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        int64_t idx = base + (int64_t)threadIdx.x * kScanItems + i;
        if (idx < n) out[idx] = off;
        off += vals[i];
    }
}

// Scratch for a scan of n items: (ntiles) int64.
inline int64_t scan_tiles_for(int64_t n) { return (n + kScanTile - 1) / kScanTile; }

template <class F>
int device_exscan(F f, int64_t n, int64_t *out, int64_t *total_dev, int64_t *tile_scratch, cudaStream_t s) {
    int64_t nt = scan_tiles_for(n);
    if (nt < 1) nt = 1;
    // the three kernels (and the next one) follow by programmatic launch
    JET_CUDA_TRY(launch_pdl(k_scan_tiles<F>, (int)nt, kTB, 0, s, true, f, n, tile_scratch));
    JET_CUDA_TRY(launch_pdl(k_scan_sums, 1, 1024, 0, s, true, tile_scratch, nt, total_dev));
    JET_CUDA_TRY(launch_pdl(k_scan_apply<F>, (int)nt, kTB, 0, s, true, f, n, (const int64_t *)tile_scratch, out));
    return JET_OK;
}

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------
struct TraceHost {
    std::vector<TraceRec> rec;
    int32_t iters = 0;
};

// What one refinement level did (for jet_stats).
struct LevelReport {
    int32_t iters = 0, kinds[3] = {0, 0, 0};
    int64_t sel_launches = 0, sel_bytes = 0, bytes_model = 0;
    float sel_ms = 0.f;
    int32_t cluster = 0;   // blocks of the cluster that ran the level loop (0: graph or host loop)
    // per refinement kernel (JET_K_*): launches, algorithmic bytes, CUDA-event ms (profiling only)
    int64_t kern_launches[JET_KERNELS] = {};
    int64_t kern_bytes[JET_KERNELS] = {};
    float kern_ms[JET_KERNELS] = {};
};

// Pinned host buffer of a context: scalar readbacks in the first 4 KB, then
// one control block per level of an uncoarsening (copied back when the level
// is enqueued, read after the last level), then the finest level's trace.
constexpr size_t kPinnedScalarBytes = 4096;
constexpr size_t kPinnedCtlStride = (sizeof(Ctl) + 255) & ~size_t(255);
constexpr size_t kPinnedCtlOff = kPinnedScalarBytes;
constexpr size_t kPinnedTraceOff = kPinnedCtlOff + kPinnedCtlStride * JET_MAX_LEVELS;
constexpr size_t kPinnedBytes = kPinnedTraceOff + sizeof(TraceRec) * (size_t)kTrace;

struct Ctx {
    int64_t launches = 0;        // kernels launched (graph-loop iterations counted per executed kernel)
    int device = 0;
    cudaStream_t stream = nullptr;
    jet_options opt{};
    int64_t *pinned = nullptr;   // pinned host buffer (layout: kPinned* below)
    cudaMemPool_t pool = nullptr; // the context's stream-ordered pool (keeps its memory between calls)
    TraceHost last_trace;
};

}  // namespace jet

struct jet_ctx {
    jet::Ctx c;
};

// hierarchy: level 0 borrows the caller's arrays (weights materialised when
// NULL), coarser levels are owned
struct jet_hier {
    jet_ctx *ctx = nullptr;
    int32_t levels = 0;
    int32_t k = 0;
    int32_t n[JET_MAX_LEVELS] = {};
    int64_t nnz[JET_MAX_LEVELS] = {};
    const int64_t *xadj[JET_MAX_LEVELS] = {};
    const int32_t *adj[JET_MAX_LEVELS] = {};
    const int32_t *vw[JET_MAX_LEVELS] = {};
    const int32_t *ew[JET_MAX_LEVELS] = {};
    const int32_t *cmap[JET_MAX_LEVELS] = {};
    std::vector<jet::DevBuf> bufs;
    float ms_coarsen = 0.f;
    int64_t launches = 0;     // kernels jet_coarsen executed
};

namespace jet {

// ----- functions implemented in the .cu files ------------------------------
// jet_refine.cu
// One level of refinement enqueued on the context's stream without a host
// wait (the host-driven loop excepted): its control block comes back into
// pinned slot `slot` (and, with want_trace, its trace into the context's
// trace area) once the stream gets there; refine_level_finish reads them
// after the caller has synchronised the stream.
struct LevelRun {
    int32_t slot = 0;
    bool want_trace = false;
    DGraph g;
    int32_t k = 0;
    int32_t cluster = 0, grid = 0, hostloop = 0;
    int nk_branch[3] = {0, 0, 0}, nk_tail = 0;
    cudaGraphExec_t exec = nullptr;   // the level's CUDA-graph loop (destroyed by refine_level_finish)
    LevelReport rep;                  // host-loop profile (kern_ms, sel_ms)
};
// W: the graph's total vertex weight (every level of a hierarchy has the same).
int refine_level_enqueue(Ctx &c, const DGraph &g, int32_t k, double eps, int32_t is_finest, uint64_t seed,
                         int32_t *part_inout, int64_t W, LevelRun &run);
int refine_level_finish(Ctx &c, LevelRun &run, int64_t *cut_out, int64_t *maxw_out, LevelReport *rep);
void refine_level_abandon(LevelRun &run);   // after an error: release what the run holds
// The batched form's small levels: one graph's chain of levels of at most
// cluster_max_n vertices, refined with those of the other chains in one
// persistent cluster launch (refine_small_chains).
struct SmallChain {
    const jet_hier *h = nullptr;
    int32_t top = 0, bottom = 0;     // the coarsest level and the finest small level (top >= bottom)
    int32_t k = 2;
    double eps = 0.03;
    uint64_t seed = 1;               // the partition's seed (level seeds derive from it)
    int64_t W = 0;                   // total vertex weight
    const int32_t *init = nullptr;   // device: start partition of level `top`
    int32_t *out = nullptr;          // device: receives the refined partition of level `bottom`
    int64_t cut = 0, maxw = 0;       // out: of level `bottom`
    int32_t status = JET_OK;         // out: of level `bottom`
};
// cluster_blocks: blocks of each cluster (0 = 4).  On success every chain's
// `out` holds its result; JET_ECUDA with *ran = 0 when the device cannot
// co-schedule one cluster (the caller refines the levels one by one).
int refine_small_chains(Ctx &c, SmallChain *chains, int32_t nchains, int32_t cluster_blocks, int *ran);
uint64_t level_seed(uint64_t seed, int32_t level);   // Jetrw seed of hierarchy level `level`

// Enqueue + synchronise + finish.  W_known: -1 = computed on the device.
int refine_level(Ctx &c, const DGraph &g, int32_t k, double eps, int32_t is_finest, uint64_t seed,
                 int32_t *part_inout, int64_t *cut_out, int64_t *maxw_out, LevelReport *rep, int64_t W_known = -1);
// Sum of the vertex weights (one device reduction and a readback).
int total_vweight(Ctx &c, const DGraph &g, int64_t &W);
int lp_pass(Ctx &c, const DGraph &g, int32_t k, const int32_t *part, const uint8_t *locked, double cval,
            uint32_t flags, int32_t *pd_out, int32_t *gain_out, uint8_t *inx_out, int32_t *f2_out,
            uint8_t *inm_out);
// The same pass with every scratch array carved out of `scratch` (at least
// lp_scratch_bytes(g.n) bytes of device memory, 256-byte aligned): no
// allocation.  Used by jet_lp_pass_noalloc.
constexpr size_t align256c(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t lp_scratch_bytes(int64_t n) {
    return 10 * align256c((size_t)(n > 0 ? n : 1) * 4) + align256c(sizeof(Ctl)) + 256 +
           align256c((size_t)JET_MAX_K * 8) + 256;
}
int lp_pass_in_scratch(Ctx &c, const DGraph &g, int32_t k, const int32_t *part, const uint8_t *locked, double cval,
                       uint32_t flags, int32_t *pd_out, int32_t *gain_out, uint8_t *inx_out, int32_t *f2_out,
                       uint8_t *inm_out, char *scratch);
int rebalance_pass(Ctx &c, const DGraph &g, int32_t k, double eps, int32_t strong, uint64_t seed, int32_t iter,
                   const int32_t *part, int32_t *dest_out, int32_t *loss_out, int64_t *nmoves, int64_t *ncand);
int cut_and_weights(Ctx &c, const DGraph &g, int32_t k, const int32_t *part, int64_t *cut_out, int64_t *pw_dev);

// jet_coarsen.cu
int hem(Ctx &c, const DGraph &g, uint64_t seed, int32_t level, int32_t rounds, int32_t *mate);
int coarsen(Ctx &c, const DGraph &g0, int32_t k, uint64_t seed, jet_hier *h);
// The greedy order behind the initial partition (component, BFS distance,
// id), for the learned initial partition's features and labels.  Device
// arrays are the caller's (any may be null); the scalars are filled on return.
struct GreedyOut {
    int32_t *dist = nullptr;   // int32[n]: BFS distance from the component's lowest id
    int64_t *S = nullptr;      // int64[n]: weight of the vertices before v in the order
    int32_t *rank = nullptr;   // int32[n]: position of v in the order
    int32_t maxdist = 0;       // deepest BFS level
    int64_t W = 0;             // total vertex weight
};
// part may be null when only the order is wanted.
int initial_partition(Ctx &c, const DGraph &g, int32_t k, int32_t *part, GreedyOut *go = nullptr);

// jet_sort.cu: stable LSD radix sort of (key, value) pairs.
struct SortScratch {
    uint64_t *key[2];
    int32_t *val[2];
    int64_t *hist, *off, *scan, *total;
};
int bits_for(int64_t x);                         // bits that hold 0..x
size_t sort_scratch_bytes(int64_t n);
void sort_scratch_carve(char *p, int64_t n, SortScratch &s);
// Sorts (key[0], val[0]) by the low kbits bits of the key, keeping the input
// order among equal keys; *which = buffer index (0/1) that holds the result.
int sort_pairs(Ctx &c, SortScratch &s, int64_t n, int kbits, int *which);

// jet_twohop.cu: two-hop matching after heavy-edge matching (Sec. 3.1);
// added[s] = vertices matched by stage s (leaves, twins, relatives).
constexpr int32_t kMatchmakerMaxDeg = 1024;
int two_hop(Ctx &c, const DGraph &g, int32_t *mate, int64_t added[3]);
int project(Ctx &c, int32_t n_fine, const int32_t *cmap, const int32_t *coarse_part, int32_t *fine_part);

// host helpers (jet_api.cu)
int64_t balance_limit(int64_t W, int32_t k, double eps, int64_t *opt);
int sync_stream(Ctx &c);
int use_device(Ctx &c);
bool bad_k_eps(int32_t k, double eps);
int check_part(Ctx &c, int32_t n, const int32_t *part, int32_t k);   // JET_EINVAL unless every part is in [0, k)
int prepare_graph(Ctx &c, int32_t n, const int64_t *xadj, const int32_t *adjncy, const int32_t *vwgt,
                  const int32_t *adjwgt, DGraph &g, DevBuf &ones, bool need_vw);
// Alg. 1 after coarsening; init_coarsest (device, n of the coarsest level)
// replaces the greedy initial partition when not null.  With top >= 0 the
// uncoarsening starts at level `top` from init_coarsest (n[top] entries):
// refined there too unless top_refined, then projected and refined on
// every finer level.
int uncoarsen(Ctx &c, const jet_hier *h, int32_t k, double eps, uint64_t seed, const int32_t *init_coarsest,
              int32_t *part_out, int64_t *cut_out, jet_stats *st, int32_t top = -1, bool top_refined = false);

}  // namespace jet
