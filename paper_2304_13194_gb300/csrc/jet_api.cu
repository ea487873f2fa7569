// C ABI of libjet (include/jet.h): context, argument checks, the multilevel
// driver of Alg. 1 and the single-pass entry points.
#include "jet_internal.cuh"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <new>
#include <thread>
#include <vector>

namespace jet {

static thread_local char g_err[512] = "";

void record_cuda_error(cudaError_t e, const char *what, const char *file, int line) {
    snprintf(g_err, sizeof(g_err), "%s: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
}

void record_error(const char *msg) { snprintf(g_err, sizeof(g_err), "%s", msg); }

const char *last_error_text() { return g_err; }

// Pool of the context whose entry point runs on this thread (set by
// use_device); null: the device's default pool.
static thread_local cudaMemPool_t t_pool = nullptr;

// Device allocations made by the library in this process (jet_alloc_count)
// and the injected failure (jet_debug_fail_alloc): the allocation whose
// count reaches g_fail_at fails; 0 = none armed.
static std::atomic<int64_t> g_alloc_count{0};
static std::atomic<int64_t> g_fail_at{0};

int dev_alloc(DevBuf &b, size_t bytes, cudaStream_t s) {
    b.release();
    b.s = s;
    const int64_t idx = g_alloc_count.fetch_add(1, std::memory_order_relaxed) + 1;
    int64_t armed = g_fail_at.load(std::memory_order_relaxed);
    if (armed != 0 && idx == armed && g_fail_at.compare_exchange_strong(armed, 0)) {
        record_error("device allocation failed (injected by jet_debug_fail_alloc)");
        return JET_ENOMEM;
    }
    bytes = std::max<size_t>(256, (bytes + 255) & ~size_t(255));
    cudaError_t e = t_pool ? cudaMallocFromPoolAsync(&b.p, bytes, t_pool, s) : cudaMallocAsync(&b.p, bytes, s);
    if (e != cudaSuccess) {
        b.p = nullptr;
        record_cuda_error(e, "cudaMallocAsync", __FILE__, __LINE__);
        cudaGetLastError();
        return JET_ENOMEM;
    }
    b.bytes = bytes;
    return JET_OK;
}

int num_sms() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

// Balance limit of Sec. 2.1 in integers: opt = ceil(W/k),
// L = floor(opt * (10^6 + round(eps * 10^6)) / 10^6).
int64_t balance_limit(int64_t W, int32_t k, double eps, int64_t *opt) {
    int64_t o = (W + k - 1) / k;
    int64_t e = llround(eps * 1e6);
    if (opt) *opt = o;
    return o * (1000000 + e) / 1000000;
}

int sync_stream(Ctx &c) {
    JET_CUDA_TRY(cudaStreamSynchronize(c.stream));
    return JET_OK;
}

static uint64_t host_splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// Seed of Jetrw's random destination on level i of the hierarchy.
uint64_t level_seed(uint64_t seed, int32_t level) {
    return host_splitmix64(seed ^ (0xA0761D6478BD642FULL * (uint64_t)(level + 1)));
}

// ---------------------------------------------------------------------------
// input checks
// ---------------------------------------------------------------------------
struct CheckOut {
    long long sum_vw, sum_ew, bad;
};

__global__ void k_check(int32_t n, const int64_t *xadj, const int32_t *adj, const int32_t *vw, const int32_t *ew,
                        int validate, CheckOut *out) {
    __shared__ long long sh[40];
    long long svw = 0, sew = 0, bad = 0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        int64_t beg = xadj[v], end = xadj[v + 1];
        svw += vw ? vw[v] : 1;
        if (validate) {
            if (end < beg) { bad = 1; continue; }
            if (vw && vw[v] <= 0) bad = 1;
        }
        for (int64_t j = beg; j < end; ++j) {
            int32_t w = ew ? ew[j] : 1;
            sew += w;
            if (!validate) continue;
            int32_t u = adj[j];
            if (u < 0 || u >= n || u == (int32_t)v || w <= 0) { bad = 1; continue; }
            // exactly one entry (v, w) in u's row: symmetric and no parallel edge
            int64_t ub = xadj[u], ue = xadj[(int64_t)u + 1];
            int cnt = 0;
            bool wok = false;
            for (int64_t t = ub; t < ue; ++t)
                if (adj[t] == (int32_t)v) { ++cnt; wok = (ew ? ew[t] : 1) == w; }
            if (cnt != 1 || !wok) bad = 1;
        }
    }
    svw = block_sum_i64(svw, sh);
    sew = block_sum_i64(sew, sh);
    bad = block_sum_i64(bad, sh);
    if (threadIdx.x == 0) {
        atomic_add_i64(reinterpret_cast<int64_t *>(&out->sum_vw), svw);
        atomic_add_i64(reinterpret_cast<int64_t *>(&out->sum_ew), sew);
        if (bad) atomic_add_i64(reinterpret_cast<int64_t *>(&out->bad), bad);
    }
}

__global__ void k_ones32(int32_t *p, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) p[i] = 1;
}

__global__ void k_check_part(int32_t n, const int32_t *part, int32_t k, int *bad) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        if (part[v] < 0 || part[v] >= k) atomicOr(bad, 1);
}

// Argument checks plus the overflow limits of jet.h (and the full graph
// check with JET_FLAG_VALIDATE).  Fills g; materialises unit vertex weights
// into `ones` when vwgt is NULL.
int prepare_graph(Ctx &c, int32_t n, const int64_t *xadj, const int32_t *adjncy, const int32_t *vwgt,
                  const int32_t *adjwgt, DGraph &g, DevBuf &ones, bool need_vw) {
    if (n < 0 || !xadj) return JET_EINVAL;
    cudaStream_t s = c.stream;
    int64_t nnz = 0;
    JET_CUDA_TRY(cudaMemcpyAsync(c.pinned, xadj + n, 8, cudaMemcpyDeviceToHost, s));
    JET_CUDA_TRY(cudaStreamSynchronize(s));
    nnz = c.pinned[0];
    if (nnz < 0) return JET_EGRAPH;
    if (nnz > 0 && !adjncy) return JET_EINVAL;
    DevBuf cb;
    JET_TRY(dev_alloc(cb, sizeof(CheckOut), s));
    JET_CUDA_TRY(cudaMemsetAsync(cb.p, 0, sizeof(CheckOut), s));
    int validate = (c.opt.flags & JET_FLAG_VALIDATE) ? 1 : 0;
    if (n > 0)
        k_check<<<std::min(num_sms() * 8, grid_for(n, kTB)), kTB, 0, s>>>(n, xadj, adjncy, vwgt, adjwgt, validate,
                                                                         cb.as<CheckOut>());
    JET_CUDA_TRY(cudaGetLastError());
    JET_CUDA_TRY(cudaMemcpyAsync(c.pinned, cb.p, sizeof(CheckOut), cudaMemcpyDeviceToHost, s));
    JET_CUDA_TRY(cudaStreamSynchronize(s));
    CheckOut h;
    memcpy(&h, c.pinned, sizeof(h));
    if (h.bad) return JET_EGRAPH;
    if (h.sum_vw >= (1LL << 31) || h.sum_ew >= (1LL << 31)) return JET_EOVERFLOW;
    g.n = n;
    g.nnz = nnz;
    g.xadj = xadj;
    g.adj = adjncy;
    g.ew = adjwgt;
    g.vw = vwgt;
    if (!vwgt && need_vw) {
        JET_TRY(dev_alloc(ones, (size_t)std::max(n, 1) * 4, s));
        if (n > 0) k_ones32<<<grid_for(n, kTB, 8192), kTB, 0, s>>>(ones.as<int32_t>(), n);
        JET_CUDA_TRY(cudaGetLastError());
        g.vw = ones.as<int32_t>();
    }
    return JET_OK;
}

int check_part(Ctx &c, int32_t n, const int32_t *part, int32_t k) {
    if (n == 0) return JET_OK;
    if (!part) return JET_EINVAL;
    DevBuf b;
    JET_TRY(dev_alloc(b, 16, c.stream));
    JET_CUDA_TRY(cudaMemsetAsync(b.p, 0, 16, c.stream));
    k_check_part<<<grid_for(n, kTB, 8192), kTB, 0, c.stream>>>(n, part, k, b.as<int>());
    JET_CUDA_TRY(cudaGetLastError());
    JET_CUDA_TRY(cudaMemcpyAsync(c.pinned, b.p, 4, cudaMemcpyDeviceToHost, c.stream));
    JET_CUDA_TRY(cudaStreamSynchronize(c.stream));
    return (c.pinned[0] & 0xFFFFFFFF) ? JET_EINVAL : JET_OK;
}

bool bad_k_eps(int32_t k, double eps) { return k < 1 || k > JET_MAX_K || !(eps >= 0.0) || !std::isfinite(eps); }

int use_device(Ctx &c) {
    JET_CUDA_TRY(cudaSetDevice(c.device));
    t_pool = c.pool;
    return JET_OK;
}

// ---------------------------------------------------------------------------
// Alg. 1 after coarsening
// ---------------------------------------------------------------------------
struct EventTimer {
    cudaEvent_t e[6] = {};
    bool ok = true;
    EventTimer() {
        for (auto &x : e)
            if (cudaEventCreate(&x) != cudaSuccess) ok = false;
    }
    ~EventTimer() {
        for (auto &x : e)
            if (x) cudaEventDestroy(x);
    }
    float ms(int a, int b) {
        float t = 0.f;
        if (!ok || cudaEventElapsedTime(&t, e[a], e[b]) != cudaSuccess) { cudaGetLastError(); return 0.f; }
        return t;
    }
};

int uncoarsen(Ctx &c, const jet_hier *h, int32_t k, double eps, uint64_t seed, const int32_t *init_coarsest,
              int32_t *part_out, int64_t *cut_out, jet_stats *st, int32_t top, bool top_refined) {
    cudaStream_t s = c.stream;
    int32_t l = top >= 0 ? top : h->levels - 1;
    if (l >= h->levels || (top >= 0 && !init_coarsest)) return JET_EINVAL;
    int32_t nmax = 1;
    for (int32_t i = 1; i <= l; ++i) nmax = std::max(nmax, h->n[i]);
    DevBuf pa, pb;
    if (l > 0) {
        JET_TRY(dev_alloc(pa, (size_t)nmax * 4, s));
        JET_TRY(dev_alloc(pb, (size_t)nmax * 4, s));
    }
    int32_t *cur = l == 0 ? part_out : pa.as<int32_t>();
    int32_t *other = pb.as<int32_t>();
    EventTimer ev;
    cudaEventRecord(ev.e[0], s);
    auto level_graph = [&](int32_t i) {
        DGraph g;
        g.n = h->n[i]; g.nnz = h->nnz[i]; g.xadj = h->xadj[i]; g.adj = h->adj[i]; g.vw = h->vw[i]; g.ew = h->ew[i];
        return g;
    };
    if (init_coarsest) {
        JET_CUDA_TRY(cudaMemcpyAsync(cur, init_coarsest, (size_t)h->n[l] * 4, cudaMemcpyDeviceToDevice, s));
    } else {
        JET_TRY(initial_partition(c, level_graph(l), k, cur));
        c.launches += 1;
    }
    cudaEventRecord(ev.e[1], s);
    int status = JET_OK;
    int64_t cut = 0, maxw = 0;
    int64_t edge_iters = 0, fin_edge_iters = 0;
    // every level has the finest graph's total vertex weight (contraction sums them)
    int64_t W = 0;
    JET_TRY(total_vweight(c, level_graph(l), W));
    // level boundaries, read once after the loop (no synchronisation per level)
    std::vector<cudaEvent_t> lev;
    struct EvFree {
        std::vector<cudaEvent_t> &v;
        ~EvFree() {
            for (cudaEvent_t e : v)
                if (e) cudaEventDestroy(e);
        }
    } lev_free{lev};
    if (st) {
        lev.assign((size_t)h->levels + 1, nullptr);
        for (auto &e : lev)
            if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); e = nullptr; }
    }
    // every level is enqueued without a host wait (the host builds the next
    // level's loop while the device refines this one); the control blocks are
    // read after the finest level
    struct Runs {
        LevelRun r[JET_MAX_LEVELS];
        int32_t lo = JET_MAX_LEVELS, hi = -1;
        cudaStream_t s = nullptr;
        bool done = false;
        ~Runs() {
            if (done || hi < lo) return;
            cudaStreamSynchronize(s);
            for (int32_t i = lo; i <= hi; ++i) refine_level_abandon(r[i]);
        }
    } runs;
    runs.s = s;
    for (int32_t i = l; i >= 0; --i) {
        DGraph g = level_graph(i);
        if (st && lev[(size_t)i + 1]) cudaEventRecord(lev[(size_t)i + 1], s);
        if (i < l) {
            int32_t *dst = i == 0 ? part_out : other;
            JET_TRY(project(c, g.n, h->cmap[i], cur, dst));
            c.launches += 1;
            other = cur;
            cur = dst;
        }
        if (i == 0) cudaEventRecord(ev.e[2], s);
        if (i == l && top_refined) continue;   // the given partition is already refined there
        LevelRun &run = runs.r[i];
        run.slot = i;
        run.want_trace = i == 0;
        runs.lo = std::min(runs.lo, i);
        runs.hi = std::max(runs.hi, i);
        JET_TRY(refine_level_enqueue(c, g, k, eps, i == 0, level_seed(seed, i), cur, W, run));
    }
    if (st && lev[0]) cudaEventRecord(lev[0], s);
    cudaEventRecord(ev.e[3], s);
    JET_CUDA_TRY(cudaStreamSynchronize(s));
    runs.done = true;
    int first_err = JET_OK;
    for (int32_t i = l; i >= 0; --i) {
        if (i == l && top_refined) continue;
        LevelReport rep;
        int r = refine_level_finish(c, runs.r[i], &cut, &maxw, &rep);
        if (r < 0) {
            if (first_err == JET_OK) first_err = r;
            continue;
        }
        status = r;
        int64_t m = h->nnz[i] / 2;
        edge_iters += (int64_t)rep.iters * m;
        if (i == 0) fin_edge_iters = (int64_t)rep.iters * m;
        if (st) {
            st->iters_lp[i] = rep.kinds[0]; st->iters_rw[i] = rep.kinds[1]; st->iters_rs[i] = rep.kinds[2];
            st->cut_level[i] = cut;
            st->sel_launches[i] = rep.sel_launches;
            st->sel_bytes[i] = rep.sel_bytes;
            st->sel_ms[i] = rep.sel_ms;
            st->cluster_blocks[i] = rep.cluster;
            st->bytes_model += rep.bytes_model;
            for (int kk = 0; kk < JET_KERNELS; ++kk) {
                st->kern_launches[i][kk] = rep.kern_launches[kk];
                st->kern_bytes[i][kk] = rep.kern_bytes[kk];
                st->kern_ms[i][kk] = rep.kern_ms[kk];
            }
        }
    }
    if (first_err != JET_OK) return first_err;
    if (st) {
        // level i ran between the events recorded at i + 1 and at i
        for (int32_t i = l; i >= 0; --i) {
            float t = 0.f;
            if (lev[(size_t)i + 1] && lev[(size_t)i] &&
                cudaEventElapsedTime(&t, lev[(size_t)i + 1], lev[(size_t)i]) == cudaSuccess)
                st->ms_level[i] = t;
            else
                cudaGetLastError();
        }
    }
    if (cut_out) *cut_out = cut;
    if (st) {
        st->levels = h->levels;
        for (int32_t i = 0; i < h->levels; ++i) { st->n[i] = h->n[i]; st->m[i] = h->nnz[i] / 2; }
        st->edge_iters = edge_iters;
        st->fin_edge_iters = fin_edge_iters;
        st->ms_init = ev.ms(0, 1);
        st->ms_refine = ev.ms(1, 3);
        st->ms_refine_finest = ev.ms(2, 3);
        st->cut = cut;
        st->max_part_w = maxw;
    }
    return status;
}

}  // namespace jet

using namespace jet;

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

void jet_options_default(jet_options *o) {
    if (!o) return;
    o->c_fine = 0.25;
    o->c_coarse = 0.75;
    o->phi = 0.999;
    o->max_no_improve = 12;
    o->weak_limit = 2;
    o->coarsen_target = 0;
    o->max_levels = JET_MAX_LEVELS;
    o->max_iters_per_level = 10000;
    o->hem_rounds = 8;
    o->flags = 0;
    o->cluster_max_n = 4096;
    o->cluster_blocks = 0;
    o->barrier_polls = 0;
    o->list_blocks_per_sm = o->list_items_per_block = o->apply_blocks_per_sm = o->scan_blocks_per_sm = 0;
    o->hub_degree = 0;
}

int jet_ctx_create(int device, void *cuda_stream, const jet_options *opt, jet_ctx **out) {
    if (!out) return JET_EINVAL;
    *out = nullptr;
    jet_options o;
    jet_options_default(&o);
    if (opt) o = *opt;
    if (!(o.c_fine >= 0 && o.c_fine <= 1 && o.c_coarse >= 0 && o.c_coarse <= 1 && o.phi > 0 && o.phi <= 1) ||
        o.max_no_improve < 0 || o.weak_limit < 0 || o.coarsen_target < 0 || o.max_levels < 1 ||
        o.max_iters_per_level < 0 || o.hem_rounds < 0 || o.hem_rounds > 64 || o.cluster_max_n < 0 ||
        o.barrier_polls < 0 || o.list_blocks_per_sm < 0 || o.list_blocks_per_sm > 64 || o.list_items_per_block < 0 ||
        o.apply_blocks_per_sm < 0 || o.apply_blocks_per_sm > 64 || o.scan_blocks_per_sm < 0 ||
        o.scan_blocks_per_sm > 64 || (o.hub_degree != 0 && o.hub_degree < 32) ||
        !(o.cluster_blocks == 0 || o.cluster_blocks == 2 || o.cluster_blocks == 4 || o.cluster_blocks == 8 ||
          o.cluster_blocks == 16))
        return JET_EINVAL;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) { cudaGetLastError(); return JET_ECUDA; }
    if (device < 0 || device >= ndev) return JET_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess) { cudaGetLastError(); return JET_ECUDA; }
    jet_ctx *c = new (std::nothrow) jet_ctx;
    if (!c) return JET_ENOMEM;
    c->c.device = device;
    c->c.stream = static_cast<cudaStream_t>(cuda_stream);
    c->c.opt = o;
    if (cudaMallocHost(&c->c.pinned, kPinnedBytes) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return JET_ENOMEM;
    }
    // a private pool that keeps its memory across synchronisations, so that
    // repeated calls of the same size reuse it instead of mapping it again
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    if (cudaMemPoolCreate(&c->c.pool, &props) == cudaSuccess) {
        uint64_t keep = ~0ULL;
        cudaMemPoolSetAttribute(c->c.pool, cudaMemPoolAttrReleaseThreshold, &keep);
    } else {
        cudaGetLastError();
        c->c.pool = nullptr;
    }
    *out = c;
    return JET_OK;
}

void jet_ctx_destroy(jet_ctx *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->c.device);
    cudaStreamSynchronize(ctx->c.stream);
    if (ctx->c.pinned) cudaFreeHost(ctx->c.pinned);
    if (t_pool == ctx->c.pool) t_pool = nullptr;
    // memory still held by hierarchies of this context returns to the
    // system when they are destroyed
    if (ctx->c.pool) cudaMemPoolDestroy(ctx->c.pool);
    delete ctx;
}

int jet_coarsen(jet_ctx *ctx, int32_t n, const int64_t *xadj, const int32_t *adjncy, const int32_t *vwgt,
                const int32_t *adjwgt, int32_t k, uint64_t seed, jet_hier **out) {
    if (!ctx || !out || bad_k_eps(k, 0.0)) return JET_EINVAL;
    *out = nullptr;
    Ctx &c = ctx->c;
    JET_TRY(use_device(c));
    DGraph g;
    DevBuf ones;
    JET_TRY(prepare_graph(c, n, xadj, adjncy, vwgt, adjwgt, g, ones, false));
    jet_hier *h = new (std::nothrow) jet_hier;
    if (!h) return JET_ENOMEM;
    h->ctx = ctx;
    EventTimer ev;
    cudaEventRecord(ev.e[0], c.stream);
    int64_t l0 = c.launches;
    int r = coarsen(c, g, k, seed, h);
    h->launches = c.launches - l0;
    cudaEventRecord(ev.e[1], c.stream);
    if (r >= 0) {
        cudaError_t e = cudaStreamSynchronize(c.stream);
        if (e != cudaSuccess) { record_cuda_error(e, "sync", __FILE__, __LINE__); r = JET_ECUDA; }
    }
    if (r < 0) { delete h; return r; }
    h->ms_coarsen = ev.ms(0, 1);
    *out = h;
    return JET_OK;
}

void jet_hier_destroy(jet_hier *h) {
    if (!h) return;
    cudaSetDevice(h->ctx->c.device);
    h->bufs.clear();
    cudaStreamSynchronize(h->ctx->c.stream);
    delete h;
}

int jet_hier_info(const jet_hier *h, int32_t *levels, int64_t *n_per_level, int64_t *m_per_level) {
    if (!h) return JET_EINVAL;
    if (levels) *levels = h->levels;
    for (int32_t i = 0; i < h->levels; ++i) {
        if (n_per_level) n_per_level[i] = h->n[i];
        if (m_per_level) m_per_level[i] = h->nnz[i] / 2;
    }
    return JET_OK;
}

int jet_hier_level(const jet_hier *h, int32_t level, int32_t *n, const int64_t **xadj, const int32_t **adjncy,
                   const int32_t **vwgt, const int32_t **adjwgt, const int32_t **cmap) {
    if (!h || level < 0 || level >= h->levels) return JET_EINVAL;
    if (n) *n = h->n[level];
    if (xadj) *xadj = h->xadj[level];
    if (adjncy) *adjncy = h->adj[level];
    if (vwgt) *vwgt = h->vw[level];
    if (adjwgt) *adjwgt = h->ew[level];
    if (cmap) *cmap = level + 1 < h->levels ? h->cmap[level] : nullptr;
    return JET_OK;
}

int jet_uncoarsen(jet_ctx *ctx, const jet_hier *h, int32_t k, double eps, uint64_t seed, int32_t *part_out,
                  int64_t *cut_out, jet_stats *stats) {
    if (!ctx || !h || bad_k_eps(k, eps) || (h->n[0] > 0 && !part_out)) return JET_EINVAL;
    Ctx &c = ctx->c;
    JET_TRY(use_device(c));
    if (stats) {
        memset(stats, 0, sizeof(*stats));
        stats->ms_coarsen = h->ms_coarsen;
    }
    if (h->n[0] == 0) {
        if (cut_out) *cut_out = 0;
        return JET_OK;
    }
    int64_t l0 = c.launches;
    int r = uncoarsen(c, h, k, eps, seed, nullptr, part_out, cut_out, stats);
    if (stats) {
        stats->ms_total = stats->ms_coarsen + stats->ms_init + stats->ms_refine;
        stats->kernel_launches = h->launches + (c.launches - l0);
    }
    return r;
}

int jet_coarsest_refined(jet_ctx *ctx, const jet_hier *h, int32_t k, double eps, uint64_t seed, int32_t *part_out,
                         int64_t *cut_out) {
    if (!ctx || !h || bad_k_eps(k, eps)) return JET_EINVAL;
    const int32_t l = h->levels - 1;
    if (h->n[l] > 0 && !part_out) return JET_EINVAL;
    Ctx &c = ctx->c;
    JET_TRY(use_device(c));
    if (h->n[l] == 0) {
        if (cut_out) *cut_out = 0;
        return JET_OK;
    }
    DGraph g;
    g.n = h->n[l]; g.nnz = h->nnz[l]; g.xadj = h->xadj[l]; g.adj = h->adj[l]; g.vw = h->vw[l]; g.ew = h->ew[l];
    JET_TRY(initial_partition(c, g, k, part_out));
    int64_t cut = 0, maxw = 0;
    LevelReport rep;
    int r = refine_level(c, g, k, eps, l == 0, level_seed(seed, l), part_out, &cut, &maxw, &rep);
    if (r < 0) return r;
    JET_TRY(sync_stream(c));
    if (cut_out) *cut_out = cut;
    return r;
}

int jet_refine(jet_ctx *ctx, int32_t n, const int64_t *xadj, const int32_t *adjncy, const int32_t *vwgt,
               const int32_t *adjwgt, int32_t k, double eps, int32_t is_finest, uint64_t seed, int32_t *part_inout,
               int64_t *cut_out) {
    if (!ctx || bad_k_eps(k, eps)) return JET_EINVAL;
    Ctx &c = ctx->c;
    JET_TRY(use_device(c));
    DGraph g;
    DevBuf ones;
    JET_TRY(prepare_graph(c, n, xadj, adjncy, vwgt, adjwgt, g, ones, true));
    JET_TRY(check_part(c, n, part_inout, k));
    if (n == 0) {
        if (cut_out) *cut_out = 0;
        c.last_trace.rec.clear();
        c.last_trace.iters = 0;
        return JET_OK;
    }
    return refine_level(c, g, k, eps, is_finest ? 1 : 0, seed, part_inout, cut_out, nullptr, nullptr);
}

int jet_last_trace(jet_ctx *ctx, int32_t cap, int32_t *kind, int64_t *nx, int64_t *nm, int64_t *cut, int64_t *maxw,
                   int32_t *iters_out) {
    if (!ctx || cap < 0) return JET_EINVAL;
    const TraceHost &t = ctx->c.last_trace;
    int32_t m = std::min<int32_t>(cap, (int32_t)t.rec.size());
    for (int32_t i = 0; i < m; ++i) {
        const TraceRec &r = t.rec[(size_t)i];
        if (kind) kind[i] = r.kind;
        if (nx) nx[i] = r.nx;
        if (nm) nm[i] = r.nm;
        if (cut) cut[i] = r.cut;
        if (maxw) maxw[i] = r.maxw;
    }
    if (iters_out) *iters_out = t.iters;
    return JET_OK;
}

int jet_partition(jet_ctx *ctx, int32_t n, const int64_t *xadj, const int32_t *adjncy, const int32_t *vwgt,
                  const int32_t *adjwgt, int32_t k, double eps, uint64_t seed, int32_t *part_out, int64_t *cut_out,
                  jet_stats *stats) {
    if (!ctx || bad_k_eps(k, eps) || (n > 0 && !part_out)) return JET_EINVAL;
    jet_hier *h = nullptr;
    int r = jet_coarsen(ctx, n, xadj, adjncy, vwgt, adjwgt, k, seed, &h);
    if (r < 0) return r;
    r = jet_uncoarsen(ctx, h, k, eps, seed, part_out, cut_out, stats);
    jet_hier_destroy(h);
    return r;
}

// Batched form.  Three stages, each bit-identical to jet_partition per item:
//  1. the workers (host threads, each with its own context, stream and pool)
//     coarsen every graph and compute the greedy start of its coarsest level;
//  2. the small levels of all graphs — each graph's chain of levels of at
//     most cluster_max_n vertices, coarsest first — are refined in one
//     persistent cluster launch that takes graphs from a work queue
//     (refine_small_chains);
//  3. the workers refine every graph's larger levels (projection + the
//     CUDA-graph loop per level).
int jet_partition_batch(jet_ctx *ctx, int32_t count, jet_batch_item *items, int32_t workers) {
    if (!ctx || count < 0 || (count > 0 && !items)) return JET_EINVAL;
    if (count == 0) return JET_OK;
    Ctx &c = ctx->c;
    JET_TRY(use_device(c));
    if (workers <= 0) workers = 8;
    workers = std::min(workers, count);
    for (int32_t i = 0; i < count; ++i)
        if (bad_k_eps(items[i].k, items[i].eps) || items[i].n < 0 || (items[i].n > 0 && !items[i].part_out))
            return JET_EINVAL;
    // the workers' streams start after the work already on the caller's stream
    cudaEvent_t start = nullptr;
    JET_CUDA_TRY(cudaEventCreateWithFlags(&start, cudaEventDisableTiming));
    struct EventFree {
        cudaEvent_t e;
        ~EventFree() { cudaEventDestroy(e); }
    } start_free{start};
    JET_CUDA_TRY(cudaEventRecord(start, c.stream));
    struct Worker {
        cudaStream_t s = nullptr;
        jet_ctx *wc = nullptr;
        ~Worker() {
            if (wc) jet_ctx_destroy(wc);
            if (s) cudaStreamDestroy(s);
        }
    };
    std::vector<Worker> wk((size_t)workers);
    jet_options wo = c.opt;
    if (workers > 1) wo.flags &= ~JET_FLAG_GRID_LOOP;   // concurrent workers: no cooperative launches
    for (auto &w : wk) {
        JET_CUDA_TRY(cudaStreamCreateWithFlags(&w.s, cudaStreamNonBlocking));
        JET_CUDA_TRY(cudaStreamWaitEvent(w.s, start, 0));
        JET_TRY(jet_ctx_create(c.device, w.s, &wo, &w.wc));
    }
    JET_TRY(use_device(c));
    struct Item {
        jet_hier *h = nullptr;
        DevBuf init;                 // greedy start of the coarsest level (worker's pool)
        int64_t W = 0;
        int32_t bottom = -1;         // finest level of the small chain (-1: none)
        int32_t chain = -1;
        bool done = false;
        double ms = 0;
        ~Item() {
            if (h) jet_hier_destroy(h);
        }
    };
    std::vector<Item> st((size_t)count);
    std::vector<int> wstat((size_t)workers, JET_OK);
    // runs fn(worker context, item) over all items on the workers
    auto run_workers = [&](auto &&fn) {
        std::atomic<int32_t> next{0};
        auto body = [&](int w) {
            jet_ctx *wc = wk[(size_t)w].wc;
            for (;;) {
                int32_t i = next.fetch_add(1);
                if (i >= count) break;
                if (st[(size_t)i].done) continue;
                auto t0 = std::chrono::steady_clock::now();
                fn(wc, i);
                st[(size_t)i].ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
            }
            if (cudaStreamSynchronize(wk[(size_t)w].s) != cudaSuccess) {
                cudaGetLastError();
                wstat[(size_t)w] = JET_ECUDA;
            }
        };
        std::vector<std::thread> pool;
        int started = 0;
        try {
            pool.reserve((size_t)workers);
            for (int w = 0; w < workers; ++w) {
                pool.emplace_back(body, w);
                ++started;
            }
        } catch (...) {   // no exception crosses the C ABI: the workers that started take every item
            if (started == 0) body(0);   // none did: the calling thread takes the whole batch
        }
        for (auto &t : pool) t.join();
    };
    const int32_t thr = c.opt.cluster_max_n;
    // stage 1: coarsening and the greedy start of the coarsest level
    run_workers([&](jet_ctx *wc, int32_t i) {
        jet_batch_item &it = items[i];
        Item &s1 = st[(size_t)i];
        it.cut = 0;
        it.status = JET_OK;
        if (it.n == 0) {
            s1.done = true;
            return;
        }
        int r = jet_coarsen(wc, it.n, it.xadj, it.adjncy, it.vwgt, it.adjwgt, it.k, it.seed, &s1.h);
        if (r < 0) { it.status = r; s1.done = true; return; }
        Ctx &w = wc->c;
        const jet_hier *h = s1.h;
        const int32_t l = h->levels - 1;
        DGraph gl;
        gl.n = h->n[l]; gl.nnz = h->nnz[l]; gl.xadj = h->xadj[l]; gl.adj = h->adj[l]; gl.vw = h->vw[l]; gl.ew = h->ew[l];
        r = use_device(w);
        if (r >= 0) r = dev_alloc(s1.init, (size_t)std::max<int32_t>(gl.n, 1) * 4, w.stream);
        if (r >= 0) r = initial_partition(w, gl, it.k, s1.init.as<int32_t>());
        if (r >= 0) r = total_vweight(w, gl, s1.W);
        if (r < 0) { it.status = r; s1.done = true; return; }
        if (thr > 0 && h->n[l] <= thr) {
            int32_t b = l;
            while (b > 0 && h->n[b - 1] <= thr) --b;
            s1.bottom = b;
        }
    });
    for (int w = 0; w < workers; ++w)
        if (wstat[(size_t)w] != JET_OK) return wstat[(size_t)w];
    // stage 2: every graph's small levels in one persistent launch
    std::vector<SmallChain> chains;
    std::vector<DevBuf> chain_out;
    for (int32_t i = 0; i < count; ++i) {
        Item &s1 = st[(size_t)i];
        if (s1.done || s1.bottom < 0) continue;
        const jet_batch_item &it = items[i];
        SmallChain ch;
        ch.h = s1.h;
        ch.top = s1.h->levels - 1;
        ch.bottom = s1.bottom;
        ch.k = it.k;
        ch.eps = it.eps;
        ch.seed = it.seed;
        ch.W = s1.W;
        ch.init = s1.init.as<int32_t>();
        if (s1.bottom == 0) {
            ch.out = it.part_out;
        } else {
            chain_out.emplace_back();
            JET_TRY(dev_alloc(chain_out.back(), (size_t)s1.h->n[s1.bottom] * 4, c.stream));
            ch.out = chain_out.back().as<int32_t>();
        }
        s1.chain = (int32_t)chains.size();
        chains.push_back(ch);
    }
    int ran = 0;
    JET_TRY(refine_small_chains(c, chains.data(), (int32_t)chains.size(), c.opt.cluster_blocks, &ran));
    // stage 3: the larger levels
    run_workers([&](jet_ctx *wc, int32_t i) {
        jet_batch_item &it = items[i];
        Item &s1 = st[(size_t)i];
        const SmallChain *ch = (ran && s1.chain >= 0) ? &chains[(size_t)s1.chain] : nullptr;
        int r;
        if (ch && ch->bottom == 0) {
            it.cut = ch->cut;
            r = ch->status;
        } else if (ch) {
            r = use_device(wc->c);
            if (r >= 0) r = uncoarsen(wc->c, s1.h, it.k, it.eps, it.seed, ch->out, it.part_out, &it.cut, nullptr,
                                      ch->bottom, true);
        } else {
            r = use_device(wc->c);
            if (r >= 0) r = uncoarsen(wc->c, s1.h, it.k, it.eps, it.seed, s1.init.as<int32_t>(), it.part_out, &it.cut,
                                      nullptr);
        }
        it.status = r;
    });
    for (int32_t i = 0; i < count; ++i) items[i].ms = (float)st[(size_t)i].ms;
    for (int w = 0; w < workers; ++w)
        if (wstat[(size_t)w] != JET_OK) return wstat[(size_t)w];
    for (int32_t i = 0; i < count; ++i)
        if (items[i].status < 0) return items[i].status;
    return JET_OK;
}

int jet_autotune(jet_ctx *ctx, int32_t count, jet_batch_item *items, int32_t reps, jet_tune_report *report) {
    if (!ctx || count <= 0 || !items) return JET_EINVAL;
    if (reps <= 0) reps = 3;
    Ctx &c = ctx->c;
    JET_TRY(use_device(c));
    jet_tune_report rep;
    memset(&rep, 0, sizeof(rep));
    // median wall time of `reps` runs of the batch after one untimed run
    auto time_batch = [&](int32_t workers, float *ms) -> int {
        std::vector<float> t;
        for (int r = 0; r <= reps; ++r) {
            auto t0 = std::chrono::steady_clock::now();
            int st = jet_partition_batch(ctx, count, items, workers);
            if (st < 0) return st;
            float dt = std::chrono::duration<float, std::milli>(std::chrono::steady_clock::now() - t0).count();
            if (r > 0) t.push_back(dt);
        }
        std::sort(t.begin(), t.end());
        *ms = t[t.size() / 2];
        return JET_OK;
    };
    int32_t workers = count > 1 ? 8 : 1;
    // One stage: each value of one choice (*target) timed with the others
    // fixed; the fastest stays.
    auto stage = [&](int32_t id, const int32_t *vals, int nv, int32_t *target) -> int {
        int32_t best_v = *target;
        float best = 0.f;
        for (int i = 0; i < nv; ++i) {
            *target = vals[i];
            float ms = 0.f;
            JET_TRY(time_batch(workers, &ms));
            if (rep.ncand < JET_TUNE_MAX_CAND) {
                rep.cand_stage[rep.ncand] = id;
                rep.cand_value[rep.ncand] = vals[i];
                rep.cand_ms[rep.ncand] = ms;
                rep.ncand += 1;
            }
            if (i == 0 || ms < best) { best = ms; best_v = vals[i]; }
        }
        *target = best_v;
        return JET_OK;
    };
    static const int32_t blocks[] = {16, 8, 4, 2};
    static const int32_t thresholds[] = {0, 1024, 2048, 4096, 8192, 16384};
    static const int32_t wcands[] = {1, 2, 4, 8, 16};
    static const int32_t list_bpsm[] = {2, 4, 8};
    static const int32_t apply_bpsm[] = {1, 2, 4};
    static const int32_t items_pb[] = {32, 64, 128};
    static const int32_t scan_bpsm[] = {4, 8, 16};
    static const int32_t hubs[] = {256, 1024, 4096};
    const jet_options saved = c.opt;
    jet_options &o = c.opt;
    o.cluster_max_n = 4096;
    o.list_blocks_per_sm = 4;
    o.apply_blocks_per_sm = 4;
    o.list_items_per_block = 64;
    o.scan_blocks_per_sm = 8;
    o.hub_degree = 1024;
    int st = stage(JET_TUNE_CLUSTER_BLOCKS, blocks, 4, &o.cluster_blocks);
    if (st >= 0) st = stage(JET_TUNE_CLUSTER_MAX_N, thresholds, 6, &o.cluster_max_n);
    if (st >= 0 && count > 1) st = stage(JET_TUNE_WORKERS, wcands, 5, &workers);
    if (st >= 0) st = stage(JET_TUNE_LIST_BLOCKS, list_bpsm, 3, &o.list_blocks_per_sm);
    if (st >= 0) st = stage(JET_TUNE_APPLY_BLOCKS, apply_bpsm, 3, &o.apply_blocks_per_sm);
    if (st >= 0) st = stage(JET_TUNE_LIST_ITEMS, items_pb, 3, &o.list_items_per_block);
    if (st >= 0) st = stage(JET_TUNE_SCAN_BLOCKS, scan_bpsm, 3, &o.scan_blocks_per_sm);
    if (st >= 0) st = stage(JET_TUNE_HUB_DEGREE, hubs, 3, &o.hub_degree);
    if (st < 0) {
        c.opt = saved;
        return st;
    }
    rep.cluster_max_n = o.cluster_max_n;
    rep.cluster_blocks = o.cluster_blocks;
    rep.workers = workers;
    rep.list_blocks_per_sm = o.list_blocks_per_sm;
    rep.apply_blocks_per_sm = o.apply_blocks_per_sm;
    rep.list_items_per_block = o.list_items_per_block;
    rep.scan_blocks_per_sm = o.scan_blocks_per_sm;
    rep.hub_degree = o.hub_degree;
    if (report) *report = rep;
    return JET_OK;
}

int jet_partition_host(jet_ctx *ctx, int32_t n, const int64_t *xadj, const int32_t *adjncy, const int32_t *vwgt,
                       const int32_t *adjwgt, int32_t k, double eps, uint64_t seed, int32_t *part_out, int64_t *cut_out,
                       jet_stats *stats) {
    if (!ctx || n < 0 || !xadj || bad_k_eps(k, eps) || (n > 0 && !part_out)) return JET_EINVAL;
    Ctx &c = ctx->c;
    JET_TRY(use_device(c));
    cudaStream_t s = c.stream;
    int64_t nnz = xadj[n];
    if (nnz < 0 || (nnz > 0 && !adjncy)) return JET_EINVAL;
    DevBuf dx, da, dv, dw, dp;
    JET_TRY(dev_alloc(dx, (size_t)(n + 1) * 8, s));
    JET_TRY(dev_alloc(da, (size_t)std::max<int64_t>(nnz, 1) * 4, s));
    JET_TRY(dev_alloc(dp, (size_t)std::max(n, 1) * 4, s));
    JET_CUDA_TRY(cudaMemcpyAsync(dx.p, xadj, (size_t)(n + 1) * 8, cudaMemcpyHostToDevice, s));
    if (nnz > 0) JET_CUDA_TRY(cudaMemcpyAsync(da.p, adjncy, (size_t)nnz * 4, cudaMemcpyHostToDevice, s));
    if (vwgt) {
        JET_TRY(dev_alloc(dv, (size_t)std::max(n, 1) * 4, s));
        JET_CUDA_TRY(cudaMemcpyAsync(dv.p, vwgt, (size_t)n * 4, cudaMemcpyHostToDevice, s));
    }
    if (adjwgt) {
        JET_TRY(dev_alloc(dw, (size_t)std::max<int64_t>(nnz, 1) * 4, s));
        if (nnz > 0) JET_CUDA_TRY(cudaMemcpyAsync(dw.p, adjwgt, (size_t)nnz * 4, cudaMemcpyHostToDevice, s));
    }
    int r = jet_partition(ctx, n, dx.as<int64_t>(), da.as<int32_t>(), vwgt ? dv.as<int32_t>() : nullptr,
                          adjwgt ? dw.as<int32_t>() : nullptr, k, eps, seed, dp.as<int32_t>(), cut_out, stats);
    if (r < 0) return r;
    if (n > 0) JET_CUDA_TRY(cudaMemcpyAsync(part_out, dp.p, (size_t)n * 4, cudaMemcpyDeviceToHost, s));
    JET_CUDA_TRY(cudaStreamSynchronize(s));
    return r;
}

int jet_cut(jet_ctx *ctx, int32_t n, const int64_t *xadj, const int32_t *adjncy, const int32_t *vwgt,
            const int32_t *adjwgt, int32_t k, const int32_t *part, int64_t *cut_out, int64_t *pw_out) {
    if (!ctx || bad_k_eps(k, 0.0)) return JET_EINVAL;
    Ctx &c = ctx->c;
    JET_TRY(use_device(c));
    DGraph g;
    DevBuf ones;
    JET_TRY(prepare_graph(c, n, xadj, adjncy, vwgt, adjwgt, g, ones, true));
    JET_TRY(check_part(c, n, part, k));
    return cut_and_weights(c, g, k, part, cut_out, pw_out);
}

int jet_lp_pass(jet_ctx *ctx, int32_t n, const int64_t *xadj, const int32_t *adjncy, const int32_t *vwgt,
                const int32_t *adjwgt, int32_t k, const int32_t *part, const uint8_t *locked, double cval,
                uint32_t flags, int32_t *pd_out, int32_t *gain_out, uint8_t *inx_out, int32_t *f2_out,
                uint8_t *inm_out) {
    if (!ctx || bad_k_eps(k, 0.0) || !(cval >= 0 && cval <= 1)) return JET_EINVAL;
    Ctx &c = ctx->c;
    JET_TRY(use_device(c));
    DGraph g;
    DevBuf ones;
    JET_TRY(prepare_graph(c, n, xadj, adjncy, vwgt, adjwgt, g, ones, true));
    JET_TRY(check_part(c, n, part, k));
    return lp_pass(c, g, k, part, locked, cval, flags, pd_out, gain_out, inx_out, f2_out, inm_out);
}

int jet_rebalance_pass(jet_ctx *ctx, int32_t n, const int64_t *xadj, const int32_t *adjncy, const int32_t *vwgt,
                       const int32_t *adjwgt, int32_t k, double eps, int32_t strong, uint64_t seed, int32_t iter,
                       const int32_t *part, int32_t *dest_out, int32_t *loss_out, int64_t *nmoves_out,
                       int64_t *ncand_out) {
    if (!ctx || bad_k_eps(k, eps) || iter < 0) return JET_EINVAL;
    Ctx &c = ctx->c;
    JET_TRY(use_device(c));
    DGraph g;
    DevBuf ones;
    JET_TRY(prepare_graph(c, n, xadj, adjncy, vwgt, adjwgt, g, ones, true));
    JET_TRY(check_part(c, n, part, k));
    return rebalance_pass(c, g, k, eps, strong, seed, iter, part, dest_out, loss_out, nmoves_out, ncand_out);
}

int jet_hem(jet_ctx *ctx, int32_t n, const int64_t *xadj, const int32_t *adjncy, const int32_t *adjwgt, uint64_t seed,
            int32_t level, int32_t rounds, int32_t *mate_out) {
    if (!ctx || rounds < 0 || rounds > 64 || level < 0 || (n > 0 && !mate_out)) return JET_EINVAL;
    Ctx &c = ctx->c;
    JET_TRY(use_device(c));
    DGraph g;
    DevBuf ones;
    JET_TRY(prepare_graph(c, n, xadj, adjncy, nullptr, adjwgt, g, ones, true));
    JET_TRY(hem(c, g, seed, level, rounds, mate_out));
    return sync_stream(c);
}

int jet_two_hop(jet_ctx *ctx, int32_t n, const int64_t *xadj, const int32_t *adjncy, int32_t *mate_inout,
                int64_t *added_out) {
    if (!ctx || (n > 0 && !mate_inout)) return JET_EINVAL;
    Ctx &c = ctx->c;
    JET_TRY(use_device(c));
    DGraph g;
    DevBuf ones;
    JET_TRY(prepare_graph(c, n, xadj, adjncy, nullptr, nullptr, g, ones, false));
    int64_t added[3] = {0, 0, 0};
    JET_TRY(two_hop(c, g, mate_inout, added));
    if (added_out) memcpy(added_out, added, sizeof(added));
    return JET_OK;
}

int jet_initial_partition(jet_ctx *ctx, int32_t n, const int64_t *xadj, const int32_t *adjncy, const int32_t *vwgt,
                          int32_t k, int32_t *part_out) {
    if (!ctx || bad_k_eps(k, 0.0) || (n > 0 && !part_out)) return JET_EINVAL;
    Ctx &c = ctx->c;
    JET_TRY(use_device(c));
    DGraph g;
    DevBuf ones;
    JET_TRY(prepare_graph(c, n, xadj, adjncy, vwgt, nullptr, g, ones, true));
    return initial_partition(c, g, k, part_out);
}

int64_t jet_alloc_count(void) { return g_alloc_count.load(std::memory_order_relaxed); }

void jet_debug_fail_alloc(int64_t nth) {
    g_fail_at.store(nth > 0 ? g_alloc_count.load(std::memory_order_relaxed) + nth : 0, std::memory_order_relaxed);
}

const char *jet_kernel_name(int32_t i) {
    static const char *const names[JET_K_COUNT] = {"k_lp_scan", "k_lp_select", "k_afterburn", "k_apply",
                                                   "k_rb_scan", "k_rb_cand", "k_rb_tilehist", "k_rb_tilescan",
                                                   "k_rb_take", "k_rb_cookie"};
    return (i >= 0 && i < JET_K_COUNT) ? names[i] : nullptr;
}

const char *jet_status_string(int s) {
    switch (s) {
    case JET_OK: return "ok";
    case JET_WUNBALANCED: return "warning: result violates the balance limit";
    case JET_WITERLIMIT: return "warning: a level hit max_iters_per_level";
    case JET_EINVAL: return "invalid argument";
    case JET_EGRAPH: return "invalid graph";
    case JET_ENOMEM: return "device allocation failed";
    case JET_ECUDA: return "CUDA error";
    case JET_ETIMEOUT: return "device wait timed out";
    case JET_EOVERFLOW: return "weight sums exceed 2^31";
    default: return "unknown status";
    }
}

/* Text of the last CUDA error recorded on this thread (diagnostics). */
const char *jet_last_error(void) { return last_error_text(); }

}  // extern "C"
