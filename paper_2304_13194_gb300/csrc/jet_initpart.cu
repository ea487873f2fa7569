// Greedy initial partition of the coarsest graph (Alg. 1 InitialPartition;
// the paper calls Metis there, Sec. 3 — this build grows parts greedily).
//
// Order the vertices by (lowest vertex id of their connected component, hop
// distance from that vertex, vertex id) and cut the sequence into k pieces by
// weight: P(v) = floor(k S(v) / W), S(v) the weight of the vertices before v.
//
// Device-wide, for any graph size (a stalled coarsening can leave millions of
// vertices here):
//  1. components by union-find, the larger root always hooked under the
//     smaller, so every tree ends at its component's lowest id whatever the
//     order of the hooks.  The hooks are sampled first (each vertex's first
//     two row entries), the root that most of an evenly spaced sample of
//     vertices reaches is taken as the large component's, and then only the
//     rows of vertices outside it are hooked in full (every edge with an
//     end outside that component is met from that end; an edge between two
//     vertices inside it joins nothing new).  Double-buffered pointer
//     jumping (a fixed number of rounds, each reading one array and writing
//     the other) then gives every vertex its root exactly — path
//     compression done in place would let a late halving store overwrite a
//     finished root with an ancestor;
//  2. breadth-first levels from all those roots at once, one frontier per
//     level (each kernel launch takes one level and exits at once when the
//     frontier is empty, so the host enqueues levels in batches); a level
//     whose frontier carries many row entries is taken bottom-up (the
//     vertices not reached yet look for a parent), the others top-down;
//  3. a stable LSD radix sort of the vertices (in id order) by the key
//     (root, distance): the id order inside a key is kept;
//  4. an exclusive scan of the weights in that order, then P.
#include "jet_internal.cuh"

#include <algorithm>

namespace jet {

namespace {

constexpr int32_t kInf = INT32_MAX;
constexpr int kBfsBatch = 16;                     // levels enqueued between host checks
constexpr int kFindCap = 1 << 26;                 // bound of every union-find loop

struct IpCtl {
    int32_t size[2];     // frontier lengths, by level parity
    int32_t level;       // level the next k_bfs_level launch expands
    int32_t ticket;      // blocks of the current launch that finished
    int32_t error;       // a union-find loop hit kFindCap
    int32_t major;       // root reached by most of the sampled vertices after the sampled hooks
    int64_t total;       // scan total (W)
    int64_t mf[2];       // row entries of the frontier, by level parity
    int64_t mv;          // row entries of the vertices reached so far
};

// Root of x with path halving.  parent[] only ever decreases (parent[x] <= x),
// so the walk is strictly decreasing and ends; the cap is a safety net.
__device__ __forceinline__ int32_t uf_find(int32_t *parent, int32_t x, int32_t *err) {
    for (int i = 0; i < kFindCap; ++i) {
        int32_t p = parent[x];
        if (p == x) return x;
        int32_t gp = parent[p];
        if (gp != p) parent[x] = gp;
        x = gp;
    }
    *err = 1;
    return x;
}

__global__ void k_uf_init(int32_t n, int32_t *parent) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        parent[v] = (int32_t)v;
}

// The edge {u, v}, u < v, hooks the two roots, the larger under the smaller
// (a failed CAS means another hook lowered the root; retry from the new one).
__device__ __forceinline__ void uf_hook_edge(int32_t *parent, int32_t u, int32_t v, int32_t *err) {
    int32_t ru = uf_find(parent, u, err), rv = uf_find(parent, v, err);
    for (int i = 0; i < kFindCap && ru != rv; ++i) {
        int32_t hi = ru > rv ? ru : rv, lo = ru > rv ? rv : ru;
        int32_t old = atomicCAS(&parent[hi], hi, lo);
        if (old == hi) break;
        ru = uf_find(parent, old, err);
        rv = uf_find(parent, lo, err);
        if (i + 1 == kFindCap) *err = 1;
    }
}

// Sampled hooks: every vertex hooks the edges of its first kSampleHooks row
// entries.
constexpr int kSampleHooks = 2;
__global__ void k_uf_hook_sample(DGraph g, int32_t *parent, IpCtl *ctl) {
    int32_t err = 0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < g.n; v += (int64_t)gridDim.x * blockDim.x) {
        const int64_t beg = ld_xadj(g.xadj, v), end = ld_xadj(g.xadj, v + 1);
        for (int64_t j = beg; j < end && j < beg + kSampleHooks; ++j) {
            const int32_t u = __ldg(g.adj + j);
            if (u != v) uf_hook_edge(parent, u, (int32_t)v, &err);
        }
    }
    if (err) ctl->error = 1;
}

// The root most of kMajorSample evenly spaced vertices reach (ties: the
// smaller root); one block of kMajorSample threads.  Only a work saving: a
// poor pick costs hooks, not correctness.
constexpr int kMajorSample = 256;
__global__ void __launch_bounds__(kMajorSample) k_uf_major(int32_t n, int32_t *parent, IpCtl *ctl) {
    __shared__ int32_t r[kMajorSample];
    __shared__ unsigned long long best;
    int32_t err = 0;
    const int32_t v = (int32_t)(((int64_t)threadIdx.x * n) / kMajorSample);
    r[threadIdx.x] = uf_find(parent, v, &err);
    if (threadIdx.x == 0) best = 0;
    __syncthreads();
    int32_t cnt = 0;
    for (int i = 0; i < kMajorSample; ++i) cnt += r[i] == r[threadIdx.x];
    // larger count first, then the smaller root
    atomicMax(&best, ((unsigned long long)cnt << 32) | (unsigned long long)(uint32_t)(INT32_MAX - r[threadIdx.x]));
    __syncthreads();
    if (threadIdx.x == 0) ctl->major = INT32_MAX - (int32_t)(uint32_t)(best & 0xffffffffull);
    if (err) ctl->error = 1;
}

// One warp per vertex v outside the major component hooks every edge of its
// row; rows longer than kHugeDeg are set aside (up to kHugeCap per block)
// and taken by the whole block at the end.
__global__ void __launch_bounds__(kTB) k_uf_hook_rest(DGraph g, int32_t *parent, IpCtl *ctl) {
    __shared__ int32_t huge[kHugeCap];
    __shared__ int nhuge;
    if (threadIdx.x == 0) nhuge = 0;
    __syncthreads();
    const int32_t major = ctl->major;
    const int warps = blockDim.x >> 5;
    const unsigned lane = lane_id();
    int32_t err = 0;
    for (int64_t v = (int64_t)blockIdx.x * warps + (threadIdx.x >> 5); v < g.n; v += (int64_t)gridDim.x * warps) {
        const int64_t beg = ld_xadj(g.xadj, v), end = ld_xadj(g.xadj, v + 1);
        if (end == beg) continue;
        int32_t rv = 0;
        if (lane == 0) rv = uf_find(parent, (int32_t)v, &err);
        rv = __shfl_sync(0xffffffffu, rv, 0);
        if (rv == major) continue;
        if (end - beg > kHugeDeg) {
            int slot = 0;
            if (lane == 0) slot = atomicAdd(&nhuge, 1);
            slot = __shfl_sync(0xffffffffu, slot, 0);
            if (slot < kHugeCap) {
                if (lane == 0) huge[slot] = (int32_t)v;
                continue;
            }
        }
        for (int64_t j = beg + lane; j < end; j += 32) {
            const int32_t u = __ldg(g.adj + j);
            if (u != v) uf_hook_edge(parent, u, (int32_t)v, &err);
        }
    }
    __syncthreads();
    const int nh = nhuge < kHugeCap ? nhuge : kHugeCap;
    for (int s = 0; s < nh; ++s) {
        const int32_t v = huge[s];
        const int64_t beg = ld_xadj(g.xadj, v), end = ld_xadj(g.xadj, (int64_t)v + 1);
        for (int64_t j = beg + threadIdx.x; j < end; j += blockDim.x) {
            const int32_t u = __ldg(g.adj + j);
            if (u != v) uf_hook_edge(parent, u, v, &err);
        }
    }
    if (err) ctl->error = 1;
}

// One round of pointer jumping: out[v] = in[in[v]] (ancestors only, so after
// ceil(log2 n) rounds every entry is its tree's root).
__global__ void k_uf_jump(int32_t n, const int32_t *in, int32_t *out) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        out[v] = in[in[v]];
}

// Distance 0 at the roots, which form the first frontier (and their row
// entries the first frontier's).
__global__ void __launch_bounds__(kTB) k_uf_finish(DGraph g, const int32_t *root, int32_t *dist, int32_t *front0,
                                                   IpCtl *ctl) {
    __shared__ long long red[40];
    const int32_t n = g.n;
    long long mf = 0;
    for (int64_t v0 = (int64_t)blockIdx.x * blockDim.x; v0 < n; v0 += (int64_t)gridDim.x * blockDim.x) {
        int64_t v = v0 + threadIdx.x;
        bool is_root = false;
        if (v < n) {
            is_root = root[v] == v;
            dist[v] = is_root ? 0 : kInf;
            if (is_root) mf += ld_xadj(g.xadj, v + 1) - ld_xadj(g.xadj, v);
        }
        int slot = warp_append(&ctl->size[0], is_root);
        if (is_root) front0[slot] = (int32_t)v;
    }
    mf = block_sum_i64(mf, red);
    if (threadIdx.x == 0 && mf) {
        atomic_add_i64(&ctl->mf[0], mf);
        atomic_add_i64(&ctl->mv, mf);
    }
}

// Bottom-up steps (Beamer's direction switch) are taken while the
// frontier's row entries exceed 1/kBottomUpAlpha of those of the vertices
// not reached yet.  4 rather than Beamer's 14: on a mesh the vertices not
// reached yet mostly have no parent in the frontier and would read their
// whole rows, so only a frontier whose rows rival theirs switches.
constexpr int64_t kBottomUpAlpha = 4;

// Whether the warp's row chunk holds a vertex of level l (whole warp).
__device__ __forceinline__ bool bfs_parent_in_chunk(const DGraph &g, const int32_t *dist, int64_t j, int64_t end,
                                                    int32_t l) {
    const int32_t w = j < end ? __ldg(g.adj + j) : -1;
    return __any_sync(0xffffffffu, w >= 0 && dist[w] == l);
}

// One breadth-first level l -> l + 1 (frontier of parity l & 1).  Distances
// are exact whichever way a level is taken:
//  * top-down: one warp per frontier vertex; a neighbour is claimed for
//    level l + 1 by a CAS on its distance;
//  * bottom-up: every vertex not reached yet looks for a neighbour at level
//    l (rows of up to 32 entries one thread each, 8 entries in flight,
//    longer rows one warp each, rows longer than kHugeDeg the whole block;
//    each stops at the first one found) and writes its own distance.
// The new frontier is appended either way; the row entries of its vertices
// are counted for the next level's choice.  The last block to finish closes
// the level.
__global__ void __launch_bounds__(kTB) k_bfs_level(DGraph g, int32_t *dist, int32_t *front0, int32_t *front1,
                                                   IpCtl *ctl) {
    const int32_t l = ctl->level;
    const int32_t cur = ctl->size[l & 1];
    if (cur == 0) return;                        // search finished: every block leaves
    const int32_t *in = (l & 1) ? front1 : front0;
    int32_t *out = (l & 1) ? front0 : front1;
    int32_t *out_size = &ctl->size[(l + 1) & 1];
    const bool bottom_up = ctl->mf[l & 1] * kBottomUpAlpha > g.nnz - ctl->mv;
    const int warps = blockDim.x >> 5;
    const unsigned lane = lane_id();
    __shared__ int32_t huge[kHugeCap];
    __shared__ int nhuge;
    __shared__ long long red[40];
    long long mf_next = 0;
    if (threadIdx.x == 0) nhuge = 0;
    __syncthreads();
    if (!bottom_up) {
        for (int64_t w0 = (int64_t)blockIdx.x * warps; w0 < cur; w0 += (int64_t)gridDim.x * warps) {
            int64_t w = w0 + (threadIdx.x >> 5);
            int64_t beg = 0, end = 0;
            int32_t v = -1;
            if (w < cur) {
                v = in[w];
                beg = ld_xadj(g.xadj, v);
                end = ld_xadj(g.xadj, (int64_t)v + 1);
            }
            if (end - beg > kHugeDeg) {              // hub row: the whole block, below
                int slot = 0;
                if (lane == 0) slot = atomicAdd(&nhuge, 1);
                slot = __shfl_sync(0xffffffffu, slot, 0);
                if (slot < kHugeCap) {
                    if (lane == 0) huge[slot] = v;
                    end = beg;
                }
            }
            for (int64_t j0 = beg; j0 < end; j0 += 32) {   // whole warp: same row
                int64_t j = j0 + lane;
                bool claim = false;
                int32_t u = -1;
                if (j < end) {
                    u = __ldg(g.adj + j);
                    claim = dist[u] == kInf && atomicCAS(&dist[u], kInf, l + 1) == kInf;
                }
                int slot = warp_append(out_size, claim);
                if (claim) {
                    out[slot] = u;
                    mf_next += ld_xadj(g.xadj, (int64_t)u + 1) - ld_xadj(g.xadj, u);
                }
            }
        }
        __syncthreads();
        const int nh = nhuge < kHugeCap ? nhuge : kHugeCap;
        for (int s = 0; s < nh; ++s) {
            const int32_t v = huge[s];
            const int64_t beg = ld_xadj(g.xadj, v), end = ld_xadj(g.xadj, (int64_t)v + 1);
            for (int64_t j0 = beg + (int64_t)(threadIdx.x >> 5) * 32; j0 < end; j0 += blockDim.x) {
                int64_t j = j0 + lane;
                bool claim = false;
                int32_t u = -1;
                if (j < end) {
                    u = __ldg(g.adj + j);
                    claim = dist[u] == kInf && atomicCAS(&dist[u], kInf, l + 1) == kInf;
                }
                int slot = warp_append(out_size, claim);
                if (claim) {
                    out[slot] = u;
                    mf_next += ld_xadj(g.xadj, (int64_t)u + 1) - ld_xadj(g.xadj, u);
                }
            }
        }
    } else {
        __shared__ int32_t stage[kTB];
        __shared__ int nstage;
        for (int64_t v0 = (int64_t)blockIdx.x * blockDim.x; v0 < g.n; v0 += (int64_t)gridDim.x * blockDim.x) {
            if (threadIdx.x == 0) nstage = 0;
            __syncthreads();
            const int64_t v = v0 + threadIdx.x;
            bool found = false;
            int64_t beg = 0, end = 0;
            if (v < g.n && dist[v] == kInf) {
                beg = ld_xadj(g.xadj, v);
                end = ld_xadj(g.xadj, v + 1);
                if (end - beg > 32) {
                    bool staged = false;
                    if (end - beg > kHugeDeg) {
                        const int slot = atomicAdd(&nhuge, 1);
                        if (slot < kHugeCap) {
                            huge[slot] = (int32_t)v;
                            staged = true;
                        }
                    }
                    if (!staged) stage[atomicAdd(&nstage, 1)] = (int32_t)v;
                } else {
                    for (int64_t j0 = beg; j0 < end && !found; j0 += 8) {
                        int32_t w[8];
#pragma unroll
                        for (int q = 0; q < 8; ++q) w[q] = j0 + q < end ? __ldg(g.adj + j0 + q) : -1;
#pragma unroll
                        for (int q = 0; q < 8; ++q) found |= w[q] >= 0 && dist[w[q]] == l;
                    }
                    if (found) {
                        dist[v] = l + 1;
                        mf_next += end - beg;
                    }
                }
            }
            const int slot = warp_append(out_size, found);
            if (found) out[slot] = (int32_t)v;
            __syncthreads();
            const int ns = nstage;
            for (int q = threadIdx.x >> 5; q < ns; q += warps) {   // staged rows, one warp each
                const int32_t sv = stage[q];
                const int64_t sb = ld_xadj(g.xadj, sv), se = ld_xadj(g.xadj, (int64_t)sv + 1);
                bool hit = false;
                for (int64_t j0 = sb; j0 < se && !hit; j0 += 32) hit = bfs_parent_in_chunk(g, dist, j0 + lane, se, l);
                if (hit && lane == 0) {
                    dist[sv] = l + 1;
                    out[atomicAdd(out_size, 1)] = sv;
                    mf_next += se - sb;
                }
            }
            __syncthreads();
        }
        const int nh = nhuge < kHugeCap ? nhuge : kHugeCap;
        for (int s = 0; s < nh; ++s) {           // hub rows, the whole block
            const int32_t hv = huge[s];
            const int64_t hb = ld_xadj(g.xadj, hv), he = ld_xadj(g.xadj, (int64_t)hv + 1);
            bool hit = false;
            for (int64_t j0 = hb; j0 < he; j0 += blockDim.x) {
                const int64_t j = j0 + threadIdx.x;
                const int32_t w = j < he ? __ldg(g.adj + j) : -1;
                hit = __syncthreads_or(w >= 0 && dist[w] == l);
                if (hit) break;
            }
            if (hit && threadIdx.x == 0) {
                dist[hv] = l + 1;
                out[atomicAdd(out_size, 1)] = hv;
                mf_next += he - hb;
            }
        }
    }
    mf_next = block_sum_i64(mf_next, red);
    if (threadIdx.x == 0 && mf_next) atomic_add_i64(&ctl->mf[(l + 1) & 1], mf_next);
    __shared__ int s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = atomicAdd(&ctl->ticket, 1);
        s_last = t == (int)gridDim.x - 1;
        if (s_last) {
            __threadfence();
            ctl->ticket = 0;
            ctl->size[l & 1] = 0;
            ctl->mv += __ldcg(reinterpret_cast<const long long *>(&ctl->mf[(l + 1) & 1]));   // from L2: other blocks added it
            ctl->mf[l & 1] = 0;
            ctl->level = l + 1;
        }
    }
}

// ---- sort keys: (root, distance) over vertices in id order ----------------
__global__ void k_sort_init(int32_t n, const int32_t *root, const int32_t *dist, int dbits, uint64_t *key,
                            int32_t *val) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        key[v] = ((uint64_t)(uint32_t)root[v] << dbits) | (uint64_t)(uint32_t)dist[v];
        val[v] = (int32_t)v;
    }
}

// Weight of the vertex at sorted position i (unit weights when vw is null).
struct SortedWeight {
    const int32_t *val;
    const int32_t *vw;
    __device__ int64_t operator()(int64_t i) const { return vw ? vw[val[i]] : 1; }
};

__global__ void k_assign(int32_t n, const int32_t *val, const int64_t *S, const IpCtl *ctl, int32_t k, int32_t *part) {
    const long long W = ctl->total;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        part[val[i]] = (int32_t)(((long long)k * S[i]) / W);
}

// The order itself, by vertex: S(v), position and distance.
__global__ void k_order_out(int32_t n, const int32_t *val, const int64_t *S, const int32_t *dist, int64_t *S_out,
                            int32_t *rank_out, int32_t *dist_out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = val[i];
        if (S_out) S_out[v] = S[i];
        if (rank_out) rank_out[v] = (int32_t)i;
        if (dist_out) dist_out[v] = dist[v];
    }
}


}  // namespace

int initial_partition(Ctx &c, const DGraph &g, int32_t k, int32_t *part, GreedyOut *go) {
    cudaStream_t s = c.stream;
    const int64_t n = g.n;
    if (n == 0) return JET_OK;
    const size_t nn = (size_t)n;
    auto a256 = [](size_t x) { return (x + 255) & ~size_t(255); };
    // parent, root, dist, front0, front1 | S | scan tiles | ctl | sort scratch
    const size_t bytes = 5 * a256(nn * 4) + a256(nn * 8) + a256((size_t)(scan_tiles_for(n) + 1) * 8) +
                         a256(sizeof(IpCtl)) + sort_scratch_bytes(n);
    DevBuf buf;
    JET_TRY(dev_alloc(buf, bytes, s));
    char *p = buf.as<char>();
    auto take = [&](size_t b) { char *r = p; p += a256(b); return r; };
    int32_t *parent = reinterpret_cast<int32_t *>(take(nn * 4));
    int32_t *rootb = reinterpret_cast<int32_t *>(take(nn * 4));
    int32_t *dist = reinterpret_cast<int32_t *>(take(nn * 4));
    int32_t *front0 = reinterpret_cast<int32_t *>(take(nn * 4));
    int32_t *front1 = reinterpret_cast<int32_t *>(take(nn * 4));
    int64_t *S = reinterpret_cast<int64_t *>(take(nn * 8));
    int64_t *scan_scr = reinterpret_cast<int64_t *>(take((size_t)(scan_tiles_for(n) + 1) * 8));
    IpCtl *ctl = reinterpret_cast<IpCtl *>(take(sizeof(IpCtl)));
    SortScratch sc;
    sort_scratch_carve(p, n, sc);
    JET_CUDA_TRY(cudaMemsetAsync(ctl, 0, sizeof(IpCtl), s));
    const int gv = std::min(num_sms() * 8, grid_for(n, kTB));
    const int gw = std::min(num_sms() * 8, grid_for(n, kTB / 32));

    // 1. components
    k_uf_init<<<gv, kTB, 0, s>>>((int32_t)n, parent);
    k_uf_hook_sample<<<gv, kTB, 0, s>>>(g, parent, ctl);
    k_uf_major<<<1, kMajorSample, 0, s>>>((int32_t)n, parent, ctl);
    k_uf_hook_rest<<<gw, kTB, 0, s>>>(g, parent, ctl);
    int32_t *ra = parent, *rb = rootb;
    const int rounds = bits_for(n);
    for (int r = 0; r < rounds; ++r) {
        k_uf_jump<<<gv, kTB, 0, s>>>((int32_t)n, ra, rb);
        std::swap(ra, rb);
    }
    const int32_t *root = ra;
    k_uf_finish<<<gv, kTB, 0, s>>>(g, root, dist, front0, ctl);
    c.launches += 5 + rounds;
    JET_CUDA_TRY(cudaGetLastError());

    // 2. breadth-first levels, kBfsBatch launches between checks
    const int gb = num_sms() * 4;
    for (int64_t batch = 0;; ++batch) {
        for (int i = 0; i < kBfsBatch; ++i) k_bfs_level<<<gb, kTB, 0, s>>>(g, dist, front0, front1, ctl);
        c.launches += kBfsBatch;
        JET_CUDA_TRY(cudaGetLastError());
        IpCtl h;
        JET_CUDA_TRY(cudaMemcpyAsync(&h, ctl, sizeof(IpCtl), cudaMemcpyDeviceToHost, s));
        JET_CUDA_TRY(cudaStreamSynchronize(s));
        if (h.error) {
            record_error("initial partition: union-find step limit reached");
            return JET_ETIMEOUT;
        }
        if (h.size[0] == 0 && h.size[1] == 0) break;
        if (batch * kBfsBatch > n + kBfsBatch) {     // more levels than vertices: impossible
            record_error("initial partition: breadth-first search did not end");
            return JET_ETIMEOUT;
        }
    }
    IpCtl h;
    JET_CUDA_TRY(cudaMemcpyAsync(&h, ctl, sizeof(IpCtl), cudaMemcpyDeviceToHost, s));
    JET_CUDA_TRY(cudaStreamSynchronize(s));
    const int32_t maxdist = std::max(h.level - 1, 0);   // deepest level reached

    // 3. stable sort of the vertices (in id order) by (root, distance)
    const int dbits = bits_for(maxdist);
    k_sort_init<<<gv, kTB, 0, s>>>((int32_t)n, root, dist, dbits, sc.key[0], sc.val[0]);
    c.launches += 1;
    int which = 0;
    JET_TRY(sort_pairs(c, sc, n, bits_for(n - 1) + dbits, &which));
    const int32_t *order = sc.val[which];

    // 4. weights before each vertex in that order, then P
    JET_TRY(device_exscan(SortedWeight{order, g.vw}, n, S, &ctl->total, scan_scr, s));
    c.launches += 3;
    if (part) {
        k_assign<<<gv, kTB, 0, s>>>((int32_t)n, order, S, ctl, k, part);
        c.launches += 1;
    }
    if (go) {
        k_order_out<<<gv, kTB, 0, s>>>((int32_t)n, order, S, dist, go->S, go->rank, go->dist);
        c.launches += 1;
        JET_CUDA_TRY(cudaMemcpyAsync(&go->W, &ctl->total, 8, cudaMemcpyDeviceToHost, s));
        go->maxdist = maxdist;
    }
    JET_CUDA_TRY(cudaGetLastError());
    JET_CUDA_TRY(cudaStreamSynchronize(s));
    return JET_OK;
}

}  // namespace jet
