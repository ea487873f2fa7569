// Coarsening (Sec. 3.1): heavy-edge matching, coarse mapping, edge
// contraction (Alg. 2), projection (Alg. 1 ProjectPartition) and the greedy
// initial partition of the coarsest graph (Alg. 1 InitialPartition).
//
// Matching is a deterministic handshake: every unmatched vertex proposes its
// heaviest unmatched neighbour (ties: smaller splitmix64 hash of the
// neighbour, then smaller id) and mutual proposals match, round after round.
// Contraction merges each coarse vertex's (at most two) fine rows, sorts the
// mapped neighbour ids and sums duplicate entries: rows of <= 32 entries in
// one thread (register bitonic network), up to 256 in one warp and longer
// rows in one block (bitonic sorts in shared memory, or in a global scratch
// segment for very long rows).
#include "jet_internal.cuh"

#include <algorithm>
#include <cstring>

namespace jet {

template <bool EW>
__device__ __forceinline__ int32_t cw(const DGraph &g, int64_t j) {
    if constexpr (EW) return __ldg(g.ew + j);
    else return 1;
}

// Phase 2 of device_exscan: exclusive scan of the tile sums (one block).
__global__ void __launch_bounds__(1024) k_scan_sums(int64_t *tile_sums, int64_t ntiles, int64_t *total_dev) {
    __shared__ long long sh[40];
    pdl_enter();
    long long carry = 0;
    for (int64_t t0 = 0; t0 < ntiles; t0 += blockDim.x) {
        int64_t t = t0 + threadIdx.x;
        long long x = t < ntiles ? tile_sums[t] : 0;
        long long tot = 0;
        long long ex = block_exscan_i64(x, sh, &tot);
        if (t < ntiles) tile_sums[t] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0 && total_dev) *total_dev = carry;
}

struct HemCtl {
    int32_t stop;
    int32_t pad;
    int64_t added[64];
};

__device__ __forceinline__ bool hem_better(int32_t w1, uint64_t h1, int32_t u1, int32_t w2, uint64_t h2, int32_t u2) {
    if (u2 < 0) return u1 >= 0;
    if (u1 < 0) return false;
    if (w1 != w2) return w1 > w2;
    if (h1 != h2) return h1 < h2;
    return u1 < u2;
}

__device__ __forceinline__ uint64_t hem_hash(uint64_t seed, uint64_t salt, int32_t u) {
    return splitmix64(seed ^ salt ^ (uint64_t)(uint32_t)u);
}

__device__ __forceinline__ bool hem_skip(const HemCtl *hc, int r) {
    return r > 0 && (hc->stop || hc->added[r - 1] == 0);
}

// One proposal round (short rows): prop[v] = chosen neighbour or -1.
template <bool EW>
__global__ void __launch_bounds__(kTB) k_hem_propose_small(DGraph g, const int32_t *mate, int32_t *prop, uint64_t seed,
                                                           uint64_t salt, int r, HemCtl *hc) {
    pdl_enter();
    if (hem_skip(hc, r)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) hc->stop = 1;
        return;
    }
    int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= g.n) return;
    int64_t beg = ld_xadj(g.xadj, v), end = ld_xadj(g.xadj, (int64_t)v + 1);
    if (end - beg > kSmallDeg) return;
    int32_t bu = -1, bw = 0;
    uint64_t bh = 0;
    if (mate[v] < 0) {
        for (int64_t j = beg; j < end; ++j) {
            int32_t u = __ldg(g.adj + j);
            if (mate[u] >= 0) continue;
            int32_t w = cw<EW>(g, j);
            uint64_t h = hem_hash(seed, salt, u);
            if (hem_better(u >= 0 ? w : 0, h, u, bw, bh, bu)) { bu = u; bw = w; bh = h; }
        }
    }
    prop[v] = bu;
}

// The heaviest unmatched neighbour over the entries first, first + step, ...
// < end of a row, U at a time (ids, then their mates, in flight together);
// folds into (bu, bw, bh).
template <bool EW, int U = 4>
__device__ __forceinline__ void hem_row(const DGraph &g, const int32_t *mate, uint64_t seed, uint64_t salt, int64_t first,
                                        int64_t end, int64_t step, int32_t &bu, int32_t &bw, uint64_t &bh) {
    for (int64_t j0 = first; j0 < end; j0 += U * step) {
        int32_t u[U], m[U];
#pragma unroll
        for (int q = 0; q < U; ++q) {
            const int64_t j = j0 + q * step;
            u[q] = j < end ? __ldg(g.adj + j) : -1;
        }
#pragma unroll
        for (int q = 0; q < U; ++q) m[q] = u[q] >= 0 ? mate[u[q]] : 0;
#pragma unroll
        for (int q = 0; q < U; ++q) {
            if (u[q] < 0 || m[q] >= 0) continue;
            const int32_t ww = cw<EW>(g, j0 + q * step);
            const uint64_t h = hem_hash(seed, salt, u[q]);
            if (hem_better(ww, h, u[q], bw, bh, bu)) { bu = u[q]; bw = ww; bh = h; }
        }
    }
}

template <bool EW>
__global__ void __launch_bounds__(kTB) k_hem_propose_big(DGraph g, const int32_t *bigv, int32_t nbig, const int32_t *mate,
                                                         int32_t *prop, uint64_t seed, uint64_t salt, int r, HemCtl *hc) {
    pdl_enter();
    if (hem_skip(hc, r)) return;
    const int warps = blockDim.x >> 5;
    const unsigned lane = lane_id();
    for (int64_t w = (int64_t)blockIdx.x * warps + (threadIdx.x >> 5); w < nbig; w += (int64_t)gridDim.x * warps) {
        int32_t v = bigv[w];
        int32_t bu = -1, bw = 0;
        uint64_t bh = 0;
        if (mate[v] < 0) {
            int64_t beg = ld_xadj(g.xadj, v), end = ld_xadj(g.xadj, (int64_t)v + 1);
            hem_row<EW>(g, mate, seed, salt, beg + lane, end, 32, bu, bw, bh);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            int32_t ou = __shfl_xor_sync(0xffffffffu, bu, o);
            int32_t ow = __shfl_xor_sync(0xffffffffu, bw, o);
            uint64_t oh = __shfl_xor_sync(0xffffffffu, bh, o);
            if (hem_better(ow, oh, ou, bw, bh, bu)) { bu = ou; bw = ow; bh = oh; }
        }
        if (lane == 0) prop[v] = bu;
    }
}

// Hub rows (longer than kHugeDeg): one block per row, the same choice.
template <bool EW>
__global__ void __launch_bounds__(kTB) k_hem_propose_huge(DGraph g, const int32_t *hugev, int32_t nhuge,
                                                          const int32_t *mate, int32_t *prop, uint64_t seed,
                                                          uint64_t salt, int r, HemCtl *hc) {
    pdl_enter();
    if (hem_skip(hc, r)) return;
    __shared__ int32_t su[32], sw[32];
    __shared__ uint64_t shh[32];
    const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
    for (int64_t t = blockIdx.x; t < nhuge; t += gridDim.x) {
        const int32_t v = hugev[t];
        int32_t bu = -1, bw = 0;
        uint64_t bh = 0;
        if (mate[v] < 0) {
            const int64_t beg = ld_xadj(g.xadj, v), end = ld_xadj(g.xadj, (int64_t)v + 1);
            hem_row<EW, 8>(g, mate, seed, salt, beg + threadIdx.x, end, blockDim.x, bu, bw, bh);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const int32_t ou = __shfl_xor_sync(0xffffffffu, bu, o);
            const int32_t ow = __shfl_xor_sync(0xffffffffu, bw, o);
            const uint64_t oh = __shfl_xor_sync(0xffffffffu, bh, o);
            if (hem_better(ow, oh, ou, bw, bh, bu)) { bu = ou; bw = ow; bh = oh; }
        }
        if (lane == 0) { su[warp] = bu; sw[warp] = bw; shh[warp] = bh; }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (unsigned i = 1; i < (blockDim.x >> 5); ++i)
                if (hem_better(sw[i], shh[i], su[i], bw, bh, bu)) { bu = su[i]; bw = sw[i]; bh = shh[i]; }
            prop[v] = bu;
        }
        __syncthreads();
    }
}

// Mutual proposals match (synchronous: every proposal of the round is read
// before any mate changes matter, since proposals only name unmatched ones).
__global__ void __launch_bounds__(kTB) k_hem_match(int32_t n, int32_t *mate, const int32_t *prop, int r, HemCtl *hc) {
    __shared__ long long red[40];
    pdl_enter();
    if (hc->stop) return;
    long long c = 0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        int32_t u = prop[v];
        if (u >= 0 && prop[u] == (int32_t)v) { mate[v] = u; ++c; }
    }
    c = block_sum_i64(c, red);
    if (threadIdx.x == 0 && c) atomic_add_i64(&hc->added[r], c);
}

// Rows longer than kSmallDeg: warp rows (up to kHugeDeg entries) into list,
// hub rows into hlist.
__global__ void k_collect_rows(DGraph g, int32_t *list, int32_t *count, int32_t *hlist, int32_t *hcount) {
    int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t d = v < g.n ? ld_xadj(g.xadj, (int64_t)v + 1) - ld_xadj(g.xadj, v) : 0;
    const bool big = d > kSmallDeg && d <= kHugeDeg, huge = d > kHugeDeg;
    int slot = warp_append(count, big);
    if (big) list[slot] = v;
    slot = warp_append(hcount, huge);
    if (huge) hlist[slot] = v;
}

__global__ void k_fill(int32_t *p, int64_t n, int32_t val) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) p[i] = val;
}

// The warp rows (list at buf) and the hub rows (list at *huge) of g.
static int big_rows(Ctx &c, const DGraph &g, DevBuf &buf, int32_t &nbig, int32_t **huge, int32_t &nhuge) {
    cudaStream_t s = c.stream;
    const size_t nb = ((size_t)std::max<int64_t>(g.n, 1) * 4 + 255) & ~size_t(255);
    JET_TRY(dev_alloc(buf, 2 * nb + 256, s));
    int32_t *list = buf.as<int32_t>();
    *huge = reinterpret_cast<int32_t *>(buf.as<char>() + nb);
    int32_t *cnt = reinterpret_cast<int32_t *>(buf.as<char>() + 2 * nb);
    JET_CUDA_TRY(cudaMemsetAsync(cnt, 0, 8, s));
    if (g.n > 0) k_collect_rows<<<grid_for(g.n, kTB), kTB, 0, s>>>(g, list, cnt, *huge, cnt + 1);
    if (g.n > 0) c.launches += 1;
    JET_CUDA_TRY(cudaGetLastError());
    JET_CUDA_TRY(cudaMemcpyAsync(c.pinned, cnt, 8, cudaMemcpyDeviceToHost, s));
    JET_CUDA_TRY(cudaStreamSynchronize(s));
    int32_t h[2];
    memcpy(h, c.pinned, 8);
    nbig = h[0];
    nhuge = h[1];
    return JET_OK;
}

int hem(Ctx &c, const DGraph &g, uint64_t seed, int32_t level, int32_t rounds, int32_t *mate) {
    cudaStream_t s = c.stream;
    if (g.n == 0) return JET_OK;
    DevBuf bigbuf, pbuf, hbuf;
    int32_t nbig = 0, nhuge = 0;
    int32_t *hugev = nullptr;
    JET_TRY(big_rows(c, g, bigbuf, nbig, &hugev, nhuge));
    JET_TRY(dev_alloc(pbuf, (size_t)g.n * 4, s));
    JET_TRY(dev_alloc(hbuf, sizeof(HemCtl), s));
    HemCtl *hc = hbuf.as<HemCtl>();
    JET_CUDA_TRY(cudaMemsetAsync(hc, 0, sizeof(HemCtl), s));
    k_fill<<<grid_for(g.n, kTB, 4096), kTB, 0, s>>>(mate, g.n, -1);
    c.launches += 1;
    rounds = std::min(rounds, 64);
    int gl = num_sms() * 8;
    // the rounds follow one another by programmatic launch (each kernel waits
    // for the previous one on the device before it reads anything)
    const bool pdl = !(c.opt.flags & JET_FLAG_NO_PDL);
    int32_t *prop = pbuf.as<int32_t>();
    const int32_t *bigv = bigbuf.as<int32_t>();
    for (int r = 0; r < rounds; ++r) {
        uint64_t salt = 0xD1B54A32D192ED03ULL * (uint64_t)(64 * (int64_t)level + r + 1);
        const int gs = grid_for(g.n, kTB);
        if (g.ew) JET_CUDA_TRY(launch_pdl(k_hem_propose_small<true>, gs, kTB, 0, s, pdl, g, (const int32_t *)mate, prop, seed, salt, r, hc));
        else JET_CUDA_TRY(launch_pdl(k_hem_propose_small<false>, gs, kTB, 0, s, pdl, g, (const int32_t *)mate, prop, seed, salt, r, hc));
        c.launches += 1;
        if (nbig > 0) {
            int gb = std::min(gl, grid_for(nbig, kTB / 32));
            if (g.ew) JET_CUDA_TRY(launch_pdl(k_hem_propose_big<true>, gb, kTB, 0, s, pdl, g, bigv, nbig, (const int32_t *)mate, prop, seed, salt, r, hc));
            else JET_CUDA_TRY(launch_pdl(k_hem_propose_big<false>, gb, kTB, 0, s, pdl, g, bigv, nbig, (const int32_t *)mate, prop, seed, salt, r, hc));
            c.launches += 1;
        }
        if (nhuge > 0) {
            int gh = std::min(gl, nhuge);
            if (g.ew) JET_CUDA_TRY(launch_pdl(k_hem_propose_huge<true>, gh, kTB, 0, s, pdl, g, (const int32_t *)hugev, nhuge, (const int32_t *)mate, prop, seed, salt, r, hc));
            else JET_CUDA_TRY(launch_pdl(k_hem_propose_huge<false>, gh, kTB, 0, s, pdl, g, (const int32_t *)hugev, nhuge, (const int32_t *)mate, prop, seed, salt, r, hc));
            c.launches += 1;
        }
        JET_CUDA_TRY(launch_pdl(k_hem_match, std::min(gl, grid_for(g.n, kTB)), kTB, 0, s, pdl, g.n, mate, (const int32_t *)prop, r, hc));
        c.launches += 1;
    }
    JET_CUDA_TRY(cudaGetLastError());
    return JET_OK;   // mate is final once the stream passes here (the scratch is freed in stream order)
}

// ---------------------------------------------------------------------------
// coarse mapping: representatives are unmatched vertices and the smaller id
// of each pair; C[v] = rank of v's representative
// ---------------------------------------------------------------------------
struct RepFlag {
    const int32_t *mate;
    __device__ int64_t operator()(int64_t v) const {
        int32_t m = mate[v];
        return (m < 0 || v < m) ? 1 : 0;
    }
};

__global__ void k_cmap(int32_t n, const int32_t *mate, const int64_t *cidx, int32_t *cmap, int32_t *crep) {
    pdl_enter();
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        int32_t m = mate[v];
        int64_t r = (m >= 0 && m < v) ? m : v;
        cmap[v] = (int32_t)cidx[r];
        if (r == v) crep[cidx[v]] = (int32_t)v;
    }
}

struct RowBound {
    const int64_t *xadj;
    const int32_t *crep, *mate;
    __device__ int64_t operator()(int64_t c) const {
        int32_t r = crep[c];
        int32_t m = mate[r];
        int64_t b = xadj[r + 1] - xadj[r];
        if (m >= 0) b += xadj[(int64_t)m + 1] - xadj[m];
        return b;
    }
};

// Longest merged row sorted in shared memory by one block; longer rows go
// through the device-wide radix sort (a launch-shape choice).
#ifndef JET_SORT_SMEM
#define JET_SORT_SMEM 4096
#endif
constexpr int kSortSmem = JET_SORT_SMEM;

__host__ __device__ inline int64_t pow2ceil(int64_t x) {
    int64_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

// Hub rows (bound > kSortSmem) are contracted through one device-wide radix
// sort of all their entries: HubBound gives each hub row's segment length
// (0 for the others), HubFlag its rank among the hub rows.
struct HubBound {
    const int32_t *crep, *mate;
    const int64_t *xadj;
    __device__ int64_t operator()(int64_t c) const {
        int32_t r = crep[c];
        int32_t m = mate[r];
        int64_t b = xadj[r + 1] - xadj[r];
        if (m >= 0) b += xadj[(int64_t)m + 1] - xadj[m];
        return b > kSortSmem ? b : 0;
    }
};
struct HubFlag {
    HubBound hb;
    __device__ int64_t operator()(int64_t c) const { return hb(c) > 0 ? 1 : 0; }
};

// Coarse vertex weights, and the coarse rows sorted into classes by their
// bound (entries of the merged fine rows): <= 16 and <= 32 (one thread),
// <= kWarpSort (one warp), longer (one block).  counts = {warp rows, block
// rows, 16-entry thread rows, 32-entry thread rows}.
constexpr int kWarpSort = 256;
__global__ void k_coarse_vw(int32_t nc, const int32_t *crep, const int32_t *mate, const int32_t *vw, int32_t *vwc,
                            int32_t *warp_list, int32_t *large_list, int32_t *t16_list, int32_t *t32_list,
                            int32_t *counts, const int64_t *boff, const int64_t *btot) {
    pdl_enter();
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < ((int64_t)nc + 31) / 32 * 32;
         c += (int64_t)gridDim.x * blockDim.x) {
        bool valid = c < nc;
        int64_t b = 0;
        if (valid) {
            int32_t r = crep[c];
            int32_t m = mate[r];
            vwc[c] = vw[r] + (m >= 0 ? vw[m] : 0);
            b = (c + 1 < nc ? boff[c + 1] : *btot) - boff[c];
        }
        const bool t16 = valid && b <= 16, t32 = valid && b > 16 && b <= 32;
        const bool wr = valid && b > 32 && b <= kWarpSort, large = valid && b > kWarpSort;
        int s0 = warp_append(&counts[2], t16);
        if (t16) t16_list[s0] = (int32_t)c;
        int s1 = warp_append(&counts[3], t32);
        if (t32) t32_list[s1] = (int32_t)c;
        int s2 = warp_append(&counts[0], wr);
        if (wr) warp_list[s2] = (int32_t)c;
        int s3 = warp_append(&counts[1], large);
        if (large) large_list[s3] = (int32_t)c;
    }
}

// Gathers entry i (0 <= i < bound) of coarse row c: (C[u] << 32) | w.
template <bool EW>
__device__ __forceinline__ unsigned long long row_entry(const DGraph &g, const int32_t *cmap, int32_t r, int32_t m,
                                                        int64_t degr, int64_t i) {
    int64_t j = i < degr ? ld_xadj(g.xadj, r) + i : ld_xadj(g.xadj, m) + (i - degr);
    int32_t cu = cmap[__ldg(g.adj + j)];
    return ((unsigned long long)(uint32_t)cu << 32) | (uint32_t)cw<EW>(g, j);
}

// Rows of <= N entries (N = 16 or 32): one thread each (32 rows of a warp in
// flight together), the keys (C[u] << 32 | w) sorted by a bitonic network
// over registers, then one pass that adds up equal coarse neighbours and
// drops the row's own vertex.  Same output as the warp and block forms.
// counts[slot] rows in list.
template <bool EW, int N>
__global__ void __launch_bounds__(kTB) k_contract_thread(DGraph g, const int32_t *cmap, const int32_t *mate,
                                                       const int32_t *crep, const int32_t *list, const int32_t *counts,
                                                       const int64_t *boff, int32_t *tadj, int32_t *tw, int32_t *rowcnt) {
    pdl_enter();
    const int32_t nrows = counts[N == 16 ? 2 : 3];
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nrows; w += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = list[w];
        const int32_t r = crep[c], m = mate[r];
        const int64_t r0 = ld_xadj(g.xadj, r), degr = ld_xadj(g.xadj, (int64_t)r + 1) - r0;
        int64_t m0 = 0, degm = 0;
        if (m >= 0) {
            m0 = ld_xadj(g.xadj, m);
            degm = ld_xadj(g.xadj, (int64_t)m + 1) - m0;
        }
        const int64_t bound = degr + degm;
        unsigned long long key[N];
#pragma unroll
        for (int t = 0; t < N; ++t) {
            key[t] = ~0ull;
            if (t < bound) {
                const int64_t j = t < degr ? r0 + t : m0 + (t - degr);
                key[t] = ((unsigned long long)(uint32_t)cmap[__ldg(g.adj + j)] << 32) | (uint32_t)cw<EW>(g, j);
            }
        }
#pragma unroll
        for (int kk = 2; kk <= N; kk <<= 1) {
#pragma unroll
            for (int j = kk >> 1; j > 0; j >>= 1) {
#pragma unroll
                for (int i = 0; i < N; ++i) {
                    const int l = i ^ j;
                    if (l > i) {
                        const unsigned long long a = key[i], b = key[l];
                        const bool swap = ((i & kk) == 0) ? (a > b) : (a < b);
                        key[i] = swap ? b : a;
                        key[l] = swap ? a : b;
                    }
                }
            }
        }
        const int64_t base = boff[c];
        int32_t cnt = 0;
        uint32_t cur = 0xFFFFFFFFu;
        long long sum = 0;
#pragma unroll
        for (int t = 0; t < N; ++t) {
            const unsigned long long kt = key[t];
            const uint32_t ck = (uint32_t)(kt >> 32);
            if (kt != ~0ull && ck != (uint32_t)c) {
                if (ck != cur) {
                    if (cur != 0xFFFFFFFFu) {
                        tadj[base + cnt] = (int32_t)cur;
                        tw[base + cnt] = (int32_t)sum;
                        ++cnt;
                    }
                    cur = ck;
                    sum = 0;
                }
                sum += (long long)(uint32_t)(kt & 0xFFFFFFFFull);
            }
        }
        if (cur != 0xFFFFFFFFu) {
            tadj[base + cnt] = (int32_t)cur;
            tw[base + cnt] = (int32_t)sum;
            ++cnt;
        }
        rowcnt[c] = cnt;
    }
}

// Rows of 33..kWarpSort entries: one warp each, bitonic sort over the warp's
// shared-memory segment (pairs of a stage split over the lanes, __syncwarp
// between stages), then heads of equal-id runs summed and written in order.
template <bool EW>
__global__ void __launch_bounds__(kTB) k_contract_warp(DGraph g, const int32_t *cmap, const int32_t *mate,
                                                       const int32_t *crep, const int32_t *list, const int32_t *counts,
                                                       const int64_t *boff, int32_t *tadj, int32_t *tw, int32_t *rowcnt) {
    __shared__ unsigned long long sk[kTB / 32][kWarpSort];
    pdl_enter();
    const int warps = blockDim.x >> 5;
    const unsigned lane = lane_id();
    unsigned long long *keys = sk[threadIdx.x >> 5];
    const int32_t nrows = counts[0];
    for (int64_t w = (int64_t)blockIdx.x * warps + (threadIdx.x >> 5); w < nrows; w += (int64_t)gridDim.x * warps) {
        const int32_t c = list[w];
        const int32_t r = crep[c], m = mate[r];
        const int64_t degr = ld_xadj(g.xadj, (int64_t)r + 1) - ld_xadj(g.xadj, r);
        const int64_t bound = degr + (m >= 0 ? ld_xadj(g.xadj, (int64_t)m + 1) - ld_xadj(g.xadj, m) : 0);
        const int P = (int)pow2ceil(bound);   // <= kWarpSort by the class
        for (int i = lane; i < P; i += 32) keys[i] = i < bound ? row_entry<EW>(g, cmap, r, m, degr, i) : ~0ull;
        __syncwarp();
        for (int kk = 2; kk <= P; kk <<= 1) {
            for (int j = kk >> 1; j > 0; j >>= 1) {
                for (int i = lane; i < P; i += 32) {
                    const int l = i ^ j;
                    if (l > i) {
                        const unsigned long long a = keys[i], b = keys[l];
                        const bool up = (i & kk) == 0;
                        if ((a > b) == up) { keys[i] = b; keys[l] = a; }
                    }
                }
                __syncwarp();
            }
        }
        const int64_t base = boff[c];
        int32_t written = 0;
        for (int i0 = 0; i0 < bound; i0 += 32) {
            const int i = i0 + (int)lane;
            bool head = false;
            uint32_t ck = 0;
            long long sum = 0;
            if (i < bound) {
                ck = (uint32_t)(keys[i] >> 32);
                head = (i == 0 || (uint32_t)(keys[i - 1] >> 32) != ck) && ck != (uint32_t)c;
                if (head)
                    for (int t = i; t < bound && (uint32_t)(keys[t] >> 32) == ck; ++t)
                        sum += (long long)(uint32_t)(keys[t] & 0xFFFFFFFFull);
            }
            const unsigned hm = __ballot_sync(0xffffffffu, head);
            const int pos = __popc(hm & ((1u << lane) - 1u));
            if (head) {
                tadj[base + written + pos] = (int32_t)ck;
                tw[base + written + pos] = (int32_t)sum;
            }
            written += __popc(hm);
        }
        if (lane == 0) rowcnt[c] = written;
        __syncwarp();
    }
}

// Rows of kWarpSort..kSortSmem entries: one block per row, bitonic sort in
// shared memory.
template <bool EW>
__global__ void __launch_bounds__(kTB) k_contract_large(DGraph g, const int32_t *cmap, const int32_t *mate,
                                                        const int32_t *crep, const int32_t *list, const int32_t *counts,
                                                        const int64_t *boff, int32_t *tadj, int32_t *tw,
                                                        int32_t *rowcnt) {
    __shared__ unsigned long long sk[kSortSmem];
    pdl_enter();
    __shared__ long long sh[40];
    const int32_t nrows = counts[1];
    for (int64_t w = blockIdx.x; w < nrows; w += gridDim.x) {
        int32_t c = list[w];
        int32_t r = crep[c], m = mate[r];
        int64_t degr = ld_xadj(g.xadj, (int64_t)r + 1) - ld_xadj(g.xadj, r);
        int64_t bound = degr + (m >= 0 ? ld_xadj(g.xadj, (int64_t)m + 1) - ld_xadj(g.xadj, m) : 0);
        if (bound > kSortSmem) continue;   // hub row: the radix-sort path (uniform over the block)
        int64_t P = pow2ceil(bound);
        unsigned long long *keys = sk;
        for (int64_t i = threadIdx.x; i < P; i += blockDim.x)
            keys[i] = i < bound ? row_entry<EW>(g, cmap, r, m, degr, i) : ~0ull;
        __syncthreads();
        for (int64_t kk = 2; kk <= P; kk <<= 1) {
            for (int64_t j = kk >> 1; j > 0; j >>= 1) {
                for (int64_t i = threadIdx.x; i < P; i += blockDim.x) {
                    int64_t ixj = i ^ j;
                    if (ixj > i) {
                        unsigned long long a = keys[i], b = keys[ixj];
                        bool up = (i & kk) == 0;
                        if ((a > b) == up) { keys[i] = b; keys[ixj] = a; }
                    }
                }
                __syncthreads();
            }
        }
        // heads of runs with equal coarse id, summed, self id dropped; written in order
        int64_t base = boff[c];
        long long written = 0;
        for (int64_t i0 = 0; i0 < bound; i0 += blockDim.x) {
            int64_t i = i0 + threadIdx.x;
            bool head = false;
            uint32_t ck = 0;
            long long sum = 0;
            if (i < bound) {
                unsigned long long key = keys[i];
                ck = (uint32_t)(key >> 32);
                head = (i == 0 || (uint32_t)(keys[i - 1] >> 32) != ck) && ck != (uint32_t)c;
                if (head) {
                    for (int64_t t = i; t < bound && (uint32_t)(keys[t] >> 32) == ck; ++t)
                        sum += (long long)(uint32_t)(keys[t] & 0xFFFFFFFFull);
                }
            }
            long long tot = 0;
            long long pos = block_exscan_i64(head ? 1 : 0, sh, &tot);
            if (head) { tadj[base + written + pos] = (int32_t)ck; tw[base + written + pos] = (int32_t)sum; }
            written += tot;
        }
        if (threadIdx.x == 0) rowcnt[c] = (int32_t)written;
        __syncthreads();
    }
}

struct CountVal {
    const int32_t *cnt;
    __device__ int64_t operator()(int64_t c) const { return cnt[c]; }
};

__global__ void k_finish_xadj(int32_t nc, const int64_t *ex, const int64_t *tot, int64_t *xadj_c) {
    pdl_enter();
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c <= nc; c += (int64_t)gridDim.x * blockDim.x)
        xadj_c[c] = c < nc ? ex[c] : *tot;
}

// Hub rows, step 1: every entry of hub row c becomes (rank(c) << 32 | C[u],
// w) at its segment hoff[c] + i (one block per row).
template <bool EW>
__global__ void __launch_bounds__(kTB) k_hub_fill(DGraph g, const int32_t *cmap, const int32_t *mate, const int32_t *crep,
                                                  const int32_t *list, const int32_t *counts, const int64_t *hoff,
                                                  const int64_t *hrank, uint64_t *key, int32_t *val,
                                                  int32_t *hub_c) {
    const int32_t nrows = counts[1];
    for (int64_t w = blockIdx.x; w < nrows; w += gridDim.x) {
        const int32_t c = list[w];
        const int32_t r = crep[c], m = mate[r];
        const int64_t degr = ld_xadj(g.xadj, (int64_t)r + 1) - ld_xadj(g.xadj, r);
        const int64_t bound = degr + (m >= 0 ? ld_xadj(g.xadj, (int64_t)m + 1) - ld_xadj(g.xadj, m) : 0);
        if (bound <= kSortSmem) continue;
        const int64_t off = hoff[c];
        const uint64_t hi = (uint64_t)hrank[c] << 32;
        if (threadIdx.x == 0) hub_c[hrank[c]] = c;
        for (int64_t i = threadIdx.x; i < bound; i += blockDim.x) {
            const unsigned long long e = row_entry<EW>(g, cmap, r, m, degr, i);
            key[off + i] = hi | (e >> 32);
            val[off + i] = (int32_t)(uint32_t)(e & 0xFFFFFFFFull);
        }
    }
}

// Hub rows, step 2 (after the stable sort by rank, then coarse id): the
// sorted entries of hub row c are the segment starting at hoff[c], in coarse
// id order.  An entry heads its output entry when it starts a run of equal
// (rank, coarse id) and the id is not the row's own; an exclusive scan of the
// head flags over all hub entries places every head (hs[p] - hs[hoff[c]]),
// so every row, however long, is spread over the whole grid.
struct HubHead {
    const uint64_t *key;
    const int32_t *hub_c;
    __device__ int64_t operator()(int64_t p) const {
        const uint64_t kp = key[p];
        if (p > 0 && key[p - 1] == kp) return 0;
        return (uint32_t)kp != (uint32_t)hub_c[kp >> 32] ? 1 : 0;
    }
};

__global__ void __launch_bounds__(kTB) k_hub_emit(int64_t htotal, const uint64_t *key, const int32_t *val,
                                                  const int32_t *hub_c, const int64_t *hoff, const int64_t *hs,
                                                  const int64_t *boff, int32_t *tadj, int32_t *tw) {
    const HubHead head{key, hub_c};
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < htotal; p += (int64_t)gridDim.x * blockDim.x) {
        if (!head(p)) continue;
        const uint64_t kp = key[p];
        const int32_t c = hub_c[kp >> 32];
        long long sum = 0;
        for (int64_t t = p; t < htotal && key[t] == kp; ++t) sum += (long long)(uint32_t)val[t];
        const int64_t q = boff[c] + (hs[p] - hs[hoff[c]]);
        tadj[q] = (int32_t)(uint32_t)kp;
        tw[q] = (int32_t)sum;
    }
}

// Hub rows, step 3: entries written per hub row (rank order; the segment of
// rank r ends where the next one starts).
__global__ void k_hub_rowcnt(int64_t nhub, int64_t htotal, const int32_t *hub_c, const int64_t *hoff, const int64_t *hs,
                             const int64_t *hs_total, int32_t *rowcnt) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nhub; r += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = hub_c[r];
        const int64_t beg = hoff[c];
        const int64_t end = r + 1 < nhub ? hoff[hub_c[r + 1]] : htotal;
        const int64_t he = end < htotal ? hs[end] : *hs_total;
        rowcnt[c] = (int32_t)(he - hs[beg]);
    }
}

// Long coarse rows (more than kWarpSort bound entries) are compacted by one
// block each; k_copy_rows leaves them out.
__global__ void __launch_bounds__(kTB) k_copy_long(const int32_t *list, const int32_t *counts, const int64_t *boff,
                                                   const int64_t *xadj_c, const int32_t *tadj, const int32_t *tw,
                                                   int32_t *adj_c, int32_t *ew_c) {
    pdl_enter();
    const int32_t nrows = counts[1];
    for (int64_t w = blockIdx.x; w < nrows; w += gridDim.x) {
        const int32_t c = list[w];
        const int64_t src = boff[c], dst = xadj_c[c], len = xadj_c[c + 1] - dst;
        for (int64_t i = threadIdx.x; i < len; i += blockDim.x) {
            adj_c[dst + i] = tadj[src + i];
            ew_c[dst + i] = tw[src + i];
        }
    }
}

// Compaction of the coarse rows: kCopyLanes lanes per row (the rows are
// short; a warp per row left most lanes idle and serialised the rows'
// round trips).
constexpr int kCopyLanes = 8;
__global__ void k_copy_rows(int32_t nc, const int64_t *boff, const int64_t *btot, const int64_t *xadj_c,
                            const int32_t *tadj, const int32_t *tw, int32_t *adj_c, int32_t *ew_c) {
    pdl_enter();
    const int64_t groups = (int64_t)gridDim.x * blockDim.x / kCopyLanes;
    const int gl = (int)(threadIdx.x % kCopyLanes);
    for (int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / kCopyLanes; c < nc; c += groups) {
        const int64_t src = boff[c], dst = xadj_c[c], len = xadj_c[c + 1] - dst;
        const int64_t bound = (c + 1 < nc ? boff[c + 1] : *btot) - src;
        if (bound > kWarpSort) continue;   // k_copy_long
        for (int64_t i = gl; i < len; i += kCopyLanes) {
            adj_c[dst + i] = tadj[src + i];
            ew_c[dst + i] = tw[src + i];
        }
    }
}

// One coarsening level: matching, map, contraction.  Returns JET_OK and sets
// stalled=true (without building the level) when n_c > 0.95 n.
static int coarsen_level(Ctx &c, const DGraph &g, uint64_t seed, int32_t level, jet_hier *h, bool &stalled) {
    cudaStream_t s = c.stream;
    stalled = false;
    int64_t n = g.n;
    DevBuf mbuf, cidxb, scan_scr, tot;
    JET_TRY(dev_alloc(mbuf, (size_t)n * 4, s));
    int32_t *mate = mbuf.as<int32_t>();
    JET_TRY(hem(c, g, seed, level, c.opt.hem_rounds, mate));
    if (c.opt.flags & JET_FLAG_TWO_HOP) {
        int64_t added[3];
        JET_TRY(two_hop(c, g, mate, added));
    }
    JET_TRY(dev_alloc(cidxb, (size_t)n * 8, s));
    JET_TRY(dev_alloc(scan_scr, (size_t)std::max<int64_t>(scan_tiles_for(n), 1) * 8 * 2 + 64, s));
    JET_TRY(dev_alloc(tot, 64, s));
    int64_t *totp = tot.as<int64_t>();
    c.launches += 3;
    JET_TRY(device_exscan(RepFlag{mate}, n, cidxb.as<int64_t>(), totp, scan_scr.as<int64_t>(), s));
    JET_CUDA_TRY(cudaMemcpyAsync(c.pinned, totp, 8, cudaMemcpyDeviceToHost, s));
    JET_CUDA_TRY(cudaStreamSynchronize(s));
    int64_t nc = c.pinned[0];
    if (100 * nc > 95 * n) { stalled = true; return JET_OK; }
    // cmap (owned by the hierarchy) and representatives
    DevBuf cmapb, crepb;
    JET_TRY(dev_alloc(cmapb, (size_t)n * 4, s));
    JET_TRY(dev_alloc(crepb, (size_t)std::max<int64_t>(nc, 1) * 4, s));
    int32_t *cmap = cmapb.as<int32_t>(), *crep = crepb.as<int32_t>();
    JET_CUDA_TRY(launch_pdl(k_cmap, grid_for(n, kTB, 8192), kTB, 0, s, true, g.n, (const int32_t *)mate,
                            (const int64_t *)cidxb.as<int64_t>(), cmap, crep));
    c.launches += 1;
    // bounds of the coarse rows
    DevBuf boffb, hoffb, hrankb;
    JET_TRY(dev_alloc(boffb, (size_t)std::max<int64_t>(nc, 1) * 8, s));
    JET_TRY(dev_alloc(hoffb, (size_t)std::max<int64_t>(nc, 1) * 8, s));
    JET_TRY(dev_alloc(hrankb, (size_t)std::max<int64_t>(nc, 1) * 8, s));
    int64_t *boff = boffb.as<int64_t>(), *hoff = hoffb.as<int64_t>(), *hrank = hrankb.as<int64_t>();
    c.launches += 9;
    JET_TRY(device_exscan(RowBound{g.xadj, crep, mate}, nc, boff, totp, scan_scr.as<int64_t>(), s));
    const HubBound hb{crep, mate, g.xadj};
    JET_TRY(device_exscan(hb, nc, hoff, totp + 1, scan_scr.as<int64_t>(), s));
    JET_TRY(device_exscan(HubFlag{hb}, nc, hrank, totp + 3, scan_scr.as<int64_t>(), s));
    JET_CUDA_TRY(cudaMemcpyAsync(c.pinned, totp, 32, cudaMemcpyDeviceToHost, s));
    JET_CUDA_TRY(cudaStreamSynchronize(s));
    int64_t btotal = c.pinned[0], htotal = c.pinned[1], nhub = c.pinned[3];
    // coarse vertex weights and row classes
    DevBuf vwcb, lists, tadjb, twb, cntb, hsortb, hubcb, hsb;
    JET_TRY(dev_alloc(vwcb, (size_t)std::max<int64_t>(nc, 1) * 4, s));
    const int64_t ncl = std::max<int64_t>(nc, 1);
    JET_TRY(dev_alloc(lists, (size_t)ncl * 16 + 64, s));
    int32_t *warp_list = lists.as<int32_t>(), *large_list = warp_list + ncl;
    int32_t *t16_list = large_list + ncl, *t32_list = t16_list + ncl;
    int32_t *counts = t32_list + ncl;
    JET_CUDA_TRY(cudaMemsetAsync(counts, 0, 16, s));
    JET_CUDA_TRY(launch_pdl(k_coarse_vw, grid_for(nc, kTB, 8192), kTB, 0, s, true, (int32_t)nc, (const int32_t *)crep,
                            (const int32_t *)mate, g.vw, vwcb.as<int32_t>(), warp_list, large_list, t16_list, t32_list,
                            counts, (const int64_t *)boff, (const int64_t *)totp));
    JET_TRY(dev_alloc(tadjb, (size_t)std::max<int64_t>(btotal, 1) * 4, s));
    JET_TRY(dev_alloc(twb, (size_t)std::max<int64_t>(btotal, 1) * 4, s));
    JET_TRY(dev_alloc(cntb, (size_t)std::max<int64_t>(nc, 1) * 4, s));
    int gl = num_sms() * 8;
    const int gwarp = std::min(gl, grid_for(nc, kTB / 32));
    const int glarge = std::min(num_sms() * 4, (int)std::max<int64_t>(1, nc));
    const int gthread = std::min(gl, grid_for(nc, kTB));
    int32_t *tadj = tadjb.as<int32_t>(), *tw = twb.as<int32_t>(), *cnt = cntb.as<int32_t>();
    {
        const int32_t *cm = cmap, *mt = mate, *cr = crep, *cts = counts;
        const int64_t *bo = boff;
        if (g.ew) {
            JET_CUDA_TRY(launch_pdl(k_contract_thread<true, 16>, gthread, kTB, 0, s, true, g, cm, mt, cr, (const int32_t *)t16_list, cts, bo, tadj, tw, cnt));
            JET_CUDA_TRY(launch_pdl(k_contract_thread<true, 32>, gthread, kTB, 0, s, true, g, cm, mt, cr, (const int32_t *)t32_list, cts, bo, tadj, tw, cnt));
            JET_CUDA_TRY(launch_pdl(k_contract_warp<true>, gwarp, kTB, 0, s, true, g, cm, mt, cr, (const int32_t *)warp_list, cts, bo, tadj, tw, cnt));
            JET_CUDA_TRY(launch_pdl(k_contract_large<true>, glarge, kTB, 0, s, true, g, cm, mt, cr, (const int32_t *)large_list, cts, bo, tadj, tw, cnt));
        } else {
            JET_CUDA_TRY(launch_pdl(k_contract_thread<false, 16>, gthread, kTB, 0, s, true, g, cm, mt, cr, (const int32_t *)t16_list, cts, bo, tadj, tw, cnt));
            JET_CUDA_TRY(launch_pdl(k_contract_thread<false, 32>, gthread, kTB, 0, s, true, g, cm, mt, cr, (const int32_t *)t32_list, cts, bo, tadj, tw, cnt));
            JET_CUDA_TRY(launch_pdl(k_contract_warp<false>, gwarp, kTB, 0, s, true, g, cm, mt, cr, (const int32_t *)warp_list, cts, bo, tadj, tw, cnt));
            JET_CUDA_TRY(launch_pdl(k_contract_large<false>, glarge, kTB, 0, s, true, g, cm, mt, cr, (const int32_t *)large_list, cts, bo, tadj, tw, cnt));
        }
    }
    c.launches += 4;
    if (nhub > 0) {
        // hub rows: all their entries in one stable radix sort by (rank, coarse id)
        JET_TRY(dev_alloc(hsortb, sort_scratch_bytes(htotal), s));
        SortScratch sc;
        sort_scratch_carve(hsortb.as<char>(), htotal, sc);
        JET_TRY(dev_alloc(hubcb, (size_t)nhub * 4, s));
        JET_TRY(dev_alloc(hsb, (size_t)htotal * 8 + (size_t)(scan_tiles_for(htotal) + 1) * 8 + 64, s));
        int32_t *hub_c = hubcb.as<int32_t>();
        int64_t *hs = hsb.as<int64_t>(), *hs_scr = hs + htotal;
        if (g.ew) k_hub_fill<true><<<glarge, kTB, 0, s>>>(g, cmap, mate, crep, large_list, counts, hoff, hrank, sc.key[0], sc.val[0], hub_c);
        else k_hub_fill<false><<<glarge, kTB, 0, s>>>(g, cmap, mate, crep, large_list, counts, hoff, hrank, sc.key[0], sc.val[0], hub_c);
        c.launches += 1;
        JET_CUDA_TRY(cudaGetLastError());
        int which = 0;
        JET_TRY(sort_pairs(c, sc, htotal, 32 + bits_for(nhub - 1), &which));
        JET_TRY(device_exscan(HubHead{sc.key[which], hub_c}, htotal, hs, totp + 4, hs_scr, s));
        k_hub_emit<<<std::min(gl, grid_for(htotal, kTB)), kTB, 0, s>>>(htotal, sc.key[which], sc.val[which], hub_c, hoff, hs,
                                                                      boff, tadj, tw);
        k_hub_rowcnt<<<grid_for(nhub, kTB, 1024), kTB, 0, s>>>(nhub, htotal, hub_c, hoff, hs, totp + 4, cnt);
        c.launches += 5;
    }
    JET_CUDA_TRY(cudaGetLastError());
    // coarse xadj
    DevBuf xcb, exb;
    JET_TRY(dev_alloc(xcb, (size_t)(nc + 1) * 8, s));
    JET_TRY(dev_alloc(exb, (size_t)std::max<int64_t>(nc, 1) * 8, s));
    c.launches += 3;
    JET_TRY(device_exscan(CountVal{cntb.as<int32_t>()}, nc, exb.as<int64_t>(), totp + 2, scan_scr.as<int64_t>(), s));
    JET_CUDA_TRY(launch_pdl(k_finish_xadj, grid_for(nc + 1, kTB, 8192), kTB, 0, s, true, (int32_t)nc,
                            (const int64_t *)exb.as<int64_t>(), (const int64_t *)(totp + 2), xcb.as<int64_t>()));
    c.launches += 1;
    JET_CUDA_TRY(cudaMemcpyAsync(c.pinned, totp + 2, 8, cudaMemcpyDeviceToHost, s));
    JET_CUDA_TRY(cudaStreamSynchronize(s));
    int64_t nnzc = c.pinned[0];
    DevBuf adjcb, ewcb;
    JET_TRY(dev_alloc(adjcb, (size_t)std::max<int64_t>(nnzc, 1) * 4, s));
    JET_TRY(dev_alloc(ewcb, (size_t)std::max<int64_t>(nnzc, 1) * 4, s));
    JET_CUDA_TRY(launch_pdl(k_copy_long, glarge, kTB, 0, s, true, (const int32_t *)large_list, (const int32_t *)counts,
                            (const int64_t *)boff, (const int64_t *)xcb.as<int64_t>(), (const int32_t *)tadjb.as<int32_t>(),
                            (const int32_t *)twb.as<int32_t>(), adjcb.as<int32_t>(), ewcb.as<int32_t>()));
    c.launches += 1;
    JET_CUDA_TRY(launch_pdl(k_copy_rows, std::min(gl, grid_for(nc, kTB / kCopyLanes)), kTB, 0, s, true, (int32_t)nc,
                            (const int64_t *)boff, (const int64_t *)totp, (const int64_t *)xcb.as<int64_t>(),
                            (const int32_t *)tadjb.as<int32_t>(), (const int32_t *)twb.as<int32_t>(), adjcb.as<int32_t>(),
                            ewcb.as<int32_t>()));
    JET_CUDA_TRY(cudaGetLastError());
    int32_t i = h->levels;
    h->cmap[i - 1] = cmap;
    h->n[i] = (int32_t)nc;
    h->nnz[i] = nnzc;
    h->xadj[i] = xcb.as<int64_t>();
    h->adj[i] = adjcb.as<int32_t>();
    h->vw[i] = vwcb.as<int32_t>();
    h->ew[i] = ewcb.as<int32_t>();
    h->levels = i + 1;
    h->bufs.push_back(std::move(cmapb));
    h->bufs.push_back(std::move(xcb));
    h->bufs.push_back(std::move(adjcb));
    h->bufs.push_back(std::move(vwcb));
    h->bufs.push_back(std::move(ewcb));
    return JET_OK;   // the next level's work follows in stream order
}

__global__ void k_ones(int32_t *p, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) p[i] = 1;
}

// MLCoarsen of Alg. 1 (see jet_coarsen in jet.h for the stop rules).
int coarsen(Ctx &c, const DGraph &g0, int32_t k, uint64_t seed, jet_hier *h) {
    cudaStream_t s = c.stream;
    h->levels = 1;
    h->k = k;
    h->n[0] = g0.n;
    h->nnz[0] = g0.nnz;
    h->xadj[0] = g0.xadj;
    h->adj[0] = g0.adj;
    h->ew[0] = g0.ew;
    if (g0.vw) {
        h->vw[0] = g0.vw;
    } else {
        DevBuf ones;
        JET_TRY(dev_alloc(ones, (size_t)std::max<int32_t>(g0.n, 1) * 4, s));
        if (g0.n > 0) k_ones<<<grid_for(g0.n, kTB, 8192), kTB, 0, s>>>(ones.as<int32_t>(), g0.n);
        if (g0.n > 0) c.launches += 1;
        JET_CUDA_TRY(cudaGetLastError());
        h->vw[0] = ones.as<int32_t>();
        h->bufs.push_back(std::move(ones));
    }
    int32_t T = c.opt.coarsen_target > 0 ? c.opt.coarsen_target : std::max(8 * k, 256);
    int32_t maxl = std::min<int32_t>(c.opt.max_levels, JET_MAX_LEVELS);
    while (h->n[h->levels - 1] > T && h->levels < maxl) {
        int32_t i = h->levels - 1;
        DGraph gi;
        gi.n = h->n[i]; gi.nnz = h->nnz[i]; gi.xadj = h->xadj[i]; gi.adj = h->adj[i]; gi.vw = h->vw[i]; gi.ew = h->ew[i];
        bool stalled = false;
        JET_TRY(coarsen_level(c, gi, seed, i, h, stalled));
        if (stalled) break;
    }
    return JET_OK;
}

// ---------------------------------------------------------------------------
// projection (Alg. 1 ProjectPartition)
// ---------------------------------------------------------------------------
__global__ void k_project(int32_t n, const int32_t *cmap, const int32_t *pc, int32_t *pf) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        pf[v] = pc[cmap[v]];
}

int project(Ctx &c, int32_t n_fine, const int32_t *cmap, const int32_t *coarse_part, int32_t *fine_part) {
    if (n_fine > 0) k_project<<<grid_for(n_fine, kTB, 8192), kTB, 0, c.stream>>>(n_fine, cmap, coarse_part, fine_part);
    if (n_fine > 0) c.launches += 1;
    JET_CUDA_TRY(cudaGetLastError());
    return JET_OK;
}

}  // namespace jet
