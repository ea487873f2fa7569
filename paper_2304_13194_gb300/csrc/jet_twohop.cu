// Two-hop matching (Sec. 3.1), added to heavy-edge matching when more than
// 25% of the vertices are still unmatched: leaves (degree-1 vertices with
// the same neighbour), twins (vertices with the same neighbourhood) and
// relatives (vertices with the same matchmaker: their lowest-id neighbour
// that is already matched and has degree <= kMatchmakerMaxDeg).  The stages
// run in that order, each only while 4u > n.  Inside a group the vertices
// pair in ascending id: first with second, third with fourth, ...
//
// Per stage, device-wide: one key per vertex (a sentinel for non-candidates;
// one warp per vertex so that hubs do not stall a thread), a stable radix
// sort of (key, vertex) with the vertices entering in id order, the group
// heads by a scan, and the pairs of even rank with their successor.
#include "jet_internal.cuh"

#include <algorithm>

namespace jet {

namespace {

constexpr uint64_t kTwinSalt = 0x2545F4914F6CDD1DULL;
constexpr uint64_t kTwinDeg = 0x9FB21C651E98DF25ULL;

__global__ void k_count_unmatched(int32_t n, const int32_t *mate, int64_t *out) {
    __shared__ long long red[40];
    long long c = 0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        c += mate[v] < 0;
    c = block_sum_i64(c, red);
    if (threadIdx.x == 0 && c) atomic_add_i64(out, c);
}

// Stage keys, one warp per vertex: the neighbour of a leaf; the order-free
// neighbourhood hash of a twin candidate (wrapping sum, so the lane order does
// not matter); the lowest eligible matchmaker of a relative.
__global__ void __launch_bounds__(kTB) k_two_hop_keys(DGraph g, int stage, const int32_t *mate, uint64_t sentinel,
                                                      uint64_t *key, int32_t *val) {
    const int warps = blockDim.x >> 5;
    const unsigned lane = lane_id();
    for (int64_t v = (int64_t)blockIdx.x * warps + (threadIdx.x >> 5); v < g.n; v += (int64_t)gridDim.x * warps) {
        uint64_t k = sentinel;
        if (mate[v] < 0) {
            const int64_t beg = ld_xadj(g.xadj, v), end = ld_xadj(g.xadj, v + 1);
            if (stage == 0) {
                if (end - beg == 1) k = (uint64_t)(uint32_t)__ldg(g.adj + beg);
            } else if (stage == 1) {
                unsigned long long h = 0;
                for (int64_t j = beg + lane; j < end; j += 32)
                    h += splitmix64((uint64_t)(uint32_t)__ldg(g.adj + j) ^ kTwinSalt);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) h += __shfl_xor_sync(0xffffffffu, h, o);
                h += splitmix64((uint64_t)(end - beg) ^ kTwinDeg);
                k = h == ~0ULL ? ~0ULL - 1 : h;
            } else {
                int32_t best = INT32_MAX;
                for (int64_t j = beg + lane; j < end; j += 32) {
                    int32_t u = __ldg(g.adj + j);
                    if (u < best && mate[u] >= 0 && ld_xadj(g.xadj, (int64_t)u + 1) - ld_xadj(g.xadj, u) <= kMatchmakerMaxDeg)
                        best = u;
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    int32_t t = __shfl_xor_sync(0xffffffffu, best, o);
                    best = t < best ? t : best;
                }
                if (best != INT32_MAX) k = (uint64_t)(uint32_t)best;
            }
        }
        if (lane == 0) {
            key[v] = k;
            val[v] = (int32_t)v;
        }
    }
}

// 1 at the first position of each group of equal (non-sentinel) keys.
struct GroupHead {
    const uint64_t *key;
    uint64_t sentinel;
    __device__ int64_t operator()(int64_t i) const {
        uint64_t k = key[i];
        return k != sentinel && (i == 0 || key[i - 1] != k) ? 1 : 0;
    }
};

__global__ void k_group_starts(int64_t n, const uint64_t *key, uint64_t sentinel, const int64_t *heads_before,
                               int64_t *start) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t k = key[i];
        if (k != sentinel && (i == 0 || key[i - 1] != k)) start[heads_before[i]] = i;
    }
}

// Position i of a group pairs with i + 1 when its rank in the group is even
// and i + 1 is in the same group.
__global__ void k_pair_groups(int64_t n, const uint64_t *key, const int32_t *val, uint64_t sentinel,
                              const int64_t *heads_before, const int64_t *start, int32_t *mate) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i + 1 < n; i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t k = key[i];
        if (k == sentinel || key[i + 1] != k) continue;
        bool head = i == 0 || key[i - 1] != k;
        int64_t gid = heads_before[i] + (head ? 1 : 0) - 1;
        if (((i - start[gid]) & 1) == 0) {
            int32_t a = val[i], b = val[i + 1];
            mate[a] = b;
            mate[b] = a;
        }
    }
}

}  // namespace

int two_hop(Ctx &c, const DGraph &g, int32_t *mate, int64_t added[3]) {
    cudaStream_t s = c.stream;
    added[0] = added[1] = added[2] = 0;
    const int64_t n = g.n;
    if (n == 0) return JET_OK;
    const size_t nn = (size_t)n;
    auto a256 = [](size_t x) { return (x + 255) & ~size_t(255); };
    // heads_before, start | scan tiles | counter | sort scratch
    const size_t bytes = 2 * a256(nn * 8) + a256((size_t)(scan_tiles_for(n) + 1) * 8) + a256(16) + sort_scratch_bytes(n);
    DevBuf buf;
    JET_TRY(dev_alloc(buf, bytes, s));
    char *p = buf.as<char>();
    auto take = [&](size_t b) { char *r = p; p += a256(b); return r; };
    int64_t *hb = reinterpret_cast<int64_t *>(take(nn * 8));
    int64_t *start = reinterpret_cast<int64_t *>(take(nn * 8));
    int64_t *scan_scr = reinterpret_cast<int64_t *>(take((size_t)(scan_tiles_for(n) + 1) * 8));
    int64_t *cnt = reinterpret_cast<int64_t *>(take(16));
    SortScratch sc;
    sort_scratch_carve(p, n, sc);
    const int gv = std::min(num_sms() * 8, grid_for(n, kTB));
    const int gw = std::min(num_sms() * 8, grid_for(n, kTB / 32));
    auto unmatched = [&](int64_t &u) -> int {
        JET_CUDA_TRY(cudaMemsetAsync(cnt, 0, 8, s));
        k_count_unmatched<<<gv, kTB, 0, s>>>((int32_t)n, mate, cnt);
        c.launches += 1;
        JET_CUDA_TRY(cudaGetLastError());
        JET_CUDA_TRY(cudaMemcpyAsync(c.pinned, cnt, 8, cudaMemcpyDeviceToHost, s));
        JET_CUDA_TRY(cudaStreamSynchronize(s));
        u = c.pinned[0];
        return JET_OK;
    };
    int64_t un = 0;
    JET_TRY(unmatched(un));
    for (int stage = 0; stage < 3; ++stage) {
        if (4 * un <= n) break;
        // keys below n for leaves and relatives (sentinel n), any 64-bit value for twins
        const uint64_t sentinel = stage == 1 ? ~0ULL : (uint64_t)n;
        const int kbits = stage == 1 ? 64 : bits_for(n);
        k_two_hop_keys<<<gw, kTB, 0, s>>>(g, stage, mate, sentinel, sc.key[0], sc.val[0]);
        c.launches += 1;
        JET_CUDA_TRY(cudaGetLastError());
        int which = 0;
        JET_TRY(sort_pairs(c, sc, n, kbits, &which));
        const uint64_t *key = sc.key[which];
        const int32_t *val = sc.val[which];
        JET_TRY(device_exscan(GroupHead{key, sentinel}, n, hb, cnt + 1, scan_scr, s));
        k_group_starts<<<gv, kTB, 0, s>>>(n, key, sentinel, hb, start);
        k_pair_groups<<<gv, kTB, 0, s>>>(n, key, val, sentinel, hb, start, mate);
        c.launches += 5;
        JET_CUDA_TRY(cudaGetLastError());
        int64_t un2 = 0;
        JET_TRY(unmatched(un2));
        added[stage] = un - un2;
        un = un2;
    }
    return JET_OK;
}

}  // namespace jet
