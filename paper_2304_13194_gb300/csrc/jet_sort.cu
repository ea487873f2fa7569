// Stable LSD radix sort of (64-bit key, int32 value) pairs, device-wide:
// per tile of kSortTile elements a digit histogram, one exclusive scan over
// all (digit, tile) counts in digit-major order, then a scatter that keeps
// the input order among equal digits (chunk by chunk, warp by warp, lane by
// lane).  Used where the method orders vertices by a key with ties broken by
// vertex id: the values enter in id order.
#include "jet_internal.cuh"

#include <algorithm>

namespace jet {

namespace {

constexpr int kSortItems = 8;                     // elements per thread and tile
constexpr int kSortTile = kTB * kSortItems;       // elements per tile
constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;

// Digit histogram of each tile, stored digit-major: hist[d * ntiles + tile].
__global__ void __launch_bounds__(kTB) k_sort_hist(const uint64_t *key, int64_t n, int shift, int64_t ntiles,
                                                   int64_t *hist) {
    __shared__ int32_t h[kRadix];
    for (int i = threadIdx.x; i < kRadix; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
#pragma unroll
    for (int i = 0; i < kSortItems; ++i) {
        int64_t e = base + (int64_t)i * blockDim.x + threadIdx.x;
        if (e < n) atomicAdd(&h[(int)((key[e] >> shift) & (kRadix - 1))], 1);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kRadix; d += blockDim.x) hist[(int64_t)d * ntiles + blockIdx.x] = h[d];
}

struct HistVal {
    const int64_t *hist;
    __device__ int64_t operator()(int64_t i) const { return hist[i]; }
};

// Scatter of one tile, chunk after chunk of blockDim elements in index order;
// inside a chunk, warp after warp and lane after lane: the rank of an element
// among the tile's equal digits keeps the input order (stable).
__global__ void __launch_bounds__(kTB) k_sort_scatter(const uint64_t *key_in, const int32_t *val_in, uint64_t *key_out,
                                                      int32_t *val_out, int64_t n, int shift, int64_t ntiles,
                                                      const int64_t *off) {
    __shared__ int32_t wcnt[kTB / 32][kRadix];    // per-warp digit counts, then warp prefixes
    __shared__ int32_t ctot[kRadix];              // this chunk's count per digit
    __shared__ int64_t run[kRadix];               // tile offset + elements placed so far, per digit
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int nwarps = blockDim.x >> 5;
    for (int d = threadIdx.x; d < kRadix; d += blockDim.x) run[d] = off[(int64_t)d * ntiles + blockIdx.x];
    for (int i = 0; i < kSortItems; ++i) {
        for (int t = threadIdx.x; t < nwarps * kRadix; t += blockDim.x) wcnt[t / kRadix][t % kRadix] = 0;
        __syncthreads();
        const int64_t e = base + (int64_t)i * blockDim.x + threadIdx.x;
        const bool ok = e < n;
        const uint64_t k = ok ? key_in[e] : 0;
        const int32_t v = ok ? val_in[e] : 0;
        const int d = ok ? (int)((k >> shift) & (kRadix - 1)) : -1;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int rank = __popc(peers & lt);
        if (ok && rank == 0) wcnt[warp][d] = __popc(peers);
        __syncthreads();
        for (int dd = threadIdx.x; dd < kRadix; dd += blockDim.x) {
            int32_t acc = 0;
            for (int w = 0; w < nwarps; ++w) {
                int32_t c = wcnt[w][dd];
                wcnt[w][dd] = acc;
                acc += c;
            }
            ctot[dd] = acc;
        }
        __syncthreads();
        if (ok) {
            const int64_t pos = run[d] + wcnt[warp][d] + rank;
            key_out[pos] = k;
            val_out[pos] = v;
        }
        __syncthreads();
        for (int dd = threadIdx.x; dd < kRadix; dd += blockDim.x) run[dd] += ctot[dd];
        __syncthreads();
    }
}

}  // namespace

int bits_for(int64_t x) {
    int b = 0;
    while (b < 63 && (x >> b) != 0) ++b;
    return b;
}

size_t sort_scratch_bytes(int64_t n) {
    const size_t nn = (size_t)std::max<int64_t>(n, 1);
    const int64_t ntiles = (n + kSortTile - 1) / kSortTile;
    const int64_t nhist = std::max<int64_t>(ntiles, 1) * kRadix;
    auto a256 = [](size_t x) { return (x + 255) & ~size_t(255); };
    return 2 * a256(nn * 8) + 2 * a256(nn * 4) + 2 * a256((size_t)nhist * 8) +
           a256((size_t)(scan_tiles_for(nhist) + 1) * 8) + a256(16);
}

void sort_scratch_carve(char *p, int64_t n, SortScratch &s) {
    const size_t nn = (size_t)std::max<int64_t>(n, 1);
    const int64_t ntiles = (n + kSortTile - 1) / kSortTile;
    const int64_t nhist = std::max<int64_t>(ntiles, 1) * kRadix;
    auto a256 = [](size_t x) { return (x + 255) & ~size_t(255); };
    auto take = [&](size_t b) { char *r = p; p += a256(b); return r; };
    s.key[0] = reinterpret_cast<uint64_t *>(take(nn * 8));
    s.key[1] = reinterpret_cast<uint64_t *>(take(nn * 8));
    s.val[0] = reinterpret_cast<int32_t *>(take(nn * 4));
    s.val[1] = reinterpret_cast<int32_t *>(take(nn * 4));
    s.hist = reinterpret_cast<int64_t *>(take((size_t)nhist * 8));
    s.off = reinterpret_cast<int64_t *>(take((size_t)nhist * 8));
    s.scan = reinterpret_cast<int64_t *>(take((size_t)(scan_tiles_for(nhist) + 1) * 8));
    s.total = reinterpret_cast<int64_t *>(take(16));
}

int sort_pairs(Ctx &c, SortScratch &sc, int64_t n, int kbits, int *which) {
    cudaStream_t s = c.stream;
    *which = 0;
    if (n <= 0) return JET_OK;
    const int64_t ntiles = (n + kSortTile - 1) / kSortTile;
    const int64_t nhist = ntiles * kRadix;
    int cur = 0;
    for (int shift = 0; shift < kbits; shift += kRadixBits) {
        k_sort_hist<<<(unsigned)ntiles, kTB, 0, s>>>(sc.key[cur], n, shift, ntiles, sc.hist);
        JET_TRY(device_exscan(HistVal{sc.hist}, nhist, sc.off, sc.total, sc.scan, s));
        k_sort_scatter<<<(unsigned)ntiles, kTB, 0, s>>>(sc.key[cur], sc.val[cur], sc.key[cur ^ 1], sc.val[cur ^ 1], n, shift,
                                                        ntiles, sc.off);
        c.launches += 5;
        JET_CUDA_TRY(cudaGetLastError());
        cur ^= 1;
    }
    *which = cur;
    return JET_OK;
}

}  // namespace jet
