// Learned initial partition of the coarsest graph.  The paper partitions the
// coarsest graph with Metis (Sec. 3); this build offers a message-passing
// network's proposal next to its greedy initial partition and keeps whichever
// gives the smaller exact cut after full Jet refinement (Alg. 1 uncoarsening).
//
// Network (rows are vertices; H0 = the 16 features, widths 16 -> 64 -> 64 -> 64):
//   A_l = mean over the neighbours of H_{l-1}
//   H_l = relu([H_{l-1}, A_l] W_l + b_l),  l = 1, 2, 3
//   logits = H_3 Wo + bo,  loss = mean softmax cross-entropy.
// Kernels:
//   k_agg_fwd / k_agg_bwd   mean aggregation over CSR and its transpose, one
//                           warp per vertex (gather form both ways: the
//                           transpose reads each neighbour's 1/deg share, so
//                           no atomics and a fixed summation order);
//   k_gemm_rows             row-parallel C = A B (+ bias, relu): 64 rows per
//                           block, A and B staged in shared memory as bf16,
//                           mma.sync m16n8k16 with float32 accumulators;
//   k_gemm_tn + k_tn_reduce weight gradients A^T B over all rows: each block
//                           reduces a fixed 512-row chunk on the tensor cores,
//                           the partial sums are added in block order
//                           (deterministic, no atomics);
//   k_softmax_ce, k_adam, the feature kernels and the balanced decode.
// All sizes here are small (the coarsest graph has a few hundred to a few
// thousand vertices, a training batch some tens of thousands): the dense
// layers are K <= 256, N <= 256 products whose cost is launch latency, so
// they use the warp-level mma.sync path rather than tcgen05 with TMEM, whose
// setup (TMEM allocation, descriptors, mbarriers) would exceed the work.
#include "jet_internal.cuh"

#include <cuda_bf16.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <new>
#include <thread>

namespace jet {

namespace {

constexpr int kF = JET_LIP_FEATURES;
constexpr int kHd = JET_LIP_HIDDEN;
constexpr int kLayers = 3;
constexpr int kGemmBM = 64;        // rows per block of k_gemm_rows (4 warps x 16 rows)
constexpr int kTnRows = 64;        // rows staged per step of k_gemm_tn
constexpr int kTnChunk = 256;      // rows per block of k_gemm_tn (a constant: the summation order is fixed)
constexpr int kTnWarps = 8;
constexpr int kTnMaxTiles = 16;    // 16x8 output tiles per warp of k_gemm_tn
constexpr int kGemmSmemMax = 100 * 1024;

int din_of(int l) { return l == 0 ? kF : kHd; }
int pad16(int x) { return (x + 15) & ~15; }

struct Offsets {
    int64_t W[kLayers + 1], b[kLayers + 1], total;
};

Offsets offsets(int32_t k) {
    Offsets o;
    int64_t p = 0;
    for (int l = 0; l < kLayers; ++l) {
        o.W[l] = p;
        p += (int64_t)2 * din_of(l) * kHd;
        o.b[l] = p;
        p += kHd;
    }
    o.W[kLayers] = p;
    p += (int64_t)kHd * k;
    o.b[kLayers] = p;
    p += k;
    o.total = p;
    return o;
}

// ---- tensor-core tile ------------------------------------------------------
// D (16x8, f32) += A (16x16, bf16, row-major) B (16x8, bf16, column-major).
// Fragments (g = lane / 4, t = lane % 4): a0 rows g / cols 2t..2t+1, a1 rows
// g+8, a2 rows g / cols 2t+8.., a3 rows g+8 / cols 2t+8..; b0 rows 2t..2t+1 /
// col g, b1 rows 2t+8..; d0,d1 row g / cols 2t, 2t+1, d2,d3 row g+8.
__device__ __forceinline__ void mma_16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Two consecutive bf16 (the lower index in the low half).
__device__ __forceinline__ uint32_t ld_pair(const __nv_bfloat16 *p) { return *reinterpret_cast<const uint32_t *>(p); }

// C = A B over M rows, bf16 operands rounded from float32 as they are staged,
// float32 accumulation.  A(r, kk) = A[r*lda + kk] for kk < Kv; B(kk, c) =
// B[kk*ldb + c], or B[c*ldb + kk] with TRANS_B, for kk < Kv and c < Nv;
// zero beyond.  Kp (multiple of 16) and Np (multiple of 8, <= 256) are the
// padded sizes.  For c < Nv: Y[r*ldy + c] = acc + bias[c] (when Y), R[r*ldr
// + c] = max(acc + bias[c], 0) (when R).  Block: 128 threads, 64 rows.
template <bool TRANS_B>
__global__ void __launch_bounds__(128) k_gemm_rows(int32_t M, int Kp, int Kv, int Np, int Nv, const float *A, int lda,
                                                   const float *B, int ldb, const float *bias, float *Y, int ldy,
                                                   float *R, int ldr) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int sk = Kp + 8;                                                  // staged row stride (bf16)
    __nv_bfloat16 *As = reinterpret_cast<__nv_bfloat16 *>(smem_raw);      // [kGemmBM][sk]
    __nv_bfloat16 *Bt = As + kGemmBM * sk;                                  // [Np][sk]: B transposed
    const int64_t r0 = (int64_t)blockIdx.x * kGemmBM;
    for (int i = threadIdx.x; i < kGemmBM * Kp; i += blockDim.x) {
        const int r = i / Kp, kk = i - r * Kp;
        const float x = (r0 + r < M && kk < Kv) ? A[(r0 + r) * lda + kk] : 0.f;
        As[r * sk + kk] = __float2bfloat16_rn(x);
    }
    for (int i = threadIdx.x; i < Np * Kp; i += blockDim.x) {
        int c, kk;
        if (TRANS_B) { c = i / Kp; kk = i - c * Kp; }   // walk the source contiguously
        else { kk = i / Np; c = i - kk * Np; }
        float x = 0.f;
        if (kk < Kv && c < Nv) x = TRANS_B ? B[(int64_t)c * ldb + kk] : B[(int64_t)kk * ldb + c];
        Bt[c * sk + kk] = __float2bfloat16_rn(x);
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int rw = warp * 16;
    for (int nc = 0; nc < Np; nc += 64) {
        const int nt = min(8, (Np - nc) >> 3);
        float acc[8][4];
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
        for (int k0 = 0; k0 < Kp; k0 += 16) {
            uint32_t a[4];
            a[0] = ld_pair(As + (rw + g) * sk + k0 + 2 * t);
            a[1] = ld_pair(As + (rw + g + 8) * sk + k0 + 2 * t);
            a[2] = ld_pair(As + (rw + g) * sk + k0 + 2 * t + 8);
            a[3] = ld_pair(As + (rw + g + 8) * sk + k0 + 2 * t + 8);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                if (j < nt) {
                    const __nv_bfloat16 *bp = Bt + (nc + j * 8 + g) * sk + k0 + 2 * t;
                    mma_16816(acc[j], a, ld_pair(bp), ld_pair(bp + 8));
                }
            }
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            if (j >= nt) continue;
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const int64_t r = r0 + rw + g + (h >> 1) * 8;
                const int col = nc + j * 8 + 2 * t + (h & 1);
                if (r < M && col < Nv) {
                    const float y = acc[j][h] + (bias ? bias[col] : 0.f);
                    if (Y) Y[r * ldy + col] = y;
                    if (R) R[r * ldr + col] = fmaxf(y, 0.f);
                }
            }
        }
    }
}

// Partial weight gradients over the rows [blockIdx.x * kTnChunk, + kTnChunk):
// P[blk][i*Np + c] = sum_r A(r, i) B(r, c) with bf16 operands and float32
// accumulation (i < Kp, c < Np; A(r, i) = A[r*lda + i] for i < Kv, B(r, c) =
// B[r*ldb + c] for c < Nv, zero beyond), and CS[blk][c] = sum_r B(r, c) in
// float32: thread t stages the columns t % 64 + 64 g of the rows t / 64 + 4 j
// and keeps their running sums, which the four row classes then add in a
// fixed order.  Requires (Kp/16) (Np/8) <= kTnWarps * kTnMaxTiles, Np <= 256
// and 256 threads.
__global__ void __launch_bounds__(256) k_gemm_tn(int32_t M, int Kp, int Kv, int Np, int Nv, const float *A, int lda,
                                                 const float *B, int ldb, float *P, float *CS) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int sr = kTnRows + 8;
    __nv_bfloat16 *At = reinterpret_cast<__nv_bfloat16 *>(smem_raw);   // [Kp][sr]
    __nv_bfloat16 *Bt = At + Kp * sr;                                    // [Np][sr]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int mt = Kp >> 4, ntiles = mt * (Np >> 3);
    float acc[kTnMaxTiles][4];
#pragma unroll
    for (int q = 0; q < kTnMaxTiles; ++q) acc[q][0] = acc[q][1] = acc[q][2] = acc[q][3] = 0.f;
    const int64_t c0 = (int64_t)blockIdx.x * kTnChunk;
    const int64_t c1 = min((int64_t)M, c0 + kTnChunk);
    const int tc = threadIdx.x & 63, tr = threadIdx.x >> 6;   // column lane, row class (0..3)
    float cs[4] = {0.f, 0.f, 0.f, 0.f};
    for (int64_t r0 = c0; r0 < c1; r0 += kTnRows) {
        __syncthreads();
        for (int i = threadIdx.x; i < kTnRows * Kp; i += blockDim.x) {
            const int r = i / Kp, kk = i - r * Kp;
            const float x = (r0 + r < c1 && kk < Kv) ? A[(r0 + r) * lda + kk] : 0.f;
            At[kk * sr + r] = __float2bfloat16_rn(x);
        }
#pragma unroll
        for (int gcol = 0; gcol < 4; ++gcol) {
            const int c = tc + 64 * gcol;
            if (c < Np) {
                for (int r = tr; r < kTnRows; r += 4) {
                    const float x = (r0 + r < c1 && c < Nv) ? B[(r0 + r) * ldb + c] : 0.f;
                    cs[gcol] += x;
                    Bt[c * sr + r] = __float2bfloat16_rn(x);
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < kTnMaxTiles; ++q) {
            const int tile = warp + q * kTnWarps;
            if (tile < ntiles) {
                const int i0 = (tile % mt) * 16, n0 = (tile / mt) * 8;
#pragma unroll
                for (int k0 = 0; k0 < kTnRows; k0 += 16) {
                    uint32_t a[4];
                    a[0] = ld_pair(At + (i0 + g) * sr + k0 + 2 * t);
                    a[1] = ld_pair(At + (i0 + g + 8) * sr + k0 + 2 * t);
                    a[2] = ld_pair(At + (i0 + g) * sr + k0 + 2 * t + 8);
                    a[3] = ld_pair(At + (i0 + g + 8) * sr + k0 + 2 * t + 8);
                    const __nv_bfloat16 *bp = Bt + (n0 + g) * sr + k0 + 2 * t;
                    mma_16816(acc[q], a, ld_pair(bp), ld_pair(bp + 8));
                }
            }
        }
    }
    float *Pb = P + (int64_t)blockIdx.x * Kp * Np;
#pragma unroll
    for (int q = 0; q < kTnMaxTiles; ++q) {
        const int tile = warp + q * kTnWarps;
        if (tile < ntiles) {
            const int i0 = (tile % mt) * 16, n0 = (tile / mt) * 8;
#pragma unroll
            for (int h = 0; h < 4; ++h) Pb[(i0 + g + (h >> 1) * 8) * Np + n0 + 2 * t + (h & 1)] = acc[q][h];
        }
    }
    // column sums: the four row classes in order
    __syncthreads();
    float *red = reinterpret_cast<float *>(smem_raw);   // [4][256], the staging tiles are no longer read
#pragma unroll
    for (int gcol = 0; gcol < 4; ++gcol) red[tr * 256 + tc + 64 * gcol] = cs[gcol];
    __syncthreads();
    for (int c = threadIdx.x; c < Np; c += blockDim.x)
        CS[(int64_t)blockIdx.x * Np + c] = ((red[c] + red[256 + c]) + red[512 + c]) + red[768 + c];
}

// gW[i*Nv + c] = sum over blocks b (in order) of P[b][i*Np + c] (i < Kv,
// c < Nv); gb[c] = sum over b of CS[b][c].
__global__ void k_tn_reduce(int nb, int Kp, int Kv, int Np, int Nv, const float *P, const float *CS, float *gW,
                            float *gb) {
    const int64_t total = (int64_t)Kv * Nv;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total + Nv;
         e += (int64_t)gridDim.x * blockDim.x) {
        float s = 0.f;
        if (e < total) {
            const int64_t i = e / Nv, c = e - i * Nv;
            for (int b = 0; b < nb; ++b) s += P[(int64_t)b * Kp * Np + i * Np + c];
            gW[e] = s;
        } else {
            const int64_t c = e - total;
            for (int b = 0; b < nb; ++b) s += CS[(int64_t)b * Np + c];
            gb[c] = s;
        }
    }
}

// ---- aggregation over CSR ---------------------------------------------------
// Z[v][0:d] = H[v] (skipped when H is Z itself), Z[v][d:2d] = mean of H[u]
// over the neighbours u of v (0 without neighbours).  H row stride ldh, Z
// row stride 2d.  One warp per vertex, lanes over the d columns.
__global__ void __launch_bounds__(kTB) k_agg_fwd(DGraph g, int d, const float *H, int ldh, float *Z) {
    const int warps = blockDim.x >> 5;
    const int lane = threadIdx.x & 31;
    const int ldz = 2 * d;
    for (int64_t v = (int64_t)blockIdx.x * warps + (threadIdx.x >> 5); v < g.n; v += (int64_t)gridDim.x * warps) {
        const int64_t beg = g.xadj[v], end = g.xadj[v + 1];
        for (int c = lane; c < d; c += 32) {
            float s = 0.f;
            for (int64_t j = beg; j < end; ++j) s += H[(int64_t)g.adj[j] * ldh + c];
            if (H != Z) Z[v * ldz + c] = H[v * ldh + c];
            Z[v * ldz + d + c] = end > beg ? s / (float)(end - beg) : 0.f;
        }
    }
}

// Transpose of the aggregation plus the direct half:
// dH[u][c] = dZ[u][c] + sum over neighbours v of dZ[v][d + c] / deg(v).
__global__ void __launch_bounds__(kTB) k_agg_bwd(DGraph g, int d, const float *dZ, float *dH) {
    const int warps = blockDim.x >> 5;
    const int lane = threadIdx.x & 31;
    const int ldz = 2 * d;
    for (int64_t u = (int64_t)blockIdx.x * warps + (threadIdx.x >> 5); u < g.n; u += (int64_t)gridDim.x * warps) {
        const int64_t beg = g.xadj[u], end = g.xadj[u + 1];
        for (int c = lane; c < d; c += 32) {
            float s = dZ[u * ldz + c];
            for (int64_t j = beg; j < end; ++j) {
                const int64_t v = g.adj[j];
                s += dZ[v * ldz + d + c] / (float)(g.xadj[v + 1] - g.xadj[v]);
            }
            dH[u * d + c] = s;
        }
    }
}

__global__ void k_relu_bwd(int64_t count, const float *dH, const float *Y, float *dY) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        dY[i] = Y[i] > 0.f ? dH[i] : 0.f;
}

// One warp per row: loss_v = logsumexp(L_v) - L_v[y_v]; dlog_v[c] =
// (softmax_c - [c = y_v]) / n.  Per-block loss sums (warps in order) in
// part[blockIdx.x]; a label outside [0, k) sets *bad and its row adds no loss.
__global__ void __launch_bounds__(kTB) k_softmax_ce(int32_t n, int k, const float *L, const int32_t *y, float *dlog,
                                                    double *part, int *bad) {
    __shared__ double wsum[kTB / 32];
    const int warps = blockDim.x >> 5, warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    double acc = 0.0;
    for (int64_t v = (int64_t)blockIdx.x * warps + warp; v < n; v += (int64_t)gridDim.x * warps) {
        const float *Lv = L + v * k;
        float mx = -INFINITY;
        for (int c = lane; c < k; c += 32) mx = fmaxf(mx, Lv[c]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        float s = 0.f;
        for (int c = lane; c < k; c += 32) s += expf(Lv[c] - mx);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        const int32_t yv = y[v];
        const bool ok = yv >= 0 && yv < k;
        for (int c = lane; c < k; c += 32) {
            float p = expf(Lv[c] - mx) / s;
            if (c == yv) p -= 1.f;
            dlog[v * k + c] = p / (float)n;
        }
        if (lane == 0) {
            if (ok) acc += (double)(logf(s) + mx - Lv[yv]);
            else *bad = 1;
        }
    }
    if (lane == 0) wsum[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < warps; ++w) t += wsum[w];
        part[blockIdx.x] = t;
    }
}

// Sum of the per-block losses over a fixed tree (thread t takes the blocks
// t, t + 256, ... in order, then pairwise halving): one block of 256 threads.
__global__ void __launch_bounds__(256) k_loss_total(int nb, const double *part, int32_t n, float *loss) {
    __shared__ double sh[256];
    double t = 0.0;
    for (int b = threadIdx.x; b < nb; b += 256) t += part[b];
    sh[threadIdx.x] = t;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = (float)(sh[0] / (double)(n > 0 ? n : 1));
}

__global__ void k_adam(int64_t count, float *p, const float *gr, float *m, float *v, float lr, float b1, float b2,
                       float c1, float c2, float eps) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = gr[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// ---- features ---------------------------------------------------------------
struct FeatStats {
    unsigned long long maxdeg, maxvw, maxwdeg;
};

// One warp per vertex: wdeg(v) = sum of its edge weights (its degree for unit
// weights); maxima of degree, vertex weight and wdeg.
__global__ void __launch_bounds__(kTB) k_feat_rows(DGraph g, int64_t *wdeg, FeatStats *st) {
    const int warps = blockDim.x >> 5;
    const int lane = threadIdx.x & 31;
    unsigned long long md = 0, mv = 0, mw = 0;
    for (int64_t v = (int64_t)blockIdx.x * warps + (threadIdx.x >> 5); v < g.n; v += (int64_t)gridDim.x * warps) {
        const int64_t beg = g.xadj[v], end = g.xadj[v + 1];
        long long s = 0;
        if (g.ew) {
            for (int64_t j = beg + lane; j < end; j += 32) s += g.ew[j];
            s = warp_sum_i64(s);
        } else {
            s = end - beg;
        }
        if (lane == 0) {
            wdeg[v] = s;
            md = max(md, (unsigned long long)(end - beg));
            mv = max(mv, (unsigned long long)g.vw[v]);
            mw = max(mw, (unsigned long long)s);
        }
    }
    if (lane == 0) {
        atomicMax(&st->maxdeg, md);
        atomicMax(&st->maxvw, mv);
        atomicMax(&st->maxwdeg, mw);
    }
}

__device__ __forceinline__ float ratio_f(long long a, long long b) {
    return __fdiv_rn((float)a, (float)(b > 0 ? b : 1));
}

__device__ __forceinline__ float tri_f(float y) {
    return fabsf(__fsub_rn(__fmul_rn(2.f, __fsub_rn(y, floorf(y))), 1.f));
}

__global__ void k_feat(DGraph g, const int64_t *wdeg, const FeatStats *st, const int32_t *dist, int32_t maxdist,
                       const int64_t *S, long long W, float *X) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < g.n; v += (int64_t)gridDim.x * blockDim.x) {
        float *x = X + v * kF;
        const long long deg = g.xadj[v + 1] - g.xadj[v];
        x[0] = 1.f;
        x[1] = ratio_f(deg, (long long)st->maxdeg);
        x[2] = ratio_f(g.vw[v], (long long)st->maxvw);
        const float s = ratio_f(S[v], W);
        x[3] = s;
        x[4] = ratio_f(dist[v], maxdist);
        x[5] = ratio_f(wdeg[v], (long long)st->maxwdeg);
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            const float y = __fmul_rn(s, (float)(1 << j));
            x[6 + j] = tri_f(y);
            x[11 + j] = tri_f(__fadd_rn(y, 0.25f));
        }
    }
}

// ---- canonical labels ----------------------------------------------------------
// Parts renumbered by the mean position of their vertices in the greedy
// order: per part the sum of positions and the count (integer atomics, so the
// result does not depend on their order), then each part's rank.
__global__ void k_lab_sum(int32_t n, const int32_t *part, const int32_t *rank, unsigned long long *sum,
                          unsigned long long *cnt) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        atomicAdd(&sum[part[v]], (unsigned long long)rank[v]);
        atomicAdd(&cnt[part[v]], 1ULL);
    }
}

// newlab[p] = number of parts before p: nonempty parts by mean position
// (compared exactly as sum_q cnt_p < sum_p cnt_q), equal means by id, empty
// parts after all others.  One block.
__global__ void k_lab_rank(int k, const unsigned long long *sum, const unsigned long long *cnt, int32_t *newlab) {
    for (int p = threadIdx.x; p < k; p += blockDim.x) {
        int c = 0;
        for (int q = 0; q < k; ++q) {
            if (q == p) continue;
            bool before;
            if (cnt[q] == 0 || cnt[p] == 0) {
                before = cnt[q] != 0 && cnt[p] == 0 ? true : (cnt[q] == 0 && cnt[p] != 0 ? false : q < p);
            } else {
                const unsigned __int128 a = (unsigned __int128)sum[q] * cnt[p], b = (unsigned __int128)sum[p] * cnt[q];
                before = a < b || (a == b && q < p);
            }
            c += before;
        }
        newlab[p] = c;
    }
}

__global__ void k_lab_apply(int32_t n, const int32_t *part, const int32_t *newlab, int32_t *out) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        out[v] = newlab[part[v]];
}

__global__ void k_fill_i32(int32_t *p, int64_t n, int32_t x) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) p[i] = x;
}

// ---- balanced decode --------------------------------------------------------
// One warp per vertex: a(v) = argmax (lowest part on ties) and the sort key
// of "margin descending": the margin is >= +0, so its bits order like its
// value and their complement sorts it descending.
__global__ void __launch_bounds__(kTB) k_decode_prep(int32_t n, int k, const float *L, int32_t *a, uint64_t *key,
                                                     int32_t *val) {
    const int warps = blockDim.x >> 5;
    const int lane = threadIdx.x & 31;
    for (int64_t v = (int64_t)blockIdx.x * warps + (threadIdx.x >> 5); v < n; v += (int64_t)gridDim.x * warps) {
        const float *Lv = L + v * k;
        float best = -INFINITY;
        int bi = INT_MAX;
        for (int c = lane; c < k; c += 32) {
            const float x = Lv[c];
            if (x > best || bi == INT_MAX) { best = x; bi = c; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        float second = -INFINITY;
        for (int c = lane; c < k; c += 32)
            if (c != bi) second = fmaxf(second, Lv[c]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) second = fmaxf(second, __shfl_xor_sync(0xffffffffu, second, o));
        const float margin = k > 1 ? __fsub_rn(best, second) : 0.f;
        if (lane == 0) {
            a[v] = bi;
            key[v] = (uint64_t)(0xFFFFFFFFu - __float_as_uint(margin));
            val[v] = (int32_t)v;
        }
    }
}

// The sequential fill, one warp: lane 0 places the vertices in sorted order;
// the whole warp searches the lightest part when the preferred one is full.
__global__ void k_decode_fill(int32_t n, int k, const int32_t *order, const int32_t *a, const int32_t *vw,
                              long long cap, int32_t *part) {
    extern __shared__ long long w[];
    const int lane = threadIdx.x & 31;
    for (int p = lane; p < k; p += 32) w[p] = 0;
    __syncwarp();
    for (int64_t i0 = 0; i0 < n; i0 += 32) {
        int32_t v = 0, pa = 0, wv = 0;
        if (i0 + lane < n) {
            v = order[i0 + lane];
            pa = a[v];
            wv = vw[v];
        }
        const int cnt = (int)min((int64_t)32, n - i0);
        for (int j = 0; j < cnt; ++j) {
            const int32_t vj = __shfl_sync(0xffffffffu, v, j);
            const int32_t pj = __shfl_sync(0xffffffffu, pa, j);
            const long long wj = __shfl_sync(0xffffffffu, wv, j);
            int p = pj;
            if (w[pj] + wj > cap) {
                long long bw = LLONG_MAX;
                int bp = INT_MAX;
                for (int q = lane; q < k; q += 32)
                    if (w[q] < bw) { bw = w[q]; bp = q; }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const long long ow = __shfl_xor_sync(0xffffffffu, bw, o);
                    const int op = __shfl_xor_sync(0xffffffffu, bp, o);
                    if (ow < bw || (ow == bw && op < bp)) { bw = ow; bp = op; }
                }
                p = bp;
            }
            if (lane == 0) {
                part[vj] = p;
                w[p] += wj;
            }
            __syncwarp();
        }
    }
}

// ---- host side --------------------------------------------------------------
int grid_rows(int64_t n) { return std::max(1, std::min(num_sms() * 8, grid_for(n, kTB / 32))); }
int grid_elems(int64_t n) { return std::max(1, std::min(num_sms() * 8, grid_for(n, kTB))); }

int gemm_rows(Ctx &c, bool trans_b, int32_t M, int Kp, int Kv, int Np, int Nv, const float *A, int lda, const float *B,
              int ldb, const float *bias, float *Y, int ldy, float *R, int ldr) {
    if (M <= 0) return JET_OK;
    const size_t smem = (size_t)(kGemmBM + Np) * (Kp + 8) * 2;
    const int grid = (int)((M + kGemmBM - 1) / kGemmBM);
    if (trans_b) {
        JET_CUDA_TRY(cudaFuncSetAttribute(k_gemm_rows<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kGemmSmemMax));
        k_gemm_rows<true><<<grid, 128, smem, c.stream>>>(M, Kp, Kv, Np, Nv, A, lda, B, ldb, bias, Y, ldy, R, ldr);
    } else {
        JET_CUDA_TRY(cudaFuncSetAttribute(k_gemm_rows<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kGemmSmemMax));
        k_gemm_rows<false><<<grid, 128, smem, c.stream>>>(M, Kp, Kv, Np, Nv, A, lda, B, ldb, bias, Y, ldy, R, ldr);
    }
    c.launches += 1;
    JET_CUDA_TRY(cudaGetLastError());
    return JET_OK;
}

int tn_blocks(int32_t M) { return std::max(1, (int)((M + kTnChunk - 1) / kTnChunk)); }

// gW (Kv x Nv) and gb (Nv) = A^T B and the column sums of B over all M rows.
int gemm_tn(Ctx &c, int32_t M, int Kp, int Kv, int Np, int Nv, const float *A, int lda, const float *B, int ldb,
            float *P, float *CS, float *gW, float *gb) {
    const int nb = tn_blocks(M);
    const size_t smem = (size_t)(Kp + Np) * (kTnRows + 8) * 2;
    JET_CUDA_TRY(cudaFuncSetAttribute(k_gemm_tn, cudaFuncAttributeMaxDynamicSharedMemorySize, kGemmSmemMax));
    k_gemm_tn<<<nb, kTnWarps * 32, smem, c.stream>>>(M, Kp, Kv, Np, Nv, A, lda, B, ldb, P, CS);
    k_tn_reduce<<<grid_elems((int64_t)Kv * Nv + Nv), kTB, 0, c.stream>>>(nb, Kp, Kv, Np, Nv, P, CS, gW, gb);
    c.launches += 2;
    JET_CUDA_TRY(cudaGetLastError());
    return JET_OK;
}

// Workspace of one forward (and backward) pass over n rows.
struct Work {
    DevBuf buf;
    float *Z[kLayers], *Y[kLayers], *H3, *logits, *dlog, *dH, *dY, *dZ, *P, *CS, *loss;
    double *lpart;
    int *bad;
    int ce_blocks;
};

int work_alloc(Ctx &c, Work &w, int32_t n, int32_t k, bool backward, float *logits_ext) {
    const size_t nn = (size_t)std::max(n, 1);
    const int kp = pad16(k);
    w.ce_blocks = grid_rows(n);
    const int nb = tn_blocks(n);
    const size_t ptile = (size_t)std::max(128 * kHd, kHd * kp);
    size_t sizes[20];
    int cnt = 0;
    sizes[cnt++] = nn * 2 * kF * 4;                 // Z0
    sizes[cnt++] = nn * 2 * kHd * 4;                // Z1
    sizes[cnt++] = nn * 2 * kHd * 4;                // Z2
    for (int l = 0; l < kLayers; ++l) sizes[cnt++] = nn * kHd * 4;   // Y
    sizes[cnt++] = nn * kHd * 4;                    // H3
    sizes[cnt++] = logits_ext ? 0 : nn * k * 4;     // logits
    if (backward) {
        sizes[cnt++] = nn * k * 4;                  // dlog
        sizes[cnt++] = nn * kHd * 4;                // dH
        sizes[cnt++] = nn * kHd * 4;                // dY
        sizes[cnt++] = nn * 2 * kHd * 4;            // dZ
        sizes[cnt++] = (size_t)nb * ptile * 4;      // P
        sizes[cnt++] = (size_t)nb * std::max(kHd, kp) * 4;   // CS
        sizes[cnt++] = (size_t)w.ce_blocks * 8;     // lpart
        sizes[cnt++] = 16;                          // loss, bad
    }
    size_t total = 0;
    for (int i = 0; i < cnt; ++i) total += align256c(sizes[i]);
    JET_TRY(dev_alloc(w.buf, total, c.stream));
    char *p = w.buf.as<char>();
    int i = 0;
    auto take = [&]() { char *r = p; p += align256c(sizes[i++]); return r; };
    for (int l = 0; l < kLayers; ++l) w.Z[l] = reinterpret_cast<float *>(take());
    for (int l = 0; l < kLayers; ++l) w.Y[l] = reinterpret_cast<float *>(take());
    w.H3 = reinterpret_cast<float *>(take());
    w.logits = logits_ext ? (take(), logits_ext) : reinterpret_cast<float *>(take());
    if (backward) {
        w.dlog = reinterpret_cast<float *>(take());
        w.dH = reinterpret_cast<float *>(take());
        w.dY = reinterpret_cast<float *>(take());
        w.dZ = reinterpret_cast<float *>(take());
        w.P = reinterpret_cast<float *>(take());
        w.CS = reinterpret_cast<float *>(take());
        w.lpart = reinterpret_cast<double *>(take());
        char *q = take();
        w.loss = reinterpret_cast<float *>(q);
        w.bad = reinterpret_cast<int *>(q + 8);
    }
    return JET_OK;
}

}  // namespace

// The model: float32 master parameters and Adam moments on the device.
struct Lip {
    int device = 0;
    int32_t k = 0;
    int64_t np = 0;
    float *P = nullptr, *M = nullptr, *V = nullptr;
    int64_t t = 0;
};

namespace {

int forward(Ctx &c, const Lip &m, const DGraph &g, const float *X, Work &w) {
    const Offsets o = offsets(m.k);
    const int32_t n = g.n;
    const int k = m.k, kp = pad16(k);
    k_agg_fwd<<<grid_rows(n), kTB, 0, c.stream>>>(g, kF, X, kF, w.Z[0]);
    c.launches += 1;
    JET_CUDA_TRY(cudaGetLastError());
    for (int l = 0; l < kLayers; ++l) {
        const int K = 2 * din_of(l);
        float *R = l + 1 < kLayers ? w.Z[l + 1] : w.H3;
        const int ldr = l + 1 < kLayers ? 2 * kHd : kHd;
        JET_TRY(gemm_rows(c, false, n, K, K, kHd, kHd, w.Z[l], K, m.P + o.W[l], kHd, m.P + o.b[l], w.Y[l], kHd, R, ldr));
        if (l + 1 < kLayers) {
            k_agg_fwd<<<grid_rows(n), kTB, 0, c.stream>>>(g, kHd, w.Z[l + 1], 2 * kHd, w.Z[l + 1]);
            c.launches += 1;
            JET_CUDA_TRY(cudaGetLastError());
        }
    }
    return gemm_rows(c, false, n, kHd, kHd, kp, k, w.H3, kHd, m.P + o.W[kLayers], k, m.P + o.b[kLayers], w.logits, k,
                     nullptr, 0);
}

// Loss (device scalar w.loss) and gradient (device, parameter order).
int backward(Ctx &c, const Lip &m, const DGraph &g, const int32_t *labels, Work &w, float *grad) {
    const Offsets o = offsets(m.k);
    const int32_t n = g.n;
    const int k = m.k, kp = pad16(k);
    JET_CUDA_TRY(cudaMemsetAsync(w.bad, 0, 4, c.stream));
    k_softmax_ce<<<w.ce_blocks, kTB, 0, c.stream>>>(n, k, w.logits, labels, w.dlog, w.lpart, w.bad);
    k_loss_total<<<1, 256, 0, c.stream>>>(w.ce_blocks, w.lpart, n, w.loss);
    c.launches += 2;
    JET_CUDA_TRY(cudaGetLastError());
    // output layer: dWo = H3^T dlog, dbo = colsum dlog, dH3 = dlog Wo^T
    JET_TRY(gemm_tn(c, n, kHd, kHd, kp, k, w.H3, kHd, w.dlog, k, w.P, w.CS, grad + o.W[kLayers], grad + o.b[kLayers]));
    JET_TRY(gemm_rows(c, true, n, kp, k, kHd, kHd, w.dlog, k, m.P + o.W[kLayers], k, nullptr, w.dH, kHd, nullptr, 0));
    for (int l = kLayers - 1; l >= 0; --l) {
        const int d = din_of(l), K = 2 * d;
        k_relu_bwd<<<grid_elems((int64_t)n * kHd), kTB, 0, c.stream>>>((int64_t)n * kHd, w.dH, w.Y[l], w.dY);
        c.launches += 1;
        JET_CUDA_TRY(cudaGetLastError());
        JET_TRY(gemm_tn(c, n, K, K, kHd, kHd, w.Z[l], K, w.dY, kHd, w.P, w.CS, grad + o.W[l], grad + o.b[l]));
        if (l > 0) {
            // dZ = dY W^T (n x 2d); dH_{l-1} = dZ[:, :d] + aggregation transpose of dZ[:, d:]
            JET_TRY(gemm_rows(c, true, n, kHd, kHd, K, K, w.dY, kHd, m.P + o.W[l], kHd, nullptr, w.dZ, K, nullptr, 0));
            k_agg_bwd<<<grid_rows(n), kTB, 0, c.stream>>>(g, d, w.dZ, w.dH);
            c.launches += 1;
            JET_CUDA_TRY(cudaGetLastError());
        }
    }
    return JET_OK;
}

// Features into X (device n x 16); *W_out (may be null) = total vertex weight.
int features(Ctx &c, const DGraph &g, float *X, int64_t *W_out = nullptr) {
    const int64_t n = g.n;
    if (n == 0) return JET_OK;
    const size_t nn = (size_t)n;
    DevBuf buf;
    JET_TRY(dev_alloc(buf, align256c(nn * 4) + 2 * align256c(nn * 8) + align256c(sizeof(FeatStats)), c.stream));
    char *p = buf.as<char>();
    int32_t *dist = reinterpret_cast<int32_t *>(p);
    p += align256c(nn * 4);
    int64_t *S = reinterpret_cast<int64_t *>(p);
    p += align256c(nn * 8);
    int64_t *wdeg = reinterpret_cast<int64_t *>(p);
    p += align256c(nn * 8);
    FeatStats *st = reinterpret_cast<FeatStats *>(p);
    GreedyOut go;
    go.dist = dist;
    go.S = S;
    JET_TRY(initial_partition(c, g, 1, nullptr, &go));
    JET_CUDA_TRY(cudaMemsetAsync(st, 0, sizeof(FeatStats), c.stream));
    k_feat_rows<<<grid_rows(n), kTB, 0, c.stream>>>(g, wdeg, st);
    k_feat<<<grid_elems(n), kTB, 0, c.stream>>>(g, wdeg, st, dist, go.maxdist, S, (long long)go.W, X);
    c.launches += 2;
    JET_CUDA_TRY(cudaGetLastError());
    if (W_out) *W_out = go.W;
    return sync_stream(c);
}

int decode(Ctx &c, int32_t n, const float *L, const int32_t *vw, int32_t k, int64_t cap, int32_t *part) {
    if (n == 0) return JET_OK;
    DevBuf buf;
    JET_TRY(dev_alloc(buf, align256c((size_t)n * 4) + sort_scratch_bytes(n), c.stream));
    int32_t *a = buf.as<int32_t>();
    SortScratch sc;
    sort_scratch_carve(buf.as<char>() + align256c((size_t)n * 4), n, sc);
    k_decode_prep<<<grid_rows(n), kTB, 0, c.stream>>>(n, k, L, a, sc.key[0], sc.val[0]);
    c.launches += 1;
    JET_CUDA_TRY(cudaGetLastError());
    int which = 0;
    JET_TRY(sort_pairs(c, sc, n, 32, &which));
    k_decode_fill<<<1, 32, (size_t)k * 8, c.stream>>>(n, k, sc.val[which], a, vw, (long long)cap, part);
    c.launches += 1;
    JET_CUDA_TRY(cudaGetLastError());
    return sync_stream(c);
}

// The network's proposal for graph g into part (device int32[n]).
int proposal(Ctx &c, const Lip &m, const DGraph &g, double eps, int32_t *part) {
    const int32_t n = g.n;
    if (n == 0) return JET_OK;
    DevBuf xb;
    JET_TRY(dev_alloc(xb, (size_t)n * kF * 4, c.stream));
    int64_t W = 0;
    JET_TRY(features(c, g, xb.as<float>(), &W));
    Work w;
    JET_TRY(work_alloc(c, w, n, m.k, false, nullptr));
    JET_TRY(forward(c, m, g, xb.as<float>(), w));
    const int64_t cap = balance_limit(W, m.k, eps, nullptr);
    return decode(c, n, w.logits, g.vw, m.k, cap, part);
}

int graph_of(Ctx &c, int32_t n, const int64_t *xadj, const int32_t *adjncy, const int32_t *vwgt, const int32_t *adjwgt,
             DGraph &g, DevBuf &ones) {
    return prepare_graph(c, n, xadj, adjncy, vwgt, adjwgt, g, ones, true);
}

}  // namespace

}  // namespace jet

struct jet_lip {
    jet::Lip m;
};

using namespace jet;

extern "C" {

int64_t jet_lip_num_params(int32_t k) {
    if (k < 2 || k > JET_LIP_MAX_K) return -1;
    return offsets(k).total;
}

int jet_lip_create(jet_ctx *ctx, int32_t k, const float *params, jet_lip **out) {
    if (!ctx || !out || !params || k < 2 || k > JET_LIP_MAX_K) return JET_EINVAL;
    *out = nullptr;
    Ctx &c = ctx->c;
    JET_TRY(use_device(c));
    jet_lip *h = new (std::nothrow) jet_lip;
    if (!h) return JET_ENOMEM;
    Lip &m = h->m;
    m.device = c.device;
    m.k = k;
    m.np = offsets(k).total;
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, (size_t)m.np * 3 * 4);
    if (e != cudaSuccess) {
        record_cuda_error(e, "cudaMalloc", __FILE__, __LINE__);
        delete h;
        return e == cudaErrorMemoryAllocation ? JET_ENOMEM : JET_ECUDA;
    }
    m.P = static_cast<float *>(p);
    m.M = m.P + m.np;
    m.V = m.M + m.np;
    int r = jet_lip_set_params(ctx, h, params);
    if (r < 0) {
        jet_lip_destroy(h);
        return r;
    }
    *out = h;
    return JET_OK;
}

void jet_lip_destroy(jet_lip *h) {
    if (!h) return;
    cudaSetDevice(h->m.device);
    if (h->m.P) {
        cudaDeviceSynchronize();
        cudaFree(h->m.P);
    }
    delete h;
}

int jet_lip_get_params(jet_ctx *ctx, const jet_lip *h, float *params_out) {
    if (!ctx || !h || !params_out) return JET_EINVAL;
    Ctx &c = ctx->c;
    JET_TRY(use_device(c));
    JET_CUDA_TRY(cudaMemcpyAsync(params_out, h->m.P, (size_t)h->m.np * 4, cudaMemcpyDeviceToHost, c.stream));
    return sync_stream(c);
}

int jet_lip_set_params(jet_ctx *ctx, jet_lip *h, const float *params) {
    if (!ctx || !h || !params) return JET_EINVAL;
    Ctx &c = ctx->c;
    JET_TRY(use_device(c));
    Lip &m = h->m;
    JET_CUDA_TRY(cudaMemcpyAsync(m.P, params, (size_t)m.np * 4, cudaMemcpyHostToDevice, c.stream));
    JET_CUDA_TRY(cudaMemsetAsync(m.M, 0, (size_t)m.np * 2 * 4, c.stream));
    m.t = 0;
    return sync_stream(c);
}

int jet_lip_features(jet_ctx *ctx, int32_t n, const int64_t *xadj, const int32_t *adjncy, const int32_t *vwgt,
                     const int32_t *adjwgt, float *x_out) {
    if (!ctx || (n > 0 && !x_out)) return JET_EINVAL;
    Ctx &c = ctx->c;
    JET_TRY(use_device(c));
    DGraph g;
    DevBuf ones;
    JET_TRY(graph_of(c, n, xadj, adjncy, vwgt, adjwgt, g, ones));
    return features(c, g, x_out);
}

int jet_lip_labels(jet_ctx *ctx, int32_t n, const int64_t *xadj, const int32_t *adjncy, int32_t k, const int32_t *part,
                   int32_t *labels_out) {
    if (!ctx || k < 1 || k > JET_MAX_K || (n > 0 && (!part || !labels_out))) return JET_EINVAL;
    Ctx &c = ctx->c;
    JET_TRY(use_device(c));
    DGraph g;
    DevBuf ones;
    JET_TRY(graph_of(c, n, xadj, adjncy, nullptr, nullptr, g, ones));
    JET_TRY(check_part(c, n, part, k));
    if (n == 0) return JET_OK;
    DevBuf buf;
    const size_t kb = align256c((size_t)k * 8);
    JET_TRY(dev_alloc(buf, align256c((size_t)n * 4) + 2 * kb + align256c((size_t)k * 4), c.stream));
    int32_t *rank = buf.as<int32_t>();
    unsigned long long *sum = reinterpret_cast<unsigned long long *>(buf.as<char>() + align256c((size_t)n * 4));
    unsigned long long *cnt = reinterpret_cast<unsigned long long *>(reinterpret_cast<char *>(sum) + kb);
    int32_t *newlab = reinterpret_cast<int32_t *>(reinterpret_cast<char *>(cnt) + kb);
    GreedyOut go;
    go.rank = rank;
    JET_TRY(initial_partition(c, g, 1, nullptr, &go));
    JET_CUDA_TRY(cudaMemsetAsync(sum, 0, 2 * kb, c.stream));
    k_lab_sum<<<grid_elems(n), kTB, 0, c.stream>>>(n, part, rank, sum, cnt);
    k_lab_rank<<<1, kTB, 0, c.stream>>>(k, sum, cnt, newlab);
    k_lab_apply<<<grid_elems(n), kTB, 0, c.stream>>>(n, part, newlab, labels_out);
    c.launches += 3;
    JET_CUDA_TRY(cudaGetLastError());
    return sync_stream(c);
}

int jet_lip_forward(jet_ctx *ctx, const jet_lip *h, int32_t n, const int64_t *xadj, const int32_t *adjncy,
                    const float *x, float *logits_out) {
    if (!ctx || !h || (n > 0 && (!x || !logits_out))) return JET_EINVAL;
    Ctx &c = ctx->c;
    JET_TRY(use_device(c));
    DGraph g;
    DevBuf ones;
    JET_TRY(graph_of(c, n, xadj, adjncy, nullptr, nullptr, g, ones));
    if (n == 0) return JET_OK;
    Work w;
    JET_TRY(work_alloc(c, w, n, h->m.k, false, logits_out));
    JET_TRY(forward(c, h->m, g, x, w));
    return sync_stream(c);
}

static int loss_grad(Ctx &c, const Lip &m, int32_t n, const int64_t *xadj, const int32_t *adjncy, const float *x,
                     const int32_t *labels, float *loss_out, float *grad) {
    DGraph g;
    DevBuf ones;
    JET_TRY(graph_of(c, n, xadj, adjncy, nullptr, nullptr, g, ones));
    if (n == 0) {
        JET_CUDA_TRY(cudaMemsetAsync(grad, 0, (size_t)m.np * 4, c.stream));
        if (loss_out) *loss_out = 0.f;
        return sync_stream(c);
    }
    Work w;
    JET_TRY(work_alloc(c, w, n, m.k, true, nullptr));
    JET_TRY(forward(c, m, g, x, w));
    JET_TRY(backward(c, m, g, labels, w, grad));
    JET_CUDA_TRY(cudaMemcpyAsync(c.pinned, w.loss, 16, cudaMemcpyDeviceToHost, c.stream));
    JET_TRY(sync_stream(c));
    float loss;
    int bad;
    memcpy(&loss, reinterpret_cast<char *>(c.pinned), 4);
    memcpy(&bad, reinterpret_cast<char *>(c.pinned) + 8, 4);
    if (bad) {
        record_error("jet_lip: label outside [0, k)");
        return JET_EINVAL;
    }
    if (loss_out) *loss_out = loss;
    return JET_OK;
}

int jet_lip_loss_grad(jet_ctx *ctx, const jet_lip *h, int32_t n, const int64_t *xadj, const int32_t *adjncy,
                      const float *x, const int32_t *labels, float *loss_out, float *grad_out) {
    if (!ctx || !h || !grad_out || (n > 0 && (!x || !labels))) return JET_EINVAL;
    Ctx &c = ctx->c;
    JET_TRY(use_device(c));
    return loss_grad(c, h->m, n, xadj, adjncy, x, labels, loss_out, grad_out);
}

int jet_lip_train_step(jet_ctx *ctx, jet_lip *h, int32_t n, const int64_t *xadj, const int32_t *adjncy, const float *x,
                       const int32_t *labels, float lr, float *loss_out) {
    if (!ctx || !h || (n > 0 && (!x || !labels)) || !(lr >= 0.f) || !std::isfinite(lr)) return JET_EINVAL;
    Ctx &c = ctx->c;
    JET_TRY(use_device(c));
    Lip &m = h->m;
    DevBuf gb;
    JET_TRY(dev_alloc(gb, (size_t)m.np * 4, c.stream));
    JET_TRY(loss_grad(c, m, n, xadj, adjncy, x, labels, loss_out, gb.as<float>()));
    m.t += 1;
    const double b1 = 0.9, b2 = 0.999;
    const float c1 = (float)(1.0 - std::pow(b1, (double)m.t)), c2 = (float)(1.0 - std::pow(b2, (double)m.t));
    k_adam<<<grid_elems(m.np), kTB, 0, c.stream>>>(m.np, m.P, gb.as<float>(), m.M, m.V, lr, (float)b1, (float)b2, c1,
                                                   c2, 1e-8f);
    c.launches += 1;
    JET_CUDA_TRY(cudaGetLastError());
    return sync_stream(c);
}

int jet_lip_decode(jet_ctx *ctx, int32_t n, const float *logits, const int32_t *vwgt, int32_t k, int64_t cap,
                   int32_t *part_out) {
    if (!ctx || n < 0 || k < 1 || k > JET_MAX_K || (n > 0 && (!logits || !part_out))) return JET_EINVAL;
    Ctx &c = ctx->c;
    JET_TRY(use_device(c));
    DevBuf ones;
    const int32_t *vw = vwgt;
    if (!vw && n > 0) {
        JET_TRY(dev_alloc(ones, (size_t)n * 4, c.stream));
        k_fill_i32<<<grid_elems(n), kTB, 0, c.stream>>>(ones.as<int32_t>(), n, 1);
        c.launches += 1;
        JET_CUDA_TRY(cudaGetLastError());
        vw = ones.as<int32_t>();
    }
    return decode(c, n, logits, vw, k, cap, part_out);
}

int jet_lip_initial_partition(jet_ctx *ctx, const jet_lip *h, int32_t n, const int64_t *xadj, const int32_t *adjncy,
                              const int32_t *vwgt, const int32_t *adjwgt, double eps, int32_t *part_out) {
    if (!ctx || !h || bad_k_eps(h->m.k, eps) || (n > 0 && !part_out)) return JET_EINVAL;
    Ctx &c = ctx->c;
    JET_TRY(use_device(c));
    DGraph g;
    DevBuf ones;
    JET_TRY(graph_of(c, n, xadj, adjncy, vwgt, adjwgt, g, ones));
    return proposal(c, h->m, g, eps, part_out);
}

int jet_partition_learned(jet_ctx *ctx, const jet_lip *h, int32_t n, const int64_t *xadj, const int32_t *adjncy,
                          const int32_t *vwgt, const int32_t *adjwgt, double eps, uint64_t seed, int32_t *part_out,
                          int64_t *cut_out, jet_stats *stats, jet_learned_info *info) {
    if (!ctx || !h || bad_k_eps(h->m.k, eps) || (n > 0 && !part_out)) return JET_EINVAL;
    Ctx &c = ctx->c;
    JET_TRY(use_device(c));
    const int32_t k = h->m.k;
    jet_learned_info inf;
    memset(&inf, 0, sizeof(inf));
    inf.cut_learned = -1;
    // ev: start, coarsened, proposal ready, plain done, all done; wv: the
    // learned uncoarsening on the second stream
    cudaEvent_t ev[5] = {}, wv[2] = {};
    struct EvGuard {
        cudaEvent_t *e, *w;
        ~EvGuard() {
            for (int i = 0; i < 5; ++i)
                if (e[i]) cudaEventDestroy(e[i]);
            for (int i = 0; i < 2; ++i)
                if (w[i]) cudaEventDestroy(w[i]);
        }
    } guard{ev, wv};
    for (auto &e : ev) JET_CUDA_TRY(cudaEventCreate(&e));
    for (auto &e : wv) JET_CUDA_TRY(cudaEventCreate(&e));
    const int64_t l0 = c.launches;
    auto ms = [](cudaEvent_t a, cudaEvent_t b) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, a, b) != cudaSuccess) { cudaGetLastError(); return 0.f; }
        return t;
    };
    JET_CUDA_TRY(cudaEventRecord(ev[0], c.stream));
    jet_hier *hier = nullptr;
    int r = jet_coarsen(ctx, n, xadj, adjncy, vwgt, adjwgt, k, seed, &hier);
    if (r < 0) return r;
    struct HierGuard {
        jet_hier *h;
        ~HierGuard() { jet_hier_destroy(h); }
    } hg{hier};
    JET_CUDA_TRY(cudaEventRecord(ev[1], c.stream));
    const int32_t l = hier->levels - 1;
    inf.n_coarsest = hier->n[l];
    const bool learned = n > 0 && hier->n[l] <= JET_LIP_MAX_N;
    DevBuf init, tmp;
    if (learned) {
        DGraph gc;
        gc.n = hier->n[l]; gc.nnz = hier->nnz[l]; gc.xadj = hier->xadj[l]; gc.adj = hier->adj[l];
        gc.vw = hier->vw[l]; gc.ew = hier->ew[l];
        JET_TRY(dev_alloc(init, (size_t)gc.n * 4, c.stream));
        JET_TRY(dev_alloc(tmp, (size_t)n * 4, c.stream));
        JET_TRY(proposal(c, h->m, gc, eps, init.as<int32_t>()));
    }
    JET_CUDA_TRY(cudaEventRecord(ev[2], c.stream));
    jet_stats st_plain, st_learned;
    memset(&st_plain, 0, sizeof(st_plain));
    memset(&st_learned, 0, sizeof(st_learned));
    // The two uncoarsenings of the hierarchy run concurrently: the plain one
    // on the caller's stream, the learned one on a second context and stream
    // (both latency-bound, so they share the GPU well).  The hierarchy is
    // only read.
    int r_learned = JET_OK;
    int64_t cut_learned = -1;
    cudaStream_t ws = nullptr;
    jet_ctx *wc = nullptr;
    // Concurrent uncoarsenings never use the cooperative level loop (a
    // cooperative launch wants the whole GPU to itself).
    struct FlagGuard {
        jet_options &o;
        uint32_t saved;
        ~FlagGuard() { o.flags = saved; }
    } grid_flag_guard{c.opt, c.opt.flags};
    if (learned) c.opt.flags &= ~JET_FLAG_GRID_LOOP;
    if (learned) {
        JET_CUDA_TRY(cudaStreamCreateWithFlags(&ws, cudaStreamNonBlocking));
        int rc = jet_ctx_create(c.device, ws, &c.opt, &wc);
        if (rc != JET_OK || cudaStreamWaitEvent(ws, ev[2], 0) != cudaSuccess) {
            if (wc) jet_ctx_destroy(wc);
            cudaStreamDestroy(ws);
            record_error("jet_partition_learned: second context");
            return rc != JET_OK ? rc : JET_ECUDA;
        }
    }
    auto learned_run = [&] {
        Ctx &w = wc->c;
        if (use_device(w) != JET_OK) { r_learned = JET_ECUDA; return; }
        cudaEventRecord(wv[0], ws);
        r_learned = uncoarsen(w, hier, k, eps, seed, init.as<int32_t>(), tmp.as<int32_t>(), &cut_learned,
                              &st_learned);
        cudaEventRecord(wv[1], ws);
    };
    std::thread worker;
    bool threaded = false;
    if (learned) {
        try {
            worker = std::thread(learned_run);
            threaded = true;
        } catch (...) {   // no thread: the learned uncoarsening runs after the plain one
        }
    }
    int64_t cut_plain = 0;
    int r_plain = n > 0 ? uncoarsen(c, hier, k, eps, seed, nullptr, part_out, &cut_plain, &st_plain) : JET_OK;
    cudaEventRecord(ev[3], c.stream);
    if (learned) {
        if (threaded) worker.join();
        else learned_run();
        use_device(c);
        cudaStreamWaitEvent(c.stream, wv[1], 0);
        c.launches += wc->c.launches;
    }
    cudaEventRecord(ev[4], c.stream);
    const int sync = sync_stream(c);
    if (learned) {
        jet_ctx_destroy(wc);
        cudaStreamDestroy(ws);
    }
    if (r_plain < 0) return r_plain;
    if (r_learned < 0) return r_learned;
    JET_TRY(sync);
    inf.cut_plain = cut_plain;
    inf.status_plain = r_plain;
    bool keep_learned = false;
    if (learned) {
        const bool bal_l = r_learned != JET_WUNBALANCED, bal_p = r_plain != JET_WUNBALANCED;
        keep_learned = (bal_l && !bal_p) || (bal_l == bal_p && cut_learned <= cut_plain);
        if (keep_learned) {
            JET_CUDA_TRY(cudaMemcpyAsync(part_out, tmp.as<int32_t>(), (size_t)n * 4, cudaMemcpyDeviceToDevice, c.stream));
            JET_TRY(sync_stream(c));
        }
    }
    inf.cut_learned = cut_learned;
    inf.status_learned = r_learned;
    inf.chosen = keep_learned ? 1 : 0;
    inf.ms_coarsen = ms(ev[0], ev[1]);
    inf.ms_proposal = ms(ev[1], ev[2]);
    inf.ms_plain = ms(ev[2], ev[3]);
    inf.ms_learned = learned ? ms(wv[0], wv[1]) : 0.f;
    if (stats) {
        *stats = keep_learned ? st_learned : st_plain;
        stats->ms_coarsen = inf.ms_coarsen;
        stats->ms_total = ms(ev[0], ev[4]);
        stats->kernel_launches = c.launches - l0;
    }
    if (info) *info = inf;
    if (cut_out) *cut_out = keep_learned ? cut_learned : cut_plain;
    return keep_learned ? r_learned : r_plain;
}

}  // extern "C"
