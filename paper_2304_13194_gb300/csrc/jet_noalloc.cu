// jet_lp_pass_noalloc: one Jetlp pass that allocates no device memory.
//
// Some callers cannot let a library allocate: a process whose device memory
// is fully reserved up front by its own pool (a server that sized its caches
// to the whole GPU), a latency-critical loop where cudaMalloc/cudaFree would
// synchronise the device or grow the CUDA memory pool at an unpredictable
// moment, or an embedding framework that only hands out memory it owns.  For
// them this entry point runs the same pass as jet_lp_pass with all of its
// scratch in the fixed array below, which the module reserves once on every
// device that loads the library and keeps until the process exits.
#include "jet_internal.cuh"

#include <mutex>

namespace jet {

constexpr size_t kNoallocCheckBytes = 256;
constexpr size_t kNoallocCheckOffset = lp_scratch_bytes(JET_NOALLOC_MAX_N);
constexpr size_t kNoallocBytes = kNoallocCheckOffset + kNoallocCheckBytes;

// The whole scratch of jet_lp_pass_noalloc (about 10 MiB), shared by every
// call on a device.  In host code this name is only a stand-in: the device
// address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

// Overflow limits of jet.h and the part range, written into the check slot at
// the end of the array (sum_vw, sum_ew, bad part).
__global__ void k_noalloc_check(int32_t n, const int64_t *xadj, const int32_t *vw, const int32_t *ew,
                                const int32_t *part, int32_t k) {
    __shared__ long long sh[40];
    long long *out = reinterpret_cast<long long *>(g_noalloc_scratch + kNoallocCheckOffset);
    long long svw = 0, sew = 0, bad = 0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        svw += vw ? vw[v] : 1;
        int64_t e = xadj[v + 1];
        for (int64_t j = xadj[v]; j < e; ++j) sew += ew ? ew[j] : 1;
        if (part[v] < 0 || part[v] >= k) bad = 1;
    }
    svw = block_sum_i64(svw, sh);
    sew = block_sum_i64(sew, sh);
    bad = block_sum_i64(bad, sh);
    if (threadIdx.x == 0) {
        atomic_add_i64(reinterpret_cast<int64_t *>(&out[0]), svw);
        atomic_add_i64(reinterpret_cast<int64_t *>(&out[1]), sew);
        if (bad) atomic_add_i64(reinterpret_cast<int64_t *>(&out[2]), bad);
    }
}

// Device address of g_noalloc_scratch, looked up once per device with that
// device current.
static std::mutex g_noalloc_mutex;
static void *g_noalloc_addr[256] = {};

static int noalloc_scratch(int device, char **out) {
    if (device < 0 || device >= 256) return JET_EINVAL;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            record_cuda_error(e, "cudaGetSymbolAddress(g_noalloc_scratch)", __FILE__, __LINE__);
            cudaGetLastError();
            return JET_ECUDA;
        }
        g_noalloc_addr[device] = p;
    }
    *out = static_cast<char *>(g_noalloc_addr[device]);
    return JET_OK;
}

}  // namespace jet

using namespace jet;

extern "C" int jet_lp_pass_noalloc(jet_ctx *ctx, int32_t n, const int64_t *xadj, const int32_t *adjncy,
                                   const int32_t *vwgt, const int32_t *adjwgt, int32_t k, const int32_t *part,
                                   const uint8_t *locked, double cval, uint32_t flags, int32_t *pd_out,
                                   int32_t *gain_out, uint8_t *inx_out, int32_t *f2_out, uint8_t *inm_out) {
    if (!ctx || !xadj || k < 1 || k > JET_MAX_K || !(cval >= 0 && cval <= 1) || n < 0) return JET_EINVAL;
    if (n > JET_NOALLOC_MAX_N) {
        record_error("jet_lp_pass_noalloc: n exceeds JET_NOALLOC_MAX_N (262144 vertices)");
        return JET_EINVAL;
    }
    Ctx &c = ctx->c;
    JET_TRY(use_device(c));
    char *scratch = nullptr;
    JET_TRY(noalloc_scratch(c.device, &scratch));
    if (n == 0) return JET_OK;
    if (!part) return JET_EINVAL;
    cudaStream_t s = c.stream;
    JET_CUDA_TRY(cudaMemcpyAsync(c.pinned, xadj + n, 8, cudaMemcpyDeviceToHost, s));
    JET_CUDA_TRY(cudaStreamSynchronize(s));
    int64_t nnz = c.pinned[0];
    if (nnz < 0) return JET_EGRAPH;
    if (nnz > 0 && !adjncy) return JET_EINVAL;
    char *check = scratch + kNoallocCheckOffset;
    JET_CUDA_TRY(cudaMemsetAsync(check, 0, kNoallocCheckBytes, s));
    k_noalloc_check<<<std::min(num_sms() * 8, grid_for(n, kTB)), kTB, 0, s>>>(n, xadj, vwgt, adjwgt, part, k);
    JET_CUDA_TRY(cudaGetLastError());
    JET_CUDA_TRY(cudaMemcpyAsync(c.pinned, check, 24, cudaMemcpyDeviceToHost, s));
    JET_CUDA_TRY(cudaStreamSynchronize(s));
    if (c.pinned[2]) return JET_EINVAL;
    if (c.pinned[0] >= (1LL << 31) || c.pinned[1] >= (1LL << 31)) return JET_EOVERFLOW;
    DGraph g;
    g.n = n;
    g.nnz = nnz;
    g.xadj = xadj;
    g.adj = adjncy;
    g.vw = vwgt;   // the Jetlp pass never reads vertex weights
    g.ew = adjwgt;
    return lp_pass_in_scratch(c, g, k, part, locked, cval, flags, pd_out, gain_out, inx_out, f2_out, inm_out, scratch);
}
