// Measurement helper: the fused multiply-add throughput of this GPU's float64
// and float32 pipes, the denominators of the solver kernels' roofline
// fractions (those kernels are bound by plain ALU arithmetic, not by HBM).
//
// Every thread runs FMA_CHAINS independent chains a_i <- a_i * b + c for
// `iters` steps, so each pipe sees enough independent work to stay full; the
// grid is FMA_BLOCKS_PER_SM blocks of 256 threads on every SM.  The chains are
// summed and stored so that nothing is dead code; b and c are runtime values.
#include <algorithm>

#include "common.cuh"

namespace mbe {

constexpr int FMA_CHAINS = 8;
constexpr int FMA_THREADS = 256;
constexpr int FMA_BLOCKS_PER_SM = 4;

template <typename T>
__global__ void __launch_bounds__(FMA_THREADS) k_fma_chain(int iters, T b, T c, T *out)
{
    T a[FMA_CHAINS];
#pragma unroll
    for (int i = 0; i < FMA_CHAINS; ++i) a[i] = (T)(threadIdx.x + i);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 16; ++r)
#pragma unroll
            for (int i = 0; i < FMA_CHAINS; ++i) a[i] = fma(a[i], b, c);
    }
    T s = 0;
#pragma unroll
    for (int i = 0; i < FMA_CHAINS; ++i) s += a[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace mbe

using namespace mbe;

extern "C" int mbe_fma_peak(mbe_ctx *ctx, int kind, int reps, double *tflops)
{
    MBE_CHECK(ctx && tflops, MBE_EINVAL, "mbe_fma_peak: NULL argument");
    MBE_CHECK(kind == 0 || kind == 1, MBE_EINVAL, "mbe_fma_peak: kind %d (0 float64, 1 float32)", kind);
    MBE_CHECK(reps >= 1 && reps <= 1000, MBE_EINVAL, "mbe_fma_peak: reps %d", reps);
    MBE_CU(cudaSetDevice(ctx->device));
    const int blocks = ctx->sm_count * FMA_BLOCKS_PER_SM;
    const size_t n = (size_t)blocks * FMA_THREADS;
    // about 20 ms per float64 launch and 10 ms per float32 launch on a GB300
    const int iters = kind == 0 ? 600 : 20000;
    void *out = nullptr;
    int rc = workspace(ctx, n * 8, &out);
    if (rc) return rc;
    cudaEvent_t e0, e1;
    MBE_CU(cudaEventCreate(&e0));
    MBE_CU(cudaEventCreate(&e1));
    double best = 0.0;
    for (int r = 0; r <= reps; ++r) {  // launch 0 is the warm-up
        cudaEventRecord(e0, ctx->stream);
        if (kind == 0)
            k_fma_chain<double><<<blocks, FMA_THREADS, 0, ctx->stream>>>(iters, 0.999999, 1e-7, (double *)out);
        else
            k_fma_chain<float><<<blocks, FMA_THREADS, 0, ctx->stream>>>(iters, 0.999999f, 1e-7f, (float *)out);
        cudaEventRecord(e1, ctx->stream);
        cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return cuda_fail(e, "mbe_fma_peak", __FILE__, __LINE__);
        }
        ++ctx->launches;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double flops = 2.0 * (double)n * FMA_CHAINS * 16.0 * iters;
        if (r > 0 && ms > 0.f) best = std::max(best, flops / (ms * 1e-3) / 1e12);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    MBE_CU(cudaGetLastError());
    *tflops = best;
    return MBE_OK;
}
