// Measurement utility (the paper has no counterpart): the fused
// multiply-add issue rate this GPU sustains in one precision, measured with
// independent FMA chains, as the denominator of the ALU roofline of the
// Gauss-point flux and reconstruction kernels.
#include <cuda_runtime.h>

#include "hgks.h"

namespace {

constexpr int NCHAIN = 8;      // independent chains per thread (hides the FMA latency)
constexpr int THREADS = 256;
constexpr int BLOCKS_PER_SM = 8;

template <typename R>
__global__ void __launch_bounds__(THREADS) k_fma_probe(R *__restrict__ out, int iters, R b, R c)
{
    R a[NCHAIN];
#pragma unroll
    for (int k = 0; k < NCHAIN; ++k) a[k] = R(threadIdx.x + k) * R(1e-3);
#pragma unroll 4
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < NCHAIN; ++k) a[k] = fma(a[k], b, c);
    }
    R s = R(0);
#pragma unroll
    for (int k = 0; k < NCHAIN; ++k) s += a[k];
    // a data-dependent store the compiler cannot drop (the chains converge
    // to c/(1 - b) > 0, so the branch is never taken)
    if (s < R(0)) out[blockIdx.x] = s;
}

template <typename R> int probe(cudaStream_t st, int iters, double *tflops)
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return HGKS_E_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return HGKS_E_CUDA;
    const int blocks = sms * BLOCKS_PER_SM;
    R *out = nullptr;
    if (cudaMalloc(&out, sizeof(R) * blocks) != cudaSuccess) return HGKS_E_NOMEM;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = HGKS_OK;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = HGKS_E_CUDA;
    if (rc == HGKS_OK) {
        const R b = R(0.999999), c = R(1e-6);
        k_fma_probe<R><<<blocks, THREADS, 0, st>>>(out, iters / 8, b, c);  // warm-up
        cudaEventRecord(e0, st);
        k_fma_probe<R><<<blocks, THREADS, 0, st>>>(out, iters, b, c);
        cudaEventRecord(e1, st);
        float ms = 0.f;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
            cudaGetLastError() != cudaSuccess || !(ms > 0.f))
            rc = HGKS_E_CUDA;
        else
            *tflops = 2.0 * NCHAIN * double(iters) * blocks * THREADS / (ms * 1e-3) / 1e12;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    return rc;
}

}  // namespace

extern "C" int hgks_alu_peak(int precision, void *cuda_stream, double *tflops)
{
    if (!tflops || (precision != HGKS_FP64 && precision != HGKS_MIXED)) return HGKS_E_INVALID;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    // about 50 ms per measurement at the GB300's rates
    return precision == HGKS_FP64 ? probe<double>(st, 16384, tflops) : probe<float>(st, 1 << 20, tflops);
}
