// FP64 fused multiply-add throughput of the current device
// (include/mrrr_probe.h): the denominator of the solver kernels' roofline.
#include <cuda_runtime.h>

#include "mrrr.h"
#include "mrrr_probe.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

// Each thread: kChains independent chains x = x * b + c of `iters` steps.
// b and c keep every chain finite and normal; the sum of the results is
// stored so that no chain is dead code.
__global__ void k_probe_dfma(double* out, int iters, double b, double c) {
    double x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = 1.0 + 1e-3 * (threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) x[k] = fma(x[k], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" int mrrr_probe_fp64_fma(int iters, double* gflops, double* ms, void* stream) {
    if (!gflops || !ms) return MRRR_ERR_ARG;
    if (iters <= 0) iters = 65536;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                   cudaSuccess) {
        cudaGetLastError();
        return MRRR_ERR_CUDA;
    }
    cudaStream_t st = (cudaStream_t)stream;
    double* out = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    int rc = MRRR_ERR_CUDA;
    float t = 0.f;
    if (cudaMalloc(&out, sizeof(double) * (size_t)sms * kThreads) != cudaSuccess) goto done;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) goto done;
    for (int rep = 0; rep < 2; ++rep) {
        if (cudaEventRecord(a, st) != cudaSuccess) goto done;
        k_probe_dfma<<<sms, kThreads, 0, st>>>(out, iters, 0.9999999999, 1e-10);
        if (cudaGetLastError() != cudaSuccess || cudaEventRecord(b, st) != cudaSuccess) goto done;
        if (cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(&t, a, b) != cudaSuccess) goto done;
    }
    *ms = t;
    *gflops = 2.0 * (double)sms * kThreads * kChains * (double)iters / (t * 1e-3) / 1e9;
    rc = MRRR_OK;
done:
    if (rc != MRRR_OK) cudaGetLastError();
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (out) cudaFree(out);
    return rc;
}
