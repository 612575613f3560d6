// peak.cu -- float64 FMA throughput of the device, measured by a kernel of
// independent FMA chains. The float64 storage form of the method (and the
// sphere-wall case that runs in it) is bound by the float64 units, so this
// measured rate is the peak of its roofline.
#include <cuda_runtime.h>

#include "../../include/lbmdem.h"
#include "launch.h"

namespace lbmdem {

// eight independent chains x <- x a + b per thread; a, b keep the values
// bounded (|a| < 1), the sum is stored so nothing is optimised away
__global__ void __launch_bounds__(256) fp64_fma_kernel(double* out, int iters, double a, double b) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    double x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = 1e-3 * (double)(t + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k];
    out[t] = s;
}

}  // namespace lbmdem

using namespace lbmdem;

extern "C" lbm_status lbm_fp64_fma_rate(int iters, double* tflops_out) {
    if (iters < 1 || !tflops_out) {
        set_global_error("lbm_fp64_fma_rate: iters must be >= 1 and tflops_out non-NULL");
        return LBM_ERR_INVALID;
    }
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        set_global_error("lbm_fp64_fma_rate: no CUDA device");
        return LBM_ERR_CUDA;
    }
    const int blocks = sms * 8, threads = 256;
    double* out = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    double best = 0.0;
    cudaError_t e = cudaMalloc(&out, sizeof(double) * (size_t)blocks * threads);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
        cudaEventRecord(e0, st);
        fp64_fma_kernel<<<blocks, threads, 0, st>>>(out, iters, 0.999999, 1e-7);
        cudaEventRecord(e1, st);
        e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaGetLastError();
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && ms > 0.f) {
            const double flops = 2.0 * 8.0 * (double)iters * blocks * threads;
            const double tf = flops / (ms * 1e-3) / 1e12;
            if (tf > best) best = tf;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    if (out) cudaFree(out);
    if (e != cudaSuccess) {
        set_global_error(std::string("lbm_fp64_fma_rate: ") + cudaGetErrorString(e));
        return LBM_ERR_CUDA;
    }
    *tflops_out = best;
    return LBM_OK;
}
