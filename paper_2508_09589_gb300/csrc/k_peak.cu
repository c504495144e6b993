// FP64 fused multiply-add rate of the GPU (a diagnostic): the outer Krylov solver's FP64 operator
// applies are bound by it, so its measured value is the denominator of their roofline.
#include <cuda_runtime.h>

#include "../../include/st.h"

namespace st {
st_status set_c_error(st_status code, const char* msg);

// Each thread runs 8 independent FMA chains of `iters` steps (enough independent work per
// warp to keep the FP64 pipe busy), then stores their sum so nothing is optimised away.
__global__ void __launch_bounds__(256) k_fma64(double* out, int iters, double a, double b) {
    double x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = (double)(threadIdx.x + k) * 1e-3;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
    }
    double s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
}  // namespace st

extern "C" st_status st_fp64_fma_rate(int device, double* tflops) {
    using namespace st;
    if (!tflops) return set_c_error(ST_ERR_ARG, "null argument");
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return set_c_error(ST_ERR_CUDA, "cudaSetDevice failed");
    }
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const int blocks = (sms > 0 ? sms : 152) * 8, threads = 256, iters = 4096;
    double* out = nullptr;
    if (cudaMalloc((void**)&out, sizeof(double) * blocks * threads) != cudaSuccess) {
        cudaGetLastError();
        return set_c_error(ST_ERR_OOM, "scratch allocation failed");
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    k_fma64<<<blocks, threads>>>(out, iters, 0.999999, 1e-7);  // warm-up
    float best = 1e30f;
    for (int r = 0; r < 5; ++r) {
        cudaEventRecord(e0);
        k_fma64<<<blocks, threads>>>(out, iters, 0.999999, 1e-7);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) best = ms;
    }
    const cudaError_t e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (e != cudaSuccess) return set_c_error(ST_ERR_CUDA, "FMA rate kernel failed");
    const double fmas = (double)blocks * threads * iters * 8.0;
    *tflops = 2.0 * fmas / (best * 1e-3) / 1e12;
    return ST_OK;
}
