// Throughput probe of the exponential unit, used to state the ALU roofline of
// the sweep: every integration (Eq. 3) costs one ex2.approx.ftz.f32.
//
// Each thread runs 8 independent chains x <- 2^(x * c) for `iters` steps
// (c < 0 keeps x in (0, 1]); the grid is sized to fill every SM.  Returns the
// sustained ex2 rate of the whole device.
#include <cuda_runtime.h>

#include "moc_device.cuh"
#include "moc_exp64.cuh"
#include "moc_internal.h"

namespace {

// one element per thread: the sweep's FP64 attenuation factor and CUDA's exp
__global__ void __launch_bounds__(256) k_eval_exp64(const double *x, int64_t n, double *y, double *y_lib) {
    __shared__ double2 tab[64];
    for (int i = threadIdx.x; i < 64; i += blockDim.x)
        tab[i] = make_double2(moc_exp64::kTable[i].hi, moc_exp64::kTable[i].lo);
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    y[i] = moc_exp64::exp_neg(x[i], tab);
    y_lib[i] = exp(-x[i]);
}

__global__ void __launch_bounds__(256) k_ex2_rate(int iters, float c, float *sink) {
    float x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = 0.25f + 0.01f * (float)((threadIdx.x + j) & 31);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            float y;
            asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x[j] * c));
            x[j] = y;
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += x[j];
    if (s == -1.0f) sink[blockIdx.x] = s;  // never true; keeps the chains alive
}

// the FP32 sweep's attenuation factor e^{-tau} = 2^{-b}, b = tau log2 e
__global__ void __launch_bounds__(256) k_eval_exp32(const float *b, int64_t n, float *e) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) e[i] = fast_exp2(-b[i]);
}

}  // namespace

extern "C" int moc_measure_ex2_rate(int32_t device, double *ex2_per_second, double *sm_count) {
    if (!ex2_per_second) { moc_set_error("NULL argument"); return MOC_ERR_INVALID_ARG; }
    if (cudaSetDevice(device) != cudaSuccess) { moc_set_error("cudaSetDevice failed"); return MOC_ERR_CUDA; }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
        moc_set_error("cudaDeviceGetAttribute failed");
        return MOC_ERR_CUDA;
    }
    const int blocks = sms * 8, threads = 256, iters = 4096;
    float *sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float ms = 0.0f;
    cudaError_t e = cudaMalloc(&sink, blocks * sizeof(float));
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {  // the last of 3 runs is timed
        k_ex2_rate<<<blocks, threads>>>(iters, -0.5f, sink);
        e = cudaEventRecord(e0);
        if (e == cudaSuccess) k_ex2_rate<<<blocks, threads>>>(iters, -0.5f, sink);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(e1);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (sink) cudaFree(sink);
    if (e != cudaSuccess || ms <= 0.0f) {
        moc_set_error(std::string("ex2 probe: ") + cudaGetErrorString(e));
        return MOC_ERR_CUDA;
    }
    *ex2_per_second = (double)blocks * threads * iters * 8.0 / (ms * 1e-3);
    if (sm_count) *sm_count = sms;
    return MOC_OK;
}

extern "C" int moc_eval_attenuation_f64(int32_t device, const double *x, int64_t n, double *y,
                                        double *y_lib) {
    if (n < 0 || (n > 0 && (!x || !y || !y_lib))) { moc_set_error("NULL argument or n < 0"); return MOC_ERR_INVALID_ARG; }
    if (n == 0) return MOC_OK;
    if (n > ((int64_t)1 << 28)) { moc_set_error("n above 2^28"); return MOC_ERR_INVALID_ARG; }
    if (cudaSetDevice(device) != cudaSuccess) { moc_set_error("cudaSetDevice failed"); return MOC_ERR_CUDA; }
    double *d = nullptr;
    const size_t bytes = (size_t)n * sizeof(double);
    cudaError_t e = cudaMalloc(&d, 3 * bytes);
    if (e == cudaSuccess) e = cudaMemcpy(d, x, bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        k_eval_exp64<<<(unsigned)((n + 255) / 256), 256>>>(d, n, d + n, d + 2 * n);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(y, d + n, bytes, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(y_lib, d + 2 * n, bytes, cudaMemcpyDeviceToHost);
    if (d) cudaFree(d);
    if (e != cudaSuccess) {
        moc_set_error(std::string("attenuation probe: ") + cudaGetErrorString(e));
        return MOC_ERR_CUDA;
    }
    return MOC_OK;
}

extern "C" int moc_eval_attenuation_f32(int32_t device, const float *b, int64_t n, float *e) {
    if (n < 0 || (n > 0 && (!b || !e))) { moc_set_error("NULL argument or n < 0"); return MOC_ERR_INVALID_ARG; }
    if (n == 0) return MOC_OK;
    if (n > ((int64_t)1 << 28)) { moc_set_error("n above 2^28"); return MOC_ERR_INVALID_ARG; }
    if (cudaSetDevice(device) != cudaSuccess) { moc_set_error("cudaSetDevice failed"); return MOC_ERR_CUDA; }
    float *d = nullptr;
    const size_t bytes = (size_t)n * sizeof(float);
    cudaError_t err = cudaMalloc(&d, 2 * bytes);
    if (err == cudaSuccess) err = cudaMemcpy(d, b, bytes, cudaMemcpyHostToDevice);
    if (err == cudaSuccess) {
        k_eval_exp32<<<(unsigned)((n + 255) / 256), 256>>>(d, n, d + n);
        err = cudaGetLastError();
    }
    if (err == cudaSuccess) err = cudaMemcpy(e, d + n, bytes, cudaMemcpyDeviceToHost);
    if (d) cudaFree(d);
    if (err != cudaSuccess) {
        moc_set_error(std::string("attenuation probe: ") + cudaGetErrorString(err));
        return MOC_ERR_CUDA;
    }
    return MOC_OK;
}
