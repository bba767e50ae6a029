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

// Throughput probes of the other units the FP32 sweep issues to (one
// kernel per unit, `iters` steps of 8 independent operations per thread,
// every SM filled with 8 blocks of 256 threads).  Each keeps its results
// alive through a store that never happens.

// FP32 fused multiply-add, scalar (one lane operation per instruction)
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__global__ void __launch_bounds__(256) k_fma_rate(int iters, float a, float b, float *sink,
                                                  long long *clk) {
    const long long c0 = clock64();
    const unsigned long long t0 = global_ns();
    float x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = 0.5f + 0.01f * (float)((threadIdx.x + j) & 31);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 8; ++j) asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(x[j]) : "f"(a), "f"(b));
    }
    float s = 0.0f;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += x[j];
    if (s == -1.0f) sink[blockIdx.x] = s;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        // the SM clock of this block: clock cycles over global-timer ns
        const long long c1 = clock64();
        const unsigned long long t1 = global_ns();
        clk[0] = c1 - c0;
        clk[1] = (long long)(t1 - t0);
    }
}

// FP32 fused multiply-add on packed pairs (fma.rn.f32x2: two lane
// operations per instruction)
__global__ void __launch_bounds__(256) k_fma2_rate(int iters, float a, float b, float *sink) {
    unsigned long long x[8], av, bv;
    asm("mov.b64 %0, {%1, %1};" : "=l"(av) : "f"(a));
    asm("mov.b64 %0, {%1, %1};" : "=l"(bv) : "f"(b));
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const float v = 0.5f + 0.01f * (float)((threadIdx.x + j) & 31);
        asm("mov.b64 %0, {%1, %1};" : "=l"(x[j]) : "f"(v));
    }
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 8; ++j) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[j]) : "l"(av), "l"(bv));
    }
    unsigned long long s = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) s ^= x[j];
    if (s == 1ull) sink[blockIdx.x] = (float)s;
}

// conflict-free shared-memory integer reductions: the 32 lanes of a warp add
// into 32 different banks (the sweep's fixed-point tally adds)
__global__ void __launch_bounds__(256) k_red_rate(int iters, float *sink) {
    __shared__ int buf[8 * 256];
    for (int i = threadIdx.x; i < 8 * 256; i += blockDim.x) buf[i] = 0;
    __syncthreads();
    const unsigned base = (unsigned)__cvta_generic_to_shared(buf) + 4u * (threadIdx.x & 255);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 8; ++j)
            asm volatile("red.shared.add.s32 [%0], %1;" ::"r"(base + 1024u * j), "r"(i) : "memory");
    }
    __syncthreads();
    if (buf[threadIdx.x] == -7) sink[blockIdx.x] = 1.0f;
}

// conflict-free 16-byte shared-memory loads (the sweep's row loads): a warp
// reads 512 contiguous bytes per instruction
__global__ void __launch_bounds__(256) k_lds_rate(int iters, float *sink) {
    __shared__ __align__(16) unsigned buf[4 * 256 * 2];
    for (int i = threadIdx.x; i < 4 * 256 * 2; i += blockDim.x) buf[i] = i;
    __syncthreads();
    const unsigned sbase = (unsigned)__cvta_generic_to_shared(buf);
    const unsigned lane_off = 16u * (threadIdx.x & 31);
    unsigned acc = 0;
    for (int i = 0; i < iters; ++i) {
        // a different 512-byte block each step (addresses the compiler
        // cannot hoist out of the loop); lanes stay 16 bytes apart.  Byte
        // offsets inside buf: lane_off + 512 k with k = (block ^ j) < 16,
        // so at most 496 + 7680 + 16 = 8192 = sizeof(buf)
        const unsigned blk = (unsigned)((i + (threadIdx.x >> 5)) & 15);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            unsigned a, b, c, d;
            const unsigned off = lane_off + 512u * (blk ^ (unsigned)j);
            asm volatile("ld.volatile.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                         : "=r"(a), "=r"(b), "=r"(c), "=r"(d)
                         : "r"(sbase + off));
            acc ^= a ^ b ^ c ^ d;
        }
    }
    if (acc == 0x12345u) sink[blockIdx.x] = 1.0f;
}

// float-to-integer conversions with rounding to nearest (the sweep rounds
// every tally contribution to the fixed-point grid with one)
__global__ void __launch_bounds__(256) k_f2i_rate(int iters, float *sink) {
    float x[8];
    int acc = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = 1.5f + (float)((threadIdx.x + j) & 31);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            int v;
            asm volatile("cvt.rni.s32.f32 %0, %1;" : "=r"(v) : "f"(x[j]));
            acc += v;
        }
    }
    if (acc == 7) sink[blockIdx.x] = 1.0f;
}

}  // namespace

extern "C" int moc_measure_unit_rates(int32_t device, double *out, int32_t n) {
    if (!out || n < 1) { moc_set_error("NULL argument or n < 1"); return MOC_ERR_INVALID_ARG; }
    if (cudaSetDevice(device) != cudaSuccess) { moc_set_error("cudaSetDevice failed"); return MOC_ERR_CUDA; }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
        moc_set_error("cudaDeviceGetAttribute failed");
        return MOC_ERR_CUDA;
    }
    const int blocks = sms * 8, threads = 256;
    float *sink = nullptr;
    long long *clk = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(&sink, blocks * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&clk, 2 * sizeof(long long));
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    // time kernel `which` (the last of three runs): milliseconds
    auto timed = [&](int which, int iters, float &ms) {
        for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
            e = cudaEventRecord(e0);
            if (e != cudaSuccess) break;
            switch (which) {
                case 0: k_fma_rate<<<blocks, threads>>>(iters, 0.999f, 0.001f, sink, clk); break;
                case 1: k_fma2_rate<<<blocks, threads>>>(iters, 0.999f, 0.001f, sink); break;
                case 2: k_red_rate<<<blocks, threads>>>(iters, sink); break;
                case 3: k_lds_rate<<<blocks, threads>>>(iters, sink); break;
                default: k_f2i_rate<<<blocks, threads>>>(iters, sink); break;
            }
            e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaEventRecord(e1);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        }
    };
    const double lanes = (double)blocks * threads * 8.0;
    float ms[5] = {0, 0, 0, 0, 0};
    const int iters[5] = {16384, 16384, 4096, 4096, 8192};
    for (int k = 0; k < 5 && e == cudaSuccess; ++k) timed(k, iters[k], ms[k]);
    long long hc[2] = {0, 0};
    if (e == cudaSuccess) {
        // the SM clock during the scalar FMA run (block 0 of its last repetition)
        timed(0, iters[0], ms[0]);
        if (e == cudaSuccess) e = cudaMemcpy(hc, clk, sizeof(hc), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && hc[1] <= 0) e = cudaErrorUnknown;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (sink) cudaFree(sink);
    if (clk) cudaFree(clk);
    for (int k = 0; k < 5; ++k)
        if (e == cudaSuccess && ms[k] <= 0.0f) e = cudaErrorUnknown;
    if (e != cudaSuccess) {
        moc_set_error(std::string("unit-rate probe: ") + cudaGetErrorString(e));
        return MOC_ERR_CUDA;
    }
    const double v[8] = {(double)sms,
                         (double)hc[0] / (double)hc[1] * 1e3,
                         lanes * iters[0] / (ms[0] * 1e-3),
                         2.0 * lanes * iters[1] / (ms[1] * 1e-3),
                         lanes * iters[2] / (ms[2] * 1e-3),
                         16.0 * lanes * iters[3] / (ms[3] * 1e-3),
                         lanes * iters[4] / (ms[4] * 1e-3),
                         0.0};
    for (int i = 0; i < n && i < 7; ++i) out[i] = v[i];
    return MOC_OK;
}

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
