// Group-wise reaction rates of the scalar flux with a scratch area that lives
// in a fixed device array of this library, so that the call allocates nothing.
//
// It is a variant of the finalize / reduce pair (k_finalize writes per-block
// FP64 partial sums into a scratch buffer of the solve state, k_reduce_k sums
// them).  Here the partials go to `g_rates_scratch` instead: a file-scope
// static device array of kRatesScratchDoubles doubles (66 KB), enough for
// kRatesMaxBlocks blocks x kRatesMaxGroups groups x 2 rates plus the 2 x G
// results.
//
// Nothing in the scratch has to start at zero: every block overwrites its
// own partials before the single-block final pass reads them, and the final
// pass overwrites the results.  Two calls that overlap in time (on two
// streams, or from two host threads) share the one scratch array and race;
// callers must serialise them.
#include <algorithm>

#include "moc_device.cuh"
#include "moc_kernels.h"

static __device__ __align__(256) double g_rates_scratch[kRatesScratchDoubles];

namespace {

__device__ __forceinline__ double block_total(double v, double *sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += sh[i];
    return r;  // valid in thread 0
}

// per block and group: sum_i V_i nuSigma_f phi_{i,g} and sum_i V_i Sigma_a phi_{i,g}
// over the block's FSRs (raw flux; the normalisation is applied at the end)
__global__ void k_rates_partial(DevLayout dl, DevState st, int32_t nfsr, double *scratch) {
    __shared__ double sh[32];
    const int G = dl.G;
    for (int g = 0; g < G; ++g) {
        double p = 0.0, a = 0.0;
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nfsr; i += gridDim.x * blockDim.x) {
            const int m = dl.fsr_mat[i];
            const double V = st.vol[i];
            const double phi = st.phi[(size_t)i * G + g];
            double sa = st.sig_t64[m * G + g];
            for (int h = 0; h < G; ++h) sa -= st.sig_s64[((size_t)m * G + g) * G + h];
            p += V * st.nsf64[m * G + g] * phi;
            a += V * sa * phi;
        }
        const double tp = block_total(p, sh);
        const double ta = block_total(a, sh);
        if (threadIdx.x == 0) {
            scratch[((size_t)blockIdx.x * G + g) * 2 + 0] = tp;
            scratch[((size_t)blockIdx.x * G + g) * 2 + 1] = ta;
        }
    }
}

// one block: sum the partials in block order (deterministic) and scale to
// the normalised flux; results at scratch[kRatesResultOffset + c * G + g]
__global__ void k_rates_final(DevState st, int G, int nblocks, double *scratch) {
    const int t = threadIdx.x;
    if (t >= 2 * G) return;
    const int c = t / G, g = t - c * G;
    double v = 0.0;
    for (int b = 0; b < nblocks; ++b) v += scratch[((size_t)b * G + g) * 2 + c];
    scratch[kRatesResultOffset + c * G + g] = v * st.scal[SC_SCALE];
}

}  // namespace

cudaError_t rates_scratch_address(double **ptr) {
    return cudaGetSymbolAddress(reinterpret_cast<void **>(ptr), g_rates_scratch);
}

cudaError_t launch_group_rates_static(const DevLayout &dl, const DevState &st, int32_t nfsr,
                                      double *scratch, cudaStream_t s) {
    const int nb = (int)std::min<int64_t>(kRatesMaxBlocks, std::max<int64_t>(1, (nfsr + 255) / 256));
    k_rates_partial<<<nb, 256, 0, s>>>(dl, st, nfsr, scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_rates_final<<<1, 64, 0, s>>>(st, dl.G, nb, scratch);
    return cudaGetLastError();
}
