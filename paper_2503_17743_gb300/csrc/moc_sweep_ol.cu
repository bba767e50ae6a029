// The transport sweep of layouts whose layer planes lie off the axial
// lattice (the local axial mesh of Sec. 2.2): Eq. 3 on every piece, Eq. 4
// tallies.
//
// With planes off the lattice the upward frame and the mirrored frame of a
// stored track no longer cross the same pieces, and the tracks r, r + cpl, ...
// of a z-stack are no longer layer shifts of one another, so neither segment
// templates nor the shared (Qr, Sigma_t) tile of the main sweep apply.  A
// persistent grid takes work units (a 2D track with all its polar stacks)
// from the same counter as the main sweep; a warp sweeps 32 / GLn directions
// (track, frame, sense) side by side, GLn lanes each over energy groups, every
// lane generating its direction's pieces on the fly (walk_ol) from the
// integer (lattice index, fraction rank) decisions, and adds each
// contribution W (psi_in - psi_out) into the FP64 FSR tally with a native
// atomic.
#include "moc_device.cuh"
#include "moc_exp64.cuh"
#include "moc_kernels.h"

namespace {

constexpr int kOLBlock = 256;

// e^{-x}: FP32 on the MUFU pipe, FP64 by the table-driven method of
// moc_exp64.cuh (tab: its table in shared memory)
template <typename real>
__device__ __forceinline__ real ol_atten(real x, const double2 *tab);
template <>
__device__ __forceinline__ float ol_atten<float>(float x, const double2 *) {
    return fast_exp2(-x * 1.4426950408889634f);
}
template <>
__device__ __forceinline__ double ol_atten<double>(double x, const double2 *tab) {
    return moc_exp64::exp_neg(x, tab);
}

template <typename real>
__global__ void __launch_bounds__(kOLBlock) k_sweep_ol(DevLayout dl, DevState st, const int32_t *order,
                                                        int32_t n_work, const real *psi_in, real *psi_out) {
    if (st.scal[SC_CONV] != 0.0) return;  // converged: later iterations are no-ops
    __shared__ int s_work;
    __shared__ double s_leak[kOLBlock / 32];
    __shared__ double2 s_exp[sizeof(real) == 8 ? 64 : 1];
    if constexpr (sizeof(real) == 8)
        for (int i = threadIdx.x; i < 64; i += blockDim.x)
            s_exp[i] = make_double2(moc_exp64::kTable[i].hi, moc_exp64::kTable[i].lo);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int G = dl.G, Ph = dl.Ph;
    // lanes per direction: the smallest power of two holding the groups (at
    // most 32, in group chunks beyond); a warp sweeps 32 / GLn directions side
    // by side, each walked by its own lanes
    int GLn = 1;
    while (GLn < G && GLn < 32) GLn <<= 1;
    const int per = 32 / GLn, sub = lane / GLn, gl = lane - sub * GLn;
    const real scale = (real)st.scal[SC_SCALE];
    const real *qr = reinterpret_cast<const real *>(st.qr);
    const real *sig = reinterpret_cast<const real *>(st.sig_t);
    double leak = 0.0;  // this lane's W psi leaving through vacuum faces
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_work = atomicAdd(st.counter, 1);
        __syncthreads();
        const int w = s_work;
        if (w >= n_work) break;
        const int T = order[w];
        for (int ph = 0; ph < Ph; ++ph) {
            const StackDesc &d = dl.desc[(int64_t)T * Ph + ph];
            const int n_dir = 4 * d.n_trk;
            const real W = (real)d.W;
            const int32_t *reg2d = dl.reg2d + d.seg2d_off;
            for (int task0 = warp * per; task0 < n_dir; task0 += nwarps * per) {
                const int task = task0 + sub;
                if (task >= n_dir) continue;
                const int k = task >> 2, v = task & 3;  // direction v = frame * 2 + sense
                const int64_t gid = d.trk_off + k;
                const int64_t dst = dl.dst ? (int64_t)__ldg(dl.dst + gid * 4 + v) : -1;
                for (int g0 = 0; g0 < G; g0 += GLn) {
                    const int g = g0 + gl;
                    const bool on = g < G;
                    real psi = (psi_in && on) ? psi_in[(gid * 4 + v) * G + g] * scale : (real)0;
                    auto visit = [&](int b, int L, real len) {
                        if (!on) return;
                        const int64_t f = fsr_of(dl, __ldg(reg2d + b), L);
                        const int m = __ldg(dl.fsr_mat + f);
                        const real x = ol_atten<real>(sig[(size_t)m * G + g] * len, s_exp);
                        // Eq. 3: psi_in - psi_out = (psi_in - Qr)(1 - e^{-Sigma_t l})
                        const real dq = psi - qr[(size_t)f * G + g];
                        const real t = fma(-dq, x, dq);
                        psi -= t;
                        atomicAdd(st.tally + (size_t)f * G + g, (double)(W * t));  // Eq. 4
                    };
                    walk_ol<real>(dl, d, d.i_lo + k, v >> 1, v & 1, visit);
                    if (on) {
                        if (dst >= 0 && dst < dl.n_slots) psi_out[dst * G + g] = psi;
                        else leak += (double)(W * psi);
                    }
                }
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) leak += __shfl_down_sync(0xffffffffu, leak, o);
    if (lane == 0) s_leak[warp] = leak;
    __syncthreads();
    if (threadIdx.x == 0) {
        double v = 0.0;
        for (int k = 0; k < nwarps; ++k) v += s_leak[k];
        if (v != 0.0) atomicAdd(st.scal + SC_LEAK, v);
    }
}

}  // namespace

int sweep_ol_block() { return kOLBlock; }

cudaError_t launch_sweep_ol(int precision, const DevLayout &dl, const DevState &st, const int32_t *order,
                            int32_t n_work, const void *psi_in, void *psi_out, int32_t *counter, int grid,
                            cudaStream_t s) {
    DevState a = st;
    a.counter = counter;
    if (precision == MOC_FP64)
        k_sweep_ol<double><<<grid, kOLBlock, 0, s>>>(dl, a, order, n_work, (const double *)psi_in,
                                                     (double *)psi_out);
    else
        k_sweep_ol<float><<<grid, kOLBlock, 0, s>>>(dl, a, order, n_work, (const float *)psi_in,
                                                    (float *)psi_out);
    return cudaGetLastError();
}
