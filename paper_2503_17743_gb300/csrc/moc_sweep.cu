// The transport sweep kernel (Eq. 3 on every segment, Eq. 4 tallies).
//
// Work decomposition.  A persistent grid; each block takes one work unit at a
// time from a global counter: a 2D track with all its polar z-stacks (units in
// decreasing work order).  A warp is split into 32/GL slots of GL lanes, the
// lanes of a slot over energy groups.  A warp task is (polar stack, class r,
// block of 32/GL consecutive tracks of the class, sense): the tracks
// r, r + cpl, r + 2 cpl, ... of a z-stack are one track shifted up by one
// layer each (Eq. 5, layer planes on the axial lattice), so the warp walks one
// segment template and slot j applies each piece at layer L_t + j.  Every
// slot sweeps both frames: its upward track and the mirrored downward track
// that shares its segments (layers NL-1-L).  The slots of a warp touch
// consecutive rows, so shared-memory accesses do not collide.
//
// Shared tally (SMEM = true): per unit the block stages one row per
// (2D segment, layer) FSR the unit crosses, holding (Qr, Sigma_t) of every
// group, plus a zeroed tally row; pieces touch only shared memory and the rows
// are flushed into the FP64 global tally once per unit.  Templates come from
// the stored set (EXP, Sec. 4.2, walked four pieces at a time with the next
// four records in flight) or are generated on the fly (OTF).  Without the
// shared tally (SMEM = false) pieces read Qr from global memory and add straight
// into the FP64 global tally.
#include <climits>

#include "moc_device.cuh"
#include "moc_kernels.h"

namespace {

constexpr float kLog2e = 1.4426950408889634f;

template <typename real>
struct Vec2;
template <>
struct Vec2<float> {
    using type = float2;
};
template <>
struct Vec2<double> {
    using type = double2;
};

template <typename real>
__device__ __forceinline__ real attenuation(real x);  // e^{-Sigma_t l}
template <>
__device__ __forceinline__ float attenuation<float>(float x) {
    return fast_exp2(-x);  // Sigma_t is pre-scaled by log2(e)
}
template <>
__device__ __forceinline__ double attenuation<double>(double x) {
    return exp(-x);
}

// per polar stack of the work unit, cached in shared memory
struct UnitStack {
    int64_t trk_off, tpl_base;
    double W;
    int32_t n_trk, i_lo, task_pre, pad;
};
constexpr int kMaxPh = 16;

template <typename real, int GL, bool SMEM>
__global__ void __launch_bounds__(256, 3) k_sweep(DevLayout dl, DevState st, const int32_t *order,
                                                  int32_t n_work, int32_t cap, const real *psi_in,
                                                  real *psi_out) {
    using vec2 = typename Vec2<real>::type;
    constexpr int SLOTS = 32 / GL;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_work, s_next, s_ntask;
    __shared__ UnitStack s_us[kMaxPh];
    __shared__ double s_leak[8];
    const int G = dl.G, NL = dl.NL, M = dl.M, Ph = dl.Ph, cpl = dl.cpl;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    const int j = lane / GL;        // slot: track of the block
    const int ql = lane & (GL - 1); // group within the chunk
    // shared layout: sig [M*GL] | rows (Qr, Sigma_t) [cap*GL] | tally [cap*GL]
    real *sig = reinterpret_cast<real *>(smem);
    size_t off = ((size_t)M * GL * sizeof(real) + 15) & ~(size_t)15;
    vec2 *rows = reinterpret_cast<vec2 *>(smem + off);
    off += (size_t)cap * GL * sizeof(vec2);
    real *tl_s = reinterpret_cast<real *>(smem + off);

    const real scale = (real)st.scal[SC_SCALE];
    const real *qr_g = reinterpret_cast<const real *>(st.qr);
    const real *sig_g = reinterpret_cast<const real *>(st.sig_t);
    const SegRec<real> *recs = reinterpret_cast<const SegRec<real> *>(dl.segs);
    double leak = 0.0;

    for (;;) {
        __syncthreads();
        if (tid == 0) s_work = atomicAdd(st.counter, 1);
        __syncthreads();
        const int w = s_work;
        if (w >= n_work) break;
        const int T = order[w];
        if (tid == 0) {
            int pre = 0;
            for (int ph = 0; ph < Ph; ++ph) {
                const StackDesc &e = dl.desc[(int64_t)T * Ph + ph];
                UnitStack u;
                u.trk_off = e.trk_off;
                u.tpl_base = e.exp_base;
                u.W = e.W;
                u.n_trk = e.n_trk;
                u.i_lo = e.i_lo;
                u.task_pre = pre;
                u.pad = 0;
                s_us[ph] = u;
                // per class: blocks of SLOTS tracks, two senses
                for (int r = 0; r < min(cpl, e.n_trk); ++r) {
                    const int cnt = (e.n_trk - r + cpl - 1) / cpl;
                    pre += 2 * ((cnt + SLOTS - 1) / SLOTS);
                }
            }
            s_ntask = pre;
        }
        __syncthreads();
        const int ntask = s_ntask;
        if (ntask == 0) continue;
        const StackDesc &d0 = dl.desc[(int64_t)T * Ph];
        const int nb = d0.nb;
        const int32_t *reg2d = dl.reg2d + d0.seg2d_off;
        for (int g0 = 0; g0 < G; g0 += GL) {
            const int gc = min(GL, G - g0);
            for (int e = tid; e < M * GL; e += blockDim.x) {
                const int m = e / GL, qq = e - m * GL;
                real v = qq < gc ? sig_g[m * G + g0 + qq] : (real)0;
                if (sizeof(real) == 4) v = (real)((float)v * kLog2e);
                sig[e] = v;
            }
            if (SMEM) {
                // rows of the (2D segment, layer) FSRs the unit crosses
                for (int b = warp; b < nb; b += nwarps) {
                    const int reg = __ldg(reg2d + b);
                    for (int x = lane; x < NL * GL; x += 32) {
                        const int L = x / GL, qq = x - L * GL;
                        const int f = reg * NL + L;
                        const int e = (b * NL + L) * GL + qq;
                        vec2 v;
                        if (qq < gc) {
                            const int m = __ldg(dl.fsr_mat + f);
                            real sg = sig_g[m * G + g0 + qq];
                            if (sizeof(real) == 4) sg = (real)((float)sg * kLog2e);
                            v.x = qr_g[(size_t)f * G + g0 + qq];
                            v.y = sg;
                        } else {
                            v.x = (real)0;
                            v.y = (real)0;
                        }
                        rows[e] = v;
                        tl_s[e] = (real)0;
                    }
                }
            }
            if (tid == 0) s_next = 0;
            __syncthreads();

            for (;;) {
                int t = 0;
                if (lane == 0) t = atomicAdd(&s_next, 1);
                t = __shfl_sync(0xffffffffu, t, 0);
                if (t >= ntask) break;
                // decode the warp task: polar stack, sense, class r, block mb
                int ph = 0;
                while (ph + 1 < Ph && t >= s_us[ph + 1].task_pre) ++ph;
                const UnitStack u = s_us[ph];
                int x = t - u.task_pre;
                const int sense = x & 1;
                x >>= 1;
                int r = 0, cnt = 0;
                for (;; ++r) {
                    cnt = (u.n_trk - r + cpl - 1) / cpl;
                    const int nmb = (cnt + SLOTS - 1) / SLOTS;
                    if (x < nmb) break;
                    x -= nmb;
                }
                const int mb = x;
                const int J = min(SLOTS, cnt - mb * SLOTS);  // tracks in this block
                const bool valid = j < J;
                const int k = r + (mb * SLOTS + j) * cpl;    // track of this slot in the stack
                const int64_t gid = u.trk_off + k;
                const real W = (real)u.W;
                real psiU = 0, psiD = 0;
                int64_t dstU = -1, dstD = -1;
                if (valid) {
                    if (psi_in && ql < gc) {
                        psiU = psi_in[(gid * 4 + 0 * 2 + sense) * G + g0 + ql] * scale;
                        psiD = psi_in[(gid * 4 + 1 * 2 + sense) * G + g0 + ql] * scale;
                    }
                    if (dl.dst) {
                        dstU = dl.dst[gid * 4 + 0 * 2 + sense];
                        dstD = dl.dst[gid * 4 + 1 * 2 + sense];
                    }
                }
                // one template piece for every slot: slot j is at layer Lt + lofs
                auto visit = [&](int b, int Lt, real len, int lofs) {
                    const int L = Lt + lofs;
                    if (!valid || (unsigned)L >= (unsigned)NL) return;
                    const int LD = NL - 1 - L;
                    if (SMEM) {
                        const int eU = (b * NL + L) * GL + ql, eD = (b * NL + LD) * GL + ql;
                        const vec2 aU = rows[eU], aD = rows[eD];
                        // Eq. 3: psi_out = Qr + (psi_in - Qr) e^{-Sigma_t l}
                        const real xU = attenuation<real>(aU.y * len);
                        const real xD = attenuation<real>(aD.y * len);
                        const real nU = aU.x + (psiU - aU.x) * xU;
                        const real nD = aD.x + (psiD - aD.x) * xD;
                        atomicAdd(tl_s + eU, (psiU - nU) * W);
                        atomicAdd(tl_s + eD, (psiD - nD) * W);
                        psiU = nU;
                        psiD = nD;
                    } else {
                        const int reg = __ldg(reg2d + b);
                        const size_t fU = (size_t)reg * NL + L, fD = (size_t)reg * NL + LD;
                        const int mU = __ldg(dl.fsr_mat + fU), mD = __ldg(dl.fsr_mat + fD);
                        const real qU = ql < gc ? qr_g[fU * G + g0 + ql] : (real)0;
                        const real qD = ql < gc ? qr_g[fD * G + g0 + ql] : (real)0;
                        const real xU = attenuation<real>(sig[mU * GL + ql] * len);
                        const real xD = attenuation<real>(sig[mD * GL + ql] * len);
                        const real nU = qU + (psiU - qU) * xU;
                        const real nD = qD + (psiD - qD) * xD;
                        if (ql < gc) {
                            atomicAdd(st.tally + fU * G + g0 + ql, (double)(psiU - nU) * (double)W);
                            atomicAdd(st.tally + fD * G + g0 + ql, (double)(psiD - nD) * (double)W);
                        }
                        psiU = nU;
                        psiD = nD;
                    }
                };
                if (u.tpl_base >= 0) {
                    // stored template of class r: line i_lo + r, slot layer offset mb*SLOTS + j
                    const int64_t tpl = u.tpl_base + r;
                    const int lofs = mb * SLOTS + j;
                    const int lo = -(mb * SLOTS + J - 1), hi = NL - mb * SLOTS;
                    const int Lmin = dl.tpl_lmin[tpl];
                    const int64_t lb = dl.tpl_loff[tpl];
                    const int nL = (int)(dl.tpl_loff[tpl + 1] - lb) - 1;
                    const int64_t tb = dl.tpl_off[tpl];
                    const int64_t p0 = tb + dl.tpl_lidx[lb + min(max(lo - Lmin, 0), nL)];
                    const int64_t p1 = tb + dl.tpl_lidx[lb + min(max(hi - Lmin, 0), nL)];
                    const int n = (int)(p1 - p0);
                    const int dir = sense == 0 ? 1 : -1;
                    int64_t p = sense == 0 ? p0 : p1 - 1;
                    int s = 0;
                    SegRec<real> c0, c1, c2, c3;
                    if (n >= 4) {
                        c0 = recs[p]; c1 = recs[p + dir]; c2 = recs[p + 2 * dir]; c3 = recs[p + 3 * dir];
                    }
                    for (; s + 4 <= n; s += 4) {
                        // the next four records in flight while these four are swept
                        SegRec<real> n0, n1, n2, n3;
                        const bool more = s + 8 <= n;
                        if (more) {
                            n0 = recs[p + 4 * dir]; n1 = recs[p + 5 * dir];
                            n2 = recs[p + 6 * dir]; n3 = recs[p + 7 * dir];
                        }
                        visit((int)(c0.key >> 16), (int)(c0.key & 0xffffu) - kTplLayerBias, c0.len, lofs);
                        visit((int)(c1.key >> 16), (int)(c1.key & 0xffffu) - kTplLayerBias, c1.len, lofs);
                        visit((int)(c2.key >> 16), (int)(c2.key & 0xffffu) - kTplLayerBias, c2.len, lofs);
                        visit((int)(c3.key >> 16), (int)(c3.key & 0xffffu) - kTplLayerBias, c3.len, lofs);
                        p += 4 * dir;
                        if (more) { c0 = n0; c1 = n1; c2 = n2; c3 = n3; }
                    }
                    for (; s < n; ++s) {
                        const SegRec<real> c = recs[p];
                        p += dir;
                        visit((int)(c.key >> 16), (int)(c.key & 0xffffu) - kTplLayerBias, c.len, lofs);
                    }
                } else {
                    // template generated on the fly: line of the block's lowest track
                    const StackDesc d = dl.desc[(int64_t)T * Ph + ph];
                    const int ibase = d.i_lo + r + mb * SLOTS * cpl;
                    const int b0 = first_seg(dl, d, ibase + (J - 1) * cpl);
                    const int b1 = last_seg(dl, d, ibase);
                    const int lo = -(J - 1);
                    TplRange<real> tr;
                    if (sense == 0) {
                        for (int b = b0; b <= b1; ++b) {
                            tpl_range(dl, d, ibase, b, tr);
                            for (int L = max(tr.La, lo); L <= min(tr.Le, NL - 1); ++L)
                                visit(b, L, tpl_len(dl, d, b, tr, L), j);
                        }
                    } else {
                        for (int b = b1; b >= b0; --b) {
                            tpl_range(dl, d, ibase, b, tr);
                            for (int L = min(tr.Le, NL - 1); L >= max(tr.La, lo); --L)
                                visit(b, L, tpl_len(dl, d, b, tr, L), j);
                        }
                    }
                }
                if (valid && ql < gc) {
                    if (dstU >= 0 && dstU < dl.n_slots) psi_out[dstU * G + g0 + ql] = psiU;
                    else leak += (double)W * (double)psiU;
                    if (dstD >= 0 && dstD < dl.n_slots) psi_out[dstD * G + g0 + ql] = psiD;
                    else leak += (double)W * (double)psiD;
                }
            }
            __syncthreads();
            if (SMEM) {
                for (int b = warp; b < nb; b += nwarps) {
                    const int reg = __ldg(reg2d + b);
                    for (int x = lane; x < NL * GL; x += 32) {
                        const int L = x / GL, qq = x - L * GL;
                        if (qq >= gc) continue;
                        const double v = (double)tl_s[(b * NL + L) * GL + qq];
                        if (v != 0.0) atomicAdd(st.tally + ((size_t)reg * NL + L) * G + g0 + qq, v);
                    }
                }
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) leak += __shfl_down_sync(0xffffffffu, leak, o);
    if (lane == 0) s_leak[warp] = leak;
    __syncthreads();
    if (tid == 0) {
        double v = 0.0;
        for (int k = 0; k < nwarps; ++k) v += s_leak[k];
        if (v != 0.0) atomicAdd(st.scal + SC_LEAK, v);
    }
}

int lanes_for_groups(int G) {
    int gl = 1;
    while (gl < G && gl < 32) gl <<= 1;
    return gl;
}

template <typename real, bool SMEM>
const void *pick(int gl) {
    switch (gl) {
        case 1: return (const void *)k_sweep<real, 1, SMEM>;
        case 2: return (const void *)k_sweep<real, 2, SMEM>;
        case 4: return (const void *)k_sweep<real, 4, SMEM>;
        case 8: return (const void *)k_sweep<real, 8, SMEM>;
        case 16: return (const void *)k_sweep<real, 16, SMEM>;
        default: return (const void *)k_sweep<real, 32, SMEM>;
    }
}

const void *sweep_fn(int precision, int tally_smem, int G) {
    const int gl = lanes_for_groups(G);
    if (precision == MOC_FP64) return tally_smem ? pick<double, true>(gl) : pick<double, false>(gl);
    return tally_smem ? pick<float, true>(gl) : pick<float, false>(gl);
}

}  // namespace

int sweep_lanes_per_track(int G) { return lanes_for_groups(G); }

size_t sweep_smem_bytes(int precision, int tally_smem, int M, int G, int cap) {
    const size_t rs = precision == MOC_FP64 ? 8 : 4;
    const size_t gl = (size_t)lanes_for_groups(G);
    size_t b = ((size_t)M * gl * rs + 15) & ~(size_t)15;
    if (tally_smem) b += (size_t)cap * gl * rs * 3;  // (Qr, Sigma_t) rows + tally rows
    return b;
}

cudaError_t sweep_occupancy(int precision, int tally_smem, int G, int block, size_t smem,
                            int *blocks_per_sm) {
    const void *f = sweep_fn(precision, tally_smem, G);
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, f, block, smem);
}

cudaError_t launch_sweep(int precision, int tally_smem, const DevLayout &dl, const DevState &st,
                         const int32_t *order, int32_t n_work, int32_t cap, const void *psi_in,
                         void *psi_out, int grid, int block, size_t smem, cudaStream_t s) {
    const void *f = sweep_fn(precision, tally_smem, dl.G);
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    DevLayout a0 = dl;
    DevState a1 = st;
    const int32_t *a2 = order;
    int32_t a3 = n_work, a4 = tally_smem ? cap : 0;
    const void *a5 = psi_in;
    void *a6 = psi_out;
    void *args[] = {&a0, &a1, &a2, &a3, &a4, &a5, &a6};
    return cudaLaunchKernel(f, dim3(grid), dim3(block), args, smem, s);
}
