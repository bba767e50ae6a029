// The transport sweep kernel (Eq. 3 on every segment, Eq. 4 tallies).
//
// Work decomposition.  A persistent grid; each block takes one work unit at a
// time from a global counter: a 2D track with all its polar z-stacks (units in
// decreasing work order).  The tracks r, r + cpl, r + 2 cpl, ... of a z-stack
// are one track shifted up by one layer each (Eq. 5 with the layer planes on
// the axial lattice), so a single segment template serves all of them: track
// r + m cpl crosses the template pieces whose layer L_t + m lies in [0, NL).
//
// A warp task is (polar stack, class r, block of SLOTS = 32/GL consecutive
// tracks of the class, sense).  Slot j (GL lanes) carries track m + j; each lane
// carries GPL energy groups, kept in GPL group planes of the shared rows.  Every
// lane sweeps both frames: the upward track and the mirrored downward track
// that shares its segments (layer NL-1-L).  For one plane the 32 lanes of a
// warp touch 32 consecutive words (SLOTS consecutive rows x GL groups), so
// their shared-memory accesses never collide on a bank.
//
// Shared tally (SMEM = true): per unit the block stages one row per
// (2D segment, layer) FSR the unit crosses, holding (Qr, Sigma_t) for every
// group, plus a zeroed tally row; pieces touch only shared memory and the rows
// are flushed into the FP64 global tally once per unit.  A slot outside the
// layer range works on a zero row in the same bank group as the row it would
// have touched (Qr = Sigma_t = 0 leaves psi exactly unchanged and adds 0), so
// pieces run without branches or bank conflicts.  Templates come from
// the stored set (EXP, Sec. 4.2; four pieces at a time with the next four
// records in flight) or are generated on the fly (OTF).  Without the shared
// tally (SMEM = false) pieces read Qr from global memory and add straight into
// the FP64 global tally.
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

// e^{-Sigma_t l} from x = Sigma_t l: FP32 on the MUFU pipe (Sigma_t pre-scaled
// by log2 e, the negation folds into the multiply), FP64 exp
template <typename real>
__device__ __forceinline__ real attenuation(real x);
template <>
__device__ __forceinline__ float attenuation<float>(float x) {
    return fast_exp2(-x);
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

// Template pieces generated on the fly, in the order of one sense, limited to
// the layers [lo, hi) of the unclipped line i0.
template <typename real>
struct TplIter {
    int i0, b, bend, L, Lend, lo, hi, dir;
    TplRange<real> r;
    bool done;

    __device__ __forceinline__ void init(const DevLayout &dl, const StackDesc &d, int i0_, int b0,
                                         int b1, int lo_, int hi_, int dir_) {
        i0 = i0_;
        lo = lo_;
        hi = hi_;
        dir = dir_;
        b = dir > 0 ? b0 : b1;
        bend = dir > 0 ? b1 : b0;
        done = b0 > b1;
        if (!done) load_b(dl, d);
    }
    // load 2D segment b, moving on while its layer range is empty
    __device__ __forceinline__ void load_b(const DevLayout &dl, const StackDesc &d) {
        for (;;) {
            tpl_range(dl, d, i0, b, r);
            const int a = max(r.La, lo), e = min(r.Le, hi - 1);
            if (a <= e) {
                L = dir > 0 ? a : e;
                Lend = dir > 0 ? e : a;
                return;
            }
            if (b == bend) {
                done = true;
                return;
            }
            b += dir;
        }
    }
    __device__ __forceinline__ void next(const DevLayout &dl, const StackDesc &d, int &ob, int &oL,
                                         real &len) {
        ob = b;
        oL = L;
        len = tpl_len(dl, d, b, r, L);
        if (L != Lend) {
            L += dir;
        } else if (b != bend) {
            b += dir;
            load_b(dl, d);
        } else {
            done = true;
        }
    }
};


template <typename real, int GL, int GPL, bool SMEM>
__global__ void __launch_bounds__(256, sizeof(real) == 4 ? 3 : 2)
    k_sweep(DevLayout dl, DevState st, const int32_t *order, int32_t n_work, int32_t cap,
            const real *psi_in, real *psi_out) {
    using vec2 = typename Vec2<real>::type;
    constexpr int GP = GL * GPL;     // groups per chunk (padded)
    constexpr int SLOTS = 32 / GL;   // tracks per warp task
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_work, s_next, s_ntask;
    __shared__ UnitStack s_us[kMaxPh];
    __shared__ double s_leak[8];
    const int G = dl.G, NL = dl.NL, M = dl.M, Ph = dl.Ph, cpl = dl.cpl;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    const int j = lane / GL;         // slot: track of the block
    const int ql = lane & (GL - 1);  // lane of the slot: groups ql, GL + ql, ...
    // shared layout: sig [M*GP] | rows (Qr, Sigma_t) [GPL][ROWS][GL] | tally [GPL][ROWS][GL]
    // with ROWS = cap + SLOTS: the last SLOTS rows are zero rows, one per bank group
    const int ROWS = cap + SLOTS;
    real *sig = reinterpret_cast<real *>(smem);
    size_t off = ((size_t)M * GP * sizeof(real) + 15) & ~(size_t)15;
    vec2 *rows = reinterpret_cast<vec2 *>(smem + off);
    off += (size_t)ROWS * GP * sizeof(vec2);
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
                for (int r = 0; r < min(cpl, e.n_trk); ++r) {  // per class: blocks of SLOTS tracks, 2 senses
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
        for (int g0 = 0; g0 < G; g0 += GP) {
            const int gc = min(GP, G - g0);
            for (int e = tid; e < M * GP; e += blockDim.x) {
                const int m = e / GP, qq = e - m * GP;
                real v = qq < gc ? sig_g[m * G + g0 + qq] : (real)0;
                if (sizeof(real) == 4) v = (real)((float)v * kLog2e);
                sig[e] = v;
            }
            if (SMEM) {
                // rows of the (2D segment, layer) FSRs the unit crosses
                for (int b = warp; b < nb; b += nwarps) {
                    const int reg = __ldg(reg2d + b);
                    for (int x = lane; x < NL * GP; x += 32) {
                        const int L = x / GP, qq = x - L * GP;
                        const int c = qq / GL, qx = qq - c * GL;
                        const int f = reg * NL + L;
                        const int e = (c * ROWS + b * NL + L) * GL + qx;
                        vec2 v;
                        v.x = (real)0;
                        v.y = (real)0;
                        if (qq < gc) {
                            const int m = __ldg(dl.fsr_mat + f);
                            real sg = sig_g[m * G + g0 + qq];
                            if (sizeof(real) == 4) sg = (real)((float)sg * kLog2e);
                            v.x = qr_g[(size_t)f * G + g0 + qq];
                            v.y = sg;
                        }
                        rows[e] = v;
                        tl_s[e] = (real)0;
                    }
                }
                for (int e = tid; e < GPL * SLOTS * GL; e += blockDim.x) {
                    const int c = e / (SLOTS * GL), x = e - c * SLOTS * GL;
                    vec2 z;
                    z.x = (real)0;
                    z.y = (real)0;
                    rows[(c * ROWS + cap) * GL + x] = z;
                    tl_s[(c * ROWS + cap) * GL + x] = (real)0;
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
                real psiU[GPL], psiD[GPL];
#pragma unroll
                for (int c = 0; c < GPL; ++c) {
                    psiU[c] = (real)0;
                    psiD[c] = (real)0;
                }
                int64_t dstU = -1, dstD = -1;
                if (valid) {
                    if (psi_in) {
#pragma unroll
                        for (int c = 0; c < GPL; ++c) {
                            const int qq = c * GL + ql;
                            if (qq < gc) {
                                psiU[c] = psi_in[(gid * 4 + 0 * 2 + sense) * G + g0 + qq] * scale;
                                psiD[c] = psi_in[(gid * 4 + 1 * 2 + sense) * G + g0 + qq] * scale;
                            }
                        }
                    }
                    if (dl.dst) {
                        dstU = dl.dst[gid * 4 + 0 * 2 + sense];
                        dstD = dl.dst[gid * 4 + 1 * 2 + sense];
                    }
                }
                // one template piece for every slot: 2D segment b (bn = b * NL),
                // slot j at layer Lt + lofs
                auto visit = [&](int bn, int Lt, real len, int lofs) {
                    const int L = Lt + lofs;
                    const bool act = valid && (unsigned)L < (unsigned)NL;
                    if (SMEM) {
                        // rows of the upward and the mirrored downward frame, or
                        // the zero row of the same bank group
                        const int rU = bn + L, rD = bn + (NL - 1 - L);
                        const int zU = act ? rU : cap + (rU & (SLOTS - 1));
                        const int zD = act ? rD : cap + (rD & (SLOTS - 1));
#pragma unroll
                        for (int c = 0; c < GPL; ++c) {
                            const int eU = (c * ROWS + zU) * GL + ql, eD = (c * ROWS + zD) * GL + ql;
                            const vec2 aU = rows[eU], aD = rows[eD];
                            // Eq. 3: psi_out = Qr + (psi_in - Qr) e^{-Sigma_t l}
                            const real xU = attenuation<real>(aU.y * len);
                            const real xD = attenuation<real>(aD.y * len);
                            const real nU = aU.x + (psiU[c] - aU.x) * xU;
                            const real nD = aD.x + (psiD[c] - aD.x) * xD;
                            atomicAdd(tl_s + eU, (psiU[c] - nU) * W);
                            atomicAdd(tl_s + eD, (psiD[c] - nD) * W);
                            psiU[c] = nU;
                            psiD[c] = nD;
                        }
                    } else {
                        if (!act) return;
                        const int LD = NL - 1 - L;
                        const int reg = __ldg(reg2d + bn / NL);
                        const size_t fU = (size_t)reg * NL + L, fD = (size_t)reg * NL + LD;
                        const int mU = __ldg(dl.fsr_mat + fU), mD = __ldg(dl.fsr_mat + fD);
#pragma unroll
                        for (int c = 0; c < GPL; ++c) {
                            const int qq = c * GL + ql;
                            const real qU = qq < gc ? qr_g[fU * G + g0 + qq] : (real)0;
                            const real qD = qq < gc ? qr_g[fD * G + g0 + qq] : (real)0;
                            const real xU = attenuation<real>(sig[mU * GP + qq] * len);
                            const real xD = attenuation<real>(sig[mD * GP + qq] * len);
                            const real nU = qU + (psiU[c] - qU) * xU;
                            const real nD = qD + (psiD[c] - qD) * xD;
                            if (qq < gc) {
                                atomicAdd(st.tally + fU * G + g0 + qq, (double)(psiU[c] - nU) * (double)W);
                                atomicAdd(st.tally + fD * G + g0 + qq, (double)(psiD[c] - nD) * (double)W);
                            }
                            psiU[c] = nU;
                            psiD[c] = nD;
                        }
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
                    const StackDesc &d = dl.desc[(int64_t)T * Ph + ph];
                    const int ibase = u.i_lo + r + mb * SLOTS * cpl;
                    TplIter<real> it;
                    it.init(dl, d, ibase, first_seg(dl, d, ibase + (J - 1) * cpl), last_seg(dl, d, ibase),
                            -(J - 1), NL, sense == 0 ? 1 : -1);
                    while (!it.done) {
                        int b, L;
                        real len;
                        it.next(dl, d, b, L, len);
                        visit(b * NL, L, len, j);
                    }
                }
                if (valid) {
#pragma unroll
                    for (int c = 0; c < GPL; ++c) {
                        const int qq = c * GL + ql;
                        if (qq >= gc) continue;
                        if (dstU >= 0 && dstU < dl.n_slots) psi_out[dstU * G + g0 + qq] = psiU[c];
                        else leak += (double)W * (double)psiU[c];
                        if (dstD >= 0 && dstD < dl.n_slots) psi_out[dstD * G + g0 + qq] = psiD[c];
                        else leak += (double)W * (double)psiD[c];
                    }
                }
            }
            __syncthreads();
            if (SMEM) {
                for (int b = warp; b < nb; b += nwarps) {
                    const int reg = __ldg(reg2d + b);
                    for (int x = lane; x < NL * GP; x += 32) {
                        const int L = x / GP, qq = x - L * GP;
                        if (qq >= gc) continue;
                        const int c = qq / GL, qx = qq - c * GL;
                        const double v = (double)tl_s[(c * ROWS + b * NL + L) * GL + qx];
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

// lanes per track: the smallest power of two that holds ceil(G / gpl) groups
int lanes_for_groups(int G, int gpl) {
    const int cap = gpl == 2 ? 16 : 32;
    const int need = (G + gpl - 1) / gpl;
    int gl = 1;
    while (gl < need && gl < cap) gl <<= 1;
    return gl;
}

template <typename real, int GPL, bool SMEM>
const void *pick(int gl) {
    switch (gl) {
        case 1: return (const void *)k_sweep<real, 1, GPL, SMEM>;
        case 2: return (const void *)k_sweep<real, 2, GPL, SMEM>;
        case 4: return (const void *)k_sweep<real, 4, GPL, SMEM>;
        case 8: return (const void *)k_sweep<real, 8, GPL, SMEM>;
        case 16: return (const void *)k_sweep<real, 16, GPL, SMEM>;
        default: return (const void *)k_sweep<real, (GPL == 1 ? 32 : 16), GPL, SMEM>;
    }
}

const void *sweep_fn(int precision, int tally_smem, int G, int gpl) {
    const int gl = lanes_for_groups(G, gpl);
    if (precision == MOC_FP64) return tally_smem ? pick<double, 1, true>(gl) : pick<double, 1, false>(gl);
    if (gpl == 2) return tally_smem ? pick<float, 2, true>(gl) : pick<float, 2, false>(gl);
    return tally_smem ? pick<float, 1, true>(gl) : pick<float, 1, false>(gl);
}

// rows of the tile rounded to whole bank groups, so that a zero row shares
// the banks of the row it stands in for
int round_cap(int cap) { return (cap + 31) & ~31; }

}  // namespace

int sweep_default_gpl(int precision, int G) {
    (void)precision;
    (void)G;
    return 1;
}

int sweep_lanes_per_track(int G, int gpl) { return lanes_for_groups(G, gpl); }

size_t sweep_smem_bytes(int precision, int tally_smem, int M, int G, int gpl, int cap) {
    const size_t rs = precision == MOC_FP64 ? 8 : 4;
    const size_t gp = (size_t)lanes_for_groups(G, gpl) * gpl;
    size_t b = ((size_t)M * gp * rs + 15) & ~(size_t)15;
    // (Qr, Sigma_t) rows + tally rows, including one zero row per slot
    if (tally_smem) b += (size_t)(round_cap(cap) + 32) * gp * rs * 3;
    return b;
}

cudaError_t sweep_occupancy(int precision, int tally_smem, int G, int gpl, int block, size_t smem,
                            int *blocks_per_sm) {
    const void *f = sweep_fn(precision, tally_smem, G, gpl);
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, f, block, smem);
}

cudaError_t launch_sweep(int precision, int tally_smem, int gpl, const DevLayout &dl,
                         const DevState &st, const int32_t *order, int32_t n_work, int32_t cap,
                         const void *psi_in, void *psi_out, int grid, int block, size_t smem,
                         cudaStream_t s) {
    const void *f = sweep_fn(precision, tally_smem, dl.G, gpl);
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    DevLayout a0 = dl;
    DevState a1 = st;
    const int32_t *a2 = order;
    int32_t a3 = n_work, a4 = tally_smem ? round_cap(cap) : 0;
    const void *a5 = psi_in;
    void *a6 = psi_out;
    void *args[] = {&a0, &a1, &a2, &a3, &a4, &a5, &a6};
    return cudaLaunchKernel(f, dim3(grid), dim3(block), args, smem, s);
}
