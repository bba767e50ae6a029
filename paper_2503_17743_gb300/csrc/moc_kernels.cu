// CUDA kernels of the GB300 3D MOC transport sweep (sm_103a).
//
//   k_count_stacks  segments per z-stack (preload planning, Sec. 4.2)
//   k_tpl_count     sizes of the stored segment templates (EXP, Sec. 4.2)
//   k_tpl_write     writes the stored templates
//   k_links         link destination of every track direction
//   k_volumes       tracked FSR volumes
//   k_source        isotropic source update, FP64
//   k_finalize      scalar flux from the tallies + FP64 block partials
//   k_reduce_k      FP64 production / absorption / k / normalisation
//   k_residual      FP64 fission-source residual partials
//   k_reduce_res    FP64 residual + convergence flag
#include <cstdio>

#include "moc_device.cuh"
#include "moc_kernels.h"

namespace {


__device__ __forceinline__ double block_sum(double v, double *sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0) {
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += sh[i];
    }
    return r;  // valid in thread 0
}

// ---------------------------------------------------------------------------
// layout kernels

__global__ void k_count_stacks(DevLayout dl, int64_t n_stacks, int64_t *stack_nseg,
                               int32_t *max_nseg, int32_t *trk_nseg) {
    __shared__ double sh[32];
    for (int64_t s = blockIdx.x; s < n_stacks; s += gridDim.x) {
        const StackDesc d = dl.desc[s];
        double acc = 0;
        int mx = 0;
        for (int k = threadIdx.x; k < d.n_trk; k += blockDim.x) {
            // planes off the lattice: both frames' pieces (else the upward
            // frame's, which the mirrored frame repeats)
            const int n = dl.offlat ? count_ol(dl, d, d.i_lo + k, 0) + count_ol(dl, d, d.i_lo + k, 1)
                                    : count_otf(dl, d, d.i_lo + k);
            trk_nseg[d.trk_off + k] = n;
            acc += n;
            mx = max(mx, n);
        }
        for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_down_sync(0xffffffffu, mx, o));
        if ((threadIdx.x & 31) == 0 && mx > 0) atomicMax(max_nseg, mx);
        double tot = block_sum(acc, sh);
        if (threadIdx.x == 0) stack_nseg[s] = (int64_t)(tot + 0.5);
        __syncthreads();
    }
}

// Stored templates (one per class r < cpl of each stored stack, template
// index desc.exp_base + r): piece count, lowest layer and layer span.
__global__ void k_tpl_count(DevLayout dl, const int32_t *exp_stacks, int64_t n_exp, int64_t *cnt,
                            int32_t *lmin, int32_t *nlay) {
    for (int64_t q = blockIdx.x; q < n_exp; q += gridDim.x) {
        const StackDesc d = dl.desc[exp_stacks[q]];
        const int ntpl = min(dl.cpl, d.n_trk);
        for (int r = threadIdx.x; r < ntpl; r += blockDim.x) {
            const int i0 = d.i_lo + r;
            int n = 0, lo = 0, hi = 0;
            TplRange<float> tr;
            for (int b = 0; b < d.nb; ++b) {
                tpl_range(dl, d, i0, b, tr);
                if (b == 0) lo = tr.La;
                if (tr.Le >= tr.La) n += tr.Le - tr.La + 1;
                hi = max(hi, tr.Le);
            }
            const int64_t t = d.exp_base + r;
            cnt[t] = n;
            lmin[t] = lo;
            nlay[t] = max(hi - lo + 1, 1);
        }
    }
}

template <typename real>
__global__ void k_tpl_write(DevLayout dl, const int32_t *exp_stacks, int64_t n_exp,
                            SegRec<real> *recs, int32_t *lidx) {
    for (int64_t q = blockIdx.x; q < n_exp; q += gridDim.x) {
        const StackDesc d = dl.desc[exp_stacks[q]];
        const int ntpl = min(dl.cpl, d.n_trk);
        for (int r = threadIdx.x; r < ntpl; r += blockDim.x) {
            const int64_t t = d.exp_base + r;
            const int i0 = d.i_lo + r;
            const int Lmin = dl.tpl_lmin[t];
            const int64_t lb = dl.tpl_loff[t];
            const int nL = (int)(dl.tpl_loff[t + 1] - lb) - 1;
            SegRec<real> *out = recs + dl.tpl_off[t];
            int pos = 0, x = 0;
            TplRange<real> tr;
            for (int b = 0; b < d.nb; ++b) {
                tpl_range(dl, d, i0, b, tr);
                for (int L = tr.La; L <= tr.Le; ++L) {
                    while (x <= L - Lmin && x <= nL) lidx[lb + x++] = pos;
                    SegRec<real> rec{};
                    rec.key = (dl.chunk_b > 0 || dl.sync_b > 1)
                                  ? (dl.matk ? tpl_key_seg_mat(b, L, dl.reg_mat[dl.reg2d[d.seg2d_off + b]])
                                             : tpl_key_seg(b, L))
                                  : dl.matk ? tpl_key_mat(b * dl.NL + L, b * dl.NL + dl.NL - 1 - L,
                                                          dl.reg_mat[dl.reg2d[d.seg2d_off + b]])
                                            : tpl_key(b * dl.NL + L, b * dl.NL + dl.NL - 1 - L);
                    rec.len = tpl_len(dl, d, b, tr, L);
                    out[pos++] = rec;
                }
            }
            while (x <= nL) lidx[lb + x++] = pos;
        }
    }
}

// destination of the outgoing flux of every stored track direction (slot
// gid*4+v of the next sweep's incoming flux, -1 at a vacuum face)
// Record window of every track of a stored stack, in the stack's sweep order
// (perm): track r + m cpl of class r is the pieces of template r whose layer
// lies in [-m, NL - m), a contiguous record range; stored as (count << 48) |
// first record.
__global__ void k_windows(DevLayout dl, int64_t n_stacks, uint64_t *win) {
    for (int64_t s = blockIdx.x; s < n_stacks; s += gridDim.x) {
        const StackDesc &d = dl.desc[s];
        if (d.exp_base < 0) continue;
        for (int q = threadIdx.x; q < d.n_slot; q += blockDim.x) {
            const int k = dl.perm[d.slot_off + q];
            if (k < 0) {  // padding of a synchronous block: no records
                win[d.slot_off + q] = 0ull;
                continue;
            }
            const int r = k % dl.cpl, m = k / dl.cpl;
            const int64_t tpl = d.exp_base + r;
            const int Lmin = dl.tpl_lmin[tpl];
            const int64_t lb = dl.tpl_loff[tpl];
            const int nL = (int)(dl.tpl_loff[tpl + 1] - lb) - 1;
            const int64_t tb = dl.tpl_off[tpl];
            const int64_t p0 = tb + dl.tpl_lidx[lb + min(max(-m - Lmin, 0), nL)];
            const int64_t p1 = tb + dl.tpl_lidx[lb + min(max(dl.NL - m - Lmin, 0), nL)];
            win[d.slot_off + q] = ((uint64_t)(p1 - p0) << 48) | (uint64_t)p0;
        }
    }
}

// Chunk tables of radially chunked units.  Tracks crossing chunk c: the
// 2D segment range [first_seg, last_seg] of track i shrinks towards lower b
// as i grows (both ends are monotone in i), so they are one index range,
// found by two bisections.  Template records are in order of the 2D segment
// of their keys.
template <typename real>
__global__ void k_chunk_tables(DevLayout dl, const int32_t *stacks, int64_t n, int64_t *tab) {
    const SegRec<real> *recs = reinterpret_cast<const SegRec<real> *>(dl.segs);
    const int cb = dl.chunk_b;
    for (int64_t x = blockIdx.x; x < n; x += gridDim.x) {
        const StackDesc &d = dl.desc[stacks[x]];
        const int C = (d.nb + cb - 1) / cb;
        const int ntpl = d.exp_base >= 0 ? min(dl.cpl, d.n_trk) : 0;
        int64_t *t = tab + d.chunk_base;
        for (int e = threadIdx.x; e < C + ntpl * (C + 1); e += blockDim.x) {
            if (e < C) {
                // first track whose last segment reaches chunk e, first whose
                // first segment does not lie beyond it
                int lo = 0, hi = d.n_trk;  // first k with last_seg < e * cb
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (last_seg(dl, d, d.i_lo + mid) < e * cb) hi = mid; else lo = mid + 1;
                }
                const int k1 = lo;
                lo = 0;
                hi = d.n_trk;  // first k with first_seg < (e + 1) * cb
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (first_seg(dl, d, d.i_lo + mid) < (e + 1) * cb) hi = mid; else lo = mid + 1;
                }
                const int k0 = lo;
                const int cnt = max(0, k1 - k0);
                t[e] = (int64_t)k0 | ((int64_t)cnt << 32);
            } else {
                const int r = (e - C) / (C + 1), c = (e - C) - r * (C + 1);
                const int64_t q = d.exp_base + r;
                int64_t lo = dl.tpl_off[q], hi = dl.tpl_off[q + 1];
                const int bb = c * cb;
                while (lo < hi) {  // first record with b >= c * cb
                    const int64_t mid = (lo + hi) >> 1;
                    const uint32_t key = recs[mid].key;
                    const int b = dl.matk ? tpl_seg_mat(key) : tpl_seg(key);
                    if (b >= bb) hi = mid; else lo = mid + 1;
                }
                t[e] = lo;
            }
        }
    }
}

__global__ void k_links(DevLayout dl, int64_t n_stacks, int32_t *dst) {
    for (int64_t s = blockIdx.x; s < n_stacks; s += gridDim.x) {
        const StackDesc d = dl.desc[s];
        for (int k = threadIdx.x; k < d.n_trk; k += blockDim.x) {
            const int i = d.i_lo + k;
            const int64_t gid = d.trk_off + k;
            for (int v = 0; v < 4; ++v) {
                int64_t t = exit_dest(dl, dl.desc, d, dl.desc + s, i, v);
                if (t >= dl.n_slots) t = -1;
                dst[gid * 4 + v] = (int32_t)t;
            }
        }
    }
}

// Tracked volumes are summed exactly, so that they do not depend on the order
// in which threads finish (every handle built from the same geometry and track
// parameters gets the same bits): each contribution v >= 0 is an integer
// number of 2^-64 units (bits below 2^-64 dropped), held as 32-bit chunks in
// four unsigned 64-bit words per FSR, value sum_k A_k 2^(32 k - 64).  Chunks
// are below 2^32, so a word takes 2^32 adds before it could wrap.
__device__ __forceinline__ void fix4_add(unsigned long long *a, double v) {
    if (!(v > 0.0)) return;
    int e = 0;
    const double m = frexp(v, &e);                                  // v = m 2^e, 1/2 <= m < 1
    unsigned long long M = (unsigned long long)ldexp(m, 53);        // exact, below 2^53
    int S = e + 11;                                                 // v = M 2^(S - 64)
    if (S < 0) {
        M = S > -64 ? M >> -S : 0ull;
        S = 0;
    }
    const int w = S >> 5;
    const unsigned __int128 x = (unsigned __int128)M << (S & 31);   // below 2^84
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const unsigned long long c = (unsigned long long)(x >> (32 * k)) & 0xffffffffull;
        if (c && w + k < 4) atomicAdd(a + w + k, c);
    }
}

template <typename real>
struct VolVisit {
    const DevLayout *dl;
    const int32_t *reg2d;
    int NL;
    unsigned long long *acc;
    double c;
    __device__ void operator()(int b, int L, real len) {
        const int reg = __ldg(reg2d + b);
        fix4_add(acc + 4 * fsr_of(*dl, reg, L), c * (double)len);
        fix4_add(acc + 4 * fsr_of(*dl, reg, NL - 1 - L), c * (double)len);
    }
};

// planes off the lattice: each frame's pieces on their own
template <typename real>
struct VolVisitOL {
    const DevLayout *dl;
    const int32_t *reg2d;
    unsigned long long *acc;
    double c;
    __device__ void operator()(int b, int L, real len) {
        fix4_add(acc + 4 * fsr_of(*dl, __ldg(reg2d + b), L), c * (double)len);
    }
};

template <typename real>
__global__ void k_volumes(DevLayout dl, int64_t n_stacks, unsigned long long *acc) {
    for (int64_t s = blockIdx.x; s < n_stacks; s += gridDim.x) {
        const StackDesc d = dl.desc[s];
        // each stored track carries two directions of equal weight, in two frames
        const double c = 2.0 * d.W / (4.0 * MOC_PI);
        if (dl.offlat) {
            VolVisitOL<real> v{&dl, dl.reg2d + d.seg2d_off, acc, c};
            for (int k = threadIdx.x; k < d.n_trk; k += blockDim.x) {
                walk_ol<real>(dl, d, d.i_lo + k, 0, 0, v);
                walk_ol<real>(dl, d, d.i_lo + k, 1, 0, v);
            }
        } else {
            VolVisit<real> v{&dl, dl.reg2d + d.seg2d_off, dl.NL, acc, c};
            for (int k = threadIdx.x; k < d.n_trk; k += blockDim.x) walk_otf<real>(dl, d, d.i_lo + k, 0, v);
        }
    }
}

// the volumes from their exact sums: carries first, then one fixed-order sum
__global__ void k_vol_value(const unsigned long long *acc, int64_t nfsr, double *vol) {
    for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < nfsr;
         f += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long w[4];
        unsigned long long carry = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const unsigned long long x = acc[4 * f + k] + carry;
            carry = k < 3 ? x >> 32 : 0ull;
            w[k] = k < 3 ? x & 0xffffffffull : x;
        }
        vol[f] = (((double)w[3] * 4294967296.0 + (double)w[2]) + (double)w[1] * 2.3283064365386963e-10) +
                 (double)w[0] * 5.421010862427522e-20;
    }
}

// segments of the stack's tracks for introspection (frame U order)
template <typename real>
struct ListVisit {
    const int32_t *reg2d;
    int NL;
    int32_t *f;
    double *l;
    __device__ void operator()(int b, int L, real ln) {
        *f++ = __ldg(reg2d + b) * NL + L;
        *l++ = (double)ln;
    }
};

// planes off the lattice: the pieces of the given frame, with the geometry's
// layers
template <typename real>
__global__ void k_stack_segments(DevLayout dl, int64_t s, int frame, const int64_t *offs, int32_t *fsr_u,
                                 double *len) {
    const StackDesc d = dl.desc[s];
    for (int k = threadIdx.x; k < d.n_trk; k += blockDim.x) {
        ListVisit<real> v{dl.reg2d + d.seg2d_off, dl.NL, fsr_u + offs[k], len + offs[k]};
        if (dl.offlat) walk_ol<real>(dl, d, d.i_lo + k, frame, 0, v);
        else walk_otf<real>(dl, d, d.i_lo + k, 0, v);
    }
}

// ---------------------------------------------------------------------------
// FSR-sized FP64 kernels

// Q = (sum_h Sigma_s[h->g] phi_h + chi_g / k sum_h nuSigma_f,h phi_h + S_g) / 4pi, with
// phi normalised on the fly by the latest scale; qr = Q / Sigma_t.
template <typename real>
__global__ void k_source(DevLayout dl, DevState st, int32_t nfsr) {
    if (st.scal[SC_CONV] != 0.0) return;  // converged: later iterations are no-ops
    const int G = dl.G;
    const double scale = st.scal[SC_SCALE];
    const bool eig = st.scal[SC_EIGEN] != 0.0;
    // chi / k of the normalised flux; 1 / (4 pi) per steradian.  Divisions are
    // replaced by products with precomputed inverses (FP64 division is slow)
    const double fis_scale = eig ? scale / st.scal[SC_K] : 0.0;
    const double per_sr = 1.0 / (4.0 * MOC_PI);
    real *qr = reinterpret_cast<real *>(st.qr);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nfsr; i += gridDim.x * blockDim.x) {
        const int m = dl.fsr_mat[i];
        const double *ph = st.phi + (size_t)i * G;
        double fis = 0.0;
        if (eig)
            for (int h = 0; h < G; ++h) fis += st.nsf64[m * G + h] * ph[h];
        for (int g = 0; g < G; ++g) {
            double sc = 0.0;
            for (int h = 0; h < G; ++h) sc += st.sig_s64[((size_t)m * G + h) * G + g] * ph[h];
            double q = sc * scale;
            if (eig) q += st.chi64[m * G + g] * fis * fis_scale;
            if (st.src64) q += st.src64[m * G + g];
            qr[(size_t)i * G + g] = (real)(q * per_sr * st.inv_st64[m * G + g]);
        }
    }
}

// phi = 4 pi Qr + tally / (V Sigma_t); tally cleared; block partials of
// production, absorption and (fixed source) the flux residual.
template <typename real>
__global__ void k_finalize(DevLayout dl, DevState st, int32_t nfsr) {
    if (st.scal[SC_CONV] != 0.0) return;
    __shared__ double sh[32];
    const int G = dl.G;
    const bool eig = st.scal[SC_EIGEN] != 0.0;
    const real *qr = reinterpret_cast<const real *>(st.qr);
    double P = 0, Ab = 0, r2 = 0, cnt = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nfsr; i += gridDim.x * blockDim.x) {
        const int m = dl.fsr_mat[i];
        const double V = st.vol[i], iV = st.inv_vol[i];
        double fis = 0.0;
        for (int g = 0; g < G; ++g) {
            const size_t q = (size_t)i * G + g;
            // Eq. 4: phi = 4 pi Qr + tally / (V Sigma_t)
            double t;
            if (dl.tally3) {
                long long *a = reinterpret_cast<long long *>(st.tally) + 3 * q;
                t = tally3_value(a[0], a[1], a[2]);
                a[0] = 0;
                a[1] = 0;
                a[2] = 0;
            } else {
                t = st.tally[q];
                st.tally[q] = 0.0;
            }
            const double phi = 4.0 * MOC_PI * (double)qr[q] + t * iV * st.inv_st64[m * G + g];
            if (!eig && phi > 0.0) {
                double rr = (phi - st.phi[q]) / phi;
                r2 += rr * rr;
                cnt += 1.0;
            }
            st.phi[q] = phi;
            fis += st.nsf64[m * G + g] * phi;
            Ab += V * st.siga64[m * G + g] * phi;
        }
        P += V * fis;
        st.fiss[i] = fis;
    }
    double v;
    v = block_sum(P, sh); if (threadIdx.x == 0) st.partial[blockIdx.x * 4 + 0] = v;
    v = block_sum(Ab, sh); if (threadIdx.x == 0) st.partial[blockIdx.x * 4 + 1] = v;
    v = block_sum(r2, sh); if (threadIdx.x == 0) st.partial[blockIdx.x * 4 + 2] = v;
    v = block_sum(cnt, sh); if (threadIdx.x == 0) st.partial[blockIdx.x * 4 + 3] = v;
}

// single block: production, absorption, k update and normalisation scale
// one warp: lane-strided partial sums, then a fixed-order shuffle tree, so
// the result is the same on every run
__device__ __forceinline__ double warp_partial_sum(const double *partial, int nblocks, int slot) {
    double v = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += 32) v += partial[b * 4 + slot];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;  // valid in lane 0
}

__global__ void k_reduce_k(DevState st, int nblocks, double integrations) {
    if (st.scal[SC_CONV] != 0.0) return;
    const double P = warp_partial_sum(st.partial, nblocks, 0);
    const double Ab = warp_partial_sum(st.partial, nblocks, 1);
    const double r2 = warp_partial_sum(st.partial, nblocks, 2);
    const double cnt = warp_partial_sum(st.partial, nblocks, 3);
    if (threadIdx.x != 0) return;
    double *s = st.scal;
    const bool eig = s[SC_EIGEN] != 0.0;
    s[SC_PROD] = P;
    s[SC_ABS] = Ab;
    s[SC_INTEG] += integrations;
    s[SC_ITER] += 1.0;
    if (eig) {
        const double kn = s[SC_K] * P;  // the swept flux was normalised to production 1
        s[SC_DK] = kn - s[SC_K];
        s[SC_K] = kn;
        s[SC_SCALE] = P > 0.0 ? 1.0 / P : 1.0;
        s[SC_LEAK_PREV] = s[SC_LEAK] * s[SC_SCALE];
    } else {
        s[SC_DK] = 0.0;
        s[SC_SCALE] = 1.0;
        s[SC_RES] = cnt > 0 ? sqrt(r2 / cnt) : 0.0;
        s[SC_LEAK_PREV] = s[SC_LEAK];
        s[SC_CONV] = (s[SC_TOLS] > 0 && s[SC_RES] < s[SC_TOLS]) ? 1.0 : 0.0;
    }
    s[SC_LEAK] = 0.0;
}

// eigenvalue residual: RMS relative change of the normalised fission rate
__global__ void k_residual(DevState st, int32_t nfsr) {
    if (st.scal[SC_CONV] != 0.0) return;
    __shared__ double sh[32];
    const double scale = st.scal[SC_SCALE];
    double r2 = 0, cnt = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nfsr; i += gridDim.x * blockDim.x) {
        const double f = st.fiss[i] * scale;
        if (f > 0.0) {
            const double r = (f - st.fiss_old[i]) / f;
            r2 += r * r;
            cnt += 1.0;
        }
        st.fiss_old[i] = f;
    }
    double v;
    v = block_sum(r2, sh); if (threadIdx.x == 0) st.partial[blockIdx.x * 4 + 2] = v;
    v = block_sum(cnt, sh); if (threadIdx.x == 0) st.partial[blockIdx.x * 4 + 3] = v;
}

__global__ void k_reduce_res(DevState st, int nblocks) {
    if (st.scal[SC_CONV] != 0.0) return;
    const double r2 = warp_partial_sum(st.partial, nblocks, 2);
    const double cnt = warp_partial_sum(st.partial, nblocks, 3);
    if (threadIdx.x != 0) return;
    double *s = st.scal;
    s[SC_RES] = cnt > 0 ? sqrt(r2 / cnt) : 0.0;
    s[SC_CONV] = (s[SC_TOLS] > 0 && s[SC_RES] < s[SC_TOLS] && fabs(s[SC_DK]) < s[SC_TOLK]) ? 1.0 : 0.0;
}

// initial state: phi = 1; production of it -> scale; fission rate reference
__global__ void k_init_state(DevLayout dl, DevState st, int32_t nfsr) {
    __shared__ double sh[32];
    const int G = dl.G;
    double P = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nfsr; i += gridDim.x * blockDim.x) {
        const int m = dl.fsr_mat[i];
        double fis = 0.0;
        for (int g = 0; g < G; ++g) {
            st.phi[(size_t)i * G + g] = 1.0;
            if (dl.tally3) {
                long long *a = reinterpret_cast<long long *>(st.tally) + 3 * ((size_t)i * G + g);
                a[0] = 0;
                a[1] = 0;
                a[2] = 0;
            } else {
                st.tally[(size_t)i * G + g] = 0.0;
            }
            fis += st.nsf64[m * G + g];
        }
        st.fiss[i] = fis;
        P += st.vol[i] * fis;
    }
    double v = block_sum(P, sh);
    if (threadIdx.x == 0) st.partial[blockIdx.x * 4 + 0] = v;
}

__global__ void k_init_finish(DevState st, int nblocks, int32_t nfsr) {
    __shared__ double s_scale;
    double P = 0.0;
    if (threadIdx.x < 32) P = warp_partial_sum(st.partial, nblocks, 0);
    if (threadIdx.x == 0) {
        double *s = st.scal;
        const bool eig = s[SC_EIGEN] != 0.0;
        s[SC_K] = 1.0;
        s[SC_DK] = 0.0;
        s[SC_SCALE] = (eig && P > 0.0) ? 1.0 / P : 1.0;
        s[SC_PROD] = P;
        s[SC_LEAK] = 0.0;
        s[SC_RES] = 0.0;
        s[SC_ITER] = 0.0;
        s[SC_CONV] = 0.0;
        s[SC_ERR] = 0.0;
        s_scale = s[SC_SCALE];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nfsr; i += blockDim.x) st.fiss_old[i] = st.fiss[i] * s_scale;
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers

#define CK(x)                                            \
    do {                                                 \
        cudaError_t e_ = (x);                            \
        if (e_ != cudaSuccess) return e_;                \
    } while (0)

cudaError_t launch_count_stacks(const DevLayout &dl, int64_t n_stacks, int64_t *stack_nseg,
                                int32_t *max_nseg, int32_t *trk_nseg, int grid, cudaStream_t s) {
    k_count_stacks<<<grid, 128, 0, s>>>(dl, n_stacks, stack_nseg, max_nseg, trk_nseg);
    return cudaGetLastError();
}

cudaError_t launch_tpl_count(const DevLayout &dl, const int32_t *exp_stacks, int64_t n_exp,
                             int64_t *cnt, int32_t *lmin, int32_t *nlay, int grid, cudaStream_t s) {
    if (n_exp == 0) return cudaSuccess;
    k_tpl_count<<<grid, 32, 0, s>>>(dl, exp_stacks, n_exp, cnt, lmin, nlay);
    return cudaGetLastError();
}

cudaError_t launch_tpl_write(int precision, const DevLayout &dl, const int32_t *exp_stacks,
                             int64_t n_exp, void *recs, int32_t *lidx, int grid, cudaStream_t s) {
    if (n_exp == 0) return cudaSuccess;
    if (precision == MOC_FP64)
        k_tpl_write<double><<<grid, 32, 0, s>>>(dl, exp_stacks, n_exp, (SegRec<double> *)recs, lidx);
    else
        k_tpl_write<float><<<grid, 32, 0, s>>>(dl, exp_stacks, n_exp, (SegRec<float> *)recs, lidx);
    return cudaGetLastError();
}

size_t segrec_size(int precision) {
    return precision == MOC_FP64 ? sizeof(SegRec<double>) : sizeof(SegRec<float>);
}

// per-track segment counts of one stack and frame (introspection)
__global__ void k_track_counts(DevLayout dl, int64_t s, int frame, int64_t *cnt) {
    const StackDesc d = dl.desc[s];
    for (int k = threadIdx.x; k < d.n_trk; k += blockDim.x)
        cnt[k + 1] = dl.offlat ? count_ol(dl, d, d.i_lo + k, frame) : count_otf(dl, d, d.i_lo + k);
}

cudaError_t launch_track_counts(const DevLayout &dl, int64_t stack, int frame, int64_t *cnt, cudaStream_t s) {
    k_track_counts<<<1, 128, 0, s>>>(dl, stack, frame, cnt);
    return cudaGetLastError();
}

cudaError_t launch_windows(const DevLayout &dl, int64_t n_stacks, uint64_t *win, int grid,
                           cudaStream_t s) {
    k_windows<<<grid, 128, 0, s>>>(dl, n_stacks, win);
    return cudaGetLastError();
}

cudaError_t launch_chunk_tables(int precision, const DevLayout &dl, const int32_t *stacks, int64_t n,
                                int64_t *tab, int grid, cudaStream_t s) {
    if (precision == MOC_FP64) k_chunk_tables<double><<<grid, 128, 0, s>>>(dl, stacks, n, tab);
    else k_chunk_tables<float><<<grid, 128, 0, s>>>(dl, stacks, n, tab);
    return cudaGetLastError();
}

cudaError_t launch_links(const DevLayout &dl, int64_t n_stacks, int32_t *dst, int grid,
                         cudaStream_t s) {
    k_links<<<grid, 128, 0, s>>>(dl, n_stacks, dst);
    return cudaGetLastError();
}

cudaError_t launch_volumes(int precision, const DevLayout &dl, int64_t n_stacks, int64_t nfsr,
                           unsigned long long *acc, double *vol, int grid, cudaStream_t s) {
    CK(cudaMemsetAsync(acc, 0, (size_t)nfsr * 4 * sizeof(unsigned long long), s));
    if (precision == MOC_FP64) k_volumes<double><<<grid, 128, 0, s>>>(dl, n_stacks, acc);
    else k_volumes<float><<<grid, 128, 0, s>>>(dl, n_stacks, acc);
    CK(cudaGetLastError());
    k_vol_value<<<grid, 256, 0, s>>>(acc, nfsr, vol);
    return cudaGetLastError();
}

cudaError_t launch_stack_segments(int precision, const DevLayout &dl, int64_t stack, int frame,
                                  const int64_t *offs, int32_t *fsr, double *len, cudaStream_t s) {
    if (precision == MOC_FP64) k_stack_segments<double><<<1, 128, 0, s>>>(dl, stack, frame, offs, fsr, len);
    else k_stack_segments<float><<<1, 128, 0, s>>>(dl, stack, frame, offs, fsr, len);
    return cudaGetLastError();
}

cudaError_t launch_source(int precision, const DevLayout &dl, const DevState &st, int32_t nfsr,
                          int grid, cudaStream_t s) {
    if (precision == MOC_FP64) k_source<double><<<grid, kSmallBlock, 0, s>>>(dl, st, nfsr);
    else k_source<float><<<grid, kSmallBlock, 0, s>>>(dl, st, nfsr);
    return cudaGetLastError();
}

cudaError_t launch_finalize(int precision, const DevLayout &dl, const DevState &st, int32_t nfsr,
                            int grid, double integrations, cudaStream_t s) {
    if (precision == MOC_FP64) k_finalize<double><<<grid, kSmallBlock, 0, s>>>(dl, st, nfsr);
    else k_finalize<float><<<grid, kSmallBlock, 0, s>>>(dl, st, nfsr);
    CK(cudaGetLastError());
    k_reduce_k<<<1, 32, 0, s>>>(st, grid, integrations);
    CK(cudaGetLastError());
    k_residual<<<grid, kSmallBlock, 0, s>>>(st, nfsr);
    CK(cudaGetLastError());
    k_reduce_res<<<1, 32, 0, s>>>(st, grid);
    return cudaGetLastError();
}

cudaError_t launch_finalize_fixed(int precision, const DevLayout &dl, const DevState &st,
                                  int32_t nfsr, int grid, double integrations, cudaStream_t s) {
    if (precision == MOC_FP64) k_finalize<double><<<grid, kSmallBlock, 0, s>>>(dl, st, nfsr);
    else k_finalize<float><<<grid, kSmallBlock, 0, s>>>(dl, st, nfsr);
    CK(cudaGetLastError());
    k_reduce_k<<<1, 32, 0, s>>>(st, grid, integrations);
    return cudaGetLastError();
}

cudaError_t launch_init_state(const DevLayout &dl, const DevState &st, int32_t nfsr, int grid,
                              cudaStream_t s) {
    k_init_state<<<grid, kSmallBlock, 0, s>>>(dl, st, nfsr);
    CK(cudaGetLastError());
    k_init_finish<<<1, 256, 0, s>>>(st, grid, nfsr);
    return cudaGetLastError();
}
