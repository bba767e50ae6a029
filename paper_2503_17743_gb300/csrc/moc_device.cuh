// Device-side data structures and the on-the-fly 3D segment generator.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "moc_internal.h"

#define MOC_PI 3.14159265358979323846

// Read-only problem data of one track layout, all device pointers.
struct DevLayout {
    const StackDesc *desc;   // [n_stacks] upward stacks
    const int32_t *zn;       // lattice boundary integer parts
    const float *zf;         // lattice boundary fractions (topology decisions, FP32 lengths)
    const double *zf64;      // the same fractions in FP64 (FP64 sweeps only)
    const int32_t *reg2d;    // radial region of each 2D segment
    const float *len2d;      // length of each 2D segment (cm)
    const double *len2d64;   // the same in FP64 (FP64 sweeps only)
    const int64_t *tpl_off;  // stored templates: record offsets [n_tpl + 1]
    const int64_t *tpl_loff; // offsets into tpl_lidx [n_tpl + 1]
    const int32_t *tpl_lmin; // lowest template layer of each template
    const int32_t *tpl_lidx; // first record of each template layer (relative), + count
    const void *segs;        // template records, SegRec<real>
    const int32_t *fsr_mat;  // material of each FSR
    const int32_t *dst;      // [n_gtrk*4] link destination of every track direction, or null (all vacuum)
    const uint64_t *win;     // [slots] stored stacks: each slot's record window (perm order)
    const int32_t *perm;     // [slots] per stack (StackDesc::slot_off), its tracks in sweep
                             // order: by decreasing segment count (ties: class by class,
                             // then by index); with synchronous blocks, blocks of sync_b
                             // consecutive tracks r + m cpl of one class, padding entries
                             // -1 - (r + m cpl) continuing the block's sequence
    int32_t sync_b;          // tracks per synchronous block (0: none)
    int32_t matk;            // 1: every radial region has one material in all layers, the
                             // stored records carry it (tpl_key_mat, tpl_key_seg_mat) and the
                             // shared rows hold Qr only (Sigma_t from the material table)
    int32_t tally3;          // 1: the FSR tally is three 64-bit fixed-point words per
                             // FSR-group (FP32 sweeps with the shared tally), else FP64
    const int32_t *reg_mat;  // per radial region: its material if the same in every layer, else -1
    int32_t Nz, cpl, NL, G, M, Ph;  // NL: the sweep's (uniform) layers
    float rcpl;              // 1 / cpl rounded to FP32 (0 when cpl = 0)
    int32_t NLr;             // the geometry's layers (FSR = region * NLr + layer)
    const int32_t *lmap;     // the geometry's layer of each sweep layer, or null (the same)
    int32_t bc_zmin, bc_zmax;
    int32_t tally_bits;      // FP32 shared tally: fixed-point bits per unit bound (0: not used)
    int64_t n_slots;         // geometric tracks * 4 variants (bound of every link)
    // radial chunks of units whose tile does not fit in shared memory
    const int64_t *chunk_tab; // see StackDesc::chunk_base
    int32_t chunk_b;         // 2D segments per chunk (0: every unit is swept whole)
    int32_t hand_trk;        // tracks per block in the chunk hand-off buffer
    void *hand;              // [grid][hand_trk][2 frames][G] real: psi between chunks
    // layer planes off the axial lattice (offlat = 1; cpl = 0): per frame f
    // the rank of each boundary's fraction (zc[f]), the mirrored frame's own
    // fractions (zfd, zfd64) and the NL + 1 planes of each frame (integer
    // part, rank, fraction; frame-major)
    int32_t offlat;
    const int16_t *zc0, *zc1;
    const float *zfd;
    const double *zfd64;
    const int32_t *pl_n, *pl_c;
    const float *pl_f;
    const double *pl_f64;
};

// State buffers of one solve.
struct DevState {
    double *phi;        // [nfsr*G] scalar flux (unnormalised after a sweep)
    void *qr;           // [nfsr*G] Q / Sigma_t per steradian, real
    double *tally;      // [nfsr*G] FP64 tally accumulator
    double *vol;        // [nfsr] tracked volumes
    void *psi_a;        // boundary fluxes, [n_gtrk*4*G] real (may be null: all vacuum)
    void *psi_b;
    double *fiss;       // [nfsr] raw fission rate of the latest flux
    double *fiss_old;   // [nfsr] normalised fission rate of the previous flux
    double *partial;    // per-block partial sums
    double *scal;       // device scalars (see ScalarSlot)
    int32_t *counter;   // work counter of the persistent sweep
    const void *sig_t;  // [M*G] real
    const double *sig_t64, *sig_s64, *nsf64, *chi64, *src64;  // [M*G(*G)] FP64 cross sections
    const double *inv_st64, *siga64;  // [M*G] 1 / Sigma_t and Sigma_a = Sigma_t - sum_h Sigma_s[g->h]
    const double *inv_vol;            // [nfsr] 1 / tracked volume (0 for an untracked FSR)
};

// slots of DevState::scal
enum ScalarSlot {
    SC_K = 0,      // current k
    SC_DK,         // last k change
    SC_SCALE,      // 1 / production of the latest flux (eigen) or 1
    SC_PROD,       // production of the latest flux (raw)
    SC_ABS,        // absorption of the latest flux (raw)
    SC_LEAK,       // leakage accumulated by the latest sweep (raw)
    SC_RES,        // residual
    SC_ITER,       // iterations done
    SC_CONV,       // 1 when converged
    SC_TOLK, SC_TOLS,
    SC_EIGEN,      // 1 for an eigenvalue problem
    SC_INTEG,      // integrations performed
    SC_LEAK_PREV,  // leakage of the latest completed sweep, normalised
    SC_ERR,        // nonzero: a sweep dropped a tally update (contention limit)
    SC_COUNT = 16
};

// ---------------------------------------------------------------------------
// On-the-fly generation of the 3D segments of one track of an upward z-stack
// (Eqs. 5-11, Alg. 1 "traceSegmentsOTF").
//
// In lattice units u = z / dz the track i of the stack is u(s) = i + zeta(s)
// (Eq. 5).  With zeta at the 2D boundaries stored as integer + fraction, the
// layer crossed inside a 2D segment and the FSR sequence follow from integer
// arithmetic only; lengths are Eq. 8 (full 2D length / sin), Eq. 11 (full
// layer, cpl * dz / cos) or a partial lattice interval times dz / cos.
// `visit(b, layer, len)` is called for every segment in traversal order:
// along the 2D track for sense 0, against it for sense 1.

// FSR of (radial region, sweep layer L): unequal geometry layers are split
// into uniform sweep layers, each mapped to the geometry layer holding it
__device__ __forceinline__ int64_t fsr_of(const DevLayout &dl, int reg, int L) {
    return (int64_t)reg * dl.NLr + (dl.lmap ? __ldg(dl.lmap + L) : L);
}

// A stored template piece: key (see tpl_key) and its length.
template <typename real>
struct SegRec;
template <>
struct __align__(8) SegRec<float> {
    uint32_t key;
    float len;
};
template <>
struct __align__(16) SegRec<double> {
    uint32_t key;
    uint32_t pad;
    double len;
};

template <typename real>
__device__ __forceinline__ real lat_frac(const DevLayout &dl, int idx);
template <>
__device__ __forceinline__ float lat_frac<float>(const DevLayout &dl, int idx) { return __ldg(dl.zf + idx); }
template <>
__device__ __forceinline__ double lat_frac<double>(const DevLayout &dl, int idx) { return __ldg(dl.zf64 + idx); }
template <typename real>
__device__ __forceinline__ real len_2d(const DevLayout &dl, int idx);
template <>
__device__ __forceinline__ float len_2d<float>(const DevLayout &dl, int idx) { return __ldg(dl.len2d + idx); }
template <>
__device__ __forceinline__ double len_2d<double>(const DevLayout &dl, int idx) { return __ldg(dl.len2d64 + idx); }
__device__ __forceinline__ float lam_of(const StackDesc &d, float) { return d.lam; }
__device__ __forceinline__ double lam_of(const StackDesc &d, double) { return d.lam64; }
__device__ __forceinline__ float isin_of(const StackDesc &d, float) { return d.inv_sin; }
__device__ __forceinline__ double isin_of(const StackDesc &d, double) { return d.inv_sin64; }

template <typename real>
struct SegRange {
    int32_t ua, ub;   // integer lattice coordinate at the piece ends (clipped to [0, Nz])
    real fa, fb;      // fractions at the ends
    bool full;        // spans the whole 2D segment (Eq. 8 applies)
    int32_t La, Le;   // first and last layer crossed
};

// Topology (integers and the sign of the FP32 fraction) is the same for both
// precisions; only the fractions that enter the lengths change type.
template <typename real>
__device__ __forceinline__ void seg_range(const DevLayout &dl, const StackDesc &d, int i, int b,
                                          SegRange<real> &r) {
    int32_t ua = i + __ldg(dl.zn + d.zoff + b);
    real fa = lat_frac<real>(dl, d.zoff + b);
    int32_t ub = i + __ldg(dl.zn + d.zoff + b + 1);
    const bool fb_pos = __ldg(dl.zf + d.zoff + b + 1) > 0.0f;
    real fb = lat_frac<real>(dl, d.zoff + b + 1);
    bool full = true;
    if (ua < 0) { ua = 0; fa = (real)0; full = false; }
    bool end_pos = fb_pos;
    if (ub > dl.Nz || (ub == dl.Nz && fb_pos)) { ub = dl.Nz; fb = (real)0; end_pos = false; full = false; }
    r.ua = ua; r.fa = fa; r.ub = ub; r.fb = fb; r.full = full;
    r.La = min(ua / dl.cpl, dl.NL - 1);
    r.Le = min((end_pos ? ub : ub - 1) / dl.cpl, dl.NL - 1);
}

template <typename real>
__device__ __forceinline__ real piece_len(const DevLayout &dl, const StackDesc &d, int b,
                                          const SegRange<real> &r, int L) {
    const real lam = lam_of(d, (real)0);
    if (r.La == r.Le) {
        if (r.full) return len_2d<real>(dl, d.seg2d_off + b) * isin_of(d, (real)0);   // Eq. 8
        return ((real)(r.ub - r.ua) + (r.fb - r.fa)) * lam;
    }
    if (L == r.La) return ((real)((r.La + 1) * dl.cpl - r.ua) - r.fa) * lam;
    if (L == r.Le) return ((real)(r.ub - r.Le * dl.cpl) + r.fb) * lam;
    return (real)dl.cpl * lam;                                                      // Eq. 11
}

// first 2D segment whose end lies above the bottom: i + zeta(b+1) > 0
__device__ __forceinline__ int first_seg(const DevLayout &dl, const StackDesc &d, int i) {
    if (i + __ldg(dl.zn + d.zoff) >= 0) return 0;
    int lo = 0, hi = d.nb - 1;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        int u = i + __ldg(dl.zn + d.zoff + mid + 1);
        bool above = u > 0 || (u == 0 && __ldg(dl.zf + d.zoff + mid + 1) > 0.0f);
        if (above) hi = mid; else lo = mid + 1;
    }
    return lo;
}

// last 2D segment: the first whose end reaches the top, i + zeta(b+1) >= Nz
__device__ __forceinline__ int last_seg(const DevLayout &dl, const StackDesc &d, int i) {
    if (i + __ldg(dl.zn + d.zoff + d.nb) < dl.Nz) return d.nb - 1;
    int lo = 0, hi = d.nb - 1;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (i + __ldg(dl.zn + d.zoff + mid + 1) >= dl.Nz) hi = mid; else lo = mid + 1;
    }
    return lo;
}

template <typename real, class Visit>
__device__ __forceinline__ void walk_otf(const DevLayout &dl, const StackDesc &d, int i, int sense,
                                         Visit &visit) {
    const int b0 = first_seg(dl, d, i), b1 = last_seg(dl, d, i);
    SegRange<real> r;
    if (sense == 0) {
        for (int b = b0; b <= b1; ++b) {
            seg_range(dl, d, i, b, r);
            for (int L = r.La; L <= r.Le; ++L) visit(b, L, piece_len(dl, d, b, r, L));
        }
    } else {
        for (int b = b1; b >= b0; --b) {
            seg_range(dl, d, i, b, r);
            for (int L = r.Le; L >= r.La; --L) visit(b, L, piece_len(dl, d, b, r, L));
        }
    }
}

// number of segments of track i (no lengths)
__device__ __forceinline__ int count_otf(const DevLayout &dl, const StackDesc &d, int i) {
    const int b0 = first_seg(dl, d, i), b1 = last_seg(dl, d, i);
    int n = 0;
    SegRange<float> r;
    for (int b = b0; b <= b1; ++b) {
        seg_range(dl, d, i, b, r);
        n += r.Le - r.La + 1;
    }
    return n;
}

// ---------------------------------------------------------------------------
// Layer planes off the axial lattice (Sec. 2.2's local axial mesh).  The
// frames no longer share their pieces: each walks its own planes (frame 1 in
// the mirrored coordinate, the same numbers as frame 0's lattice coordinate,
// its layer L standing for the geometry's NL - 1 - L).  A point is the pair
// (integer part, rank of its fraction in that frame); every decision is a
// comparison of such pairs, the lengths use the fractions.

struct OLPoint {
    int32_t n, c;
};
__device__ __forceinline__ bool ol_le(int32_t an, int32_t ac, int32_t bn, int32_t bc) {
    return an < bn || (an == bn && ac <= bc);
}
__device__ __forceinline__ bool ol_lt(int32_t an, int32_t ac, int32_t bn, int32_t bc) {
    return an < bn || (an == bn && ac < bc);
}

template <typename real>
__device__ __forceinline__ real ol_zf(const DevLayout &dl, int frame, int idx);
template <>
__device__ __forceinline__ float ol_zf<float>(const DevLayout &dl, int frame, int idx) {
    return __ldg((frame ? dl.zfd : dl.zf) + idx);
}
template <>
__device__ __forceinline__ double ol_zf<double>(const DevLayout &dl, int frame, int idx) {
    return __ldg((frame ? dl.zfd64 : dl.zf64) + idx);
}
template <typename real>
__device__ __forceinline__ real ol_pf(const DevLayout &dl, int k);
template <>
__device__ __forceinline__ float ol_pf<float>(const DevLayout &dl, int k) { return __ldg(dl.pl_f + k); }
template <>
__device__ __forceinline__ double ol_pf<double>(const DevLayout &dl, int k) { return __ldg(dl.pl_f64 + k); }

// The layer of frame `frame` holding the point (n, c): the largest L < NL
// whose lower plane lies at or below it (upper = false: the start of a piece,
// a point on a plane belongs to the layer above) or strictly below it
// (upper = true: the end of a piece, a point on a plane ends the layer below)
__device__ __forceinline__ int ol_layer(const DevLayout &dl, int frame, int32_t n, int32_t c, bool upper) {
    const int32_t *pn = dl.pl_n + frame * (dl.NL + 1), *pc = dl.pl_c + frame * (dl.NL + 1);
    int lo = 0, hi = dl.NL - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        const int32_t mn = __ldg(pn + mid), mc = __ldg(pc + mid);
        const bool below = upper ? ol_lt(mn, mc, n, c) : ol_le(mn, mc, n, c);
        if (below) lo = mid; else hi = mid - 1;
    }
    return lo;
}

template <typename real>
struct OLRange {
    int32_t ua, ub;   // integer parts at the piece ends (clipped to [0, Nz])
    real fa, fb;      // fractions at the ends (this frame's)
    bool full;        // spans the whole 2D segment (Eq. 8 applies)
    int32_t La, Le;   // first and last layer of this frame crossed
};

template <typename real>
__device__ __forceinline__ void ol_range(const DevLayout &dl, const StackDesc &d, int i, int b, int frame,
                                         OLRange<real> &r) {
    const int z = d.zoff + b;
    const int16_t *zc = frame ? dl.zc1 : dl.zc0;
    int32_t ua = i + __ldg(dl.zn + z), ca = __ldg(zc + z);
    int32_t ub = i + __ldg(dl.zn + z + 1), cb = __ldg(zc + z + 1);
    real fa = ol_zf<real>(dl, frame, z), fb = ol_zf<real>(dl, frame, z + 1);
    bool full = true;
    // rank 1 is the fraction 0 in both frames
    if (ua < 0) { ua = 0; ca = 1; fa = (real)0; full = false; }
    if (ub > dl.Nz || (ub == dl.Nz && cb > 1)) { ub = dl.Nz; cb = 1; fb = (real)0; full = false; }
    r.ua = ua; r.fa = fa; r.ub = ub; r.fb = fb; r.full = full;
    r.La = ol_layer(dl, frame, ua, ca, false);
    r.Le = ol_layer(dl, frame, ub, cb, true);
}

template <typename real>
__device__ __forceinline__ real ol_len(const DevLayout &dl, const StackDesc &d, int b, int frame,
                                       const OLRange<real> &r, int L) {
    const real lam = lam_of(d, (real)0);
    if (r.La == r.Le) {
        if (r.full) return len_2d<real>(dl, d.seg2d_off + b) * isin_of(d, (real)0);   // Eq. 8
        return ((real)(r.ub - r.ua) + (r.fb - r.fa)) * lam;
    }
    const int k = frame * (dl.NL + 1);
    if (L == r.La)
        return ((real)(__ldg(dl.pl_n + k + L + 1) - r.ua) + (ol_pf<real>(dl, k + L + 1) - r.fa)) * lam;
    if (L == r.Le) return ((real)(r.ub - __ldg(dl.pl_n + k + L)) + (r.fb - ol_pf<real>(dl, k + L))) * lam;
    return ((real)(__ldg(dl.pl_n + k + L + 1) - __ldg(dl.pl_n + k + L)) +                  // Eq. 11
            (ol_pf<real>(dl, k + L + 1) - ol_pf<real>(dl, k + L))) * lam;
}

// the pieces of track i of frame `frame`, in the order of `sense`:
// visit(b, the geometry's layer, length)
template <typename real, class Visit>
__device__ __forceinline__ void walk_ol(const DevLayout &dl, const StackDesc &d, int i, int frame,
                                        int sense, Visit &visit) {
    const int b0 = first_seg(dl, d, i), b1 = last_seg(dl, d, i);
    const int NL = dl.NL;
    OLRange<real> r;
    if (sense == 0) {
        for (int b = b0; b <= b1; ++b) {
            ol_range(dl, d, i, b, frame, r);
            for (int L = r.La; L <= r.Le; ++L) visit(b, frame ? NL - 1 - L : L, ol_len(dl, d, b, frame, r, L));
        }
    } else {
        for (int b = b1; b >= b0; --b) {
            ol_range(dl, d, i, b, frame, r);
            for (int L = r.Le; L >= r.La; --L) visit(b, frame ? NL - 1 - L : L, ol_len(dl, d, b, frame, r, L));
        }
    }
}

__device__ __forceinline__ int count_ol(const DevLayout &dl, const StackDesc &d, int i, int frame) {
    const int b0 = first_seg(dl, d, i), b1 = last_seg(dl, d, i);
    int n = 0;
    OLRange<float> r;
    for (int b = b0; b <= b1; ++b) {
        ol_range(dl, d, i, b, frame, r);
        n += r.Le - r.La + 1;
    }
    return n;
}

// Exit of track i of a stack in variant v (frame = v >> 1, sense = v & 1):
// returns the destination geometric track * 4 + variant, -1 for a vacuum
// face.  Exit type from the integer lattice at the exit end: radial (per-stack
// rule), axial (same stack, other frame, index -/+ Nz) or an edge shared with
// an axial face (both reflective: the track reverses).
__device__ __forceinline__ int64_t exit_dest(const DevLayout &dl, const StackDesc *descs,
                                             const StackDesc &d, const StackDesc *dg, int i, int v) {
    const int frame = v >> 1, sense = v & 1;
    const int z = d.zoff + (sense == 0 ? d.nb : 0);
    const int32_t ui = i + __ldg(dl.zn + z);
    const float uf = __ldg(dl.zf + z);
    int kind;
    int abc;
    if (sense == 0) {
        kind = ui < dl.Nz ? 0 : ((ui == dl.Nz && uf == 0.0f) ? 2 : 1);
        abc = frame == 0 ? dl.bc_zmax : dl.bc_zmin;
    } else {
        kind = (ui > 0 || (ui == 0 && uf > 0.0f)) ? 0 : ((ui == 0 && uf == 0.0f) ? 2 : 1);
        abc = frame == 0 ? dl.bc_zmin : dl.bc_zmax;
    }
    const int64_t gid = d.trk_off + (i - d.i_lo);
    // per-variant link fields are read from global memory (dg) so that the
    // register copy `d` is never indexed dynamically
    const int rbc = dg->rad_bc[v];
    if (kind == 2) return (abc && rbc) ? gid * 4 + (frame * 2 + (1 - sense)) : -1;
    if (kind == 1) {
        if (!abc) return -1;
        const int j = sense == 0 ? i - dl.Nz : i + dl.Nz;
        return (d.trk_off + (j - d.i_lo)) * 4 + ((1 - frame) * 2 + sense);
    }
    if (!rbc) return -1;
    const int dst = dg->rad_dst[v];
    const int j = (int)dg->rad_sign[v] * i + dg->rad_shift[v];
    return (descs[dst].trk_off + (j - descs[dst].i_lo)) * 4 + dg->rad_var[v];
}

// The FSR tally of FP32 sweeps with the shared tally: per FSR-group three
// signed 64-bit words (A0, A1, A2) holding (A0 + A1 2^42 + A2 2^84) 2^-64.
// A unit flushes each tile word as an integer w times its power-of-two
// fixed-point unit 2^(sh - 64); w 2^sh is split at 42-bit boundaries into a
// non-negative low part and a signed high part, each added with a native
// 64-bit integer atomic (no carry between the words; fewer than 2^21 adds per
// word keep every word in range).  Integer adds are exact and associative, so
// the tally does not depend on the order in which units finish: a solve gives
// the same tallies on every run and in any mix of solves.  Returns false for
// a unit beyond the representable range (|value| >= 2^51).
__device__ __forceinline__ bool tally3_add(long long *acc, int w, int sh) {
    unsigned long long *a = reinterpret_cast<unsigned long long *>(acc);
    const long long v = w;
    if (sh < 0) {  // below 2^-64: truncated
        atomicAdd(a, (unsigned long long)(v >> min(-sh, 63)));
        return true;
    }
    if (sh >= 84) {
        if (sh > 115) return false;
        atomicAdd(a + 2, (unsigned long long)(v << (sh - 84)));
        return true;
    }
    const int k = sh >= 42 ? 1 : 0, r = sh - 42 * k, s2 = 42 - r;
    const long long hi = v >> s2;                          // floor(w 2^r / 2^42)
    const long long lo = (v & ((1ll << s2) - 1)) << r;     // w 2^r - hi 2^42, in [0, 2^42)
    if (lo) atomicAdd(a + k, (unsigned long long)lo);
    if (hi) atomicAdd(a + k + 1, (unsigned long long)hi);
    return true;
}
__host__ __device__ __forceinline__ double tally3_value(long long a0, long long a1, long long a2) {
    // 2^-64, 2^-22, 2^20
    return (double)a0 * 5.421010862427522e-20 + (double)a1 * 2.384185791015625e-07 + (double)a2 * 1048576.0;
}

__device__ __forceinline__ float fast_exp2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// ---------------------------------------------------------------------------
// Segment templates.  Because the layer planes lie on the axial lattice, track
// i + cpl of a z-stack is track i shifted up by exactly one layer (Eq. 5 with
// i -> i + cpl): same 2D segments, same lengths, layer + 1.  The unclipped line
// u(s) = i0 + zeta(s) of a stack therefore serves as a template for every
// track i0 + m cpl: that track's segments are the template pieces whose layer
// L_t + m lies in [0, NL).  The domain faces z = 0 and z = H are layer planes,
// so clipping a track to the domain never cuts a template piece.

__device__ __forceinline__ int floor_div(int a, int c) { return a >= 0 ? a / c : -((-a + c - 1) / c); }
// the same from rc = 1 / c rounded to FP32: for |a| < 2^22 the estimate
// floor(a rc) is off by at most one, and one correction step makes it exact;
// larger |a| take the integer division
__device__ __forceinline__ int floor_div_rc(int a, int c, float rc) {
    if (a >= (1 << 22) || a <= -(1 << 22)) return floor_div(a, c);
    int q = __float2int_rd((float)a * rc);
    const int r = a - q * c;
    q += (r >= c ? 1 : 0) - (r < 0 ? 1 : 0);
    return q;
}

// pieces of the unclipped line u = i0 + zeta(s) inside 2D segment b
template <typename real>
struct TplRange {
    int32_t ua, ub;
    real fa, fb;
    int32_t La, Le;
};

template <typename real>
__device__ __forceinline__ void tpl_range(const DevLayout &dl, const StackDesc &d, int i0, int b,
                                          TplRange<real> &r) {
    r.ua = i0 + __ldg(dl.zn + d.zoff + b);
    r.fa = lat_frac<real>(dl, d.zoff + b);
    r.ub = i0 + __ldg(dl.zn + d.zoff + b + 1);
    r.fb = lat_frac<real>(dl, d.zoff + b + 1);
    const bool fb_pos = __ldg(dl.zf + d.zoff + b + 1) > 0.0f;
    r.La = floor_div_rc(r.ua, dl.cpl, dl.rcpl);
    r.Le = floor_div_rc(fb_pos ? r.ub : r.ub - 1, dl.cpl, dl.rcpl);
}

template <typename real>
__device__ __forceinline__ real tpl_len(const DevLayout &dl, const StackDesc &d, int b,
                                        const TplRange<real> &r, int L) {
    const real lam = lam_of(d, (real)0);
    if (r.La == r.Le) return len_2d<real>(dl, d.seg2d_off + b) * isin_of(d, (real)0);      // Eq. 8
    if (L == r.La) return ((real)((r.La + 1) * dl.cpl - r.ua) - r.fa) * lam;
    if (L == r.Le) return ((real)(r.ub - r.Le * dl.cpl) + r.fb) * lam;
    return (real)dl.cpl * lam;                                                              // Eq. 11
}

// A stored template piece (b the 2D segment, L_t the template layer; track
// r + m cpl of the class meets the piece in tile rows b NL + L_t + m in the
// upward frame and b NL + NL - 1 - L_t - m in the mirrored one).  Two key
// formats:
// * units swept whole (every tile row < 2^15): the two rows of the class's
//   own line, A = b NL + L_t and B = b NL + NL - 1 - L_t, as signed 16-bit
//   numbers (A low, B high): the sweep adds m and subtracts m;
// * layouts with radial chunks (large units): b << 16 | L_t (b < 2^16, L_t
//   signed 16 bits).
__host__ __device__ __forceinline__ uint32_t tpl_key(int A, int B) {
    return (uint32_t)(uint16_t)(int16_t)A | ((uint32_t)(uint16_t)(int16_t)B << 16);
}
__device__ __forceinline__ int tpl_row_up(uint32_t key) { return (int)(int16_t)(key & 0xffffu); }
__device__ __forceinline__ int tpl_row_down(uint32_t key) { return (int)key >> 16; }
// Layouts with one material per radial region (DevLayout::matk): the upward
// row in bits 0-15 as above, the mirrored row in bits 16-29 (signed, |B| <
// 2^13) and the piece's material in bits 30-31 (M <= 4)
__host__ __device__ __forceinline__ uint32_t tpl_key_mat(int A, int B, int mat) {
    return (uint32_t)(uint16_t)(int16_t)A | (((uint32_t)B & 0x3fffu) << 16) | ((uint32_t)mat << 30);
}
__device__ __forceinline__ int tpl_row_down_mat(uint32_t key) { return (int)(key << 2) >> 18; }
__device__ __forceinline__ int tpl_mat(uint32_t key) { return (int)(key >> 30); }
// the same for the keys of radially chunked layouts: 2D segment b < 2^14 in
// bits 16-29, the template layer in bits 0-15, the material in bits 30-31
__host__ __device__ __forceinline__ uint32_t tpl_key_seg_mat(int b, int L, int mat) {
    return (((uint32_t)b & 0x3fffu) << 16) | (uint32_t)(uint16_t)(int16_t)L | ((uint32_t)mat << 30);
}
__device__ __forceinline__ int tpl_seg_mat(uint32_t key) { return (int)((key >> 16) & 0x3fffu); }
__host__ __device__ __forceinline__ uint32_t tpl_key_seg(int b, int L) {
    return ((uint32_t)b << 16) | (uint32_t)(uint16_t)(int16_t)L;
}
__device__ __forceinline__ int tpl_seg(uint32_t key) { return (int)(key >> 16); }
__device__ __forceinline__ int tpl_layer(uint32_t key) { return (int)(int16_t)(key & 0xffffu); }
