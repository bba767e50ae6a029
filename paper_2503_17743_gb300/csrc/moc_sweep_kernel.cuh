// The transport sweep kernel (Eq. 3 on every segment, Eq. 4 tallies).
//
// Work decomposition.  A persistent grid; each block takes one work unit at a
// time from a global counter: a 2D track with all its polar z-stacks (units in
// decreasing work order).  The tracks r, r + cpl, r + 2 cpl, ... of a z-stack
// are one track shifted up by one layer each (Eq. 5 with the layer planes on
// the axial lattice), so a single segment template serves all of them: track
// r + m cpl crosses the template pieces whose layer L_t + m lies in [0, NL).
// The layer never decreases along an upward line, so those pieces are one
// contiguous range of the template's records.
//
// A warp task is (polar stack, class r, block of SLOTS = 32/GL tracks m of the
// class, sense).  Slot j (GL lanes) walks its own track's record range; each
// lane carries GPL energy groups, kept in GPL group planes of the shared rows.
// Every lane sweeps both frames: the upward track and the mirrored downward
// track that shares its segments (layer NL-1-L).  Slots of one warp run the
// same number of steps except where a track is clipped by the top or bottom
// face, so nearly every lane does useful work.
//
// Shared tally (SMEM = true): per unit the block stages one row per
// (2D segment, layer) FSR the unit crosses, holding (Qr, Sigma_t) for every
// group, plus a zeroed tally row; pieces touch only shared memory and the rows
// are flushed into the FP64 global tally once per unit.  Templates come from
// the stored set (EXP, Sec. 4.2; four records at a time with the next four in
// flight) or each track is generated on the fly (OTF).  Without the shared
// tally (SMEM = false) pieces read Qr from global memory and add straight into
// the FP64 global tally.
//
// psi is carried multiplied by the track weight W and by the group's
// fixed-point tally scale S (1 without a fixed-point tile): with
// d = W S (psi - Qr) the attenuated change W S (psi_in - psi_out) =
// d (1 - e^{-Sigma_t l}) is both the psi update and the tally contribution in
// tally units (Eq. 3, Eq. 4), rounded to an integer by one conversion.
#pragma once

#include <climits>
#include <type_traits>

#include "moc_device.cuh"
#include "moc_exp64.cuh"
#include "moc_kernels.h"

namespace {

constexpr float kLog2e = 1.4426950408889634f;

// e^{-Sigma_t l} from x = Sigma_t l: FP32 on the MUFU pipe (Sigma_t pre-scaled
// by log2 e, the negation folds into the multiply), FP64 by the table-driven
// method of moc_exp64.cuh (tab: its table in shared memory)
template <typename real>
__device__ __forceinline__ real attenuation(real x, const double2 *tab);
template <>
__device__ __forceinline__ float attenuation<float>(float x, const double2 *) {
    return fast_exp2(-x);
}
template <>
__device__ __forceinline__ double attenuation<double>(double x, const double2 *tab) {
    return moc_exp64::exp_neg(x, tab);
}

// k / d for 0 <= k and 1 <= d, from the FP32 reciprocal rd ~ 1 / d: exact
// below 2^24 after one correction step (the estimate is off by at most one
// there); larger k take the integer division
__device__ __forceinline__ int div_by(int k, int d, float rd) {
    if (k >= (1 << 24)) return k / d;
    int q = __float2int_rz((float)k * rd);
    const int r = k - q * d;
    q += (r >= d ? 1 : 0) - (r < 0 ? 1 : 0);
    return q;
}

// per polar stack of the work unit, cached in shared memory
// (the track weight and its inverse in both precisions: the sweep's hot path
// does no FP64 arithmetic in FP32 mode)
struct UnitStack {
    int64_t trk_off, tpl_base, cbase, slot_off;
    double W, invW;
    float Wf, invWf;
    int32_t n_trk, i_lo, task_pre, n_slot;
};
constexpr int kMaxPh = 16;

// Template pieces generated on the fly (Eqs. 8-11 on the integer lattice), in
// the order of one sense, layers [0, NL) of the unclipped line i0.  The
// iterator keeps the stack's constants and the lattice coordinates of the
// current 2D segment's two boundaries (integer part, fraction, fraction > 0
// in the FP32 table); moving to the next 2D segment reuses the boundary the
// two share, so each step loads one boundary.  Pieces, lengths and layer
// ranges are those of tpl_range / tpl_len (the stored templates).
template <typename real>
struct TplIter {
    int i0, b, bend, L, Lend, dir;
    int zoff, soff;    // the stack's first boundary entry and first 2D segment
    real lam, isin;    // 3D length per lattice unit; 1 / sin(theta)
    int ua, ub, La, Le;
    real fa, fb;
    bool pa, pb;
    bool done;

    __device__ __forceinline__ void bound(const DevLayout &dl, int k, int &u, real &f, bool &p) {
        u = i0 + __ldg(dl.zn + zoff + k);
        f = lat_frac<real>(dl, zoff + k);
        p = __ldg(dl.zf + zoff + k) > 0.0f;
    }
    __device__ __forceinline__ void init(const DevLayout &dl, const StackDesc &d, int i0_, int b0, int b1,
                                         int dir_) {
        i0 = i0_;
        dir = dir_;
        zoff = d.zoff;
        soff = d.seg2d_off;
        lam = lam_of(d, (real)0);
        isin = isin_of(d, (real)0);
        b = dir > 0 ? b0 : b1;
        bend = dir > 0 ? b1 : b0;
        done = b0 > b1;
        if (!done) {
            bound(dl, b, ua, fa, pa);
            bound(dl, b + 1, ub, fb, pb);
            settle(dl);
        }
    }
    // to 2D segment b + dir, reusing the boundary the two segments share
    __device__ __forceinline__ void step(const DevLayout &dl) {
        if (dir > 0) {
            ua = ub; fa = fb; pa = pb;
            ++b;
            bound(dl, b + 1, ub, fb, pb);
        } else {
            ub = ua; fb = fa; pb = pa;
            --b;
            bound(dl, b, ua, fa, pa);
        }
    }
    // the layer range of 2D segment b; moving on while it holds no layer in [0, NL)
    __device__ __forceinline__ void settle(const DevLayout &dl) {
        for (;;) {
            La = floor_div_rc(ua, dl.cpl, dl.rcpl);
            Le = floor_div_rc(pb ? ub : ub - 1, dl.cpl, dl.rcpl);
            const int a = max(La, 0), e = min(Le, dl.NL - 1);
            if (a <= e) {
                L = dir > 0 ? a : e;
                Lend = dir > 0 ? e : a;
                return;
            }
            if (b == bend) {
                done = true;
                return;
            }
            step(dl);
        }
    }
    __device__ __forceinline__ void next(const DevLayout &dl, int &ob, int &oL, real &len) {
        ob = b;
        oL = L;
        if (La == Le) len = len_2d<real>(dl, soff + b) * isin;                          // Eq. 8
        else if (L == La) len = ((real)((La + 1) * dl.cpl - ua) - fa) * lam;
        else if (L == Le) len = ((real)(ub - Le * dl.cpl) + fb) * lam;
        else len = (real)dl.cpl * lam;                                                   // Eq. 11
        if (L != Lend) {
            L += dir;
        } else if (b != bend) {
            step(dl);
            settle(dl);
        } else {
            done = true;
        }
    }
};


// The (Qr, Sigma_t) pairs of a lane's GPL groups in one shared row, read at a
// 32-bit shared-memory address with one vector load
template <typename real, int GPL>
struct RowLoadS;
template <>
struct RowLoadS<float, 1> {
    static __device__ __forceinline__ void get(unsigned a, float (&q)[1], float (&s)[1]) {
        asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(q[0]), "=f"(s[0]) : "r"(a));
    }
};
// (with two or more groups per lane a row keeps each pair of groups as
// Qr_0 Qr_1 Sigma_0 Sigma_1, so that the pairs load as packed operands)
template <>
struct RowLoadS<float, 2> {
    static __device__ __forceinline__ void get(unsigned a, float (&q)[2], float (&s)[2]) {
        asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                     : "=f"(q[0]), "=f"(q[1]), "=f"(s[0]), "=f"(s[1])
                     : "r"(a));
    }
};
template <>
struct RowLoadS<float, 4> {
    static __device__ __forceinline__ void get(unsigned a, float (&q)[4], float (&s)[4]) {
        asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                     : "=f"(q[0]), "=f"(q[1]), "=f"(s[0]), "=f"(s[1])
                     : "r"(a));
        asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                     : "=f"(q[2]), "=f"(q[3]), "=f"(s[2]), "=f"(s[3])
                     : "r"(a + 16u));
    }
};

// Packed FP32 pairs (two groups of a lane) for the sm_100-family f32x2
// instructions (one issue slot for two operations): the rows keep each pair
// of groups as Qr_0 Qr_1 Sigma_0 Sigma_1, loaded as two float2 values
// the same pairs as float2 values (for the packed-pair intrinsics)
__device__ __forceinline__ void row_load_f2(unsigned a, float2 &q, float2 &s) {
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(q.x), "=f"(q.y), "=f"(s.x), "=f"(s.y)
                 : "r"(a));
}
__device__ __forceinline__ void lds_f2(unsigned a, float2 &v) {
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a));
}
// (split tile of synchronous blocks: Qr and Sigma_t of a row in two arrays,
// a lane's pair of groups as one float2 load from each)
template <>
struct RowLoadS<double, 1> {
    static __device__ __forceinline__ void get(unsigned a, double (&q)[1], double (&s)[1]) {
        asm volatile("ld.shared.v2.f64 {%0, %1}, [%2];" : "=d"(q[0]), "=d"(s[0]) : "r"(a));
    }
};

// fixed-point tally += v at a 32-bit shared-memory address (native integer add)
__device__ __forceinline__ void shared_red_add(unsigned a, int v) {
    asm volatile("red.shared.add.s32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}

// FP64 sweeps: tally += t on shared memory with one compare-and-swap of the
// 64-bit word per attempt (floating-point adds on shared memory have no
// single-instruction form; FP32 sweeps use the fixed-point tally instead).  A
// word is retried only when another lane changed it in between; after
// kCasLimit attempts the update is dropped and *err set, which the host
// reports as an error.
constexpr int kCasLimit = 1 << 16;

template <typename real, int GPL>
struct TallyAdd;
template <>
struct TallyAdd<double, 1> {
    static __device__ __forceinline__ void add(double *p, const double (&t)[1], double *err) {
        unsigned long long *w = reinterpret_cast<unsigned long long *>(p);
        unsigned long long old = *w;
        for (int it = 0; it < kCasLimit; ++it) {
            const unsigned long long nw = __double_as_longlong(__longlong_as_double(old) + t[0]);
            const unsigned long long prev = atomicCAS(w, old, nw);
            if (prev == old) return;
            old = prev;
        }
        *err = 1.0;
    }
};

// threads per sweep block, three blocks per SM in FP32: ten warps with one
// group per lane, nine with more (their extra registers), eight in FP64; the
// material-keyed kernel (rows of Qr only: a smaller tile) runs four blocks of
// eight warps (64 registers)
__host__ __device__ constexpr int sweep_block(bool fp32, int GPL, bool matk = false, bool chunk = false) {
    return fp32 ? (GPL == 1 ? 320 : (matk || chunk) ? 256 : 288) : 256;
}
__host__ __device__ constexpr int sweep_min_blocks(bool fp32, bool matk) { return fp32 ? (matk ? 4 : 3) : 2; }
constexpr int kMaxSweepBlock = 320;

// words per shared tally row (FP64 tally tile: row-major, [row][TS])
__host__ __device__ constexpr int tally_stride(int GL, int GPL) { return GL * GPL + (GPL > 1 ? 1 : 0); }

// FP32 fixed-point tally tile of units swept whole: group-major, [group][RS]
// with RS >= cap rows
// and RS GPL = 32 / GL (mod 32), so that the GL lanes of a slot, whose
// groups are GPL apart, land 32 / GL banks apart: two slots of a warp then
// meet in a bank only when their rows agree modulo 32 / GL (row-major rows
// of GL GPL words collide whenever their windows overlap)
__host__ __device__ constexpr int tally_rows(int cap, int GL, int GPL) {
    return cap + ((((32 / (GL * GPL)) % (32 / GPL)) - cap % (32 / GPL)) + (32 / GPL)) % (32 / GPL);
}

// Guard rows on both sides of the split tile of a layout with synchronous
// blocks: a block's idle tracks read rows at most 7 past the rows of its
// active ones (see the SYNC step loop), and the guard rows hold finite values
constexpr int kSyncGuard = 8;

// BATCH: one launch sweeps several solves of one layout (their states in
// items[n_items]); work index w is unit order[w / n_items] of solve
// w % n_items, so the solves' units interleave, largest first.
// SYNC (FP32, two groups per lane, units swept whole): the stored stacks are
// swept in synchronous blocks of dl.sync_b tracks r + m cpl (consecutive m)
// of one segment template.  The tracks of a block step through the
// template's records together, each active while the record lies in its own
// window (else length 0: psi unchanged, tally + 0).  Their tile rows are then
// consecutive, so the Qr loads and tally adds of a block meet no bank
// conflicts, and the record is read once per block.  The tile keeps Qr and
// Sigma_t in separate arrays, with Sigma_t also once per 2D segment when the
// segment's region has one material in every layer.
// MATK (layouts with DevLayout::matk; FP32, two groups per lane, no
// synchronous blocks): the shared rows hold Qr only and a piece's
// Sigma_t log2 e comes from the material table, the material read from the
// record's key (one 8-byte table load serves both frames: a 2D segment lies
// in one region, and the region has one material in every layer).
template <typename real, int GL, int GPL, bool SMEM, bool CHUNK, bool BATCH, bool SYNC = false,
          bool MATK = false>
__global__ void __launch_bounds__(sweep_block(sizeof(real) == 4, GPL, MATK && !CHUNK, CHUNK && !MATK),
                                  sweep_min_blocks(sizeof(real) == 4, MATK && !CHUNK))
    k_sweep(DevLayout dl, DevState st, const int32_t *order, int32_t n_work, int32_t cap,
            const real *psi_in_p, real *psi_out_p, const BatchItem *items, int32_t n_items) {
    constexpr int GP = GL * GPL;     // groups per chunk (padded)
    constexpr int SLOTS = 32 / GL;   // tracks per warp task
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_work, s_work_next, s_next, s_ntask;
    __shared__ UnitStack s_us[kMaxPh];
    __shared__ double s_leak[kMaxSweepBlock / 32];
    __shared__ float s_scl[32];      // FP32 fixed-point tally: scale of each group of the chunk
    __shared__ float s_inv[32];      // and its inverse
    __shared__ int s_sh[32];         // the tally unit s_inv = 2^(s_sh - 64)
    __shared__ unsigned s_bmax[32];  // bound of |W psi| and |W Qr| per group (float bits)
    __shared__ unsigned s_ubnd[32];  // max |psi_in| over the unit's tracks per group (float bits)
    __shared__ unsigned s_hmax[32];  // max |psi| handed to the next radial chunk (float bits)
    __shared__ float s_wmax;
    __shared__ BatchItem s_item;     // BATCH: the solve of the current unit
    __shared__ double2 s_exp[sizeof(real) == 8 ? 64 : 1];  // FP64: 2^{j/64} as hi, lo
    constexpr bool kFixed = sizeof(real) == 4;  // FP32 sweeps tally in fixed point
    const int G = dl.G, NL = dl.NL, M = dl.M, Ph = dl.Ph, cpl = dl.cpl;
    const float rcpl = 1.0f / (float)max(cpl, 1);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    const int j = lane / GL;         // slot: track of the warp task
    const int ql = lane & (GL - 1);  // lane of the slot: groups ql * GPL + c, c < GPL
    // shared layout: sig [M][GP] | rows [cap][GP][2] (Qr, Sigma_t) | tally:
    // [GP][RS] (tally_rows) or [cap][TS] with rows padded by one word when a
    // lane holds several groups
    constexpr int TS = tally_stride(GL, GPL);
    // tally word of (tile row, group q): group-major for the FP32 fixed-point
    // tile of units swept whole, row-major otherwise (FP64; and radial
    // chunks, whose kernel is short of registers for the stride);
    // CS = words from group q to q + 1 of the same row
    constexpr bool kGM = kFixed && (!CHUNK || MATK);
    // units swept whole without synchronous blocks: a warp task takes SLOTS
    // consecutive slots of the unit's stacks laid end to end (tracks of two
    // polar stacks may share a warp), so that only the unit's last task per
    // sense has idle slots instead of every stack's last
    constexpr bool FLAT = !CHUNK && !SYNC;
    const int RS = kGM ? tally_rows(cap, GL, GPL) : 0;
    const int CS = kGM ? RS : 1;
    auto tix = [&](int row, int q) { return kGM ? q * RS + row : row * TS + q; };
    static_assert(!SYNC || (sizeof(real) == 4 && GPL == 2 && SMEM && !CHUNK), "synchronous blocks: FP32 pairs");
    static_assert(!MATK || (sizeof(real) == 4 && GPL == 2 && SMEM && !SYNC), "material keys: FP32 pairs");
    if (!BATCH && st.scal[SC_CONV] != 0.0) return;  // converged: later iterations are no-ops
    real *sig = reinterpret_cast<real *>(smem);
    size_t off = ((size_t)M * GP * sizeof(real) + 15) & ~(size_t)15;
    real *rows = reinterpret_cast<real *>(smem + off);
    // split tile (SYNC): Qr [row][GP] and Sigma_t log2 e [row][GP], each with
    // kSyncGuard guard rows before and after; Sigma_t of each 2D segment
    // [cap / NL][GP] (-1: the segment's region changes material with the layer)
    float *qr_t = nullptr, *sg_t = nullptr, *sb_t = nullptr;
    if constexpr (SYNC) {
        qr_t = reinterpret_cast<float *>(smem + off) + kSyncGuard * GP;
        off += (size_t)(cap + 2 * kSyncGuard) * GP * 4;
        sg_t = reinterpret_cast<float *>(smem + off) + kSyncGuard * GP;
        off += (size_t)(cap + 2 * kSyncGuard) * GP * 4;
        sb_t = reinterpret_cast<float *>(smem + off);
        off += ((size_t)(cap / NL) * GP * 4 + 15) & ~(size_t)15;
    } else {
        off += (size_t)cap * GP * (MATK ? 1 : 2) * sizeof(real);
    }
    real *tl_s = reinterpret_cast<real *>(smem + off);
    int *tl_i = reinterpret_cast<int *>(smem + off);  // the same tally rows in fixed point
    const unsigned rows_sa = (unsigned)__cvta_generic_to_shared(rows);
    const unsigned sig_sa = (unsigned)__cvta_generic_to_shared(sig);
    const unsigned tl_sa = (unsigned)__cvta_generic_to_shared(tl_s);
    const unsigned qr_sa = SYNC ? (unsigned)__cvta_generic_to_shared(qr_t) : 0u;
    const unsigned sg_sa = SYNC ? (unsigned)__cvta_generic_to_shared(sg_t) : 0u;
    const unsigned sb_sa = SYNC ? (unsigned)__cvta_generic_to_shared(sb_t) : 0u;
    if constexpr (SYNC) {
        // every row of the split tile holds finite values from here on (the
        // guard rows stay 0; unit rows are restaged per unit)
        for (int i = tid - kSyncGuard * GP; i < (cap + kSyncGuard) * GP; i += blockDim.x) {
            qr_t[i] = 0.0f;
            sg_t[i] = 0.0f;
        }
    }

    const real *sig_g = reinterpret_cast<const real *>(st.sig_t);
    const SegRec<real> *recs = reinterpret_cast<const SegRec<real> *>(dl.segs);
    real leak = (real)0;  // this lane's W psi leaving through vacuum faces
    if (tid < 32) {
        s_hmax[tid] = 0u;
        s_ubnd[tid] = 0u;
    }
    if constexpr (sizeof(real) == 8)
        for (int i = tid; i < 64; i += blockDim.x) s_exp[i] = make_double2(moc_exp64::kTable[i].hi, moc_exp64::kTable[i].lo);
    // the next unit is taken one unit ahead: thread 0 takes it from the
    // counter when the unit's tasks start (its wait for the atomic then only
    // delays its own warp's first task) and publishes it when the unit ends
    if (tid == 0) s_work = atomicAdd(st.counter, 1);

    for (;;) {
        __syncthreads();
        const int w = s_work;
        if (w >= n_work) break;
        const int T = BATCH ? order[w / n_items] : order[w];
        if constexpr (BATCH) {
            if (tid < (int)(sizeof(BatchItem) / 8))
                reinterpret_cast<uint64_t *>(&s_item)[tid] =
                    reinterpret_cast<const uint64_t *>(items + w % n_items)[tid];
            __syncthreads();
            if (s_item.scal[SC_CONV] != 0.0) {  // that solve has converged
                __syncthreads();  // every thread has read s_work and s_item
                if (tid == 0) s_work = atomicAdd(st.counter, 1);
                continue;
            }
        }
        // the unit's solve (one solve unless batched)
        const real *psi_in = BATCH ? reinterpret_cast<const real *>(s_item.psi_in) : psi_in_p;
        real *psi_out = BATCH ? reinterpret_cast<real *>(s_item.psi_out) : psi_out_p;
        double *scal_u = BATCH ? s_item.scal : st.scal;
        const real scale = (real)scal_u[SC_SCALE];
        const real *qr_g = reinterpret_cast<const real *>(BATCH ? s_item.qr : st.qr);
        double *tally_g = BATCH ? s_item.tally : st.tally;
        double *err = scal_u + SC_ERR;
        if (warp == 0) {
            // the unit's polar stacks, one lane each (Ph <= 16), stored field by
            // field; task offsets by a prefix sum over the warp
            int cnt = 0;
            float wl = 0.0f;
            if (lane < Ph) {
                const StackDesc &e = dl.desc[(int64_t)T * Ph + lane];
                UnitStack &u = s_us[lane];
                u.trk_off = e.trk_off;
                u.tpl_base = e.exp_base;
                u.cbase = e.chunk_base;
                u.slot_off = e.slot_off;
                u.n_slot = e.n_slot;
                u.W = e.W;
                u.invW = e.invW;
                u.Wf = (float)e.W;
                u.invWf = (float)e.invW;
                u.n_trk = e.n_trk;
                u.i_lo = e.i_lo;
                // FLAT: slots counted across the stacks; else blocks of SLOTS
                // slots per stack, 2 senses
                cnt = FLAT ? e.n_slot : 2 * ((e.n_slot + SLOTS - 1) / SLOTS);
                wl = (float)e.W;
            }
            int incl = cnt;
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            for (int o = 16; o > 0; o >>= 1) wl = fmaxf(wl, __shfl_xor_sync(0xffffffffu, wl, o));
            if (lane < Ph) s_us[lane].task_pre = incl - cnt;
            if (lane == Ph - 1) s_ntask = FLAT ? 2 * ((incl + SLOTS - 1) / SLOTS) : incl;
            if (lane == 0) s_wmax = wl;
            s_bmax[lane] = 0u;
        }
        __syncthreads();
        const int ntask = s_ntask;
        if (ntask == 0) {
            if (tid == 0) s_work = atomicAdd(st.counter, 1);
            continue;
        }
        const StackDesc &d0 = dl.desc[(int64_t)T * Ph];
        const int nb = d0.nb;
        const int32_t *reg2d = dl.reg2d + d0.seg2d_off;
        // A unit whose tile does not fit is swept in C radial chunks of
        // chunk_b 2D segments: first every track in sense 0, chunk by chunk
        // along the 2D track, then in sense 1 back again; a track's psi passes
        // from chunk to chunk through this block's hand-off buffer.
        const int C = (CHUNK && nb > dl.chunk_b) ? (nb + dl.chunk_b - 1) / dl.chunk_b : 1;
        real *hand = CHUNK ? reinterpret_cast<real *>(dl.hand) + (size_t)blockIdx.x * dl.hand_trk * 2 * G
                           : nullptr;
        const int64_t unit_trk0 = s_us[0].trk_off;
        for (int g0 = 0; g0 < G; g0 += GP)
        for (int pass = 0; pass < (C > 1 ? 2 : 1); ++pass)
        for (int ci = 0; ci < C; ++ci) {
            const int c_ch = pass ? C - 1 - ci : ci;             // radial chunk
            const int b0 = C > 1 ? c_ch * dl.chunk_b : 0;       // its 2D segments [b0, b1)
            const int b1 = C > 1 ? min(nb, b0 + dl.chunk_b) : nb;
            const int rowoff = b0 * NL;                          // tile row of (b0, layer 0)
            __syncthreads();  // the previous chunk's flush is done with the tile
            const int gc = min(GP, G - g0);
            float bmax = 0.0f;  // this thread's bound for group tid % GP of the chunk
            for (int e = tid; e < M * GP; e += blockDim.x) {
                const int m = e / GP, qq = e - m * GP;
                real v = qq < gc ? sig_g[m * G + g0 + qq] : (real)0;
                if (sizeof(real) == 4) v = (real)((float)v * kLog2e);
                sig[e] = v;
            }
            if (C > 1 && warp == 0) {
                // this chunk's warp tasks: per polar stack, blocks of SLOTS of the
                // tracks that cross the chunk (one sense per pass)
                int cnt = 0;
                if (lane < Ph) cnt = (int)(__ldg(dl.chunk_tab + s_us[lane].cbase + c_ch) >> 32);
                cnt = (cnt + SLOTS - 1) / SLOTS;
                int incl = cnt;
                for (int o = 1; o < 32; o <<= 1) {
                    const int v = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += v;
                }
                if (lane < Ph) s_us[lane].task_pre = incl - cnt;
                if (lane == 31) s_ntask = incl;
            }
            if (kFixed && SMEM && pass == 0 && ci == 0) {
                // the unit's incoming fluxes psi_in[(gid 4 + v) G + g], its tracks
                // gid one contiguous range of 4 G floats each: read as float4, a
                // thread taking every S-th float4 with 4 S a multiple of G, so
                // that its four elements always belong to the same four groups
                // (4 tid + k) mod G; s_ubnd is zero here (cleared after its
                // last use)
                if (psi_in) {
                    const int S = (blockDim.x / G) * G;
                    const int64_t trk_end = s_us[Ph - 1].trk_off + s_us[Ph - 1].n_trk;
                    const int64_t n4 = (trk_end - unit_trk0) * G;
                    const float4 *p4 = reinterpret_cast<const float4 *>(psi_in + unit_trk0 * 4 * G);
                    float m4[4] = {0.0f, 0.0f, 0.0f, 0.0f};
                    if (tid < S) {
#pragma unroll 4
                        for (int64_t i = tid; i < n4; i += S) {
                            const float4 v = __ldg(p4 + i);
                            m4[0] = fmaxf(m4[0], fabsf(v.x));
                            m4[1] = fmaxf(m4[1], fabsf(v.y));
                            m4[2] = fmaxf(m4[2], fabsf(v.z));
                            m4[3] = fmaxf(m4[3], fabsf(v.w));
                        }
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            const int gq = (4 * tid + k) % G - g0;
                            if (gq >= 0 && gq < gc && m4[k] > 0.0f) atomicMax(&s_ubnd[gq], __float_as_uint(m4[k]));
                        }
                    }
                }
            }
            __syncthreads();  // sig (below: Sigma_t from shared memory) and s_ubnd are complete
            if constexpr (SMEM && kFixed && !SYNC && GPL >= 2) {
                // rows of the (2D segment, layer) FSRs the unit (chunk) crosses:
                // one thread per (row, pair of groups), so that a row's FSR and
                // material are found once for two groups; the pair's Qr (and
                // Sigma_t log2 e) go out in one vector store and its two tally
                // words are cleared (the block size is a multiple of the pairs
                // per row, so a thread keeps its pair)
                constexpr int NP = GP / 2;
                const int nrow = (b1 - b0) * NL, q0 = 2 * (tid % NP);
                const float rNL = 1.0f / (float)NL;
                float bm0 = 0.0f, bm1 = 0.0f;
                for (int rr = tid / NP; rr < nrow; rr += (int)blockDim.x / NP) {
                    const int bb = div_by(rr, NL, rNL), L = rr - bb * NL;
                    const int64_t f = fsr_of(dl, __ldg(reg2d + b0 + bb), L);
                    const float *qs = reinterpret_cast<const float *>(qr_g) + (size_t)f * G + g0 + q0;
                    const float qa = q0 < gc ? qs[0] : 0.0f, qb = q0 + 1 < gc ? qs[1] : 0.0f;
                    const int e = rr * GP + q0;
                    if constexpr (MATK) {
                        *reinterpret_cast<float2 *>(reinterpret_cast<float *>(rows) + e) = make_float2(qa, qb);
                    } else {
                        const int mt = __ldg(dl.fsr_mat + f);
                        const float2 sg = *reinterpret_cast<const float2 *>(reinterpret_cast<const float *>(sig) + mt * GP + q0);
                        *reinterpret_cast<float4 *>(reinterpret_cast<float *>(rows) + 2 * e) =
                            make_float4(qa, qb, sg.x, sg.y);
                    }
                    tl_i[tix(rr, q0)] = 0;
                    tl_i[tix(rr, q0 + 1)] = 0;
                    bm0 = fmaxf(bm0, fabsf(qa));
                    bm1 = fmaxf(bm1, fabsf(qb));
                }
                if (bm0 > 0.0f) atomicMax(&s_bmax[q0], __float_as_uint(bm0));
                if (bm1 > 0.0f) atomicMax(&s_bmax[q0 + 1], __float_as_uint(bm1));
                if (tid < GP) {
                    // incoming fluxes and psi handed over from the previous chunk
                    // enter the bound too (see below)
                    float v = 0.0f;
                    if (psi_in && tid < gc) v = __uint_as_float(s_ubnd[tid]) * fabsf((float)scale);
                    if (C > 1 && ci > 0) v = fmaxf(v, __uint_as_float(s_hmax[tid]));
                    if (v > 0.0f) atomicMax(&s_bmax[tid], __float_as_uint(v));
                }
            } else if (SMEM) {
                // rows of the (2D segment, layer) FSRs the unit (chunk) crosses
                for (int bb = warp; bb < b1 - b0; bb += nwarps) {
                    const int b = b0 + bb;
                    const int reg = __ldg(reg2d + b);
                    for (int x = lane; x < NL * GP; x += 32) {
                        const int L = x / GP, qq = x - L * GP;
                        const int64_t f = fsr_of(dl, reg, L);
                        const int e = (bb * NL + L) * GP + qq;
                        const int et = tix(bb * NL + L, qq);
                        real q = (real)0, sg = (real)0;
                        if (qq < gc) {
                            sg = sig[__ldg(dl.fsr_mat + f) * GP + qq];  // FP32: times log2 e
                            q = qr_g[(size_t)f * G + g0 + qq];
                        }
                        if constexpr (SYNC) {
                            qr_t[e] = (float)q;
                            sg_t[e] = (float)sg;
                        } else if constexpr (GPL >= 2) {
                            const int pe = 2 * (e - (qq & 1));  // the pair's Qr_0 Qr_1 Sigma_0 Sigma_1
                            rows[pe + (qq & 1)] = q;
                            rows[pe + 2 + (qq & 1)] = sg;
                        } else {
                            rows[2 * e] = q;
                            rows[2 * e + 1] = sg;
                        }
                        tl_s[et] = (real)0;
                        if (kFixed) bmax = fmaxf(bmax, fabsf((float)q));
                    }
                    if constexpr (SYNC) {
                        // Sigma_t once per 2D segment where its region has one material
                        const int rm = __ldg(dl.reg_mat + reg);
                        for (int qq = lane; qq < GP; qq += 32)
                            sb_t[bb * GP + qq] = rm < 0 ? -1.0f : (qq < gc ? (float)sig[rm * GP + qq] : 0.0f);
                    }
                }
                if (kFixed) {
                    // incoming fluxes enter the bound too (psi along a track stays
                    // between its incoming value and Qr): the largest |psi_in| of
                    // the unit's own tracks, so that a unit far from the peak flux
                    // gets a fine grid
                    const int qq = tid % GP;
                    if (psi_in && qq < gc) bmax = fmaxf(bmax, __uint_as_float(s_ubnd[qq]) * fabsf((float)scale));
                    // and psi handed over from the previous chunk of this pass
                    if (C > 1 && ci > 0) bmax = fmaxf(bmax, __uint_as_float(s_hmax[qq]));
                    atomicMax(&s_bmax[qq], __float_as_uint(bmax));
                }
            }
            __syncthreads();
            if (tid == 0) s_next = 0;
            if (C > 1 && tid < 32) s_hmax[tid] = 0u;  // read above; refilled by this chunk's tasks
            const int ntask_c = C > 1 ? s_ntask : ntask;
            if (kFixed && SMEM && tid < GP) {
                // one unit of the fixed-point tally = 2^-bits of a bound of every
                // contribution: W |psi - Qr| <= W max(psi, Qr), since psi and Qr
                // are never negative (sources, fluxes and boundary fluxes
                // are non-negative and the library refuses negative inputs;
                // psi moves between its incoming value and Qr, Eq. 3).  The
                // bound is rounded up to a power of two 2^e, so that scaling by
                // the unit is exact and a flushed word is an exact shift.
                const float B = s_wmax * __uint_as_float(s_bmax[tid]);
                int e = 0;
                if (B > 0.0f) frexpf(B, &e);
                s_scl[tid] = B > 0.0f ? ldexpf(1.0f, dl.tally_bits - e) : 1.0f;
                s_inv[tid] = B > 0.0f ? ldexpf(1.0f, e - dl.tally_bits) : 1.0f;
                s_sh[tid] = B > 0.0f ? e - dl.tally_bits + 64 : 64;
            }
            __syncthreads();
            if (tid == 0 && g0 == 0 && pass == 0 && ci == 0) s_work_next = atomicAdd(st.counter, 1);

            float hmx[GPL];  // this lane's max |psi| handed to the next chunk
#pragma unroll
            for (int c = 0; c < GPL; ++c) hmx[c] = 0.0f;
            for (;;) {
                int t = 0;
                if (lane == 0) t = atomicAdd(&s_next, 1);
                t = __shfl_sync(0xffffffffu, t, 0);
                if (t >= ntask_c) break;
                // warp task: polar stack ph, sense, block of SLOTS tracks taken in
                // decreasing segment count
                // FLAT: slot gs of the unit's slots across its stacks (each slot
                // finds its own stack); else the stack of task t
                const int gs = FLAT ? (t >> 1) * SLOTS + j : t;
                int ph = 0;
                while (ph + 1 < Ph && gs >= s_us[ph + 1].task_pre) ++ph;
                const UnitStack u = s_us[ph];
                const int x = t - u.task_pre;
                int sense, q, k, widx;
                bool valid;
                if (C > 1) {
                    // tracks k0 .. k0 + count - 1 of the stack cross this chunk
                    // (index order), one sense per pass
                    const int64_t rng = __ldg(dl.chunk_tab + u.cbase + c_ch);
                    sense = pass;
                    q = x * SLOTS + j;
                    valid = q < (int)(rng >> 32);
                    k = valid ? (int)(rng & 0xffffffff) + q : 0;
                    widx = k;
                } else {
                    sense = FLAT ? (t & 1) : (x & 1);
                    q = FLAT ? gs - u.task_pre : (x >> 1) * SLOTS + j;
                    // the slot's track in the stack; a padding slot of a
                    // synchronous block holds -1 - (the track its block's
                    // sequence would continue with): idle, but with its m
                    const int kk = q < u.n_slot ? __ldg(dl.perm + u.slot_off + q) : 0;
                    valid = q < u.n_slot && kk >= 0;
                    k = kk >= 0 ? kk : -1 - kk;
                    widx = q;
                }
                const int m = div_by(k, cpl, rcpl);          // shift of the track within its class
                const int64_t gid = u.trk_off + k;
                // the track's part in this chunk: records [p0, p0 + n) of its
                // window (stored) or 2D segments [sb0, sb1] (on the fly), and
                // whether its first / last piece lies here (psi from psi_in /
                // to its successor) or it continues across a chunk boundary
                bool first_in = true, last_out = true;
                int64_t p0 = 0;
                int n = 0, sb0 = 0, sb1 = -1;
                if (CHUNK && C > 1 && u.tpl_base >= 0) {
                    const uint64_t wn = valid ? __ldg(dl.win + u.trk_off + widx) : 0ull;  // chunked: index order
                    p0 = (int64_t)(wn & 0xffffffffffffull);
                    n = (int)(wn >> 48);
                    if (valid) {
                        const int64_t *cb = dl.chunk_tab + u.cbase + C + (int64_t)(k - m * cpl) * (C + 1) + c_ch;
                        const int64_t lo = max(p0, __ldg(cb)), hi = min(p0 + n, __ldg(cb + 1));
                        first_in = sense == 0 ? lo == p0 : hi == p0 + n;
                        last_out = sense == 0 ? hi == p0 + n : lo == p0;
                        p0 = lo;
                        n = hi > lo ? (int)(hi - lo) : 0;
                    }
                } else if (CHUNK && C > 1 && valid) {
                    const StackDesc &dsk = dl.desc[(int64_t)T * Ph + ph];
                    const int i_trk = u.i_lo + k;
                    const int fb = first_seg(dl, dsk, i_trk), lb = last_seg(dl, dsk, i_trk);
                    sb0 = max(fb, b0);
                    sb1 = min(lb, b1 - 1);
                    first_in = sense == 0 ? fb >= b0 : lb < b1;
                    last_out = sense == 0 ? lb < b1 : fb >= b0;
                }
                const bool active = valid && (C == 1 || (u.tpl_base >= 0 ? n > 0 : sb0 <= sb1));
                const int64_t lt = gid - unit_trk0;  // hand-off slot of the track
                // psi is carried pre-multiplied by the track weight W, so that the
                // tally contribution W (psi_in - psi_out) is the psi change itself
                const real W = sizeof(real) == 4 ? (real)u.Wf : (real)u.W;
                const real invW = sizeof(real) == 4 ? (real)u.invWf : (real)u.invW;
                const int qlo = ql * GPL;                    // first group of this lane in the chunk
                float scl[GPL];
#pragma unroll
                for (int c = 0; c < GPL; ++c) scl[c] = kFixed && SMEM ? s_scl[ql * GPL + c] : 1.0f;
                // psi is carried as W S psi, S the group's fixed-point scale (1 when
                // the tally is not in fixed point), so that the change of the
                // carried value is the tally contribution in tally units
                real WS[GPL], iWS[GPL], iS[GPL];
#pragma unroll
                for (int c = 0; c < GPL; ++c) {
                    const real is = kFixed && SMEM ? (real)s_inv[ql * GPL + c] : (real)1;
                    WS[c] = W * (real)scl[c];
                    iWS[c] = invW * is;
                    iS[c] = is;
                }
                real psiU[GPL], psiD[GPL];
#pragma unroll
                for (int c = 0; c < GPL; ++c) {
                    psiU[c] = (real)0;
                    psiD[c] = (real)0;
                }
                int64_t dstU = -1, dstD = -1;
                if (active) {
                    if (!first_in) {
                        // psi left by the previous chunk of this pass
#pragma unroll
                        for (int c = 0; c < GPL; ++c) {
                            const int qq = ql * GPL + c;
                            if (qq < gc) {
                                psiU[c] = hand[(lt * 2 + 0) * G + g0 + qq] * WS[c];
                                psiD[c] = hand[(lt * 2 + 1) * G + g0 + qq] * WS[c];
                            }
                        }
                    } else if (psi_in) {
#pragma unroll
                        for (int c = 0; c < GPL; ++c) {
                            const int qq = ql * GPL + c;
                            if (qq < gc) {
                                psiU[c] = psi_in[(gid * 4 + 0 * 2 + sense) * G + g0 + qq] * (scale * WS[c]);
                                psiD[c] = psi_in[(gid * 4 + 1 * 2 + sense) * G + g0 + qq] * (scale * WS[c]);
                            }
                        }
                    }
                    if (last_out && dl.dst) {
                        dstU = dl.dst[gid * 4 + 0 * 2 + sense];
                        dstD = dl.dst[gid * 4 + 1 * 2 + sense];
                    }
                }
                // one segment of this slot's track, in tile rows rU (upward frame,
                // row b * NL + L) and rD (mirrored frame, row b * NL + NL-1-L)
                auto visit = [&](int rU, int rD, real len, int mat) {
                    real tU[GPL], tD[GPL];
                    if (SMEM) {
                        const int eU = rU * GP + qlo, eD = rD * GP + qlo;
                        const int tU_ = tix(rU, qlo), tD_ = tix(rD, qlo);
                        real qU[GPL], sU[GPL], qD[GPL], sD[GPL];
                        if constexpr (MATK) {
                            float2 a, sg;
                            lds_f2(rows_sa + (unsigned)eU * 4u, a);
                            qU[0] = a.x; qU[1] = a.y;
                            lds_f2(rows_sa + (unsigned)eD * 4u, a);
                            qD[0] = a.x; qD[1] = a.y;
                            lds_f2(sig_sa + (unsigned)(mat * GP + qlo) * 4u, sg);
                            sU[0] = sg.x; sU[1] = sg.y; sD[0] = sg.x; sD[1] = sg.y;
                        } else if constexpr (SYNC) {
                            float2 a, b;
                            lds_f2(qr_sa + eU * 4u, a);
                            lds_f2(sg_sa + eU * 4u, b);
                            qU[0] = a.x; qU[1] = a.y; sU[0] = b.x; sU[1] = b.y;
                            lds_f2(qr_sa + eD * 4u, a);
                            lds_f2(sg_sa + eD * 4u, b);
                            qD[0] = a.x; qD[1] = a.y; sD[0] = b.x; sD[1] = b.y;
                        } else {
                            RowLoadS<real, GPL>::get(rows_sa + eU * (unsigned)(2 * sizeof(real)), qU, sU);
                            RowLoadS<real, GPL>::get(rows_sa + eD * (unsigned)(2 * sizeof(real)), qD, sD);
                        }
#pragma unroll
                        for (int c = 0; c < GPL; ++c) {
                            // Eq. 3 on W S psi: d = W S (psi_in - Qr),
                            // W S (psi_in - psi_out) = d (1 - e^{-Sigma_t l})
                            const real xU = attenuation<real>(sU[c] * len, s_exp);
                            const real xD = attenuation<real>(sD[c] * len, s_exp);
                            const real dU = fma(-WS[c], qU[c], psiU[c]), dD = fma(-WS[c], qD[c], psiD[c]);
                            tU[c] = fma(-dU, xU, dU);
                            tD[c] = fma(-dD, xD, dD);
                            psiU[c] -= tU[c];
                            psiD[c] -= tD[c];
                        }
                        if constexpr (kFixed) {
                            // round to the fixed-point grid (|t scl| <= 2^bits <= 2^24)
#pragma unroll
                            for (int c = 0; c < GPL; ++c) {
                                shared_red_add(tl_sa + (tU_ + c * CS) * 4u,
                                               __float2int_rn((float)tU[c]));
                                shared_red_add(tl_sa + (tD_ + c * CS) * 4u,
                                               __float2int_rn((float)tD[c]));
                            }
                        } else {
                            TallyAdd<real, GPL>::add(tl_s + tU_, tU, err);
                            TallyAdd<real, GPL>::add(tl_s + tD_, tD, err);
                        }
                    } else {
                        const int b = rU / NL, L = rU - b * NL, LD = NL - 1 - L;
                        const int reg = __ldg(reg2d + b);
                        const size_t fU = (size_t)fsr_of(dl, reg, L), fD = (size_t)fsr_of(dl, reg, LD);
                        const int mU = __ldg(dl.fsr_mat + fU), mD = __ldg(dl.fsr_mat + fD);
#pragma unroll
                        for (int c = 0; c < GPL; ++c) {
                            const int qq = qlo + c;
                            const real qU = qq < gc ? qr_g[fU * G + g0 + qq] : (real)0;
                            const real qD = qq < gc ? qr_g[fD * G + g0 + qq] : (real)0;
                            const real xU = attenuation<real>(sig[mU * GP + qq] * len, s_exp);
                            const real xD = attenuation<real>(sig[mD * GP + qq] * len, s_exp);
                            const real dU = fma(-WS[c], qU, psiU[c]), dD = fma(-WS[c], qD, psiD[c]);
                            tU[c] = fma(-dU, xU, dU);
                            tD[c] = fma(-dD, xD, dD);
                            if (qq < gc) {
                                atomicAdd(tally_g + fU * G + g0 + qq, (double)tU[c]);
                                atomicAdd(tally_g + fD * G + g0 + qq, (double)tD[c]);
                            }
                            psiU[c] -= tU[c];
                            psiD[c] -= tD[c];
                        }
                    }
                };
                // the packed-pair body of four consecutive pieces (two groups per
                // lane, FP32 fixed-point tally): per frame and piece one mul
                // (-Sigma l), two ex2, then d = psi - W S Qr, t = d (1 - e^{-tau})
                // (1 - x is exact in FP32 for x >= 1/2), psi -= t in three paired
                // operations; aTU / aTD: byte addresses of the group-0 tally words
                // (group 1 lies cs4 bytes further)
                const unsigned cs4 = (unsigned)CS * 4u;
                auto packed_core = [&](float2 (&QU)[4], float2 (&SU)[4], float2 (&QD)[4], float2 (&SD)[4],
                                       const real (&len)[4], const unsigned (&aTU)[4],
                                       const unsigned (&aTD)[4]) {
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const float nl = -(float)len[i];
                        const float2 xu = __fmul2_rn(SU[i], make_float2(nl, nl));
                        const float2 xd = __fmul2_rn(SD[i], make_float2(nl, nl));
                        SU[i] = make_float2(fast_exp2(xu.x), fast_exp2(xu.y));  // now e^{-Sigma_t l}
                        SD[i] = make_float2(fast_exp2(xd.x), fast_exp2(xd.y));
                    }
                    const float2 nws = make_float2(-(float)WS[0], -(float)WS[1]);
                    float2 PU = make_float2((float)psiU[0], (float)psiU[1]);
                    float2 PD = make_float2((float)psiD[0], (float)psiD[1]);
                    int vU[4][2], vD[4][2];
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        // d = W S (psi - Qr); t = d (1 - e) as d - d e with one
                        // rounding; psi -= t
                        const float2 dU = __ffma2_rn(nws, QU[i], PU);
                        const float2 dD = __ffma2_rn(nws, QD[i], PD);
                        const float2 tU = __ffma2_rn(make_float2(-dU.x, -dU.y), SU[i], dU);
                        const float2 tD = __ffma2_rn(make_float2(-dD.x, -dD.y), SD[i], dD);
                        PU = __fadd2_rn(PU, make_float2(-tU.x, -tU.y));
                        PD = __fadd2_rn(PD, make_float2(-tD.x, -tD.y));
                        vU[i][0] = __float2int_rn(tU.x);
                        vU[i][1] = __float2int_rn(tU.y);
                        vD[i][0] = __float2int_rn(tD.x);
                        vD[i][1] = __float2int_rn(tD.y);
                    }
                    psiU[0] = (real)PU.x;
                    psiU[1] = (real)PU.y;
                    psiD[0] = (real)PD.x;
                    psiD[1] = (real)PD.y;
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        shared_red_add(aTU[i], vU[i][0]);
                        shared_red_add(aTU[i] + cs4, vU[i][1]);
                        shared_red_add(aTD[i], vD[i][0]);
                        shared_red_add(aTD[i] + cs4, vD[i][1]);
                    }
                };
                // four consecutive segments of the track at once (shared tally):
                // all row loads and exponentials first, then the psi recurrence,
                // then the tally updates, so that the loads overlap each other
                auto visit4 = [&](const int (&rU)[4], const int (&rD)[4], const real (&len)[4],
                                  const int (&bs)[4]) {
                    if constexpr (!SMEM) {
#pragma unroll
                        for (int i = 0; i < 4; ++i) visit(rU[i], rD[i], len[i], 0);
                    } else {
                        int eU[4], eD[4], fU[4], fD[4];
                        if constexpr (kFixed && GPL == 2) {
                            // both groups of the lane as packed pairs: per frame and
                            // piece one mul (-Sigma l), two ex2, then
                            // d = psi - W S Qr, t = d (1 - e^{-tau}) (1 - x is exact in
                            // FP32 for x >= 1/2), psi -= t in three paired operations
                            float2 QU[4], SU[4], QD[4], SD[4];
                            unsigned aTU[4], aTD[4];
#pragma unroll
                            for (int i = 0; i < 4; ++i) {
                                eU[i] = rU[i] * GP + qlo;
                                eD[i] = rD[i] * GP + qlo;
                                fU[i] = tix(rU[i], qlo);
                                fD[i] = tix(rD[i], qlo);
                                if constexpr (SYNC) {
                                    // Qr of both frames; Sigma_t of the 2D segment when its
                                    // region has one material (both frames), else per row
                                    lds_f2(qr_sa + eU[i] * 4u, QU[i]);
                                    lds_f2(qr_sa + eD[i] * 4u, QD[i]);
                                    float2 sb;
                                    lds_f2(sb_sa + (unsigned)(bs[i] * GP + qlo) * 4u, sb);
                                    if (sb.x < 0.0f) {
                                        lds_f2(sg_sa + eU[i] * 4u, SU[i]);
                                        lds_f2(sg_sa + eD[i] * 4u, SD[i]);
                                    } else {
                                        SU[i] = sb;
                                        SD[i] = sb;
                                    }
                                } else if constexpr (MATK) {
                                    // Qr of both frames; Sigma_t of the piece's material
                                    // (bs: the material from the record's key)
                                    lds_f2(rows_sa + (unsigned)eU[i] * 4u, QU[i]);
                                    lds_f2(rows_sa + (unsigned)eD[i] * 4u, QD[i]);
                                    lds_f2(sig_sa + (unsigned)(bs[i] * GP + qlo) * 4u, SU[i]);
                                    SD[i] = SU[i];
                                } else {
                                    row_load_f2(rows_sa + eU[i] * 8u, QU[i], SU[i]);
                                    row_load_f2(rows_sa + eD[i] * 8u, QD[i], SD[i]);
                                }
                            }
#pragma unroll
                            for (int i = 0; i < 4; ++i) {
                                aTU[i] = tl_sa + (unsigned)fU[i] * 4u;
                                aTD[i] = tl_sa + (unsigned)fD[i] * 4u;
                            }
                            packed_core(QU, SU, QD, SD, len, aTU, aTD);
                        } else {
                            real qU[4][GPL], sU[4][GPL], qD[4][GPL], sD[4][GPL];
#pragma unroll
                            for (int i = 0; i < 4; ++i) {
                                eU[i] = rU[i] * GP + qlo;
                                eD[i] = rD[i] * GP + qlo;
                                fU[i] = tix(rU[i], qlo);
                                fD[i] = tix(rD[i], qlo);
                                RowLoadS<real, GPL>::get(rows_sa + eU[i] * (unsigned)(2 * sizeof(real)), qU[i], sU[i]);
                                RowLoadS<real, GPL>::get(rows_sa + eD[i] * (unsigned)(2 * sizeof(real)), qD[i], sD[i]);
                            }
                            real tU[4][GPL], tD[4][GPL];
#pragma unroll
                            for (int i = 0; i < 4; ++i)
#pragma unroll
                                for (int c = 0; c < GPL; ++c) {
                                    sU[i][c] = attenuation<real>(sU[i][c] * len[i], s_exp);  // now e^{-Sigma_t l}
                                    sD[i][c] = attenuation<real>(sD[i][c] * len[i], s_exp);
                                }
#pragma unroll
                            for (int i = 0; i < 4; ++i)
#pragma unroll
                                for (int c = 0; c < GPL; ++c) {
                                    const real dU = fma(-WS[c], qU[i][c], psiU[c]), dD = fma(-WS[c], qD[i][c], psiD[c]);
                                    tU[i][c] = fma(-dU, sU[i][c], dU);
                                    tD[i][c] = fma(-dD, sD[i][c], dD);
                                    psiU[c] -= tU[i][c];
                                    psiD[c] -= tD[i][c];
                                }
#pragma unroll
                            for (int i = 0; i < 4; ++i) {
                                if constexpr (kFixed) {
#pragma unroll
                                    for (int c = 0; c < GPL; ++c) {
                                        shared_red_add(tl_sa + (fU[i] + c * CS) * 4u,
                                                       __float2int_rn((float)tU[i][c]));
                                        shared_red_add(tl_sa + (fD[i] + c * CS) * 4u,
                                                       __float2int_rn((float)tD[i][c]));
                                    }
                                } else {
                                    TallyAdd<real, GPL>::add(tl_s + fU[i], tU[i], err);
                                    TallyAdd<real, GPL>::add(tl_s + fD[i], tD[i], err);
                                }
                            }
                        }
                    }
                };
                if (SYNC && u.tpl_base >= 0) {
                    // synchronous block of B slots (lanes [h B GL, (h + 1) B GL)): the
                    // union [lo, hi) of its tracks' record windows, stepped together
                    const int B = dl.sync_b;
                    const uint64_t wn = valid ? __ldg(dl.win + u.slot_off + widx) : 0ull;
                    p0 = (int64_t)(wn & 0xffffffffffffull);
                    n = (int)(wn >> 48);
                    long long lo = n > 0 ? (long long)p0 : LLONG_MAX, hi = n > 0 ? (long long)(p0 + n) : LLONG_MIN;
                    for (int o = GL; o < B * GL; o <<= 1) {
                        const long long l2 = __shfl_xor_sync(0xffffffffu, lo, o);
                        const long long h2 = __shfl_xor_sync(0xffffffffu, hi, o);
                        lo = l2 < lo ? l2 : lo;
                        hi = h2 > hi ? h2 : hi;
                    }
                    const int steps = hi > lo ? (int)(hi - lo) : 0;
                    const int nmax = __reduce_max_sync(0xffffffffu, steps);
                    // this slot's own steps [sa, se) in sweep order
                    int sa = 0, se = 0;
                    if (n > 0) {
                        const int a = (int)(p0 - lo), e = a + n;
                        sa = sense == 0 ? a : steps - e;
                        se = sense == 0 ? e : steps - a;
                    }
                    const int dir = sense == 0 ? 1 : -1;
                    const SegRec<real> *pr = recs + (steps > 0 ? (sense == 0 ? lo : hi - 1) : 0);
                    // every slot of the block reads the same record; past its own
                    // window a slot takes length 0.  Its rows then lie within 7 of
                    // an active slot's (|m - m'| < B <= 8, the record in that
                    // slot's window), inside the guard rows.  A block with no
                    // track reads tile rows 0 and NL - 1.
                    auto fetch4s = [&](SegRec<real> (&c)[4], int s0) {
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const int s1 = s0 + i;
                            if (steps > 0) {
                                c[i] = pr[min(s1, steps - 1) * dir];
                                if ((unsigned)(s1 - sa) >= (unsigned)(se - sa)) c[i].len = (real)0;
                            } else {
                                c[i].key = tpl_key_seg(0, -m);
                                c[i].len = (real)0;
                            }
                        }
                    };
                    auto sweep4s = [&](const SegRec<real> (&c)[4]) {
                        int ru[4], rd[4], bs[4];
                        real ln[4];
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            bs[i] = tpl_seg(c[i].key);
                            const int bN = bs[i] * NL, Lt = tpl_layer(c[i].key);
                            ru[i] = bN + Lt + m;
                            rd[i] = bN + (NL - 1 - m) - Lt;
                            ln[i] = c[i].len;
                        }
                        visit4(ru, rd, ln, bs);
                    };
                    SegRec<real> ra[4], rb[4];
                    fetch4s(ra, 0);
                    for (int s1 = 0; s1 < nmax; s1 += 8) {
                        fetch4s(rb, s1 + 4);
                        sweep4s(ra);
                        if (s1 + 4 >= nmax) break;
                        fetch4s(ra, s1 + 8);
                        sweep4s(rb);
                    }
                } else if (u.tpl_base >= 0) {
                    if (!(CHUNK && C > 1)) {
                        // stored template of class r (line i_lo + r): this track is
                        // its pieces with template layer in [-m, NL - m), a contiguous
                        // record range because the layer never decreases along an
                        // upward line (per track in sweep order: count << 48 | first)
                        const uint64_t wn = valid ? __ldg(dl.win + u.slot_off + widx) : 0ull;
                        p0 = (int64_t)(wn & 0xffffffffffffull);
                        n = (int)(wn >> 48);
                    }
                    const int64_t p1 = p0 + n;
                    const int dir = sense == 0 ? 1 : -1;
                    const SegRec<real> *pr = recs + (sense == 0 ? p0 : p1 - 1);
                    // all slots step together to the longest track of the warp; a
                    // slot past its own end repeats its last record with length 0,
                    // which leaves psi unchanged and adds exactly 0 to the tally
                    const int nmax = __reduce_max_sync(0xffffffffu, n);
                    auto fetch4 = [&](SegRec<real> (&c)[4], int s0) {
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            if (n > 0) {
                                c[i] = pr[min(s0 + i, n - 1) * dir];
                                if (s0 + i >= n) c[i].len = (real)0;
                            } else {
                                // tile rows 0 and NL - 1 (0 and 0 for whole units)
                                c[i].key = CHUNK ? tpl_key_seg(b0, -m) : tpl_key(-m, m);
                                c[i].len = (real)0;
                            }
                        }
                    };
                    auto sweep4 = [&](const SegRec<real> (&c)[4]) {
                        int ru[4], rd[4];
                        real ln[4];
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            if constexpr (CHUNK) {
                                const int bN = (MATK ? tpl_seg_mat(c[i].key) : tpl_seg(c[i].key)) * NL,
                                          Lt = tpl_layer(c[i].key);
                                ru[i] = bN + Lt + (m - rowoff);
                                rd[i] = bN - Lt + (NL - 1 - m - rowoff);
                            } else {
                                ru[i] = tpl_row_up(c[i].key) + m;
                                rd[i] = (MATK ? tpl_row_down_mat(c[i].key) : tpl_row_down(c[i].key)) - m;
                            }
                            ln[i] = c[i].len;
                        }
                        if constexpr (GPL >= 4) {
                            // eight recurrences per segment already: no batching
#pragma unroll
                            for (int i = 0; i < 4; ++i) visit(ru[i], rd[i], ln[i], 0);
                        } else {
                            int bs[4];
#pragma unroll
                            for (int i = 0; i < 4; ++i) bs[i] = MATK ? tpl_mat(c[i].key) : 0;
                            visit4(ru, rd, ln, bs);
                        }
                    };
                    // two sets of four records: one set in flight while the other
                    // is swept; in units swept whole the last nmax mod 4 steps go
                    // one record at a time (the same arithmetic, so the same
                    // bits), so that a warp does not sweep up to three steps of
                    // zero-length pieces (radially chunked units keep the
                    // rounded steps: the extra code costs their kernel spills)
                    const int nq = CHUNK ? nmax : (nmax & ~3);
                    SegRec<real> ra[4], rb[4];
                    fetch4(ra, 0);
                    for (int s = 0; s < nq; s += 8) {
                        fetch4(rb, s + 4);
                        sweep4(ra);
                        if (s + 4 >= nq) break;
                        fetch4(ra, s + 8);
                        sweep4(rb);
                    }
                    if constexpr (!CHUNK)
                    for (int s = nq; s < nmax; ++s) {
                        int ru, rd;
                        real ln = (real)0;
                        uint32_t key;
                        if (n > 0) {
                            const SegRec<real> c = pr[min(s, n - 1) * dir];
                            key = c.key;
                            if (s < n) ln = c.len;
                        } else {
                            key = CHUNK ? tpl_key_seg(b0, -m) : tpl_key(-m, m);
                        }
                        if constexpr (CHUNK) {
                            const int bN = (MATK ? tpl_seg_mat(key) : tpl_seg(key)) * NL, Lt = tpl_layer(key);
                            ru = bN + Lt + (m - rowoff);
                            rd = bN - Lt + (NL - 1 - m - rowoff);
                        } else {
                            ru = tpl_row_up(key) + m;
                            rd = (MATK ? tpl_row_down_mat(key) : tpl_row_down(key)) - m;
                        }
                        visit(ru, rd, ln, MATK ? tpl_mat(key) : 0);
                    }
                } else if constexpr (MATK) {
                    // (no unit of a material-keyed layout is generated on the fly:
                    // the mode needs every unit stored)
                } else if (active) {
                    // generated on the fly: this track's own line, layers [0, NL),
                    // 2D segments [sb0, sb1]
                    const StackDesc &dsk = dl.desc[(int64_t)T * Ph + ph];
                    const int i_trk = u.i_lo + k;
                    TplIter<real> it;
                    if (CHUNK && C > 1) it.init(dl, dsk, i_trk, sb0, sb1, sense == 0 ? 1 : -1);
                    else it.init(dl, dsk, i_trk, first_seg(dl, dsk, i_trk), last_seg(dl, dsk, i_trk),
                                 sense == 0 ? 1 : -1);
                    while (!it.done) {
                        int b, L;
                        real len;
                        it.next(dl, b, L, len);
                        visit((b - b0) * NL + L, (b - b0) * NL + NL - 1 - L, len, 0);
                    }
                }
                if (active && !last_out) {
                    // the track goes on in the next chunk of this pass
#pragma unroll
                    for (int c = 0; c < GPL; ++c) {
                        const int qq = ql * GPL + c;
                        if (qq >= gc) continue;
                        const real vU = psiU[c] * iWS[c], vD = psiD[c] * iWS[c];
                        hand[(lt * 2 + 0) * G + g0 + qq] = vU;
                        hand[(lt * 2 + 1) * G + g0 + qq] = vD;
                        hmx[c] = fmaxf(hmx[c], fmaxf(fabsf((float)vU), fabsf((float)vD)));
                    }
                } else if (active) {
#pragma unroll
                    for (int c = 0; c < GPL; ++c) {
                        const int qq = ql * GPL + c;
                        if (qq >= gc) continue;
                        if (dstU >= 0 && dstU < dl.n_slots) psi_out[dstU * G + g0 + qq] = psiU[c] * iWS[c];
                        else leak += psiU[c] * iS[c];
                        if (dstD >= 0 && dstD < dl.n_slots) psi_out[dstD * G + g0 + qq] = psiD[c] * iWS[c];
                        else leak += psiD[c] * iS[c];
                    }
                }
            }
            if (kFixed && C > 1) {
                // the next chunk's bound covers the psi handed over to it
#pragma unroll
                for (int c = 0; c < GPL; ++c) {
                    float v = hmx[c];
                    for (int o = GL; o < 32; o <<= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
                    if (j == 0 && ql * GPL + c < gc && v > 0.0f) atomicMax(&s_hmax[ql * GPL + c], __float_as_uint(v));
                }
            }
            __syncthreads();
            if constexpr (SMEM && kFixed && GPL >= 2) {
                // one thread per (row, pair of groups), as in the staging
                constexpr int NP = GP / 2;
                const int nrow = (b1 - b0) * NL, q0 = 2 * (tid % NP);
                const int sh0 = s_sh[q0], sh1 = s_sh[q0 + 1];
                const float rNL = 1.0f / (float)NL;
                for (int rr = tid / NP; rr < nrow; rr += (int)blockDim.x / NP) {
                    const int bb = div_by(rr, NL, rNL), L = rr - bb * NL;
                    const size_t gi = (size_t)fsr_of(dl, __ldg(reg2d + b0 + bb), L) * G + g0 + q0;
                    const int iv0 = tl_i[tix(rr, q0)], iv1 = tl_i[tix(rr, q0 + 1)];
                    // into the three-word fixed-point tally: exact, so the order of
                    // the units does not matter
                    long long *t3 = reinterpret_cast<long long *>(tally_g) + 3 * gi;
                    if (iv0 != 0 && q0 < gc && !tally3_add(t3, iv0, sh0)) *err = 2.0;
                    if (iv1 != 0 && q0 + 1 < gc && !tally3_add(t3 + 3, iv1, sh1)) *err = 2.0;
                }
            }
            if (SMEM) {
                if (!(kFixed && GPL >= 2))
                for (int bb = warp; bb < b1 - b0; bb += nwarps) {
                    const int reg = __ldg(reg2d + b0 + bb);
                    for (int x = lane; x < NL * GP; x += 32) {
                        const int L = x / GP, qq = x - L * GP;
                        if (qq >= gc) continue;
                        const int e = tix(bb * NL + L, qq);
                        const size_t gi = (size_t)fsr_of(dl, reg, L) * G + g0 + qq;
                        if constexpr (kFixed) {
                            // into the three-word fixed-point tally: exact, so the
                            // order of the units does not matter
                            const int iv = tl_i[e];
                            if (iv != 0 && !tally3_add(reinterpret_cast<long long *>(tally_g) + 3 * gi, iv, s_sh[qq]))
                                *err = 2.0;
                        } else {
                            const double v = (double)tl_s[e];
                            if (v != 0.0) atomicAdd(tally_g + gi, v);
                        }
                    }
                }
                if (tid < 32) s_bmax[tid] = 0u;  // next chunk's bound (read only before its tasks)
                // the unit's incoming-flux bound, read by every chunk's staging:
                // cleared once the unit's last chunk is done
                if (kFixed && tid < 32 && pass == (C > 1 ? 1 : 0) && ci == C - 1) s_ubnd[tid] = 0u;
            }
        }
        if constexpr (BATCH) {
            // the next unit may belong to another solve: publish this one's
            // leakage now
            double lk = (double)leak;
            for (int o = 16; o > 0; o >>= 1) lk += __shfl_down_sync(0xffffffffu, lk, o);
            if (lane == 0) s_leak[warp] = lk;
            leak = (real)0;
            __syncthreads();
            if (tid == 0) {
                double v = 0.0;
                for (int k = 0; k < nwarps; ++k) v += s_leak[k];
                if (v != 0.0) atomicAdd(scal_u + SC_LEAK, v);
            }
        }
        if (tid == 0) s_work = s_work_next;  // read after the next loop-top barrier
    }
    if (BATCH) return;
    double leak64 = (double)leak;
    for (int o = 16; o > 0; o >>= 1) leak64 += __shfl_down_sync(0xffffffffu, leak64, o);
    if (lane == 0) s_leak[warp] = leak64;
    __syncthreads();
    if (tid == 0) {
        double v = 0.0;
        for (int k = 0; k < nwarps; ++k) v += s_leak[k];
        if (v != 0.0) atomicAdd(st.scal + SC_LEAK, v);
    }
}

// the kernel for gl lanes per track; only shapes with gl * GPL <= 32 exist
// (each translation unit of the sweep instantiates its share)
template <typename real, int GPL, bool SMEM, bool CHUNK, bool BATCH, int GL = 32 / GPL, bool SYNC = false,
          bool MATK = false>
const void *pick(int gl) {
    if constexpr (GL > 1) {
        if (gl < GL) return pick<real, GPL, SMEM, CHUNK, BATCH, GL / 2, SYNC, MATK>(gl);
    }
    return (const void *)k_sweep<real, GL, GPL, SMEM, CHUNK, BATCH, SYNC, MATK>;
}

template <typename real, int GPL>
const void *pick_tally(int tally_smem, int chunk, int gl) {
    if (!tally_smem) return pick<real, GPL, false, false>(gl);
    return chunk ? pick<real, GPL, true, true>(gl) : pick<real, GPL, true, false>(gl);
}

// chunk: some units are swept in radial chunks (shared tally only)

}  // namespace
