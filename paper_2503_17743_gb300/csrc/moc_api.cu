// C ABI of the GB300 3D MOC library (include/moc.h): device memory, the
// track generation pipeline and the outer iteration.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <memory>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "moc_kernels.h"
#include "moc_serve.h"

namespace {

struct DevBuf {
    void *p = nullptr;
    size_t n = 0;
    bool borrowed = false;  // another handle's buffer (a solve state sharing a layout)
    ~DevBuf() { release(); }
    void release() {
        if (p && !borrowed) cudaFree(p);
        p = nullptr;
        n = 0;
        borrowed = false;
    }
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
};

}  // namespace

struct moc_tracks {
    moc_geometry geom;
    Layout L;
    int precision = MOC_FP32;
    int device = 0;
    cudaStream_t stream = nullptr;
    int sms = 0;
    // device buffers
    DevBuf d_desc, d_zn, d_zf, d_zf64, d_reg2d, d_len2d, d_len2d64, d_segs, d_fsr_mat, d_order;
    DevBuf d_tpl_off, d_tpl_loff, d_tpl_lmin, d_tpl_lidx;
    DevBuf d_dst, d_perm, d_win, d_chunk, d_hand, d_batch, d_lmap, d_reg_mat;
    DevBuf d_zc0, d_zc1, d_zfd, d_zfd64, d_pl_n, d_pl_c, d_pl_f, d_pl_f64;  // planes off the lattice
    DevBuf d_phi, d_qr, d_tally, d_vol, d_psi[2], d_fiss, d_fiss_old, d_partial, d_scal, d_counter;
    DevBuf d_sigt, d_sigt64, d_sigs64, d_nsf64, d_chi64, d_src64, d_inv_st64, d_siga64, d_inv_vol;
    double *h_scal = nullptr;  // pinned mirror of the device scalars
    int cur = 0;               // psi buffer holding the next incoming fluxes
    bool has_psi = false;
    // layout numbers
    std::vector<int64_t> stack_nseg;
    std::vector<int32_t> order;
    int64_t n_segments3d = 0;   // both frames
    int64_t n_stored = 0;
    int64_t n_exp_stacks = 0;
    int32_t max_nseg = 0;
    int nb_max = 0;
    double integrations = 0;    // per sweep
    size_t bytes = 0;
    size_t h2d = 0;             // bytes copied from host arrays while generating
    // sweep launch
    int tally_smem = 0;
    int gpl = 1;                // energy groups per lane
    int tally_bits = 0;         // fixed-point bits of the FP32 shared tally
    int tile_cap = 0;
    int chunk_b = 0;            // 2D segments per radial chunk (0: units swept whole)
    int sync_b = 0;             // tracks per synchronous block of the stored stacks (0: none)
    int matk = 0;               // stored records carry materials, rows hold Qr only (DevLayout::matk)
    int64_t n_slots = 0;        // sweep slots of all stacks (perm / win entries)
    int64_t hand_trk = 0;       // tracks of the largest chunked unit
    int block = 256;
    int grid = 0;
    size_t smem = 0;
    int red_grid = 0;
    // host copies
    std::vector<double> vol;
    // graphs, one per psi parity
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    DevLayout dl{};
    DevState ds{};
    // solve states sharing this handle's layout (moc_state_create): a state
    // points at its owner; an owner destroyed while states live is freed with
    // the last of them
    moc_tracks *owner = nullptr;
    int live_states = 0;
    bool destroy_pending = false;
    ~moc_tracks() {
        for (auto &g : graph) if (g) cudaGraphExecDestroy(g);
        if (h_scal) cudaFreeHost(h_scal);
        if (stream) cudaStreamDestroy(stream);
    }
};

namespace {

// sources, fluxes and boundary fluxes given by a caller must be finite and
// non-negative (the FP32 sweep's fixed-point tally bound relies on it)
bool all_nonneg(const double *v, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (!(v[i] >= 0.0) || !std::isfinite(v[i])) return false;
    return true;
}

int cuda_fail(cudaError_t e, const char *what) {
    moc_set_error(std::string(what) + ": " + cudaGetErrorString(e));
    if (e == cudaErrorMemoryAllocation) return MOC_ERR_OUT_OF_MEMORY;
    return MOC_ERR_CUDA;
}

#define TRY(x, what)                                      \
    do {                                                  \
        cudaError_t e_ = (x);                             \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

cudaError_t dalloc(moc_tracks *h, DevBuf &b, size_t bytes) {
    b.n = bytes;
    if (bytes == 0) return cudaSuccess;
    cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e == cudaSuccess) h->bytes += bytes;
    return e;
}

template <typename T>
cudaError_t upload(moc_tracks *h, DevBuf &b, const std::vector<T> &v) {
    cudaError_t e = dalloc(h, b, v.size() * sizeof(T));
    if (e != cudaSuccess || v.empty()) return e;
    h->h2d += v.size() * sizeof(T);
    return cudaMemcpyAsync(b.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, h->stream);
}

size_t real_size(int precision) { return precision == MOC_FP64 ? 8 : 4; }

void fill_views(moc_tracks *h) {
    DevLayout &dl = h->dl;
    dl.desc = (const StackDesc *)h->d_desc.p;
    dl.zn = (const int32_t *)h->d_zn.p;
    dl.zf = (const float *)h->d_zf.p;
    dl.zf64 = (const double *)h->d_zf64.p;
    dl.reg2d = (const int32_t *)h->d_reg2d.p;
    dl.len2d = (const float *)h->d_len2d.p;
    dl.len2d64 = (const double *)h->d_len2d64.p;
    dl.tpl_off = (const int64_t *)h->d_tpl_off.p;
    dl.tpl_loff = (const int64_t *)h->d_tpl_loff.p;
    dl.tpl_lmin = (const int32_t *)h->d_tpl_lmin.p;
    dl.tpl_lidx = (const int32_t *)h->d_tpl_lidx.p;
    dl.segs = h->d_segs.p;
    dl.fsr_mat = (const int32_t *)h->d_fsr_mat.p;
    dl.dst = (const int32_t *)h->d_dst.p;
    dl.perm = (const int32_t *)h->d_perm.p;
    dl.win = (const uint64_t *)h->d_win.p;
    dl.Ph = h->L.Ph;
    dl.Nz = h->L.Nz;
    dl.cpl = h->L.cpl;
    dl.NL = h->L.nlv;
    dl.NLr = h->geom.nl;
    dl.lmap = (const int32_t *)h->d_lmap.p;
    dl.G = h->geom.G;
    dl.M = h->geom.M;
    dl.bc_zmin = h->geom.bc[FACE_ZMIN];
    dl.bc_zmax = h->geom.bc[FACE_ZMAX];
    dl.n_slots = h->L.n_gtrk * 4;
    dl.tally_bits = h->tally_bits;
    dl.tally3 = (h->precision == MOC_FP32 && h->tally_smem) ? 1 : 0;
    dl.chunk_tab = (const int64_t *)h->d_chunk.p;
    dl.chunk_b = h->chunk_b;
    dl.sync_b = h->sync_b;
    dl.matk = h->matk;
    dl.rcpl = dl.cpl > 0 ? 1.0f / (float)dl.cpl : 0.0f;
    dl.reg_mat = (const int32_t *)h->d_reg_mat.p;
    dl.hand_trk = (int32_t)h->hand_trk;
    dl.hand = h->d_hand.p;
    dl.offlat = h->L.offlat;
    dl.zc0 = (const int16_t *)h->d_zc0.p;
    dl.zc1 = (const int16_t *)h->d_zc1.p;
    dl.zfd = (const float *)h->d_zfd.p;
    dl.zfd64 = (const double *)h->d_zfd64.p;
    dl.pl_n = (const int32_t *)h->d_pl_n.p;
    dl.pl_c = (const int32_t *)h->d_pl_c.p;
    dl.pl_f = (const float *)h->d_pl_f.p;
    dl.pl_f64 = (const double *)h->d_pl_f64.p;
    DevState &s = h->ds;
    s.phi = (double *)h->d_phi.p;
    s.qr = h->d_qr.p;
    s.tally = (double *)h->d_tally.p;
    s.vol = (double *)h->d_vol.p;
    s.psi_a = h->d_psi[0].p;
    s.psi_b = h->d_psi[1].p;
    s.fiss = (double *)h->d_fiss.p;
    s.fiss_old = (double *)h->d_fiss_old.p;
    s.partial = (double *)h->d_partial.p;
    s.scal = (double *)h->d_scal.p;
    s.counter = (int32_t *)h->d_counter.p;
    s.sig_t = h->d_sigt.p;
    s.sig_t64 = (const double *)h->d_sigt64.p;
    s.sig_s64 = (const double *)h->d_sigs64.p;
    s.nsf64 = (const double *)h->d_nsf64.p;
    s.chi64 = (const double *)h->d_chi64.p;
    s.src64 = (const double *)h->d_src64.p;
    s.inv_st64 = (const double *)h->d_inv_st64.p;
    s.siga64 = (const double *)h->d_siga64.p;
    s.inv_vol = (const double *)h->d_inv_vol.p;
}

// The per-iteration kernels are no-ops once SC_CONV is set (a converged
// solve); the single-step entry points below clear it first on their stream.
cudaError_t clear_conv(moc_tracks *h, cudaStream_t s) {
    return cudaMemsetAsync((double *)h->d_scal.p + SC_CONV, 0, sizeof(double), s);
}

cudaError_t set_scalar(moc_tracks *h, int slot, double v) {
    return cudaMemcpyAsync((double *)h->d_scal.p + slot, &v, sizeof(double), cudaMemcpyHostToDevice,
                           h->stream);
}

// Per psi buffer p, one 16-byte block of d_counter: the work counter of the
// sweep that writes buffer p
size_t sweep_block_bytes(const moc_tracks *) { return 16; }
int32_t *sweep_counter(moc_tracks *h, int p) {
    return (int32_t *)((char *)h->d_counter.p + (size_t)p * sweep_block_bytes(h));
}

// one sweep into the other psi buffer (no source update, no finalize)
cudaError_t enqueue_sweep(moc_tracks *h, cudaStream_t s, int cur) {
    const int out = h->has_psi ? 1 - cur : 0;
    cudaError_t e = cudaMemsetAsync(sweep_counter(h, out), 0, 4, s);
    if (e != cudaSuccess) return e;
    const void *pin = h->has_psi ? h->d_psi[cur].p : nullptr;
    void *pout = h->has_psi ? h->d_psi[1 - cur].p : nullptr;
    return launch_sweep(h->precision, h->tally_smem, h->gpl, h->dl, h->ds, (const int32_t *)h->d_order.p,
                        (int32_t)h->order.size(), h->tile_cap, pin, pout, sweep_counter(h, out), h->grid,
                        h->block, h->smem, s);
}

cudaError_t enqueue_finalize(moc_tracks *h, cudaStream_t s) {
    const int nfsr = h->geom.nfsr;
    if (h->geom.src.empty())
        return launch_finalize(h->precision, h->dl, h->ds, nfsr, h->red_grid, h->integrations, s);
    return launch_finalize_fixed(h->precision, h->dl, h->ds, nfsr, h->red_grid, h->integrations, s);
}

// one outer iteration: source, sweep, flux update, k / residual; the scalars
// are copied to the pinned host mirror at the end
cudaError_t enqueue_iteration(moc_tracks *h, cudaStream_t s, int cur) {
    cudaError_t e = launch_source(h->precision, h->dl, h->ds, h->geom.nfsr, h->red_grid, s);
    if (e != cudaSuccess) return e;
    e = enqueue_sweep(h, s, cur);
    if (e != cudaSuccess) return e;
    e = enqueue_finalize(h, s);
    if (e != cudaSuccess) return e;
    return cudaMemcpyAsync(h->h_scal, h->d_scal.p, SC_COUNT * sizeof(double), cudaMemcpyDeviceToHost, s);
}

cudaError_t build_graphs(moc_tracks *h) {
    for (int c = 0; c < 2; ++c) {
        if (h->graph[c]) continue;
        cudaGraph_t g;
        cudaError_t e = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return e;
        e = enqueue_iteration(h, h->stream, c);
        cudaError_t e2 = cudaStreamEndCapture(h->stream, &g);
        if (e != cudaSuccess) return e;
        if (e2 != cudaSuccess) return e2;
        e = cudaGraphInstantiate(&h->graph[c], g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

void fill_result(moc_tracks *h, moc_result *r, double seconds, int iters) {
    if (!r) return;
    const double *s = h->h_scal;
    const bool eig = h->geom.src.empty();
    r->k = eig ? s[SC_K] : 1.0;
    r->residual = s[SC_RES];
    r->dk = s[SC_DK];
    r->production = eig ? 1.0 : s[SC_PROD];
    r->absorption = eig ? s[SC_ABS] * s[SC_SCALE] : s[SC_ABS];
    r->leakage = s[SC_LEAK_PREV];
    r->seconds = seconds;
    r->integrations = (double)iters * h->integrations;
    r->iterations = iters;
    r->converged = s[SC_CONV] != 0.0 ? 1 : 0;
}

// the sweep sets SC_ERR to 1 when a shared tally update gave up after its
// retry limit (never expected: it needs that many consecutive lost races), to
// 2 when a unit's tally scale lay outside the fixed-point tally's range
int check_sweep_flag(moc_tracks *h) {
    if (h->h_scal[SC_ERR] == 2.0) {
        moc_set_error("sweep: a tally contribution beyond 2^51 (fixed-point tally range); results are invalid");
        return MOC_ERR_CUDA;
    }
    if (h->h_scal[SC_ERR] != 0.0) {
        moc_set_error("sweep: a shared tally update exceeded its retry limit; results are invalid");
        return MOC_ERR_CUDA;
    }
    return MOC_OK;
}

// bytes of one FSR-group's tally entry: the three 64-bit fixed-point words
// of FP32 shared-tally layouts, else FP64
size_t tally_entry_bytes(const moc_tracks *h) {
    return (h->precision == MOC_FP32 && h->tally_smem) ? 24 : 8;
}

// the tally [n] copied to host FP64 values (synchronises the stream)
cudaError_t tally_to_host(moc_tracks *h, double *out, size_t n) {
    if (tally_entry_bytes(h) == 8) {
        cudaError_t e = cudaMemcpyAsync(out, h->d_tally.p, n * 8, cudaMemcpyDeviceToHost, h->stream);
        return e == cudaSuccess ? cudaStreamSynchronize(h->stream) : e;
    }
    std::vector<long long> w(3 * n);
    cudaError_t e = cudaMemcpyAsync(w.data(), h->d_tally.p, n * 24, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return e;
    for (size_t i = 0; i < n; ++i) out[i] = tally3_value(w[3 * i], w[3 * i + 1], w[3 * i + 2]);
    return cudaSuccess;
}

// Runs up to n outer iterations.  With stop_on_conv the scalars are checked
// every kSyncEvery iterations: the iteration that converges sets SC_CONV on the
// device and every later one is a no-op there, so the result does not depend
// on how often the host looks.
constexpr int kSyncEvery = 16;

int run_iterations(moc_tracks *h, int n, bool stop_on_conv, bool graph, moc_result *res) {
    TRY(cudaSetDevice(h->device), "cudaSetDevice");
    if (graph) TRY(build_graphs(h), "graph capture");
    TRY(cudaMemcpyAsync(h->h_scal, h->d_scal.p, SC_COUNT * sizeof(double), cudaMemcpyDeviceToHost,
                        h->stream), "scalars");
    TRY(cudaStreamSynchronize(h->stream), "scalars");
    const int iter0 = (int)h->h_scal[SC_ITER];
    const int cur0 = h->cur;
    cudaEvent_t e0, e1;
    TRY(cudaEventCreate(&e0), "event");
    TRY(cudaEventCreate(&e1), "event");
    TRY(cudaEventRecord(e0, h->stream), "event");
    int it = 0;
    for (; it < n;) {
        if (graph) TRY(cudaGraphLaunch(h->graph[h->cur], h->stream), "graph launch");
        else TRY(enqueue_iteration(h, h->stream, h->cur), "iteration");
        if (h->has_psi) h->cur = 1 - h->cur;
        ++it;
        if (stop_on_conv && (it % kSyncEvery == 0 || it == n)) {
            TRY(cudaStreamSynchronize(h->stream), "iteration");
            if (h->h_scal[SC_CONV] != 0.0) break;
        }
    }
    TRY(cudaEventRecord(e1, h->stream), "event");
    TRY(cudaEventSynchronize(e1), "event");
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // iterations that did work; the no-ops after convergence left psi in place
    const int done = (int)h->h_scal[SC_ITER] - iter0;
    if (h->has_psi) h->cur = (cur0 + done) & 1;
    fill_result(h, res, ms * 1e-3, done);
    return check_sweep_flag(h);
}

int init_state(moc_tracks *h) {
    TRY(cudaMemsetAsync(h->d_tally.p, 0, h->d_tally.n, h->stream), "memset");
    TRY(cudaMemsetAsync(h->d_counter.p, 0, h->d_counter.n, h->stream), "memset");  // psi = 0: bounds 0
    for (int c = 0; c < 2; ++c)
        if (h->d_psi[c].p) TRY(cudaMemsetAsync(h->d_psi[c].p, 0, h->d_psi[c].n, h->stream), "memset");
    h->cur = 0;
    TRY(set_scalar(h, SC_INTEG, 0.0), "scalar");
    TRY(set_scalar(h, SC_LEAK_PREV, 0.0), "scalar");
    TRY(set_scalar(h, SC_TOLS, 0.0), "scalar");  // no convergence test unless a solve sets one
    TRY(set_scalar(h, SC_TOLK, 0.0), "scalar");
    TRY(launch_init_state(h->dl, h->ds, h->geom.nfsr, h->red_grid, h->stream), "init state");
    TRY(cudaMemcpyAsync(h->h_scal, h->d_scal.p, SC_COUNT * sizeof(double), cudaMemcpyDeviceToHost,
                        h->stream), "scalars");
    TRY(cudaStreamSynchronize(h->stream), "init state");
    return MOC_OK;
}

// map (2D track t, polar p over both hemispheres, lattice index i) to the
// stored stack, frame and stored index
bool map_track(const moc_tracks *h, int t, int p, int64_t i, int64_t &stack, int &frame, int64_t &j) {
    const Layout &L = h->L;
    if (t < 0 || t >= L.nt || p < 0 || p >= L.P) return false;
    stack = (int64_t)t * L.Ph + (p % L.Ph);
    frame = p < L.Ph ? 0 : 1;
    if (frame == 0) j = i;
    else {
        // mirrored: height at the start of t is H - dz (j + zeta0) = z_0' + i dz
        const bool zero = L.zf[L.zoff[stack]] == 0.0f && L.zn[L.zoff[stack]] == 0;
        j = (int64_t)L.Nz - i - (zero ? 0 : 1);
    }
    const StackDesc &d = L.desc[stack];
    return j >= d.i_lo && j < (int64_t)d.i_lo + d.n_trk;
}

}  // namespace

// ---------------------------------------------------------------------------

extern "C" int moc_query_footprint(const moc_geometry *g, const moc_track_params *p,
                                   int64_t *resident, int64_t *preload_all) {
    if (!g || !p) { moc_set_error("NULL argument"); return MOC_ERR_INVALID_ARG; }
    Layout L;
    std::string err;
    moc_track_params hp = *p;
    hp.trace_on_device = 0;  // a host-only query
    int rc = moc_build_layout(*g, hp, L, err);
    if (rc) { moc_set_error(err); return rc; }
    const size_t rs = real_size(p->precision);
    const int64_t G = g->G;
    int64_t b = 0;
    b += (int64_t)L.desc.size() * sizeof(StackDesc) + (int64_t)L.zn.size() * 8;
    // planes off the lattice: per boundary two 16-bit ranks and the mirrored
    // frame's fraction (FP32, and FP64 for FP64 sweeps)
    if (L.offlat) b += (int64_t)L.zn.size() * (rs == 8 ? 16 : 8);
    b += (int64_t)L.seg_reg.size() * 8 + (int64_t)g->nfsr * 4 + (int64_t)L.desc.size() * 4;
    b += (int64_t)g->nfsr * G * (8 + rs + 8) + (int64_t)g->nfsr * 8 * 3;
    bool refl = false;
    for (int f = 0; f < 6; ++f) refl |= g->bc[f] != 0;
    if (refl) b += 2 * L.n_gtrk * 4 * G * (int64_t)rs + L.n_gtrk * 4 * 4;  // boundary fluxes, links
    b += L.n_gtrk * (4 + 8);  // sweep order and record windows
    b += (int64_t)g->nreg * 4;  // the material of each radial region (material-keyed records)
    if (resident) *resident = b;
    if (preload_all && L.offlat) *preload_all = 0;  // planes off the lattice: nothing is stored
    if (preload_all && !L.offlat) {
        // an upper estimate from the 2D segments: each 3D track crosses its 2D
        // segments plus the layer planes it passes
        double segs = 0;
        for (int64_t s = 0; s < L.n_stacks; ++s) {
            const StackDesc &d = L.desc[s];
            const double planes = (double)(L.zn[d.zoff + d.nb] - L.zn[d.zoff] + 1) / L.cpl + 1;
            segs += (double)d.n_trk * (d.nb + planes);
        }
        *preload_all = (int64_t)(segs * 8 + (double)L.n_gtrk * 8);
    }
    return MOC_OK;
}

extern "C" int moc_generate_tracks(const moc_geometry *g, const moc_track_params *prm,
                                   moc_tracks **out) {
    if (!g || !prm || !out) { moc_set_error("NULL argument"); return MOC_ERR_INVALID_ARG; }
    *out = nullptr;
    if (prm->precision != MOC_FP32 && prm->precision != MOC_FP64) {
        moc_set_error("precision must be MOC_FP32 or MOC_FP64");
        return MOC_ERR_INVALID_ARG;
    }
    std::unique_ptr<moc_tracks> h(new moc_tracks());
    h->geom = *g;
    h->precision = prm->precision;
    h->device = prm->device;
    std::string err;
    int rc = moc_build_layout(h->geom, *prm, h->L, err);
    if (rc) { moc_set_error(err); return rc; }
    Layout &L = h->L;
    const moc_geometry &geo = h->geom;
    const int G = geo.G;
    if ((int64_t)geo.nfsr * G > 0x7fffffffLL) { moc_set_error("too many FSR-groups"); return MOC_ERR_UNSUPPORTED; }
    for (int t = 0; t < L.nt; ++t) h->nb_max = std::max(h->nb_max, L.seg_off[t + 1] - L.seg_off[t]);
    if (h->nb_max >= 65536) { moc_set_error("a 2D track has too many segments"); return MOC_ERR_UNSUPPORTED; }
    {
        // link destinations are 32-bit track-direction indices (reflective faces only)
        bool has_links = false;
        for (int f = 0; f < 6; ++f) has_links |= geo.bc[f] != 0;
        if (has_links && L.n_gtrk * 4 >= (int64_t)1 << 31) {
            moc_set_error("too many 3D tracks with reflective faces (at most 2^29)");
            return MOC_ERR_UNSUPPORTED;
        }
        if (L.n_gtrk * 4 >= (int64_t)1 << 40) { moc_set_error("too many 3D tracks"); return MOC_ERR_UNSUPPORTED; }
    }
    if (L.Ph > 16) { moc_set_error("at most 32 polar angles"); return MOC_ERR_UNSUPPORTED; }
    // tally mode: a shared tile of every (2D segment, layer) row of one unit
    // when it fits
    h->tile_cap = h->nb_max * L.nlv;
    if (prm->groups_per_lane < 0 || prm->groups_per_lane > 4 || prm->groups_per_lane == 3 ||
        (prm->groups_per_lane > 1 && h->precision == MOC_FP64)) {
        moc_set_error("groups_per_lane must be 0, 1, 2 or 4 (2 and 4 for FP32 sweeps only)");
        return MOC_ERR_INVALID_ARG;
    }
    h->gpl = prm->groups_per_lane > 0 ? prm->groups_per_lane : sweep_default_gpl(h->precision, G);
    {
        // a unit whose tile exceeds kWholeTile is swept in radial chunks of
        // chunk_b 2D segments, sized for three blocks per SM; GLOBAL when not
        // even one 2D segment's layers fit
        constexpr size_t kWholeTile = 100 * 1024, kChunkTile = 72 * 1024;
        int mode = prm->tally_mode;
        if (prm->chunk_segments < 0) {
            moc_set_error("chunk_segments must be >= 0");
            return MOC_ERR_INVALID_ARG;
        }
        // FP64 sweeps: a shared tile would add with compare-and-swap loops,
        // which measured slower than the native FP64 adds of the global tally
        if (mode == MOC_TALLY_AUTO) mode = h->precision == MOC_FP64 ? MOC_TALLY_GLOBAL : MOC_TALLY_SHARED;
        // planes off the lattice: the frames' pieces differ, so the sweep of
        // moc_sweep_ol.cu (FP64 global tally) takes every layout
        if (L.offlat) mode = MOC_TALLY_GLOBAL;
        if (mode == MOC_TALLY_SHARED &&
            (prm->chunk_segments > 0 ||
             sweep_smem_bytes(h->precision, 1, 0, geo.M, G, h->gpl, h->tile_cap) > kWholeTile)) {
            int cb = 0;
            while (cb < h->nb_max &&
                   sweep_smem_bytes(h->precision, 1, 1, geo.M, G, h->gpl, (cb + 1) * L.nlv) <= kChunkTile)
                ++cb;
            if (prm->chunk_segments > 0) cb = std::min(cb, (int)prm->chunk_segments);
            if (cb >= h->nb_max) {
                cb = 0;  // every unit fits whole
            } else if (cb >= 1) {
                h->chunk_b = cb;
                h->tile_cap = cb * L.nlv;
            } else {
                mode = MOC_TALLY_GLOBAL;
            }
        }
        h->tally_smem = mode == MOC_TALLY_SHARED ? 1 : 0;
        if (!h->tally_smem) h->chunk_b = 0;
    }
    // FP32 shared tally in fixed point: each contribution t becomes an
    // integer multiple of 2^-bits of its unit's bound B (|t| <= B, so at most
    // 2^bits in magnitude) and is added with a native integer atomic.  The
    // adds wrap modulo 2^32, so partial sums may overflow as long as the
    // final sum of one row of one unit lies in [-2^31, 2^31): pieces that
    // reach one row x 2^bits < 2^31.  Pieces that reach one row of one unit:
    // per polar stack, 2 senses x 2 frames x the tracks crossing one layer
    // inside one 2D segment (at most cpl plus the segment's lattice span
    // plus 2).  At most 24 bits: the grid then matches the FP32 precision of
    // the contributions themselves.
    if (h->tally_smem && h->precision == MOC_FP32) {
        int64_t nmax = 1;
        for (int t = 0; t < L.nt; ++t) {
            const int nb = L.seg_off[t + 1] - L.seg_off[t];
            int64_t n = 0;
            for (int ph = 0; ph < L.Ph; ++ph) {
                const int32_t z = L.zoff[(size_t)t * L.Ph + ph];
                double span = 0.0;
                for (int b = 0; b < nb; ++b)
                    span = std::max(span, (L.zn[z + b + 1] + (double)L.zf[z + b + 1]) -
                                              (L.zn[z + b] + (double)L.zf[z + b]));
                n += 4 * (L.cpl + (int64_t)std::ceil(span) + 2);
            }
            nmax = std::max(nmax, n);
        }
        int bits = 24;
        while (bits > 0 && (nmax << bits) >= ((int64_t)1 << 31)) --bits;
        if (bits < 12) {  // too many pieces per row: FP64 global tally instead
            h->tally_smem = 0;
            h->chunk_b = 0;
        }
        else h->tally_bits = bits;
    }
    // synchronous blocks of the stored stacks: FP32, two groups per lane,
    // shared tally, every unit swept whole; at most the tracks of one warp
    if (prm->sync_block < 0 || prm->sync_block > 8 || (prm->sync_block & (prm->sync_block - 1))) {
        moc_set_error("sync_block must be 0, 1, 2, 4 or 8");
        return MOC_ERR_INVALID_ARG;
    }
    if (h->precision == MOC_FP32 && h->gpl == 2 && h->tally_smem && h->chunk_b == 0) {
        const int slots = 32 / sweep_lanes_per_track(G, 2);
        h->sync_b = std::min(prm->sync_block > 0 ? (int)prm->sync_block : 1, slots);
        if (h->sync_b < 2) h->sync_b = 0;
    }
    TRY(cudaSetDevice(h->device), "cudaSetDevice");
    TRY(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking), "stream");
    TRY(cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device), "attribute");
    TRY(cudaMallocHost(&h->h_scal, SC_COUNT * sizeof(double)), "pinned scalars");
    // layout tables
    std::vector<int32_t> reg2d(L.seg_reg.begin(), L.seg_reg.end());
    std::vector<float> len2d(L.seg_len.begin(), L.seg_len.end());
    TRY(upload(h.get(), h->d_zn, L.zn), "upload");
    TRY(upload(h.get(), h->d_zf, L.zf), "upload");
    if (!L.lmap.empty()) TRY(upload(h.get(), h->d_lmap, L.lmap), "upload");
    if (L.offlat) {
        TRY(upload(h.get(), h->d_zc0, L.zc[0]), "upload");
        TRY(upload(h.get(), h->d_zc1, L.zc[1]), "upload");
        TRY(upload(h.get(), h->d_zfd, L.zfd), "upload");
        TRY(upload(h.get(), h->d_pl_n, L.pl_n), "upload");
        TRY(upload(h.get(), h->d_pl_c, L.pl_c), "upload");
        std::vector<float> pf(L.pl_f.begin(), L.pl_f.end());
        TRY(upload(h.get(), h->d_pl_f, pf), "upload");
        TRY(upload(h.get(), h->d_pl_f64, L.pl_f), "upload");
        if (h->precision == MOC_FP64) TRY(upload(h.get(), h->d_zfd64, L.zfd64), "upload");
    }
    TRY(upload(h.get(), h->d_reg2d, reg2d), "upload");
    TRY(upload(h.get(), h->d_len2d, len2d), "upload");
    TRY(upload(h.get(), h->d_fsr_mat, geo.fsr_mat), "upload");
    // material keys (DevLayout::matk): FP32, two groups per lane, shared tally
    // (units swept whole or in radial chunks), no synchronous blocks, at most
    // 4 materials and one material per radial region; the stored templates
    // must cover every unit (checked once they are planned)
    bool matk_cand = h->precision == MOC_FP32 && h->gpl == 2 && h->tally_smem && h->sync_b == 0 &&
                     !L.offlat && geo.M <= 4 && !(prm->schedule & MOC_SCHED_ROWS_WITH_SIGMA);
    if (h->sync_b || matk_cand) {
        // per radial region: its material when every layer has the same one
        // (then Sigma_t is one value per 2D segment of a unit), else -1
        std::vector<int32_t> reg_mat(geo.nreg);
        for (int r = 0; r < geo.nreg; ++r) {
            int m = geo.fsr_mat[(size_t)r * geo.nl];
            for (int l = 1; l < geo.nl && m >= 0; ++l)
                if (geo.fsr_mat[(size_t)r * geo.nl + l] != m) m = -1;
            reg_mat[r] = m;
            if (m < 0) matk_cand = false;
        }
        TRY(upload(h.get(), h->d_reg_mat, reg_mat), "upload");
    }
    if (h->precision == MOC_FP64) {
        TRY(upload(h.get(), h->d_zf64, L.zf64), "upload");
        TRY(upload(h.get(), h->d_len2d64, L.seg_len), "upload");
    }
    TRY(upload(h.get(), h->d_desc, L.desc), "upload");
    fill_views(h.get());
    // segment counts per stack
    const int64_t ns = L.n_stacks;
    DevBuf d_nseg, d_max, d_tseg;
    TRY(dalloc(h.get(), d_nseg, ns * sizeof(int64_t)), "alloc");
    TRY(dalloc(h.get(), d_max, sizeof(int32_t)), "alloc");
    TRY(dalloc(h.get(), d_tseg, std::max<int64_t>(1, L.n_gtrk) * sizeof(int32_t)), "alloc");
    TRY(cudaMemsetAsync(d_max.p, 0, sizeof(int32_t), h->stream), "memset");
    const int lgrid = (int)std::max<int64_t>(1, std::min<int64_t>(ns, (int64_t)h->sms * 16));
    TRY(launch_count_stacks(h->dl, ns, (int64_t *)d_nseg.p, (int32_t *)d_max.p, (int32_t *)d_tseg.p,
                            lgrid, h->stream), "count");
    h->stack_nseg.resize(ns);
    std::vector<int32_t> tseg(L.n_gtrk);
    TRY(cudaMemcpyAsync(h->stack_nseg.data(), d_nseg.p, ns * sizeof(int64_t), cudaMemcpyDeviceToHost, h->stream), "copy");
    TRY(cudaMemcpyAsync(&h->max_nseg, d_max.p, sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream), "copy");
    if (L.n_gtrk > 0)
        TRY(cudaMemcpyAsync(tseg.data(), d_tseg.p, L.n_gtrk * sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream), "copy");
    TRY(cudaStreamSynchronize(h->stream), "count");
    h->bytes -= d_nseg.n + d_max.n + d_tseg.n;
    int64_t segs_up = 0;
    for (auto v : h->stack_nseg) segs_up += v;
    // (the counts of layouts off the lattice hold both frames)
    h->n_segments3d = L.offlat ? segs_up : 2 * segs_up;
    h->integrations = (double)h->n_segments3d * 2.0 * G;
    // Stored segments (EXP, Sec. 4.2).  What is stored is one template per
    // class r < cpl of a stack (the tracks r, r + cpl, ... are one-layer shifts
    // of each other); the work unit of the sweep is a 2D track with all its
    // polar stacks.  Template sizes first, for every stack:
    const int Ph = L.Ph;
    const int cpl = L.cpl;
    std::vector<int64_t> tpl_first(ns, 0);
    int64_t n_tpl_all = 0;
    for (int64_t s = 0; s < ns; ++s) {
        tpl_first[s] = n_tpl_all;
        L.desc[s].exp_base = n_tpl_all;
        n_tpl_all += std::min(cpl, L.desc[s].n_trk);
    }
    std::vector<int64_t> tcnt(n_tpl_all);
    std::vector<int32_t> tlmin(n_tpl_all), tnlay(n_tpl_all);
    if (n_tpl_all > 0) {
        DevBuf d_all, d_cnt, d_lmin, d_nlay;
        std::vector<int32_t> all(ns);
        std::iota(all.begin(), all.end(), 0);
        TRY(cudaMemcpyAsync(h->d_desc.p, L.desc.data(), ns * sizeof(StackDesc), cudaMemcpyHostToDevice, h->stream), "upload");
        TRY(upload(h.get(), d_all, all), "upload");
        TRY(dalloc(h.get(), d_cnt, n_tpl_all * 8), "alloc");
        TRY(dalloc(h.get(), d_lmin, n_tpl_all * 4), "alloc");
        TRY(dalloc(h.get(), d_nlay, n_tpl_all * 4), "alloc");
        TRY(launch_tpl_count(h->dl, (const int32_t *)d_all.p, ns, (int64_t *)d_cnt.p, (int32_t *)d_lmin.p,
                             (int32_t *)d_nlay.p, lgrid, h->stream), "template sizes");
        TRY(cudaMemcpyAsync(tcnt.data(), d_cnt.p, n_tpl_all * 8, cudaMemcpyDeviceToHost, h->stream), "copy");
        TRY(cudaMemcpyAsync(tlmin.data(), d_lmin.p, n_tpl_all * 4, cudaMemcpyDeviceToHost, h->stream), "copy");
        TRY(cudaMemcpyAsync(tnlay.data(), d_nlay.p, n_tpl_all * 4, cudaMemcpyDeviceToHost, h->stream), "copy");
        TRY(cudaStreamSynchronize(h->stream), "template sizes");
        h->bytes -= d_all.n + d_cnt.n + d_lmin.n + d_nlay.n;
    }
    // plan: units (2D tracks) by decreasing work; store a unit's templates
    // while the budget lasts (largest first), generate the rest on the fly
    std::vector<int64_t> unit_nseg(L.nt, 0);
    for (int t = 0; t < L.nt; ++t)
        for (int ph = 0; ph < Ph; ++ph) unit_nseg[t] += h->stack_nseg[(int64_t)t * Ph + ph];
    std::vector<int32_t> by_size(L.nt);
    std::iota(by_size.begin(), by_size.end(), 0);
    std::stable_sort(by_size.begin(), by_size.end(),
                     [&](int32_t a, int32_t b) { return unit_nseg[a] > unit_nseg[b]; });
    const int64_t rec_bytes = (int64_t)segrec_size(h->precision);
    const int64_t budget = prm->preload_budget_bytes;
    int64_t used = 0;
    std::vector<int32_t> exp_stacks;
    std::vector<int64_t> off_h(1, 0), loff_h(1, 0);
    std::vector<int32_t> lmin_h;
    for (int32_t t : by_size) {
        int64_t need = 0;
        bool ok = true;
        for (int ph = 0; ph < Ph; ++ph) {
            const int64_t s = (int64_t)t * Ph + ph;
            for (int r = 0; r < std::min(cpl, L.desc[s].n_trk); ++r) {
                const int64_t q = tpl_first[s] + r;
                need += tcnt[q] * rec_bytes + (int64_t)(tnlay[q] + 1) * 4 + 20;
                // stored keys: the template layer as a signed 16-bit number
                // (chunked and synchronous layouts), else both tile rows as
                // 16-bit numbers
                ok = ok && tlmin[q] > -32768 && tlmin[q] + tnlay[q] < 32767;
                if (h->chunk_b == 0 && h->sync_b == 0)
                    ok = ok && tlmin[q] > -2000 && tlmin[q] + tnlay[q] < 2000 &&
                         (int64_t)(L.desc[s].nb + 1) * L.nlv + 2000 < 32768;
            }
        }
        ok = ok && h->max_nseg < 65536;  // record windows hold the count in 16 bits
        ok = ok && !L.offlat;            // no templates off the lattice
        if (!ok || (budget >= 0 && used + need > budget)) {
            for (int ph = 0; ph < Ph; ++ph) L.desc[(int64_t)t * Ph + ph].exp_base = -1;
            continue;
        }
        used += need;
        for (int ph = 0; ph < Ph; ++ph) {
            const int64_t s = (int64_t)t * Ph + ph;
            L.desc[s].exp_base = (int64_t)lmin_h.size();
            for (int r = 0; r < std::min(cpl, L.desc[s].n_trk); ++r) {
                const int64_t q = tpl_first[s] + r;
                off_h.push_back(off_h.back() + tcnt[q]);
                loff_h.push_back(loff_h.back() + tnlay[q] + 1);
                lmin_h.push_back(tlmin[q]);
            }
            exp_stacks.push_back((int32_t)s);
        }
    }
    h->n_exp_stacks = (int64_t)exp_stacks.size();
    // sweep slots of every stack (perm; the record windows follow the same
    // order).  Tracks by decreasing segment count, so that the tracks a warp
    // sweeps side by side take the same number of steps; among equal counts
    // class by class (tracks r, r + cpl, ... are whole-layer shifts of one
    // another and rarely meet in the same FSR at the same step, so the shared
    // tally updates of one warp seldom collide).  Radially chunked units: in
    // index order (the tracks crossing one chunk are one range).  Stored
    // stacks of layouts with synchronous blocks: blocks of sync_b consecutive
    // tracks r + m cpl of one class (padded with entries -1 - k that continue
    // the block's sequence), blocks by decreasing segment count.
    {
        std::vector<int32_t> perm;
        perm.reserve((size_t)L.n_gtrk);
        const int B = h->sync_b;
        for (int64_t s = 0; s < ns; ++s) {
            StackDesc &d = L.desc[s];
            const int64_t o = d.trk_off;
            const int n = d.n_trk;
            d.slot_off = (int64_t)perm.size();
            if (L.offlat || (h->chunk_b > 0 && d.nb > h->chunk_b)) {
                for (int k = 0; k < n; ++k) perm.push_back(k);
            } else if (B > 1 && d.exp_base >= 0) {
                std::vector<std::pair<int32_t, std::vector<int32_t>>> blocks;
                for (int r = 0; r < std::min(cpl, n); ++r)
                    for (int k0 = r; k0 < n; k0 += B * cpl) {
                        std::vector<int32_t> e(B);
                        int32_t est = 0;
                        for (int j = 0; j < B; ++j) {
                            const int k = k0 + j * cpl;
                            e[j] = k < n ? k : -1 - k;
                            if (k < n) est = std::max(est, tseg[o + k]);
                        }
                        blocks.emplace_back(est, std::move(e));
                    }
                if (!(prm->schedule & MOC_SCHED_TRACKS_NATURAL))
                    std::stable_sort(blocks.begin(), blocks.end(),
                                     [](const auto &a, const auto &b) { return a.first > b.first; });
                for (auto &bl : blocks) perm.insert(perm.end(), bl.second.begin(), bl.second.end());
            } else {
                const size_t q0 = perm.size();
                for (int r = 0; r < std::min(cpl, n); ++r)
                    for (int k = r; k < n; k += cpl) perm.push_back(k);
                if (!(prm->schedule & MOC_SCHED_TRACKS_NATURAL))
                    std::stable_sort(perm.begin() + q0, perm.end(),
                                     [&](int32_t a, int32_t b) { return tseg[o + a] > tseg[o + b]; });
            }
            d.n_slot = (int32_t)((int64_t)perm.size() - d.slot_off);
        }
        h->n_slots = (int64_t)perm.size();
        TRY(upload(h.get(), h->d_perm, perm), "upload");
        fill_views(h.get());
    }
    TRY(cudaMemcpyAsync(h->d_desc.p, L.desc.data(), ns * sizeof(StackDesc), cudaMemcpyHostToDevice, h->stream), "upload");
    if (matk_cand) {
        // every unit stored, and the mirrored tile rows b NL + NL-1-L_t of the
        // keys within 14 signed bits (radially chunked layouts: the 2D
        // segment index within 14 unsigned bits)
        for (int64_t s = 0; s < ns && matk_cand; ++s) {
            const StackDesc &d = L.desc[s];
            if (d.exp_base < 0) { matk_cand = false; break; }
            if (h->chunk_b > 0) {
                if (d.nb >= 16000) matk_cand = false;
                continue;
            }
            for (int r = 0; r < std::min(cpl, d.n_trk); ++r) {
                const int64_t q = tpl_first[s] + r;
                if ((int64_t)d.nb * L.nlv - tlmin[q] >= 8000 || tlmin[q] + tnlay[q] >= 8000) matk_cand = false;
            }
        }
        h->matk = matk_cand ? 1 : 0;
        if (h->matk && h->chunk_b > 0) {
            // rows of Qr only: wider radial chunks in the same shared memory
            // (the keys name 2D segments, so the stored records do not change)
            constexpr size_t kChunkTile = 72 * 1024;
            int cb = h->chunk_b;
            while (cb < h->nb_max &&
                   sweep_smem_bytes(h->precision, 1, 1, geo.M, G, h->gpl, (cb + 1) * L.nlv, 0, 1, 1) <= kChunkTile)
                ++cb;
            if (prm->chunk_segments > 0) cb = std::min(cb, (int)prm->chunk_segments);
            h->chunk_b = cb;
            h->tile_cap = cb * L.nlv;
        }
        fill_views(h.get());
    }
    if (!exp_stacks.empty()) {
        DevBuf d_exp_stacks;
        TRY(upload(h.get(), d_exp_stacks, exp_stacks), "upload");
        TRY(upload(h.get(), h->d_tpl_off, off_h), "upload");
        TRY(upload(h.get(), h->d_tpl_loff, loff_h), "upload");
        TRY(upload(h.get(), h->d_tpl_lmin, lmin_h), "upload");
        h->n_stored = off_h.back();
        TRY(dalloc(h.get(), h->d_segs, (size_t)std::max<int64_t>(h->n_stored, 1) * rec_bytes), "alloc templates");
        TRY(dalloc(h.get(), h->d_tpl_lidx, (size_t)loff_h.back() * 4), "alloc template index");
        fill_views(h.get());
        const int egrid = (int)std::max<int64_t>(1, std::min<int64_t>(h->n_exp_stacks, (int64_t)h->sms * 16));
        TRY(launch_tpl_write(h->precision, h->dl, (const int32_t *)d_exp_stacks.p, h->n_exp_stacks,
                             h->d_segs.p, (int32_t *)h->d_tpl_lidx.p, egrid, h->stream), "templates");
        TRY(dalloc(h.get(), h->d_win, (size_t)std::max<int64_t>(h->n_slots, 1) * 8), "alloc record windows");
        fill_views(h.get());
        TRY(launch_windows(h->dl, ns, (uint64_t *)h->d_win.p, lgrid, h->stream), "record windows");
        TRY(cudaStreamSynchronize(h->stream), "templates");
        h->bytes -= d_exp_stacks.n;
    }
    fill_views(h.get());
    if (h->chunk_b > 0) {
        // chunk tables of the radially chunked units (see StackDesc::chunk_base)
        const int cb = h->chunk_b;
        std::vector<int32_t> cst;
        int64_t n_ent = 0;
        for (int t = 0; t < L.nt; ++t) {
            const int64_t s0 = (int64_t)t * Ph;
            if (L.desc[s0].nb <= cb) continue;
            const int64_t C = (L.desc[s0].nb + cb - 1) / cb;
            int64_t trk = 0;
            for (int ph = 0; ph < Ph; ++ph) {
                StackDesc &d = L.desc[s0 + ph];
                const int64_t ntpl = d.exp_base >= 0 ? std::min(cpl, d.n_trk) : 0;
                d.chunk_base = n_ent;
                n_ent += C + ntpl * (C + 1);
                trk += d.n_trk;
                cst.push_back((int32_t)(s0 + ph));
            }
            h->hand_trk = std::max(h->hand_trk, trk);
        }
        if (!cst.empty()) {
            DevBuf d_cst;
            TRY(cudaMemcpyAsync(h->d_desc.p, L.desc.data(), ns * sizeof(StackDesc), cudaMemcpyHostToDevice,
                                h->stream), "upload");
            TRY(upload(h.get(), d_cst, cst), "upload");
            TRY(dalloc(h.get(), h->d_chunk, (size_t)n_ent * 8), "alloc chunk tables");
            fill_views(h.get());
            const int cgrid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)cst.size(), (int64_t)h->sms * 16));
            TRY(launch_chunk_tables(h->precision, h->dl, (const int32_t *)d_cst.p, (int64_t)cst.size(),
                                    (int64_t *)h->d_chunk.p, cgrid, h->stream), "chunk tables");
            TRY(cudaStreamSynchronize(h->stream), "chunk tables");
            h->bytes -= d_cst.n;
        }
    }
    fill_views(h.get());
    // cross sections
    if (geo.M > 65535) { moc_set_error("too many materials"); return MOC_ERR_UNSUPPORTED; }
    if (h->precision == MOC_FP64) {
        TRY(upload(h.get(), h->d_sigt, geo.sigt), "upload");
    } else {
        std::vector<float> s32(geo.sigt.begin(), geo.sigt.end());
        TRY(upload(h.get(), h->d_sigt, s32), "upload");
    }
    TRY(upload(h.get(), h->d_sigt64, geo.sigt), "upload");
    TRY(upload(h.get(), h->d_sigs64, geo.sigs), "upload");
    TRY(upload(h.get(), h->d_nsf64, geo.nsf), "upload");
    TRY(upload(h.get(), h->d_chi64, geo.chi), "upload");
    if (!geo.src.empty()) TRY(upload(h.get(), h->d_src64, geo.src), "upload");
    {
        // inverses and absorption per material and group, so that the
        // per-iteration kernels multiply instead of dividing in FP64
        std::vector<double> inv_st((size_t)geo.M * G), siga((size_t)geo.M * G);
        for (int m = 0; m < geo.M; ++m)
            for (int g = 0; g < G; ++g) {
                const size_t mg = (size_t)m * G + g;
                inv_st[mg] = 1.0 / geo.sigt[mg];
                double a = geo.sigt[mg];
                for (int hh = 0; hh < G; ++hh) a -= geo.sigs[mg * G + hh];
                siga[mg] = a;
            }
        TRY(upload(h.get(), h->d_inv_st64, inv_st), "upload");
        TRY(upload(h.get(), h->d_siga64, siga), "upload");
    }
    // state
    const size_t nfg = (size_t)geo.nfsr * G;
    const size_t rs = real_size(h->precision);
    TRY(dalloc(h.get(), h->d_phi, nfg * 8), "alloc flux");
    TRY(dalloc(h.get(), h->d_qr, nfg * rs), "alloc source");
    TRY(dalloc(h.get(), h->d_tally, nfg * tally_entry_bytes(h.get())), "alloc tally");
    TRY(dalloc(h.get(), h->d_vol, (size_t)geo.nfsr * 8), "alloc volumes");
    TRY(dalloc(h.get(), h->d_fiss, (size_t)geo.nfsr * 8), "alloc");
    TRY(dalloc(h.get(), h->d_fiss_old, (size_t)geo.nfsr * 8), "alloc");
    h->red_grid = (int)std::max<int64_t>(
        1, std::min<int64_t>((geo.nfsr + kSmallBlock - 1) / kSmallBlock, (int64_t)h->sms * 8));
    TRY(dalloc(h.get(), h->d_partial, (size_t)h->red_grid * 4 * 8), "alloc");
    TRY(dalloc(h.get(), h->d_scal, SC_COUNT * 8), "alloc");
    TRY(dalloc(h.get(), h->d_counter, 2 * sweep_block_bytes(h.get())), "alloc");
    bool refl = false;
    for (int f = 0; f < 6; ++f) refl |= geo.bc[f] != 0;
    h->has_psi = refl;
    if (refl) {
        // every reflective link must land on a track direction, and no
        // direction may be fed twice; a failure here is an internal error
        std::vector<uint8_t> hit((size_t)L.n_gtrk * 4, 0);
        for (int64_t s = 0; s < ns; ++s) {
            const StackDesc &d = L.desc[s];
            for (int k = 0; k < d.n_trk; ++k)
                for (int v = 0; v < 4; ++v) {
                    const int64_t dst = moc_layout_link(geo, L, s, (int64_t)d.i_lo + k, v);
                    if (dst == -1) continue;
                    if (dst < 0 || dst >= (int64_t)hit.size() || hit[dst]) {
                        moc_set_error("internal: 3D link outside the track set or not one-to-one");
                        return MOC_ERR_INVALID_ARG;
                    }
                    hit[dst] = 1;
                }
        }
        TRY(dalloc(h.get(), h->d_dst, (size_t)L.n_gtrk * 4 * sizeof(int32_t)), "alloc links");
        fill_views(h.get());
        TRY(launch_links(h->dl, ns, (int32_t *)h->d_dst.p, lgrid, h->stream), "links");
        const size_t pb = (size_t)L.n_gtrk * 4 * G * rs;
        TRY(dalloc(h.get(), h->d_psi[0], pb), "alloc boundary fluxes");
        TRY(dalloc(h.get(), h->d_psi[1], pb), "alloc boundary fluxes");
    }
    fill_views(h.get());
    std::vector<double> init(SC_COUNT, 0.0);
    init[SC_EIGEN] = geo.src.empty() ? 1.0 : 0.0;
    init[SC_SCALE] = 1.0;
    init[SC_K] = 1.0;
    TRY(cudaMemcpyAsync(h->d_scal.p, init.data(), SC_COUNT * 8, cudaMemcpyHostToDevice, h->stream), "upload");
    {
        DevBuf d_vacc;  // exact sums, freed once the volumes are read
        TRY(dalloc(h.get(), d_vacc, (size_t)geo.nfsr * 4 * 8), "alloc volume sums");
        TRY(launch_volumes(h->precision, h->dl, ns, geo.nfsr, (unsigned long long *)d_vacc.p,
                           (double *)h->d_vol.p, lgrid, h->stream), "volumes");
        h->vol.resize(geo.nfsr);
        TRY(cudaMemcpyAsync(h->vol.data(), h->d_vol.p, geo.nfsr * 8, cudaMemcpyDeviceToHost, h->stream), "copy");
        TRY(cudaStreamSynchronize(h->stream), "volumes");
        h->bytes -= d_vacc.n;
    }
    {
        std::vector<double> inv_vol(geo.nfsr);
        for (int i = 0; i < geo.nfsr; ++i) inv_vol[i] = h->vol[i] > 0.0 ? 1.0 / h->vol[i] : 0.0;
        TRY(upload(h.get(), h->d_inv_vol, inv_vol), "upload");
    }
    // schedule: work units (2D tracks) in decreasing work, largest first
    h->order = by_size;
    if (prm->schedule & MOC_SCHED_UNITS_NATURAL) std::sort(h->order.begin(), h->order.end());
    TRY(upload(h.get(), h->d_order, h->order), "upload");
    fill_views(h.get());
    // sweep launch shape (tally mode chosen above)
    h->smem = sweep_smem_bytes(h->precision, h->tally_smem, h->chunk_b > 0, geo.M, G, h->gpl, h->tile_cap,
                               h->sync_b, L.nlv, h->matk);
    {
        const int bmax = sweep_block_threads(h->precision, h->gpl, h->matk && h->chunk_b == 0,
                                             h->chunk_b > 0 && !h->matk);
        h->block = prm->block_threads > 0 ? std::max(32, std::min(prm->block_threads, bmax) / 32 * 32) : bmax;
    }
    int bps = 0;
    TRY(sweep_occupancy(h->precision, h->tally_smem, h->chunk_b > 0, G, h->gpl, h->block, h->smem, &bps,
                        h->sync_b > 0, h->matk != 0),
        "occupancy");
    if (bps < 1) { moc_set_error("sweep kernel does not fit on an SM"); return MOC_ERR_UNSUPPORTED; }
    if (prm->blocks_per_sm > 0) bps = std::min(bps, prm->blocks_per_sm);
    h->grid = std::max(1, std::min<int>(h->sms * bps, (int)std::min<int64_t>(ns, 1 << 30)));
    if (L.offlat) {
        // the off-lattice sweep: fixed blocks, eight per SM
        h->block = sweep_ol_block();
        h->grid = std::max(1, std::min(h->sms * 8, L.nt));
    }
    if (h->chunk_b > 0) {
        // psi of the tracks between radial chunks: one region per block
        TRY(dalloc(h.get(), h->d_hand, (size_t)h->grid * h->hand_trk * 2 * G * real_size(h->precision)),
            "alloc chunk hand-off");
        fill_views(h.get());
    }
    rc = init_state(h.get());
    if (rc) return rc;
    *out = h.release();
    return MOC_OK;
}

std::mutex g_states_mu;  // live-state counts of layout owners

namespace {
// drop one state's hold on a layout owner; frees the owner when it was
// destroyed while states lived and this was the last of them
void release_owner(moc_tracks *o) {
    bool free_it = false;
    {
        std::lock_guard<std::mutex> lk(g_states_mu);
        free_it = --o->live_states == 0 && o->destroy_pending;
    }
    if (free_it) delete o;
}
}  // namespace

extern "C" void moc_destroy_tracks(moc_tracks *h) {
    if (!h) return;
    cudaSetDevice(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    moc_tracks *owner = h->owner;
    if (!owner) {
        std::lock_guard<std::mutex> lk(g_states_mu);
        if (h->live_states > 0) {
            h->destroy_pending = true;  // its states still use the layout
            return;
        }
    }
    delete h;
    if (owner) release_owner(owner);
}

extern "C" void moc_state_destroy(moc_tracks *state) { moc_destroy_tracks(state); }

namespace {
void borrow(DevBuf &d, const DevBuf &s) {
    d.p = s.p;
    d.n = s.n;
    d.borrowed = true;
}
}  // namespace

extern "C" int moc_state_create(const moc_tracks *t, const double *ext_source, moc_tracks **out) {
    if (!t || !out) { moc_set_error("NULL argument"); return MOC_ERR_INVALID_ARG; }
    *out = nullptr;
    moc_tracks *base = t->owner ? t->owner : const_cast<moc_tracks *>(t);
    {
        // hold the layout from here on, so that a concurrent destroy of its
        // owner cannot free the buffers this state borrows while it is built
        std::lock_guard<std::mutex> lk(g_states_mu);
        if (base->destroy_pending) { moc_set_error("the layout was destroyed"); return MOC_ERR_INVALID_ARG; }
        ++base->live_states;
    }
    struct Hold {
        moc_tracks *o;
        bool kept = false;
        ~Hold() {
            if (!kept) release_owner(o);
        }
    } hold{base};
    const int G = base->geom.G, M = base->geom.M;
    if (ext_source)
        for (int i = 0; i < M * G; ++i)
            if (!(ext_source[i] >= 0.0) || !std::isfinite(ext_source[i])) {
                moc_set_error("ext_source must be finite and non-negative");
                return MOC_ERR_INVALID_ARG;
            }
    TRY(cudaSetDevice(base->device), "cudaSetDevice");
    std::unique_ptr<moc_tracks> h(new moc_tracks());
    h->geom = base->geom;
    if (ext_source) h->geom.src.assign(ext_source, ext_source + (size_t)M * G);
    h->L = base->L;
    h->precision = base->precision;
    h->device = base->device;
    h->sms = base->sms;
    h->has_psi = base->has_psi;
    h->stack_nseg = base->stack_nseg;
    h->order = base->order;
    h->n_segments3d = base->n_segments3d;
    h->n_stored = base->n_stored;
    h->n_exp_stacks = base->n_exp_stacks;
    h->max_nseg = base->max_nseg;
    h->nb_max = base->nb_max;
    h->integrations = base->integrations;
    h->tally_smem = base->tally_smem;
    h->gpl = base->gpl;
    h->tally_bits = base->tally_bits;
    h->tile_cap = base->tile_cap;
    h->chunk_b = base->chunk_b;
    h->sync_b = base->sync_b;
    h->matk = base->matk;
    h->n_slots = base->n_slots;
    h->hand_trk = base->hand_trk;
    h->block = base->block;
    h->grid = base->grid;
    h->smem = base->smem;
    h->red_grid = base->red_grid;
    h->vol = base->vol;
    // the layout: shared
    borrow(h->d_desc, base->d_desc); borrow(h->d_zn, base->d_zn); borrow(h->d_zf, base->d_zf);
    borrow(h->d_zf64, base->d_zf64); borrow(h->d_reg2d, base->d_reg2d); borrow(h->d_len2d, base->d_len2d);
    borrow(h->d_len2d64, base->d_len2d64); borrow(h->d_segs, base->d_segs);
    borrow(h->d_fsr_mat, base->d_fsr_mat); borrow(h->d_order, base->d_order);
    borrow(h->d_tpl_off, base->d_tpl_off); borrow(h->d_tpl_loff, base->d_tpl_loff);
    borrow(h->d_tpl_lmin, base->d_tpl_lmin); borrow(h->d_tpl_lidx, base->d_tpl_lidx);
    borrow(h->d_dst, base->d_dst); borrow(h->d_perm, base->d_perm); borrow(h->d_win, base->d_win);
    borrow(h->d_chunk, base->d_chunk); borrow(h->d_vol, base->d_vol); borrow(h->d_inv_vol, base->d_inv_vol);
    borrow(h->d_sigt, base->d_sigt); borrow(h->d_sigt64, base->d_sigt64); borrow(h->d_sigs64, base->d_sigs64);
    borrow(h->d_nsf64, base->d_nsf64); borrow(h->d_chi64, base->d_chi64);
    borrow(h->d_inv_st64, base->d_inv_st64); borrow(h->d_siga64, base->d_siga64);
    borrow(h->d_lmap, base->d_lmap); borrow(h->d_reg_mat, base->d_reg_mat);
    borrow(h->d_zc0, base->d_zc0); borrow(h->d_zc1, base->d_zc1); borrow(h->d_zfd, base->d_zfd);
    borrow(h->d_zfd64, base->d_zfd64); borrow(h->d_pl_n, base->d_pl_n); borrow(h->d_pl_c, base->d_pl_c);
    borrow(h->d_pl_f, base->d_pl_f); borrow(h->d_pl_f64, base->d_pl_f64);
    // the solve state: its own
    TRY(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking), "stream");
    TRY(cudaMallocHost(&h->h_scal, SC_COUNT * sizeof(double)), "pinned scalars");
    if (ext_source) TRY(upload(h.get(), h->d_src64, h->geom.src), "upload");
    else borrow(h->d_src64, base->d_src64);
    const size_t nfg = (size_t)h->geom.nfsr * G, rs = real_size(h->precision);
    TRY(dalloc(h.get(), h->d_phi, nfg * 8), "alloc flux");
    TRY(dalloc(h.get(), h->d_qr, nfg * rs), "alloc source");
    TRY(dalloc(h.get(), h->d_tally, nfg * tally_entry_bytes(h.get())), "alloc tally");
    TRY(dalloc(h.get(), h->d_fiss, (size_t)h->geom.nfsr * 8), "alloc");
    TRY(dalloc(h.get(), h->d_fiss_old, (size_t)h->geom.nfsr * 8), "alloc");
    TRY(dalloc(h.get(), h->d_partial, (size_t)h->red_grid * 4 * 8), "alloc");
    TRY(dalloc(h.get(), h->d_scal, SC_COUNT * 8), "alloc");
    TRY(dalloc(h.get(), h->d_counter, 2 * sweep_block_bytes(h.get())), "alloc");
    if (h->has_psi) {
        TRY(dalloc(h.get(), h->d_psi[0], base->d_psi[0].n), "alloc boundary fluxes");
        TRY(dalloc(h.get(), h->d_psi[1], base->d_psi[1].n), "alloc boundary fluxes");
    }
    if (h->chunk_b > 0) TRY(dalloc(h.get(), h->d_hand, base->d_hand.n), "alloc chunk hand-off");
    fill_views(h.get());
    std::vector<double> init(SC_COUNT, 0.0);
    init[SC_EIGEN] = h->geom.src.empty() ? 1.0 : 0.0;
    init[SC_SCALE] = 1.0;
    init[SC_K] = 1.0;
    TRY(cudaMemcpyAsync(h->d_scal.p, init.data(), SC_COUNT * 8, cudaMemcpyHostToDevice, h->stream), "upload");
    const int rc = init_state(h.get());
    if (rc) return rc;
    h->owner = base;  // the hold taken above now belongs to the state
    hold.kept = true;
    *out = h.release();
    return MOC_OK;
}

extern "C" int moc_reset(moc_tracks *h) {
    if (!h) { moc_set_error("NULL handle"); return MOC_ERR_INVALID_ARG; }
    TRY(cudaSetDevice(h->device), "cudaSetDevice");
    return init_state(h);
}

extern "C" int moc_update_source(moc_tracks *h, double k, void *stream) {
    if (!h) { moc_set_error("NULL handle"); return MOC_ERR_INVALID_ARG; }
    TRY(cudaSetDevice(h->device), "cudaSetDevice");
    cudaStream_t s = stream ? (cudaStream_t)stream : h->stream;
    double kk = k;
    TRY(cudaMemcpyAsync((double *)h->d_scal.p + SC_K, &kk, 8, cudaMemcpyHostToDevice, s), "scalar");
    TRY(clear_conv(h, s), "scalar");
    TRY(launch_source(h->precision, h->dl, h->ds, h->geom.nfsr, h->red_grid, s), "source");
    TRY(cudaStreamSynchronize(s), "source");
    return MOC_OK;
}

extern "C" int moc_sweep(moc_tracks *h, void *stream) {
    if (!h) { moc_set_error("NULL handle"); return MOC_ERR_INVALID_ARG; }
    TRY(cudaSetDevice(h->device), "cudaSetDevice");
    cudaStream_t s = stream ? (cudaStream_t)stream : h->stream;
    TRY(clear_conv(h, s), "scalar");
    TRY(enqueue_sweep(h, s, h->cur), "sweep");
    if (h->has_psi) h->cur = 1 - h->cur;
    TRY(enqueue_finalize(h, s), "finalize");
    TRY(cudaMemcpyAsync(h->h_scal, h->d_scal.p, SC_COUNT * 8, cudaMemcpyDeviceToHost, s), "scalars");
    TRY(cudaStreamSynchronize(s), "sweep");
    return MOC_OK;
}

extern "C" int moc_enqueue_source(moc_tracks *h, void *stream) {
    if (!h) { moc_set_error("NULL handle"); return MOC_ERR_INVALID_ARG; }
    TRY(cudaSetDevice(h->device), "cudaSetDevice");
    cudaStream_t s = stream ? (cudaStream_t)stream : h->stream;
    TRY(clear_conv(h, s), "scalar");
    TRY(launch_source(h->precision, h->dl, h->ds, h->geom.nfsr, h->red_grid, s), "source");
    return MOC_OK;
}

extern "C" int moc_enqueue_sweep(moc_tracks *h, void *stream) {
    if (!h) { moc_set_error("NULL handle"); return MOC_ERR_INVALID_ARG; }
    TRY(cudaSetDevice(h->device), "cudaSetDevice");
    cudaStream_t s = stream ? (cudaStream_t)stream : h->stream;
    TRY(clear_conv(h, s), "scalar");
    TRY(enqueue_sweep(h, s, h->cur), "sweep");
    if (h->has_psi) h->cur = 1 - h->cur;
    return MOC_OK;
}

extern "C" int moc_enqueue_update(moc_tracks *h, void *stream) {
    if (!h) { moc_set_error("NULL handle"); return MOC_ERR_INVALID_ARG; }
    TRY(cudaSetDevice(h->device), "cudaSetDevice");
    cudaStream_t s = stream ? (cudaStream_t)stream : h->stream;
    TRY(clear_conv(h, s), "scalar");
    TRY(enqueue_finalize(h, s), "finalize");
    TRY(cudaMemcpyAsync(h->h_scal, h->d_scal.p, SC_COUNT * 8, cudaMemcpyDeviceToHost, s), "scalars");
    return MOC_OK;
}

extern "C" int moc_batch_step(moc_tracks *const *solves, int32_t n, void *stream) {
    if (!solves || n < 1) { moc_set_error("bad arguments"); return MOC_ERR_INVALID_ARG; }
    for (int i = 0; i < n; ++i)
        if (!solves[i]) { moc_set_error("NULL solve"); return MOC_ERR_INVALID_ARG; }
    moc_tracks *base = solves[0]->owner ? solves[0]->owner : solves[0];
    for (int i = 0; i < n; ++i) {
        const moc_tracks *o = solves[i]->owner ? solves[i]->owner : solves[i];
        if (o != base) { moc_set_error("moc_batch_step: the solves must share one layout"); return MOC_ERR_INVALID_ARG; }
        for (int k = 0; k < i; ++k)
            if (solves[k] == solves[i]) { moc_set_error("moc_batch_step: a solve appears twice"); return MOC_ERR_INVALID_ARG; }
    }
    TRY(cudaSetDevice(base->device), "cudaSetDevice");
    cudaStream_t s = stream ? (cudaStream_t)stream : solves[0]->stream;
    // one outer iteration each, no convergence test (like moc_iterate)
    for (int i = 0; i < n; ++i) {
        double *sc = (double *)solves[i]->d_scal.p;
        TRY(cudaMemsetAsync(sc + SC_CONV, 0, sizeof(double), s), "scalar");
        TRY(cudaMemsetAsync(sc + SC_TOLS, 0, sizeof(double), s), "scalar");
        TRY(cudaMemsetAsync(sc + SC_TOLK, 0, sizeof(double), s), "scalar");
    }
    if (!base->tally_smem || base->chunk_b > 0) {
        // the batched kernel needs whole units on the shared tally: one
        // iteration per solve instead
        for (int i = 0; i < n; ++i) {
            moc_tracks *h = solves[i];
            TRY(enqueue_iteration(h, s, h->cur), "iteration");
            if (h->has_psi) h->cur = 1 - h->cur;
        }
    } else {
        std::vector<BatchItem> it(n);
        for (int i = 0; i < n; ++i) {
            moc_tracks *h = solves[i];
            const int c = h->cur;
            it[i].qr = h->d_qr.p;
            it[i].tally = (double *)h->d_tally.p;
            it[i].scal = (double *)h->d_scal.p;
            it[i].psi_in = h->has_psi ? h->d_psi[c].p : nullptr;
            it[i].psi_out = h->has_psi ? h->d_psi[1 - c].p : nullptr;
        }
        if (base->d_batch.n < (size_t)n * sizeof(BatchItem)) {
            base->bytes -= base->d_batch.n;
            base->d_batch.release();
            TRY(dalloc(base, base->d_batch, (size_t)n * sizeof(BatchItem)), "alloc batch table");
        }
        TRY(cudaMemcpyAsync(base->d_batch.p, it.data(), (size_t)n * sizeof(BatchItem), cudaMemcpyHostToDevice, s),
            "upload");
        for (int i = 0; i < n; ++i) {
            moc_tracks *h = solves[i];
            TRY(launch_source(h->precision, h->dl, h->ds, h->geom.nfsr, h->red_grid, s), "source");
        }
        // one persistent sweep over the units of every solve
        moc_tracks *h0 = solves[0];
        int32_t *counter = sweep_counter(h0, h0->has_psi ? 1 - h0->cur : 0);
        TRY(cudaMemsetAsync(counter, 0, 4, s), "memset");
        TRY(launch_sweep_batch(base->precision, base->gpl, h0->dl, h0->ds, (const int32_t *)base->d_order.p,
                               (int32_t)base->order.size(), base->tile_cap, counter,
                               (const BatchItem *)base->d_batch.p, n, base->grid, base->block, base->smem, s),
            "batched sweep");
        for (int i = 0; i < n; ++i) {
            moc_tracks *h = solves[i];
            TRY(enqueue_finalize(h, s), "finalize");
            TRY(cudaMemcpyAsync(h->h_scal, h->d_scal.p, SC_COUNT * 8, cudaMemcpyDeviceToHost, s), "scalars");
            if (h->has_psi) h->cur = 1 - h->cur;
        }
    }
    TRY(cudaStreamSynchronize(s), "batch step");
    for (int i = 0; i < n; ++i) {
        const int rc = check_sweep_flag(solves[i]);
        if (rc) return rc;
    }
    return MOC_OK;
}

extern "C" int moc_read_result(moc_tracks *h, void *stream, moc_result *res) {
    if (!h || !res) { moc_set_error("NULL argument"); return MOC_ERR_INVALID_ARG; }
    TRY(cudaSetDevice(h->device), "cudaSetDevice");
    cudaStream_t s = stream ? (cudaStream_t)stream : h->stream;
    TRY(cudaStreamSynchronize(s), "synchronize");
    fill_result(h, res, 0.0, (int)h->h_scal[SC_ITER]);
    return check_sweep_flag(h);
}

extern "C" int moc_iterate(moc_tracks *h, int32_t n, int32_t use_graph, moc_result *res) {
    if (!h || n < 0) { moc_set_error("bad arguments"); return MOC_ERR_INVALID_ARG; }
    TRY(cudaSetDevice(h->device), "cudaSetDevice");
    // exactly n iterations: no convergence test, and a converged state resumes
    TRY(set_scalar(h, SC_TOLS, 0.0), "scalar");
    TRY(set_scalar(h, SC_CONV, 0.0), "scalar");
    return run_iterations(h, n, false, use_graph != 0, res);
}

static int solve(moc_tracks *h, const moc_solve_params *p, moc_result *res, bool eigen) {
    if (!h || !p || p->max_iter < 1) { moc_set_error("bad arguments"); return MOC_ERR_INVALID_ARG; }
    if (eigen != h->geom.src.empty()) {
        moc_set_error(eigen ? "moc_solve_eigen: the geometry has an external source"
                            : "moc_solve_fixed_source: the geometry has no external source");
        return MOC_ERR_INVALID_ARG;
    }
    int rc = init_state(h);
    if (rc) return rc;
    TRY(set_scalar(h, SC_TOLK, p->tol_k), "scalar");
    TRY(set_scalar(h, SC_TOLS, p->tol_src), "scalar");
    rc = run_iterations(h, p->max_iter, p->tol_src > 0, p->use_graph != 0, res);
    if (rc) return rc;
    if (p->tol_src > 0 && h->h_scal[SC_CONV] == 0.0) {
        moc_set_error("not converged within max_iter");
        return MOC_ERR_NOT_CONVERGED;
    }
    return MOC_OK;
}

extern "C" int moc_solve_eigen(moc_tracks *h, const moc_solve_params *p, moc_result *res) {
    return solve(h, p, res, true);
}

extern "C" int moc_solve_fixed_source(moc_tracks *h, const moc_solve_params *p, moc_result *res) {
    return solve(h, p, res, false);
}

extern "C" int moc_get_flux(moc_tracks *h, double *phi, double *k) {
    if (!h) { moc_set_error("NULL handle"); return MOC_ERR_INVALID_ARG; }
    TRY(cudaSetDevice(h->device), "cudaSetDevice");
    TRY(cudaMemcpyAsync(h->h_scal, h->d_scal.p, SC_COUNT * 8, cudaMemcpyDeviceToHost, h->stream), "copy");
    const size_t n = (size_t)h->geom.nfsr * h->geom.G;
    if (phi) TRY(cudaMemcpyAsync(phi, h->d_phi.p, n * 8, cudaMemcpyDeviceToHost, h->stream), "copy");
    TRY(cudaStreamSynchronize(h->stream), "copy");
    const double sc = h->h_scal[SC_SCALE];
    if (phi && sc != 1.0)
        for (size_t q = 0; q < n; ++q) phi[q] *= sc;
    if (k) *k = h->geom.src.empty() ? h->h_scal[SC_K] : 1.0;
    return MOC_OK;
}

extern "C" int moc_get_flux_device(moc_tracks *h, const double **phi, const double **scale,
                                   int64_t *n_fsr, int32_t *G) {
    if (!h || !phi) { moc_set_error("NULL argument"); return MOC_ERR_INVALID_ARG; }
    // no copy, no synchronisation: the library's own buffers, read-only for
    // the caller (phi is the flux iterate of Eq. 4; scale its normalisation)
    *phi = static_cast<const double *>(h->d_phi.p);
    if (scale) *scale = static_cast<const double *>(h->d_scal.p) + SC_SCALE;
    if (n_fsr) *n_fsr = h->geom.nfsr;
    if (G) *G = h->geom.G;
    return MOC_OK;
}

extern "C" int moc_set_flux(moc_tracks *h, const double *phi, double k) {
    if (!h || !phi) { moc_set_error("NULL argument"); return MOC_ERR_INVALID_ARG; }
    TRY(cudaSetDevice(h->device), "cudaSetDevice");
    const moc_geometry &g = h->geom;
    const size_t n = (size_t)g.nfsr * g.G;
    if (!all_nonneg(phi, n)) { moc_set_error("phi must be finite and non-negative"); return MOC_ERR_INVALID_ARG; }
    if (!(k > 0.0) || !std::isfinite(k)) { moc_set_error("k must be finite and positive"); return MOC_ERR_INVALID_ARG; }
    std::vector<double> fiss(g.nfsr, 0.0);
    double P = 0;
    for (int i = 0; i < g.nfsr; ++i) {
        const int m = g.fsr_mat[i];
        for (int gr = 0; gr < g.G; ++gr) fiss[i] += g.nsf[(size_t)m * g.G + gr] * phi[(size_t)i * g.G + gr];
        P += h->vol[i] * fiss[i];
    }
    const bool eig = g.src.empty();
    const double scale = (eig && P > 0) ? 1.0 / P : 1.0;
    for (auto &f : fiss) f *= scale;
    TRY(cudaMemcpyAsync(h->d_phi.p, phi, n * 8, cudaMemcpyHostToDevice, h->stream), "upload");
    TRY(cudaMemcpyAsync(h->d_fiss_old.p, fiss.data(), g.nfsr * 8, cudaMemcpyHostToDevice, h->stream), "upload");
    TRY(set_scalar(h, SC_SCALE, scale), "scalar");
    TRY(set_scalar(h, SC_K, k), "scalar");
    TRY(cudaStreamSynchronize(h->stream), "upload");
    return MOC_OK;
}

extern "C" int moc_get_volumes(moc_tracks *h, double *v) {
    if (!h || !v) { moc_set_error("NULL argument"); return MOC_ERR_INVALID_ARG; }
    std::memcpy(v, h->vol.data(), h->vol.size() * 8);
    return MOC_OK;
}

extern "C" int moc_tracks_info(const moc_tracks *h, int64_t *out, int32_t n) {
    if (!h || !out) { moc_set_error("NULL argument"); return MOC_ERR_INVALID_ARG; }
    const int64_t v[28] = {h->geom.nfsr, h->geom.G, h->L.nt, 2 * h->L.n_stacks, 2 * h->L.n_gtrk,
                           h->n_segments3d, (int64_t)h->integrations, h->n_stored, h->n_exp_stacks,
                           (int64_t)h->bytes, h->L.Nz, h->L.cpl, h->grid, h->block,
                           h->tally_smem ? MOC_TALLY_SHARED : MOC_TALLY_GLOBAL, h->precision,
                           (int64_t)h->smem, h->tile_cap, sweep_lanes_per_track(h->geom.G, h->gpl),
                           h->max_nseg, (int64_t)h->h2d, h->gpl, h->chunk_b, h->sync_b > 1 ? h->sync_b : 1,
                           h->n_slots, h->L.offlat,
                           (h->tally_smem && h->precision == MOC_FP32) ? h->tally_bits : 0, h->matk};
    for (int i = 0; i < n && i < 28; ++i) out[i] = v[i];
    return MOC_OK;
}

extern "C" int moc_get_segments2d(const moc_tracks *h, int32_t t, int64_t cap, int32_t *region,
                                  double *length, double *position, int64_t *n) {
    if (!h || !n) { moc_set_error("NULL argument"); return MOC_ERR_INVALID_ARG; }
    const Layout &L = h->L;
    if (t < 0 || t >= L.nt) { moc_set_error("2D track out of range"); return MOC_ERR_INVALID_ARG; }
    const int64_t a = L.seg_off[t], b = L.seg_off[t + 1];
    *n = b - a;
    if (cap < b - a) return MOC_OK;  // sizes only
    for (int64_t q = a; q < b; ++q) {
        if (region) region[q - a] = L.seg_reg[q];
        if (length) length[q - a] = L.seg_len[q];
        if (position) position[q - a] = L.seg_pos[q + t];
    }
    if (position) position[b - a] = L.seg_pos[b + t];
    return MOC_OK;
}

extern "C" int moc_get_stack_segments(moc_tracks *h, int32_t t, int32_t p, int64_t cap_tracks,
                                      int64_t cap_segments, int64_t *track_index, int32_t *n_seg,
                                      int32_t *fsr, double *length, int64_t *n_tracks,
                                      int64_t *n_segments) {
    if (!h) { moc_set_error("NULL handle"); return MOC_ERR_INVALID_ARG; }
    const Layout &L = h->L;
    if (t < 0 || t >= L.nt || p < 0 || p >= L.P) { moc_set_error("stack out of range"); return MOC_ERR_INVALID_ARG; }
    TRY(cudaSetDevice(h->device), "cudaSetDevice");
    const int64_t s = (int64_t)t * L.Ph + (p % L.Ph);
    const int frame = p < L.Ph ? 0 : 1;
    const StackDesc &d = L.desc[s];
    // per-track counts by the device generator
    DevBuf d_cnt;
    TRY(dalloc(h, d_cnt, (size_t)(d.n_trk + 1) * sizeof(int64_t)), "alloc");
    TRY(cudaMemsetAsync(d_cnt.p, 0, d_cnt.n, h->stream), "memset");
    TRY(launch_track_counts(h->dl, s, frame, (int64_t *)d_cnt.p, h->stream), "count");
    std::vector<int64_t> cnt(d.n_trk + 1, 0);
    TRY(cudaMemcpyAsync(cnt.data(), d_cnt.p, cnt.size() * 8, cudaMemcpyDeviceToHost, h->stream), "copy");
    TRY(cudaStreamSynchronize(h->stream), "count");
    h->bytes -= d_cnt.n;
    std::vector<int64_t> offs(d.n_trk + 1, 0);
    for (int k = 0; k < d.n_trk; ++k) offs[k + 1] = offs[k] + cnt[k + 1];
    const int64_t tot = offs[d.n_trk];
    *n_tracks = d.n_trk;
    *n_segments = tot;
    if (cap_tracks < d.n_trk || cap_segments < tot) {
        moc_set_error("capacity too small");
        return MOC_ERR_INVALID_ARG;
    }
    DevBuf d_offs, d_f, d_l;
    TRY(upload(h, d_offs, offs), "upload");
    TRY(dalloc(h, d_f, (size_t)std::max<int64_t>(tot, 1) * 4), "alloc");
    TRY(dalloc(h, d_l, (size_t)std::max<int64_t>(tot, 1) * 8), "alloc");
    TRY(launch_stack_segments(h->precision, h->dl, s, frame, (const int64_t *)d_offs.p, (int32_t *)d_f.p,
                              (double *)d_l.p, h->stream), "segments");
    std::vector<int32_t> f(tot);
    std::vector<double> l(tot);
    if (tot) {
        TRY(cudaMemcpyAsync(f.data(), d_f.p, tot * 4, cudaMemcpyDeviceToHost, h->stream), "copy");
        TRY(cudaMemcpyAsync(l.data(), d_l.p, tot * 8, cudaMemcpyDeviceToHost, h->stream), "copy");
    }
    TRY(cudaStreamSynchronize(h->stream), "copy");
    h->bytes -= d_offs.n + d_f.n + d_l.n;
    const int NL = L.nlv, NLr = h->geom.nl;
    const bool zero = L.zf[d.zoff] == 0.0f && L.zn[d.zoff] == 0;
    int64_t q = 0;
    for (int kk = 0; kk < d.n_trk; ++kk) {
        // frame D: list by increasing physical index = decreasing stored index
        const int k = frame == 0 ? kk : d.n_trk - 1 - kk;
        const int64_t j = d.i_lo + k;
        track_index[kk] = frame == 0 ? j : (int64_t)L.Nz - j - (zero ? 0 : 1);
        n_seg[kk] = (int32_t)(offs[k + 1] - offs[k]);
        for (int64_t a = offs[k]; a < offs[k + 1]; ++a, ++q) {
            // the device lists (region, sweep layer) of the upward frame; the
            // mirrored frame flips the layer, then the geometry's layer (planes
            // off the lattice: the frame's own pieces, the geometry's layers)
            const int reg = f[a] / NL, Lv = f[a] % NL;
            const int Lm = (frame == 1 && !L.offlat) ? NL - 1 - Lv : Lv;
            fsr[q] = reg * NLr + (L.lmap.empty() ? Lm : L.lmap[Lm]);
            length[q] = l[a];
        }
    }
    return MOC_OK;
}

extern "C" int moc_track_psi(moc_tracks *h, int32_t t, int32_t p, int64_t i, int32_t sense,
                             double *values, int32_t set) {
    if (!h || !values || sense < 0 || sense > 1) { moc_set_error("bad arguments"); return MOC_ERR_INVALID_ARG; }
    if (!h->has_psi) { moc_set_error("all faces are vacuum: no boundary fluxes are stored"); return MOC_ERR_UNSUPPORTED; }
    int64_t s, j;
    int frame;
    if (!map_track(h, t, p, i, s, frame, j)) { moc_set_error("track out of range"); return MOC_ERR_INVALID_ARG; }
    TRY(cudaSetDevice(h->device), "cudaSetDevice");
    const StackDesc &d = h->L.desc[s];
    const int G = h->geom.G;
    const int64_t gid = d.trk_off + (j - d.i_lo);
    const int v = frame * 2 + sense;
    const size_t rs = real_size(h->precision);
    char *base = (char *)h->d_psi[h->cur].p + ((size_t)(gid * 4 + v) * G) * rs;
    if (set && !all_nonneg(values, (size_t)G)) {
        moc_set_error("boundary flux values must be finite and non-negative");
        return MOC_ERR_INVALID_ARG;
    }
    TRY(cudaMemcpyAsync(h->h_scal, h->d_scal.p, SC_COUNT * 8, cudaMemcpyDeviceToHost, h->stream), "copy");
    TRY(cudaStreamSynchronize(h->stream), "copy");
    const double sc = h->h_scal[SC_SCALE];
    if (set) {
        if (rs == 8) {
            std::vector<double> tmp(G);
            for (int g = 0; g < G; ++g) tmp[g] = values[g] / sc;
            TRY(cudaMemcpy(base, tmp.data(), G * 8, cudaMemcpyHostToDevice), "copy");
        } else {
            std::vector<float> tmp(G);
            for (int g = 0; g < G; ++g) tmp[g] = (float)(values[g] / sc);
            TRY(cudaMemcpy(base, tmp.data(), G * 4, cudaMemcpyHostToDevice), "copy");
        }
    } else {
        if (rs == 8) {
            TRY(cudaMemcpy(values, base, G * 8, cudaMemcpyDeviceToHost), "copy");
            for (int g = 0; g < G; ++g) values[g] *= sc;
        } else {
            std::vector<float> tmp(G);
            TRY(cudaMemcpy(tmp.data(), base, G * 4, cudaMemcpyDeviceToHost), "copy");
            for (int g = 0; g < G; ++g) values[g] = tmp[g] * sc;
        }
    }
    return MOC_OK;
}

extern "C" int moc_sweep_from_source(moc_tracks *h, const double *Q, double *tally, double *leakage) {
    if (!h || !Q) { moc_set_error("NULL argument"); return MOC_ERR_INVALID_ARG; }
    TRY(cudaSetDevice(h->device), "cudaSetDevice");
    const moc_geometry &g = h->geom;
    const size_t n = (size_t)g.nfsr * g.G;
    if (!all_nonneg(Q, n)) { moc_set_error("Q must be finite and non-negative"); return MOC_ERR_INVALID_ARG; }
    const size_t rs = real_size(h->precision);
    std::vector<double> qr(n);
    for (int i = 0; i < g.nfsr; ++i)
        for (int gr = 0; gr < g.G; ++gr)
            qr[(size_t)i * g.G + gr] = Q[(size_t)i * g.G + gr] / g.sigt[(size_t)g.fsr_mat[i] * g.G + gr];
    if (rs == 8) {
        TRY(cudaMemcpyAsync(h->d_qr.p, qr.data(), n * 8, cudaMemcpyHostToDevice, h->stream), "upload");
        TRY(cudaStreamSynchronize(h->stream), "upload");
    } else {
        std::vector<float> q32(qr.begin(), qr.end());
        TRY(cudaMemcpyAsync(h->d_qr.p, q32.data(), n * 4, cudaMemcpyHostToDevice, h->stream), "upload");
        TRY(cudaStreamSynchronize(h->stream), "upload");
    }
    TRY(cudaMemsetAsync(h->d_tally.p, 0, h->d_tally.n, h->stream), "memset");
    TRY(set_scalar(h, SC_LEAK, 0.0), "scalar");
    TRY(clear_conv(h, h->stream), "scalar");
    TRY(enqueue_sweep(h, h->stream, h->cur), "sweep");
    if (h->has_psi) h->cur = 1 - h->cur;
    if (tally) TRY(tally_to_host(h, tally, n), "copy");
    TRY(cudaMemcpyAsync(h->h_scal, h->d_scal.p, SC_COUNT * 8, cudaMemcpyDeviceToHost, h->stream), "copy");
    TRY(cudaStreamSynchronize(h->stream), "sweep");
    if (leakage) *leakage = h->h_scal[SC_LEAK];
    if (check_sweep_flag(h)) return MOC_ERR_CUDA;
    TRY(cudaMemsetAsync(h->d_tally.p, 0, h->d_tally.n, h->stream), "memset");
    TRY(set_scalar(h, SC_LEAK, 0.0), "scalar");
    // the outgoing fluxes are physical values: the next sweep reads them as is
    TRY(set_scalar(h, SC_SCALE, 1.0), "scalar");
    TRY(cudaStreamSynchronize(h->stream), "sweep");
    return MOC_OK;
}

// ---------------------------------------------------------------------------
// Group-wise reaction rates with no allocation.  For callers that cannot
// allocate device memory when they need the rates: a serving loop that has
// handed the free HBM to resident solves (admission by footprint) would see
// cudaMalloc fail, and cudaFree can synchronise the whole device and stall
// the other solves' work.  The scratch is the library's static device array
// (moc_static.cu); its address is resolved once per device, with that device
// current, on the first call.

namespace {
constexpr int kRatesMaxDevices = 64;
std::mutex g_rates_mu;
double *g_rates_scratch_ptr[kRatesMaxDevices] = {};
}  // namespace

extern "C" int moc_group_rates_static(moc_tracks *h, void *stream, double *rates) {
    if (!h || !rates) { moc_set_error("NULL argument"); return MOC_ERR_INVALID_ARG; }
    const int G = h->geom.G;
    if (G > kRatesMaxGroups) {
        moc_set_error("moc_group_rates_static: at most 32 energy groups (fixed scratch of 128 blocks "
                      "x 32 groups x 2 rates)");
        return MOC_ERR_UNSUPPORTED;
    }
    if (h->device < 0 || h->device >= kRatesMaxDevices) {
        moc_set_error("moc_group_rates_static: device ordinal above 63");
        return MOC_ERR_UNSUPPORTED;
    }
    TRY(cudaSetDevice(h->device), "cudaSetDevice");
    double *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_rates_mu);
        if (!g_rates_scratch_ptr[h->device]) {
            double *p = nullptr;
            TRY(rates_scratch_address(&p), "cudaGetSymbolAddress");
            if (!p) { moc_set_error("cudaGetSymbolAddress returned NULL"); return MOC_ERR_CUDA; }
            g_rates_scratch_ptr[h->device] = p;
        }
        scratch = g_rates_scratch_ptr[h->device];
    }
    cudaStream_t s = stream ? (cudaStream_t)stream : h->stream;
    TRY(launch_group_rates_static(h->dl, h->ds, h->geom.nfsr, scratch, s), "rates");
    TRY(cudaMemcpyAsync(rates, scratch + kRatesResultOffset, 2 * (size_t)G * sizeof(double),
                        cudaMemcpyDeviceToHost, s), "copy");
    TRY(cudaStreamSynchronize(s), "rates");
    return MOC_OK;
}

extern "C" int moc_sweep_units_from_source(moc_tracks *h, const double *Q, int32_t t0, int32_t t1,
                                           double *tally, double *leakage) {
    if (!h || !Q || !tally) { moc_set_error("NULL argument"); return MOC_ERR_INVALID_ARG; }
    if (t0 < 0 || t1 > h->L.nt || t0 > t1) { moc_set_error("2D track range out of bounds"); return MOC_ERR_INVALID_ARG; }
    TRY(cudaSetDevice(h->device), "cudaSetDevice");
    const moc_geometry &g = h->geom;
    const size_t n = (size_t)g.nfsr * g.G;
    if (!all_nonneg(Q, n)) { moc_set_error("Q must be finite and non-negative"); return MOC_ERR_INVALID_ARG; }
    std::vector<double> qr(n);
    for (int i = 0; i < g.nfsr; ++i)
        for (int gr = 0; gr < g.G; ++gr)
            qr[(size_t)i * g.G + gr] = Q[(size_t)i * g.G + gr] / g.sigt[(size_t)g.fsr_mat[i] * g.G + gr];
    if (real_size(h->precision) == 8) {
        TRY(cudaMemcpyAsync(h->d_qr.p, qr.data(), n * 8, cudaMemcpyHostToDevice, h->stream), "upload");
        TRY(cudaStreamSynchronize(h->stream), "upload");
    } else {
        std::vector<float> q32(qr.begin(), qr.end());
        TRY(cudaMemcpyAsync(h->d_qr.p, q32.data(), n * 4, cudaMemcpyHostToDevice, h->stream), "upload");
        TRY(cudaStreamSynchronize(h->stream), "upload");
    }
    std::vector<int32_t> units;
    for (int32_t t : h->order)
        if (t >= t0 && t < t1) units.push_back(t);
    DevBuf d_units;
    TRY(upload(h, d_units, units.empty() ? std::vector<int32_t>(1, 0) : units), "upload");
    TRY(cudaMemsetAsync(h->d_tally.p, 0, h->d_tally.n, h->stream), "memset");
    TRY(set_scalar(h, SC_LEAK, 0.0), "scalar");
    TRY(set_scalar(h, SC_SCALE, 1.0), "scalar");
    TRY(clear_conv(h, h->stream), "scalar");
    const int out = h->has_psi ? 1 - h->cur : 0;
    TRY(cudaMemsetAsync(sweep_counter(h, out), 0, 4, h->stream), "memset");
    void *pout = h->has_psi ? h->d_psi[1 - h->cur].p : nullptr;
    TRY(launch_sweep(h->precision, h->tally_smem, h->gpl, h->dl, h->ds, (const int32_t *)d_units.p,
                     (int32_t)units.size(), h->tile_cap, nullptr, pout, sweep_counter(h, out), h->grid,
                     h->block, h->smem, h->stream),
        "sweep");
    TRY(tally_to_host(h, tally, n), "copy");
    TRY(cudaMemcpyAsync(h->h_scal, h->d_scal.p, SC_COUNT * 8, cudaMemcpyDeviceToHost, h->stream), "copy");
    TRY(cudaStreamSynchronize(h->stream), "sweep");
    h->bytes -= d_units.n;
    if (leakage) *leakage = h->h_scal[SC_LEAK];
    if (check_sweep_flag(h)) return MOC_ERR_CUDA;
    TRY(cudaMemsetAsync(h->d_tally.p, 0, h->d_tally.n, h->stream), "memset");
    TRY(set_scalar(h, SC_LEAK, 0.0), "scalar");
    TRY(cudaStreamSynchronize(h->stream), "sweep");
    return MOC_OK;
}

// ---------------------------------------------------------------------------
// Pieces of a solve for the serving engine (moc_server.cu): start a solve,
// enqueue iterations without waiting, read the state once the stream is idle.
// A converged solve's later iterations are no-ops on the device, so how many
// iterations the engine enqueues between looks does not change the result.

int tracks_start_solve(moc_tracks *h, const moc_solve_params *p) {
    if (!h || !p || p->max_iter < 1) { moc_set_error("bad arguments"); return MOC_ERR_INVALID_ARG; }
    TRY(cudaSetDevice(h->device), "cudaSetDevice");
    int rc = init_state(h);
    if (rc) return rc;
    TRY(set_scalar(h, SC_TOLK, p->tol_k), "scalar");
    TRY(set_scalar(h, SC_TOLS, p->tol_src), "scalar");
    TRY(build_graphs(h), "graph capture");
    return MOC_OK;
}

int tracks_enqueue_iterations(moc_tracks *h, int n, cudaEvent_t done) {
    TRY(cudaSetDevice(h->device), "cudaSetDevice");
    for (int i = 0; i < n; ++i) {
        TRY(cudaGraphLaunch(h->graph[h->cur], h->stream), "graph launch");
        if (h->has_psi) h->cur = 1 - h->cur;
    }
    TRY(cudaEventRecord(done, h->stream), "event");
    return MOC_OK;
}

int tracks_read_state(moc_tracks *h, moc_result *res, int *converged) {
    // the scalars were copied to the pinned mirror by the last iteration
    const int done = (int)h->h_scal[SC_ITER];
    *converged = h->h_scal[SC_CONV] != 0.0 ? 1 : 0;
    if (*converged && h->has_psi) h->cur = done & 1;
    fill_result(h, res, 0.0, done);
    return check_sweep_flag(h);
}
