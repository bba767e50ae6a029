/*
 * moc.h -- C ABI of the GB300 3D method-of-characteristics transport sweep.
 *
 * The library solves the multigroup neutron transport equation (Eq. 1 of
 * "Neutron particle transport 3D method of characteristic Multi GPU platform
 * Parallel Computing", arXiv 2503.17743) on an axially extruded pin lattice
 * with the method of characteristics: 2D cyclic tracks are expanded on the
 * GPU into axially stacked 3D tracks (Sec. 2.2, Eqs. 5-11), every segment is
 * attenuated per group and polar angle with the flat-source solution (Eq. 3)
 * and tallied into flat-source-region (FSR) scalar fluxes (Eq. 4), inside a
 * power iteration for k-eff (Sec. 3.1, "iterative solving").
 *
 * Conventions for every entry point:
 *   - Every call returns MOC_OK (0) or one of the MOC_ERR_* codes below;
 *     moc_last_error() returns a thread-local message for the last failure.
 *   - All pointers in descriptors are HOST pointers; the library copies what
 *     it needs during the call and never keeps a caller pointer.
 *   - Handles are opaque and owned by the library; each create/generate has
 *     a destroy.  Device memory is allocated by the library with cudaMalloc
 *     on the device named in moc_track_params.device.
 *   - `stream` arguments are cudaStream_t values passed as void*; NULL means
 *     the handle's own stream.  Calls that return results to host memory
 *     synchronise that stream before returning.
 *   - Arrays indexed by FSR use the FSR numbering of the geometry: radial
 *     regions numbered cell by cell (cell c = cy*ncx + cx; a pin cell has the
 *     region inside the circle then the moderator around it, any other cell
 *     one region), FSR = region * n_layers + layer.  Group index is fastest:
 *     phi[fsr * G + g].
 */
#ifndef MOC3D_MOC_H
#define MOC3D_MOC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define MOC_OK 0
#define MOC_ERR_INVALID_ARG 1
#define MOC_ERR_OUT_OF_MEMORY 2
#define MOC_ERR_CUDA 3
#define MOC_ERR_NOT_CONVERGED 4
#define MOC_ERR_TIMEOUT 5
#define MOC_ERR_UNSUPPORTED 6

/* moc_track_params.schedule flags (load balancing, Sec. 4.3; default 0 uses both) */
#define MOC_SCHED_UNITS_NATURAL 1   /* work units (2D tracks) in index order, not largest first */
#define MOC_SCHED_TRACKS_NATURAL 2  /* a stack's tracks in index order, not by segment count */
/* the shared rows of the FP32 sweep carry Sigma_t beside Qr even where the
 * stored segments could carry their material (see moc_tracks_info entry 27) */
#define MOC_SCHED_ROWS_WITH_SIGMA 4

/* arithmetic of the sweep */
#define MOC_FP32 0
#define MOC_FP64 1

/* FSR tally strategy of the sweep kernel */
#define MOC_TALLY_AUTO 0   /* FP32: shared-memory tile (radial chunks if needed); FP64: global */
#define MOC_TALLY_SHARED 1 /* per-stack tile privatised in shared memory, flushed in FP64 */
#define MOC_TALLY_GLOBAL 2 /* atomics straight into the FP64 global tally */

typedef struct moc_geometry moc_geometry;
typedef struct moc_tracks moc_tracks;

/* Axially extruded pin lattice (Sec. 2.2: every axial plane has the same
 * radial geometry; materials may change from layer to layer).
 *   ncx, ncy      cells along x and y, square cells of side `pitch` (cm)
 *   fuel_radius   radius (cm) of the circle of a pin cell, < pitch/2
 *   height        axial extent (cm), split into n_layers equal layers
 *   has_pin       [ncy*ncx] 1 = cell holds a pin (circle), 0 = one region
 *   mat_in        [ncy*ncx*n_layers] material inside the circle, per layer
 *   mat_out       [ncy*ncx*n_layers] material outside the circle (whole cell
 *                 for has_pin = 0), per layer
 *   bc            faces xmin, xmax, ymin, ymax, zmin, zmax: 1 reflective, 0 vacuum
 *   fuel_rings    finer flat source regions of a pin cell (0 is read as 1):
 *                 rings of equal area inside the fuel circle,
 *   moderator_rings  (0 or more) circles of equal area steps between the
 *                 fuel circle and the cell's inscribed circle (radius pitch/2,
 *                 itself not a boundary),
 *   sectors       (0 is read as 1) equal angular sectors about the cell
 *                 centre, sector s covering [2 pi s / S, 2 pi (s+1) / S)
 *                 counterclockwise from +x, applied to every ring and to the
 *                 region outside the last circle.
 * Radial regions are numbered cell by cell; within a pin cell region
 * ring * sectors + sector, rings from the centre outwards and the region
 * outside every circle last.  Rings inside the fuel circle take mat_in, the
 * others mat_out.  With 1, 0, 1 a pin cell has two regions (circle, then
 * moderator).  Cells without a pin stay one region.
 *   layer_z       NULL (n_layers equal layers) or [n_layers + 1] layer planes
 *                 rising from 0 to height: unequal layers (the local axial
 *                 mesh of Sec. 2.2).  Planes may lie anywhere on the axial
 *                 line: when every plane is a whole number of axial spacings
 *                 the sweep uses segment templates and the shared tally;
 *                 otherwise (also equal layers that are not whole spacings)
 *                 each track direction is generated on its own against the
 *                 planes (ties of a track end with a plane decided exactly,
 *                 within 1e-10 of a spacing) and tallied into the FP64 FSR
 *                 tally; a plane within 1e-9 of a spacing is on it. */
typedef struct {
    int32_t ncx, ncy;
    double pitch, fuel_radius, height;
    int32_t n_layers;
    const int32_t *has_pin;
    const int32_t *mat_in;
    const int32_t *mat_out;
    int32_t bc[6];
    int32_t fuel_rings, moderator_rings, sectors;
    const double *layer_z;
} moc_geometry_desc;

/* Multigroup macroscopic cross sections (1/cm), host arrays:
 *   sigma_t     [M*G]     total
 *   sigma_s     [M*G*G]   scattering from group g into group h at [m][g][h]
 *   nu_sigma_f  [M*G]     nu times fission
 *   chi         [M*G]     fission spectrum
 *   ext_source  [M*G]     isotropic volumetric source density, or NULL */
typedef struct {
    int32_t num_materials, num_groups;
    const double *sigma_t;
    const double *sigma_s;
    const double *nu_sigma_f;
    const double *chi;
    const double *ext_source;
} moc_materials;

/* Track layout and sweep configuration.
 *   n_azim             azimuthal angles over [0, 2 pi), multiple of 4
 *   n_polar            polar angles over (0, pi), even (Gauss-Legendre in
 *                      cos(theta), n_polar/2 per hemisphere)
 *   radial_spacing     desired 2D track spacing (cm); corrected for cycles
 *   axial_spacing      desired z-stack spacing dz (cm, Eq. 5); the layer
 *                      height must be a whole number of spacings
 *   precision          MOC_FP32 or MOC_FP64 sweep arithmetic
 *   preload_budget_bytes  device bytes for stored (EXP) segments, Sec. 4.2:
 *                      < 0 store every segment, 0 generate every segment on
 *                      the fly (OTF), > 0 store the largest stacks first
 *                      until the budget is used
 *   tally_mode         MOC_TALLY_*
 *   block_threads      threads per block of the sweep (0 = tuned default)
 *   blocks_per_sm      resident sweep blocks per SM (0 = occupancy maximum)
 *   device             CUDA device ordinal
 *   groups_per_lane    energy groups one thread carries along a track: 1, 2
 *                      or 4 (2 and 4 for FP32 sweeps only; 0 = tuned default)
 *   schedule           0, or MOC_SCHED_* flags that switch off a load-balancing
 *                      step (Sec. 4.3) or the material-keyed rows, for ablations
 *   chunk_segments     shared tally only: sweep a unit (2D track) in radial
 *                      chunks of at most this many 2D segments; 0 = only the
 *                      units whose tile does not fit in shared memory, in the
 *                      largest chunks that keep three blocks per SM.  A
 *                      track's psi passes from chunk to chunk; results equal
 *                      the whole-unit sweep up to FP rounding.
 *   trace_on_device    1: trace the 2D tracks through the lattice on the GPU
 *                      (one thread per track; the same pieces as the host
 *                      tracer, bit for bit), 0: on the host (Sec. 3.1).
 *   sync_block         warp schedule of the stored (EXP) stacks, FP32 sweeps
 *                      with two groups per lane, shared tally, units swept
 *                      whole: 1 = each track of a warp walks its own records
 *                      (tracks by decreasing segment count); 4 or 8 = blocks
 *                      of that many tracks of one segment template (tracks
 *                      r + m cpl, consecutive m) step through the
 *                      template's records together, so that their tally rows
 *                      are consecutive (no shared-memory bank conflicts) and
 *                      the record is read once per block, at the price of idle
 *                      tracks where the block's windows do not overlap; 0 = the
 *                      default, 1 (the autotuner times 1, 4 and 8).  Other
 *                      layouts ignore it. */
typedef struct {
    int32_t n_azim, n_polar;
    double radial_spacing, axial_spacing;
    int32_t precision;
    int64_t preload_budget_bytes;
    int32_t tally_mode;
    int32_t block_threads;
    int32_t blocks_per_sm;
    int32_t device;
    int32_t groups_per_lane;
    int32_t schedule;
    int32_t chunk_segments;
    int32_t trace_on_device;
    int32_t sync_block;
} moc_track_params;

/* Stopping rule of a solve: |k_n - k_(n-1)| < tol_k (eigenvalue problems
 * only) and residual < tol_src, or max_iter iterations.  tol_src <= 0 runs
 * exactly max_iter iterations.  use_graph = 1 captures one outer iteration
 * as a CUDA graph and replays it. */
typedef struct {
    double tol_k, tol_src;
    int32_t max_iter;
    int32_t use_graph;
} moc_solve_params;

/* Result of a solve or of moc_iterate. */
typedef struct {
    double k;               /* k-eff (1 for fixed-source problems) */
    double residual;        /* RMS relative change of the fission source (eigen) or flux (fixed) */
    double dk;              /* k change over the last iteration */
    double production;      /* sum V nu-Sigma_f phi of the normalised flux */
    double absorption;      /* sum V Sigma_a phi */
    double leakage;         /* outgoing weighted flux at vacuum faces, last sweep */
    double seconds;         /* device time of the iterations */
    double integrations;    /* segment-group integrations performed */
    int32_t iterations;
    int32_t converged;
} moc_result;

/* thread-local message of the last error */
const char *moc_last_error(void);

/* Create a geometry from a lattice and cross sections (host only, no GPU
 * work).  Errors: MOC_ERR_INVALID_ARG for NULL arrays, non-positive or NaN
 * Sigma_t, negative cross sections, scattering row sums >= Sigma_t, material
 * indices out of range, a circle that does not fit its cell. */
int moc_create_geometry(const moc_geometry_desc *desc, const moc_materials *mat,
                        moc_geometry **out);
void moc_destroy_geometry(moc_geometry *geom);

/* Device bytes moc_generate_tracks would allocate for this layout, without
 * allocating (host work only): `resident` excludes stored segments,
 * `preload_all` is the extra for storing every segment. */
int moc_query_footprint(const moc_geometry *geom, const moc_track_params *params,
                        int64_t *resident, int64_t *preload_all);

/* 2D cyclic tracking on the host (Sec. 3.1 keeps it on the CPU), z-stack
 * tables (Sec. 3.2 Z-STACK), then on the device: per-track segment counts,
 * the preload plan (Sec. 4.2) and the stored segments, tracked FSR volumes,
 * and the initial state (phi = 1, boundary fluxes 0, k = 1).  Errors:
 * MOC_ERR_UNSUPPORTED when a problem with reflective faces has more than
 * 2^29 3D tracks (link destinations are 32-bit track-direction indices),
 * more than 32 polar angles are asked for, or layer planes off the axial
 * lattice have more than 4000 distinct fractions of a spacing,
 * MOC_ERR_OUT_OF_MEMORY when the device cannot hold the state, MOC_ERR_CUDA on
 * a CUDA failure. */
int moc_generate_tracks(const moc_geometry *geom, const moc_track_params *params,
                        moc_tracks **out);
void moc_destroy_tracks(moc_tracks *tracks);

/* One transport sweep (Eq. 3 on every segment, both directions, all groups
 * and polar angles; tallies of Eq. 4) from the current source, followed by
 * the scalar-flux update phi = (4 pi Q + tally / V) / Sigma_t.  Boundary
 * fluxes advance by one Jacobi step. */
int moc_sweep(moc_tracks *tracks, void *stream);

/* Isotropic source from the current flux:
 * Q = (sum_h Sigma_s[h->g] phi_h + chi_g / k * sum_h nuSigma_f,h phi_h + S_g) / (4 pi). */
int moc_update_source(moc_tracks *tracks, double k, void *stream);

/* Power iteration to convergence (eigenvalue problem; the geometry must have
 * no external source).  Returns MOC_ERR_NOT_CONVERGED (with `res` filled)
 * when max_iter is reached first. */
int moc_solve_eigen(moc_tracks *tracks, const moc_solve_params *params, moc_result *res);

/* Source iteration to convergence of a fixed-source problem (the geometry
 * must have an external source). */
int moc_solve_fixed_source(moc_tracks *tracks, const moc_solve_params *params,
                           moc_result *res);

/* Reset the state to phi = 1, zero boundary fluxes, k = 1. */
int moc_reset(moc_tracks *tracks);

/* Run exactly n outer iterations (source, sweep, flux update, k update) from
 * the current state; eigenvalue or fixed-source by the geometry. */
int moc_iterate(moc_tracks *tracks, int32_t n, int32_t use_graph, moc_result *res);

/* Non-blocking pieces of one outer iteration, enqueued on `stream` (NULL: the
 * handle's stream) in this order: the source update (moc_update_source with
 * the device-resident k), one sweep (Eq. 3 / Eq. 4 tallies, boundary fluxes
 * advance one Jacobi step), and the flux, k and residual update (FP64
 * reductions; the scalars are copied to a pinned host mirror).  They return
 * after enqueueing; moc_read_result synchronises `stream` and fills `res`
 * (seconds = 0, iterations = outer iterations so far, integrations = those of
 * that many sweeps).  Errors: MOC_ERR_INVALID_ARG for NULL, MOC_ERR_CUDA. */
int moc_enqueue_source(moc_tracks *tracks, void *stream);
int moc_enqueue_sweep(moc_tracks *tracks, void *stream);
int moc_enqueue_update(moc_tracks *tracks, void *stream);
int moc_read_result(moc_tracks *tracks, void *stream, moc_result *res);

/* Copy the normalised scalar flux [n_fsr*G] (FP64, host) and k. */
int moc_get_flux(moc_tracks *tracks, double *phi, double *k);

/* The scalar flux where it lives on the device, without a copy: for a
 * consumer on the same device (a PyTorch tensor made from the pointer, a
 * caller's kernel) that should not round-trip through host memory.
 *   phi    out: device pointer to phi[n_fsr*G] (FP64, group fastest), the
 *          flux iterate of the Eq. 4 update before normalisation
 *   scale  out (may be NULL): device pointer to one FP64 value; the
 *          normalised flux (what moc_get_flux returns) is phi * (*scale)
 *          (1 for fixed-source problems, 1 / production for eigenvalue
 *          problems)
 *   n_fsr, G  out (may be NULL): the array's shape
 * Both buffers are owned by the library and READ-ONLY for the caller.  They
 * stay allocated until the handle is destroyed; their values change with
 * every outer iteration, so read them on the handle's stream (or after
 * synchronising it) and before the next iteration is enqueued.  No GPU work
 * and no synchronisation happen in the call.  Errors: MOC_ERR_INVALID_ARG for
 * NULL tracks or phi. */
int moc_get_flux_device(moc_tracks *tracks, const double **phi, const double **scale,
                        int64_t *n_fsr, int32_t *G);

/* Set the scalar flux [n_fsr*G] and k (host FP64 input).  Errors:
 * MOC_ERR_INVALID_ARG for NULL, a flux value negative or not finite, k not
 * positive. */
int moc_set_flux(moc_tracks *tracks, const double *phi, double k);

/* Tracked FSR volumes [n_fsr] (FP64, host). */
int moc_get_volumes(moc_tracks *tracks, double *volumes);

/* A second, independent solve on the layout of `tracks` (Sec. 4.2: the
 * stored segments, links and tables are shared, not copied): its own flux,
 * source, boundary fluxes and scalars, in the initial state.  ext_source
 * [M*G] (host, copied; NULL = the geometry's own) gives it a different
 * external source, which makes it a fixed-source problem.  The returned
 * handle is a moc_tracks and takes every call a moc_tracks takes; it holds a
 * host copy of the layout tables.  Destroy it with moc_state_destroy (or
 * moc_destroy_tracks); the layout's memory lives until its owner and all its
 * states are destroyed.  Errors: MOC_ERR_INVALID_ARG (NULL, a source value
 * negative or not finite, an owner already destroyed), MOC_ERR_OUT_OF_MEMORY,
 * MOC_ERR_CUDA. */
int moc_state_create(const moc_tracks *tracks, const double *ext_source, moc_tracks **state);
void moc_state_destroy(moc_tracks *state);

/* One outer iteration (source, sweep, flux / k update, Sec. 5.1) of each of n
 * solves that share one layout (the moc_tracks and its states), with the
 * sweeps of all of them in ONE persistent launch whose work list takes every
 * unit of every solve, the solves' units interleaved, largest first.  Like
 * moc_iterate(solve, 1): no convergence test, and a converged solve resumes.
 * Layouts without the shared tally, or with radially chunked units, run one
 * iteration per solve instead.  Enqueued on `stream` (NULL: the first
 * solve's stream) and synchronised before returning.  Calls on solves of one
 * layout must not overlap in time (they share the batch table).  Errors:
 * MOC_ERR_INVALID_ARG (NULL, n < 1, a solve twice, different layouts),
 * MOC_ERR_CUDA. */
int moc_batch_step(moc_tracks *const *solves, int32_t n, void *stream);

/* The 2D segments of 2D track t (Sec. 3.1 ray tracing, host copy): *n
 * segments; when cap >= *n, region[*n], length[*n] (cm) and position[*n + 1]
 * (distance of each boundary from the track's start, the last = its length)
 * are written (each may be NULL).  Errors: MOC_ERR_INVALID_ARG (NULL n, t
 * out of range). */
int moc_get_segments2d(const moc_tracks *tracks, int32_t t, int64_t cap, int32_t *region,
                       double *length, double *position, int64_t *n);

/* Layout counts, int64 values written to out[0..n-1]:
 *   0 n_fsr, 1 groups, 2 2D tracks, 3 z-stacks (both hemispheres), 4 3D tracks,
 *   5 3D segments, 6 segment-group integrations per sweep, 7 stored segments,
 *   8 preloaded stacks, 9 device bytes held, 10 axial lattice cells Nz,
 *   11 lattice cells per layer, 12 sweep blocks, 13 sweep threads per block,
 *   14 tally mode in use, 15 precision, 16 sweep shared memory bytes per block,
 *   17 shared tile entries, 18 lanes per track, 19 most segments on one
 *   track, 20 bytes copied host to device while generating, 21 energy
 *   groups per lane, 22 2D segments per radial chunk (0: no unit is
 *   chunked), 23 tracks per synchronous block of the stored stacks (1: none,
 *   see moc_track_params.sync_block), 24 sweep slots (tracks plus the
 *   padding of synchronous blocks), 25 1 when layer planes lie off the
 *   axial lattice (11 is then 0), 26 fixed-point bits of the FP32 shared
 *   tally per unit bound (0: not used), 27 1 when the stored segments carry
 *   their material and the shared rows hold Qr only (FP32, two groups per
 *   lane, shared tally, every unit stored, no synchronous blocks, one
 *   material per radial region, at most 4 materials; Sigma_t then comes from
 *   the material table) */
int moc_tracks_info(const moc_tracks *tracks, int64_t *out, int32_t n);

/* 3D segments of z-stack (t, p) as the device generator produces them
 * (lengths in the sweep's precision, returned as FP64):
 * t = 2D track, p = polar index in [0, n_polar) (p < n_polar/2 upward, p - n_polar/2
 * the downward mirror).  Tracks are listed by their lattice index i (the
 * track whose height at the start of t is z_0 + i dz with 0 <= z_0 < dz), in
 * increasing i; segments in traversal order along t.  Capacities are in
 * elements; on return *n_tracks and *n_segments hold the sizes (also when a
 * capacity was too small, with MOC_ERR_INVALID_ARG). */
int moc_get_stack_segments(moc_tracks *tracks, int32_t t, int32_t p, int64_t cap_tracks,
                           int64_t cap_segments, int64_t *track_index, int32_t *n_seg,
                           int32_t *fsr, double *length, int64_t *n_tracks,
                           int64_t *n_segments);

/* Incoming boundary flux of one track direction (t, p, i, sense = 0 along t,
 * 1 against it) for the next sweep, get (set = 0) or set (set = 1), G values
 * (set: finite and non-negative, else MOC_ERR_INVALID_ARG). */
int moc_track_psi(moc_tracks *tracks, int32_t t, int32_t p, int64_t i, int32_t sense,
                  double *values, int32_t set);

/* Sweep from a caller-given source Q [n_fsr*G] (per steradian, host FP64,
 * finite and non-negative, else MOC_ERR_INVALID_ARG) with the current
 * boundary fluxes; returns the FSR tally [n_fsr*G] and leakage. */
int moc_sweep_from_source(moc_tracks *tracks, const double *Q, double *tally, double *leakage);

/* One sweep of only the 2D tracks t in [t0, t1) (every polar angle, both
 * senses) from the isotropic source Q [n_fsr*G] (per steradian, FP64, host)
 * with zero incoming boundary fluxes: a bounded sample of a sweep that an
 * oracle can reproduce on large problems (Q finite and non-negative, else
 * MOC_ERR_INVALID_ARG).  tally [n_fsr*G] (host, FP64) gets
 * sum over those tracks' segments of W (psi_in - psi_out) (Eq. 4 before the
 * division by volume); *leakage (may be NULL) their W psi leaving through
 * vacuum faces.  Afterwards the stored boundary fluxes are undefined: call
 * moc_reset before iterating.  Errors: MOC_ERR_INVALID_ARG (NULL, range
 * outside [0, 2D tracks]), MOC_ERR_CUDA. */
int moc_sweep_units_from_source(moc_tracks *tracks, const double *Q, int32_t t0, int32_t t1,
                                double *tally, double *leakage);

/* Group-wise reaction rates of the normalised scalar flux (the flux
 * moc_get_flux returns), computed on the device without allocating any
 * memory.  The paper has no counterpart: it is a library service for callers
 * that cannot allocate device memory at that moment (for example a serving
 * loop that has handed the free HBM to resident solves).
 *   rates   host array of 2*G doubles, written on return:
 *           rates[g]     = sum_i V_i nuSigma_f[m_i][g] phi_{i,g}
 *           rates[G + g] = sum_i V_i (Sigma_t - sum_h Sigma_s[g->h])[m_i] phi_{i,g}
 *           (their sums are moc_result.production and .absorption)
 *   stream  cudaStream_t as void*, NULL = the handle's stream; the call
 *           synchronises it before returning.
 * Scratch: a fixed device array inside the library (8256 doubles, 66 KB per
 * device) instead of an allocation; nothing in it has to start at zero.  Limit:
 * G <= 32 (MOC_ERR_UNSUPPORTED beyond).  The first call on each device
 * resolves the scratch address (cudaGetSymbolAddress, with that device
 * current); make that first call before any stream capture begins.  Every
 * call synchronises `stream` and copies the rates into host memory before
 * it returns.  Calls that overlap in time (two streams or two host threads)
 * share the scratch and race: serialise them.  Errors: MOC_ERR_INVALID_ARG for NULL,
 * MOC_ERR_UNSUPPORTED, MOC_ERR_CUDA. */
int moc_group_rates_static(moc_tracks *tracks, void *stream, double *rates);

/* Sustained rate of the device's exponential unit (ex2.approx.ftz.f32, one
 * per integration of Eq. 3): 8 independent chains per thread on every SM,
 * the last of three runs timed with CUDA events.  Measurement support for
 * the sweep's ALU roofline; the paper has no counterpart.  Allocates and
 * frees a small device buffer.
 *   ex2_per_second  out: exponentials per second over the whole device
 *   sm_count        out (may be NULL): multiprocessors of the device
 * Errors: MOC_ERR_INVALID_ARG for NULL, MOC_ERR_CUDA. */
int moc_measure_ex2_rate(int32_t device, double *ex2_per_second, double *sm_count);

/* Sustained throughput of the other units the FP32 sweep issues to, each
 * probed by its own kernel (8 independent operations per thread and step,
 * 8 blocks of 256 threads on every SM, the last of three runs timed with
 * CUDA events).  Measurement support for the sweep's roofline; the paper has
 * no counterpart.  Allocates and frees a small device buffer.
 *   out[0]  multiprocessors of the device
 *   out[1]  SM clock (MHz) during the scalar FMA run (clock64 over its time)
 *   out[2]  FP32 fused multiply-adds per second, scalar (fma.rn.f32),
 *           counted as lane operations
 *   out[3]  FP32 lane operations per second as packed pairs
 *           (fma.rn.f32x2, two per lane and instruction)
 *   out[4]  conflict-free shared-memory 32-bit integer reductions per second
 *           (red.shared.add.s32, 32 banks per warp instruction)
 *   out[5]  conflict-free shared-memory load bytes per second (16-byte loads,
 *           512 contiguous bytes per warp instruction)
 *   out[6]  float-to-integer conversions with rounding per second
 *           (cvt.rni.s32.f32)
 *   n       entries of out to write (at most 7)
 * Errors: MOC_ERR_INVALID_ARG for NULL or n < 1, MOC_ERR_CUDA. */
int moc_measure_unit_rates(int32_t device, double *out, int32_t n);

/* The attenuation factor e^{-x} of Eq. 3 as the FP64 sweep computes it
 * (table-driven: 2^{j/64} in hi + lo parts, degree-5 polynomial on
 * |r| <= ln2/128; within 1 ulp for |x| < 700, 0 for x >= 700), evaluated on
 * the device next to CUDA's exp(-x) for comparison.  Synchronous; allocates
 * and frees 24 n bytes of device memory.
 *   x      host [n]: arguments (optical lengths Sigma_t l)
 *   n      0 <= n <= 2^28
 *   y      host out [n]: the sweep's e^{-x}
 *   y_lib  host out [n]: CUDA's exp(-x)
 * Errors: MOC_ERR_INVALID_ARG for NULL pointers with n > 0 or n out of
 * range, MOC_ERR_CUDA. */
int moc_eval_attenuation_f64(int32_t device, const double *x, int64_t n, double *y, double *y_lib);

/* The attenuation factor e^{-tau} of Eq. 3 as the FP32 sweep computes it:
 * 2^{-b} with b = tau log2 e (the sweep pre-scales Sigma_t by log2 e) on the
 * hardware ex2.approx.ftz.f32; the sweep's escape fraction is 1 minus this
 * value.  Evaluated on the device.  Synchronous; allocates and frees 8 n
 * bytes of device memory.
 *   b  host [n]: tau log2 e, >= 0
 *   n  0 <= n <= 2^28
 *   e  host out [n]: 2^{-b}
 * Errors: MOC_ERR_INVALID_ARG for NULL pointers with n > 0 or n out of
 * range, MOC_ERR_CUDA. */
int moc_eval_attenuation_f32(int32_t device, const float *b, int64_t n, float *e);

/* Autotuner of the sweep's launch schedule: generates the tracks of `geom`
 * under every candidate schedule (energy groups per lane 1, 2, 4 for FP32
 * sweeps; shared-memory or global tally; preload budget: everything stored,
 * base->preload_budget_bytes when >= 0, nothing stored; with two groups per
 * lane and stored templates, sync_block 1, 4 and 8), times `iterations`
 * outer iterations of each after 2 warm-up iterations (CUDA events), and
 * writes the fastest schedule to *best (base's other fields unchanged, the
 * tally mode and the synchronous block resolved).  *seconds_per_iteration
 * (may be NULL) is its time; report (may be NULL) gets up to max_report rows
 * of 6 doubles: groups per lane, tally mode in use, preload budget, stored
 * template pieces, seconds per iteration, tracks per synchronous block in use
 * (1: none); *n_report the rows written.  The paper fixes its launch shape by
 * hand; this tunes it per problem.  Runs on base->device and frees
 * everything it generated.  Errors: MOC_ERR_INVALID_ARG (NULL, iterations <
 * 1), MOC_ERR_UNSUPPORTED (no candidate could be generated), errors of
 * moc_generate_tracks and moc_iterate. */
int moc_autotune(const moc_geometry *geom, const moc_track_params *base, int32_t iterations,
                 moc_track_params *best, double *seconds_per_iteration, int32_t max_report,
                 double *report, int32_t *n_report);

/* ---------------------------------------------------------------------------
 * Serving engine: independent eigenvalue and fixed-source solves of different
 * geometries, group counts and track layouts, kept resident on one device and
 * advanced together as they arrive (continuous batching).  The paper solves
 * one problem at a time; this is a library service around that solver.
 *
 * Requests queue in arrival order and are admitted while a slot is free and
 * their device footprint (moc_query_footprint: resident state plus stored
 * templates) fits next to the resident solves in the memory budget; a
 * request whose footprint alone exceeds the budget is not admitted and
 * finishes with MOC_ERR_OUT_OF_MEMORY.  A request that fails (track
 * generation, for example MOC_ERR_UNSUPPORTED for more than 32 polar
 * angles; an enqueue; a kernel) finishes with its own status while the other
 * resident solves go on.  Each resident solve
 * owns a stream and captured iteration graphs; a step enqueues a quantum of
 * outer iterations on every idle solve (their kernels overlap on the device),
 * waits for the oldest quantum in flight and retires every solve whose
 * stopping rule held or that reached max_iter.  Iterations after convergence
 * are no-ops on the device, so a solve's result does not depend on the mix it
 * ran in.  Track generation of admitted requests runs on 4 host worker
 * threads inside the engine, so it overlaps the resident solves' work.  One
 * host thread drives an engine; calls on one engine must not overlap. */
typedef struct {
    int32_t device;
    int32_t max_active;           /* resident solves at most (0 = 16) */
    int64_t memory_budget_bytes;  /* device bytes for resident solves (0 = 80% of free memory) */
    int32_t iterations_per_poll;  /* outer iterations per solve between host checks (0 = 8) */
} moc_server_params;

typedef struct moc_server moc_server;

int moc_server_create(const moc_server_params *params, moc_server **out);
void moc_server_destroy(moc_server *server);

/* Queue one solve.  The geometry and both parameter sets are copied, so the
 * caller may destroy them after the call; eigenvalue or fixed source follows
 * the geometry (external source present or not); solve->use_graph is ignored
 * (graphs are always used).  *ticket identifies the request.  Errors:
 * MOC_ERR_INVALID_ARG (NULL, max_iter < 1, track parameters naming another
 * device), errors of moc_query_footprint. */
int moc_server_submit(moc_server *server, const moc_geometry *geom, const moc_track_params *tracks,
                      const moc_solve_params *solve, int64_t *ticket);

/* One engine step: admit, enqueue, wait for the oldest quantum in flight,
 * retire finished solves, admit and enqueue again.  *finished = requests
 * finished by this call (retired or failed), *pending = queued + resident
 * requests left (either may be NULL; both are written also on failure).
 * Blocks at most until one quantum completes.  Errors: MOC_ERR_INVALID_ARG
 * for NULL; MOC_ERR_CUDA only when the device context reports a sticky error
 * (one failing solve is reported through its own ticket instead). */
int moc_server_step(moc_server *server, int32_t *finished, int32_t *pending);

/* Result of a ticket: *ready = 0 while it is queued or resident.  Once ready,
 * fills res (may be NULL), phi (n_fsr*G normalised flux, may be NULL; phi_len
 * its capacity) and times[2] (may be NULL: seconds queued before admission and
 * seconds from submission to retirement), then forgets the ticket.  Returns
 * the solve's own status (MOC_ERR_NOT_CONVERGED when the stopping rule never
 * held).  MOC_ERR_INVALID_ARG for an unknown or already fetched ticket. */
int moc_server_result(moc_server *server, int64_t ticket, moc_result *res, double *phi,
                      int64_t phi_len, double *times, int32_t *ready);

/* Counters, int64 values written to out[0..n-1]: 0 queued, 1 resident,
 * 2 admitted so far, 3 retired so far, 4 device bytes held by resident
 * solves (footprint estimates), 5 memory budget, 6 most solves resident at
 * once. */
int moc_server_stats(const moc_server *server, int64_t *out, int32_t n);

#ifdef __cplusplus
}
#endif
#endif /* MOC3D_MOC_H */
