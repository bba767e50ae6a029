// Launchers of the CUDA kernels (moc_kernels.cu).
#pragma once

#include <cuda_runtime.h>

#include "moc_device.cuh"

// segments per stack (stack_nseg), their maximum, and per geometric track (trk_nseg)
cudaError_t launch_count_stacks(const DevLayout &dl, int64_t n_stacks, int64_t *stack_nseg,
                                int32_t *max_nseg, int32_t *trk_nseg, int grid, cudaStream_t s);
cudaError_t launch_tpl_count(const DevLayout &dl, const int32_t *exp_stacks, int64_t n_exp,
                             int64_t *cnt, int32_t *lmin, int32_t *nlay, int grid, cudaStream_t s);
cudaError_t launch_tpl_write(int precision, const DevLayout &dl, const int32_t *exp_stacks,
                             int64_t n_exp, void *recs, int32_t *lidx, int grid, cudaStream_t s);
size_t segrec_size(int precision);
cudaError_t launch_track_counts(const DevLayout &dl, int64_t stack, int frame, int64_t *cnt, cudaStream_t s);
// per track of the stored stacks, in sweep order: (record count << 48) | first record
cudaError_t launch_windows(const DevLayout &dl, int64_t n_stacks, uint64_t *win, int grid,
                           cudaStream_t s);
// chunk tables of the stacks of radially chunked units (StackDesc::chunk_base)
cudaError_t launch_chunk_tables(int precision, const DevLayout &dl, const int32_t *stacks, int64_t n,
                                int64_t *tab, int grid, cudaStream_t s);
cudaError_t launch_links(const DevLayout &dl, int64_t n_stacks, int32_t *dst, int grid,
                         cudaStream_t s);
// tracked volumes, summed exactly in acc (scratch of nfsr * 4 words) and
// written to vol [nfsr]
cudaError_t launch_volumes(int precision, const DevLayout &dl, int64_t n_stacks, int64_t nfsr,
                           unsigned long long *acc, double *vol, int grid, cudaStream_t s);
cudaError_t launch_stack_segments(int precision, const DevLayout &dl, int64_t stack, int frame,
                                  const int64_t *offs, int32_t *fsr, double *len, cudaStream_t s);
// the sweep (moc_sweep.cu); gpl = energy groups per lane (1 or 2, FP32 only)
int sweep_default_gpl(int precision, int G);
int sweep_lanes_per_track(int G, int gpl);
// threads per sweep block the kernel is compiled for (its launch bound)
int sweep_block_threads(int precision, int gpl, int matk = 0, int chunk = 0);
// sync: tracks per synchronous block (0: none; the split tile), NL: sweep layers
// matk: rows of Qr only (layouts whose records carry materials)
size_t sweep_smem_bytes(int precision, int tally_smem, int chunk, int M, int G, int gpl, int cap,
                        int sync = 0, int NL = 1, int matk = 0);
// The state of one solve of a batched sweep (pointers into device memory)
struct BatchItem {
    const void *qr;             // Q / Sigma_t, real
    double *tally;              // FP64 tally
    double *scal;               // device scalars
    const void *psi_in;         // boundary fluxes in / out (null: all vacuum)
    void *psi_out;
};
// counter: the work counter (zero at launch)
cudaError_t launch_sweep(int precision, int tally_smem, int gpl, const DevLayout &dl,
                         const DevState &st, const int32_t *order, int32_t n_work, int32_t cap,
                         const void *psi_in, void *psi_out, int32_t *counter, int grid, int block,
                         size_t smem, cudaStream_t s);
// The sweep of layouts with layer planes off the axial lattice
// (moc_sweep_ol.cu): block sweep_ol_block() threads, no dynamic shared memory
int sweep_ol_block();
cudaError_t launch_sweep_ol(int precision, const DevLayout &dl, const DevState &st, const int32_t *order,
                            int32_t n_work, const void *psi_in, void *psi_out, int32_t *counter, int grid,
                            cudaStream_t s);
// One sweep of n solves sharing the layout dl (shared tally, no radial
// chunks): items[n] (device) hold their states; n_units = units in order.
cudaError_t launch_sweep_batch(int precision, int gpl, const DevLayout &dl, const DevState &st,
                               const int32_t *order, int32_t n_units, int32_t cap, int32_t *counter,
                               const BatchItem *items, int32_t n, int grid, int block, size_t smem,
                               cudaStream_t s);
// the sweep kernel for one lane shape (moc_sweep_f32g1/g2/g4.cu, moc_sweep_f64.cu);
// batch: the variant that sweeps several solves of one layout (shared tally,
// units swept whole)
const void *sweep_kernel_f32_gpl1(int tally_smem, int chunk, int batch, int gl);
// sync: the synchronous-block variant (layouts with dl.sync_b > 0)
const void *sweep_kernel_f32_gpl2(int tally_smem, int chunk, int batch, int gl, int sync);
const void *sweep_kernel_f32_gpl4(int tally_smem, int chunk, int batch, int gl);
// the variant for layouts whose records carry materials (moc_sweep_f32g2m.cu:
// two groups per lane, shared tally; chunk: some units in radial chunks)
const void *sweep_kernel_f32_gpl2_matk(int chunk, int batch, int gl);
const void *sweep_kernel_f64(int tally_smem, int chunk, int batch, int gl);
cudaError_t sweep_occupancy(int precision, int tally_smem, int chunk, int G, int gpl, int block,
                            size_t smem, int *blocks_per_sm, bool sync = false, bool matk = false);
// threads per block of the per-FSR kernels (source, finalize, residual, init):
// small blocks spread a few thousand FSRs over many SMs
constexpr int kSmallBlock = 64;
cudaError_t launch_source(int precision, const DevLayout &dl, const DevState &st, int32_t nfsr,
                          int grid, cudaStream_t s);
cudaError_t launch_finalize(int precision, const DevLayout &dl, const DevState &st, int32_t nfsr,
                            int grid, double integrations, cudaStream_t s);
cudaError_t launch_finalize_fixed(int precision, const DevLayout &dl, const DevState &st,
                                  int32_t nfsr, int grid, double integrations, cudaStream_t s);
cudaError_t launch_init_state(const DevLayout &dl, const DevState &st, int32_t nfsr, int grid,
                              cudaStream_t s);

// group-wise reaction rates with a fixed library-owned scratch array
// (moc_static.cu): at most kRatesMaxGroups groups; partials of up to
// kRatesMaxBlocks blocks, then 2 x G results at kRatesResultOffset
constexpr int kRatesMaxBlocks = 128;
constexpr int kRatesMaxGroups = 32;
constexpr int kRatesResultOffset = kRatesMaxBlocks * kRatesMaxGroups * 2;
constexpr int kRatesScratchDoubles = kRatesResultOffset + 2 * kRatesMaxGroups;
cudaError_t rates_scratch_address(double **ptr);
cudaError_t launch_group_rates_static(const DevLayout &dl, const DevState &st, int32_t nfsr,
                                      double *scratch, cudaStream_t s);
