// Dispatch and launch of the transport sweep (the kernel: moc_sweep_kernel.cuh;
// its instantiations: moc_sweep_f32g1/g2/g4.cu, moc_sweep_f64.cu, compiled in
// parallel).
#include "moc_sweep_kernel.cuh"

namespace {

// lanes per track: the smallest power of two that holds ceil(G / gpl) groups
int lanes_for_groups(int G, int gpl) {
    const int cap = 32 / gpl;
    const int need = (G + gpl - 1) / gpl;
    int gl = 1;
    while (gl < need && gl < cap) gl <<= 1;
    return gl;
}

// chunk: some units are swept in radial chunks (shared tally only)
// matk: the layout's records carry materials (DevLayout::matk)
const void *sweep_fn(int precision, int tally_smem, int chunk, int G, int gpl, int batch = 0, int sync = 0,
                     int matk = 0) {
    const int gl = lanes_for_groups(G, gpl);
    if (precision == MOC_FP64) return sweep_kernel_f64(tally_smem, chunk, batch, gl);
    if (matk) return sweep_kernel_f32_gpl2_matk(chunk, batch, gl);
    if (gpl == 4) return sweep_kernel_f32_gpl4(tally_smem, chunk, batch, gl);
    if (gpl == 2) return sweep_kernel_f32_gpl2(tally_smem, chunk, batch, gl, sync);
    return sweep_kernel_f32_gpl1(tally_smem, chunk, batch, gl);
}

// The kernel's dynamic shared-memory limit is per function and shared by
// every thread of the process: solves of different tile sizes launched from
// several threads (the serving engine) would race on it.  So every caller
// sets the same value, the device's opt-in maximum, and checks its own size.
cudaError_t allow_dynamic_smem(const void *f, size_t smem) {
    int dev = 0, cap = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&cap, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    if (smem > (size_t)cap) return cudaErrorInvalidValue;
    // the opt-in maximum less the kernel's static shared memory
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, f);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, cap - (int)fa.sharedSizeBytes);
}

}  // namespace

// two groups per lane in FP32 (half the per-segment bookkeeping per
// integration; the autotuner's usual pick), one in FP64
int sweep_default_gpl(int precision, int G) {
    return (precision == MOC_FP32 && G > 1) ? 2 : 1;
}

int sweep_lanes_per_track(int G, int gpl) { return lanes_for_groups(G, gpl); }

int sweep_block_threads(int precision, int gpl, int matk, int chunk) {
    return sweep_block(precision != MOC_FP64, gpl, matk != 0, chunk != 0);
}

size_t sweep_smem_bytes(int precision, int tally_smem, int chunk, int M, int G, int gpl, int cap,
                        int sync, int NL, int matk) {
    const size_t rs = precision == MOC_FP64 ? 8 : 4;
    const size_t gp = (size_t)lanes_for_groups(G, gpl) * gpl;
    size_t b = ((size_t)M * gp * rs + 15) & ~(size_t)15;
    if (!tally_smem) return b;
    if (sync) {
        // split tile (Qr, Sigma_t with guard rows), Sigma_t per 2D segment,
        // then the tally with a guard of kSyncGuard words after it
        b += 2 * (size_t)(cap + 2 * kSyncGuard) * gp * 4;
        b += ((size_t)(cap / NL) * gp * 4 + 15) & ~(size_t)15;
        b += ((size_t)tally_rows(cap, (int)(gp / gpl), gpl) * gp + kSyncGuard) * 4;
        return b;
    }
    // (Qr, Sigma_t) rows (Qr only with material keys) + tally rows
    b += (size_t)cap * gp * rs * (matk ? 1 : 2) +
         (precision == MOC_FP64 || (chunk && !matk) ? (size_t)cap * tally_stride((int)(gp / gpl), gpl)
                                                    : (size_t)tally_rows(cap, (int)(gp / gpl), gpl) * gp) * rs;
    return b;
}

cudaError_t sweep_occupancy(int precision, int tally_smem, int chunk, int G, int gpl, int block,
                            size_t smem, int *blocks_per_sm, bool sync, bool matk) {
    const void *f = sweep_fn(precision, tally_smem, chunk, G, gpl, 0, sync ? 1 : 0, matk ? 1 : 0);
    cudaError_t e = allow_dynamic_smem(f, smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, f, block, smem);
}

cudaError_t launch_sweep(int precision, int tally_smem, int gpl, const DevLayout &dl,
                         const DevState &st, const int32_t *order, int32_t n_work, int32_t cap,
                         const void *psi_in, void *psi_out, int32_t *counter, int grid, int block,
                         size_t smem, cudaStream_t s) {
    if (dl.offlat) return launch_sweep_ol(precision, dl, st, order, n_work, psi_in, psi_out, counter, grid, s);
    const void *f = sweep_fn(precision, tally_smem, tally_smem && dl.chunk_b > 0, dl.G, gpl, 0,
                             tally_smem && dl.sync_b > 0 ? 1 : 0, tally_smem ? dl.matk : 0);
    cudaError_t e = allow_dynamic_smem(f, smem);
    if (e != cudaSuccess) return e;
    DevLayout a0 = dl;
    DevState a1 = st;
    a1.counter = counter;
    const int32_t *a2 = order;
    int32_t a3 = n_work, a4 = tally_smem ? cap : 0;
    const void *a5 = psi_in;
    void *a6 = psi_out;
    const BatchItem *a7 = nullptr;
    int32_t a8 = 0;
    void *args[] = {&a0, &a1, &a2, &a3, &a4, &a5, &a6, &a7, &a8};
    return cudaLaunchKernel(f, dim3(grid), dim3(block), args, smem, s);
}

cudaError_t launch_sweep_batch(int precision, int gpl, const DevLayout &dl, const DevState &st,
                               const int32_t *order, int32_t n_units, int32_t cap, int32_t *counter,
                               const BatchItem *items, int32_t n, int grid, int block, size_t smem,
                               cudaStream_t s) {
    const void *f = sweep_fn(precision, 1, 0, dl.G, gpl, 1, dl.sync_b > 0 ? 1 : 0, dl.matk);
    cudaError_t e = allow_dynamic_smem(f, smem);
    if (e != cudaSuccess) return e;
    DevLayout a0 = dl;
    DevState a1 = st;
    a1.counter = counter;
    const int32_t *a2 = order;
    int32_t a3 = n_units * n, a4 = cap;
    const void *a5 = nullptr;
    void *a6 = nullptr;
    const BatchItem *a7 = items;
    int32_t a8 = n;
    void *args[] = {&a0, &a1, &a2, &a3, &a4, &a5, &a6, &a7, &a8};
    return cudaLaunchKernel(f, dim3(grid), dim3(block), args, smem, s);
}
