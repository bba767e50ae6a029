// Sweep kernel instantiations: FP64, 1 energy group per lane
// (the kernel is in moc_sweep_kernel.cuh; the dispatch in moc_sweep.cu).
#include "moc_sweep_kernel.cuh"

const void *sweep_kernel_f64(int tally_smem, int chunk, int batch, int gl) {
    if (batch) return pick<double, 1, true, false, true>(gl);
    if (!tally_smem) return pick<double, 1, false, false, false>(gl);
    return chunk ? pick<double, 1, true, true, false>(gl) : pick<double, 1, true, false, false>(gl);
}
