// Sweep kernel instantiations: FP32, 1 energy group per lane
// (the kernel is in moc_sweep_kernel.cuh; the dispatch in moc_sweep.cu).
#include "moc_sweep_kernel.cuh"

const void *sweep_kernel_f32_gpl1(int tally_smem, int chunk, int batch, int gl) {
    if (batch) return pick<float, 1, true, false, true>(gl);
    if (!tally_smem) return pick<float, 1, false, false, false>(gl);
    return chunk ? pick<float, 1, true, true, false>(gl) : pick<float, 1, true, false, false>(gl);
}
