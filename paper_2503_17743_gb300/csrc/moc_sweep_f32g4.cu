// Sweep kernel instantiations: FP32, 4 energy groups per lane
// (the kernel is in moc_sweep_kernel.cuh; the dispatch in moc_sweep.cu).
#include "moc_sweep_kernel.cuh"

const void *sweep_kernel_f32_gpl4(int tally_smem, int chunk, int batch, int gl) {
    if (batch) return pick<float, 4, true, false, true>(gl);
    if (!tally_smem) return pick<float, 4, false, false, false>(gl);
    return chunk ? pick<float, 4, true, true, false>(gl) : pick<float, 4, true, false, false>(gl);
}
