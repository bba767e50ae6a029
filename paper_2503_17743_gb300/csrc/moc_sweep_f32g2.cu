// Sweep kernel instantiations: FP32, 2 energy groups per lane
// (the kernel is in moc_sweep_kernel.cuh; the dispatch in moc_sweep.cu).
#include "moc_sweep_kernel.cuh"

const void *sweep_kernel_f32_gpl2(int tally_smem, int chunk, int batch, int gl, int sync) {
    if (sync) return batch ? pick<float, 2, true, false, true, 16, true>(gl)
                           : pick<float, 2, true, false, false, 16, true>(gl);
    if (batch) return pick<float, 2, true, false, true>(gl);
    if (!tally_smem) return pick<float, 2, false, false, false>(gl);
    return chunk ? pick<float, 2, true, true, false>(gl) : pick<float, 2, true, false, false>(gl);
}
