// Sweep kernel instantiations: FP32, 2 energy groups per lane, layouts whose
// records carry the material of every piece (rows of Qr only), units swept
// whole or in radial chunks
// (the kernel is in moc_sweep_kernel.cuh; the dispatch in moc_sweep.cu).
#include "moc_sweep_kernel.cuh"

const void *sweep_kernel_f32_gpl2_matk(int chunk, int batch, int gl) {
    if (chunk) return pick<float, 2, true, true, false, 16, false, true>(gl);
    return batch ? pick<float, 2, true, false, true, 16, false, true>(gl)
                 : pick<float, 2, true, false, false, 16, false, true>(gl);
}
