// Polar resampling and ring FFT launchers: the FP32-output instantiations
// and the dispatcher (the 16-bit-output ones are in k_polar16.cu).  The
// kernel itself is in polar_impl.cuh.
#include "polar_impl.cuh"

namespace mra {

cudaError_t launch_polar16(const Geometry &g, const PolarArgs &a, cudaStream_t st);

size_t polar_smem_one_row(const Geometry &g, bool taps, bool out16) {
  return polar_smem_bytes(g, taps, out16, 1);
}

cudaError_t launch_polar(const Geometry &g, const PolarArgs &a, cudaStream_t st) {
  if (a.n_imgs <= 0 || a.rows_per_img <= 0) return cudaSuccess;
  if (a.out16) return launch_polar16(g, a, st);
  return g.taps ? launch_polar_t<true, kOutF32>(g, a, st) : launch_polar_t<false, kOutF32>(g, a, st);
}

}  // namespace mra
