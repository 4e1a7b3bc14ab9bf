// Polar resampling and ring FFT launchers with 16-bit (BF16 / FP16) mma
// fragment output for the precision-split path.  The kernel itself is in
// polar_impl.cuh.
#include "polar_impl.cuh"

namespace mra {

cudaError_t launch_polar16(const Geometry &g, const PolarArgs &a, cudaStream_t st) {
  if (a.fp16) return g.taps ? launch_polar_t<true, kOutF16>(g, a, st) : launch_polar_t<false, kOutF16>(g, a, st);
  return g.taps ? launch_polar_t<true, kOutBF16>(g, a, st) : launch_polar_t<false, kOutBF16>(g, a, st);
}

}  // namespace mra
