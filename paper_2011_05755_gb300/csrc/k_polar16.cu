// Polar resampling and ring FFT launchers with 16-bit (BF16 / FP16) output
// for the precision-split path: mma.sync fragments, or the k-step tiles of
// the tcgen05 kernel (M = 256).  The kernel itself is in
// polar_impl.cuh.
#include "polar_impl.cuh"

namespace mra {

cudaError_t launch_polar16(const Geometry &g, const PolarArgs &a, cudaStream_t st) {
  if (a.umma) {
    if (a.fp16) return g.taps ? launch_polar_t<true, kOutUF16>(g, a, st) : launch_polar_t<false, kOutUF16>(g, a, st);
    return g.taps ? launch_polar_t<true, kOutUBF16>(g, a, st) : launch_polar_t<false, kOutUBF16>(g, a, st);
  }
  if (a.fp16) return g.taps ? launch_polar_t<true, kOutF16>(g, a, st) : launch_polar_t<false, kOutF16>(g, a, st);
  return g.taps ? launch_polar_t<true, kOutBF16>(g, a, st) : launch_polar_t<false, kOutBF16>(g, a, st);
}

}  // namespace mra
