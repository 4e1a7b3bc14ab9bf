// Host helper: raise a kernel's dynamic shared-memory limit to at least a
// launch's need, never lowering it.  Handles of different geometries (and
// host threads) share one kernel instantiation, so the limit a launch sees
// must be the largest any launch asked for; the check and the update run
// under one process-wide lock.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <mutex>

namespace mra {

inline std::mutex &smem_limit_mutex() {
  static std::mutex m;
  return m;
}

// `granted` is the caller's per-kernel record of the limit already set.
template <class Kernel>
cudaError_t raise_smem_limit(Kernel *kernel, size_t bytes, size_t &granted) {
  std::lock_guard<std::mutex> lock(smem_limit_mutex());
  if (granted >= bytes) return cudaSuccess;
  const cudaError_t e =
      cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(bytes));
  if (e == cudaSuccess) granted = bytes;
  return e;
}

}  // namespace mra
