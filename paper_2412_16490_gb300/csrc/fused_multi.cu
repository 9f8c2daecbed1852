// The several-job step kernel (bodex_kernels.cuh).
#include "bodex_kernels.cuh"

int launch_multi(bool adapt, bool exact, const MultiArgs& MA, int total, size_t bytes, cudaStream_t st) {
  auto go = [&](auto kernel) -> int {
    if (int r = ensure_smem(kernel, bytes)) return r;
    kernel<<<total, CTA_LANES, bytes, st>>>(MA);
    return launch_err("multi_kernel launch");
  };
  if (exact) return go(multi_kernel<false, true>);
  return adapt ? go(multi_kernel<true>) : go(multi_kernel<false>);
}
