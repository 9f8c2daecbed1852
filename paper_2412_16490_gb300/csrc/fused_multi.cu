// The several-job step kernel (bodex_kernels.cuh).
#include "bodex_kernels.cuh"

int launch_multi(bool adapt, const MultiArgs& MA, int total, size_t bytes, cudaStream_t st) {
  int r = adapt ? ensure_smem(multi_kernel<true>, bytes) : ensure_smem(multi_kernel<false>, bytes);
  if (r != BODEX_OK) return r;
  if (adapt) multi_kernel<true><<<total, CTA_LANES, bytes, st>>>(MA);
  else multi_kernel<false><<<total, CTA_LANES, bytes, st>>>(MA);
  return launch_err("multi_kernel launch");
}
