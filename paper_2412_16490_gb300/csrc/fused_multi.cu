// The several-job step kernel (bodex_kernels.cuh).
#include "bodex_kernels.cuh"

// pull: one CTA per resident slot (SMs x CTAs that fit per SM at `bytes`
// of shared memory), at most one per work item, pulling items until none is
// left; otherwise one CTA per work item.
int launch_multi(bool adapt, bool exact, bool pull, const MultiArgs& MA, size_t bytes, cudaStream_t st) {
  auto go = [&](auto kernel) -> int {
    if (int r = ensure_smem(kernel, bytes)) return r;
    int grid = MA.total;
    if (pull) {
      int dev = 0, sms = 0, per_sm = 0;
      if (cudaGetDevice(&dev) != cudaSuccess ||
          cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, CTA_LANES, bytes) != cudaSuccess)
        return launch_err("multi_kernel occupancy query");
      grid = std::max(1, std::min(MA.total, sms * std::max(per_sm, 1)));
    }
    kernel<<<grid, CTA_LANES, bytes, st>>>(MA);
    return launch_err("multi_kernel launch");
  };
  if (pull) {
    if (exact) return go(multi_kernel<false, true, true>);
    return adapt ? go(multi_kernel<true, false, true>) : go(multi_kernel<false, false, true>);
  }
  if (exact) return go(multi_kernel<false, true>);
  return adapt ? go(multi_kernel<true>) : go(multi_kernel<false>);
}
