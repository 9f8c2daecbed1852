// The batched-QP kernels (bodex_kernels.cuh).
#include "bodex_kernels.cuh"

int launch_qp(int m, const float* G, int B, const float* T, int s, const AdmmCfg& cfg, int warm, float* y, float* z,
              float* lam, float* Q, int32_t* iters, int32_t* status, float* res, cudaStream_t st) {
  switch (m) {
    case 3: return run_qp<3>(G, B, T, s, cfg, warm, y, z, lam, Q, iters, status, res, st);
    case 4: return run_qp<4>(G, B, T, s, cfg, warm, y, z, lam, Q, iters, status, res, st);
    case 5: return run_qp<5>(G, B, T, s, cfg, warm, y, z, lam, Q, iters, status, res, st);
    default: return fail(BODEX_ERR_INVALID, "m must be 3, 4 or 5");
  }
}
