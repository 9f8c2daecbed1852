// The fused step kernels for hands with 5 contacts (bodex_kernels.cuh).
#include "bodex_kernels.cuh"

int launch_fused_m5(int mode, const FusedArgs& A, cudaStream_t st) { return run_fused<5>(mode, A, st); }
