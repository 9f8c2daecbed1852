// The fused step kernels for hands with 4 contacts (bodex_kernels.cuh).
#include "bodex_kernels.cuh"

int launch_fused_m4(int mode, const FusedArgs& A, cudaStream_t st) { return run_fused<4>(mode, A, st); }
