// The fused step kernels for hands with 3 contacts (bodex_kernels.cuh).
#include "bodex_kernels.cuh"

int launch_fused_m3(int mode, const FusedArgs& A, cudaStream_t st) { return run_fused<3>(mode, A, st); }
