// Float-float complex128 tile passes, K = 10 tile qubits.
#define VQG_DF_DEFINE
#include "k_fused_df.cuh"

using namespace vqg;
VQG_DF_INSTANTIATE(10)
