// Step, import, export, macroscopic and mass kernels for bf16 PDF storage.
#include "psm_kernels.cuh"

PSM_DEFINE_STORAGE(bf16, __nv_bfloat16)
#include "psm_adjoint.cuh"

PSM_DEFINE_ADJOINT(bf16, __nv_bfloat16)
