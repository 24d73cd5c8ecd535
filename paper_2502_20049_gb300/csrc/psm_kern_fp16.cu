// Step, import, export, macroscopic and mass kernels for fp16 PDF storage.
#include "psm_kernels.cuh"

PSM_DEFINE_STORAGE(fp16, __half)
#include "psm_adjoint.cuh"

PSM_DEFINE_ADJOINT(fp16, __half)
