// Step, import, export, macroscopic and mass kernels for fp32 PDF storage.
#include "psm_kernels.cuh"

PSM_DEFINE_STORAGE(fp32, float)
#include "psm_adjoint.cuh"

PSM_DEFINE_ADJOINT(fp32, float)
