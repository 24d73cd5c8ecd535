// Step, import, export, macroscopic and mass kernels for fp64 PDF storage.
#include "psm_kernels.cuh"

PSM_DEFINE_STORAGE(fp64, double)
#include "psm_adjoint.cuh"

PSM_DEFINE_ADJOINT(fp64, double)
