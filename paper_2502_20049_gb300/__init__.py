"""PSM lattice Boltzmann hot path (arXiv 2502.20049) for NVIDIA GB300 (sm_103a).

The compute path is the CUDA library ``libpsm.so`` (C ABI in ``include/psm.h``);
:mod:`.psm` is its Python binding and :mod:`.workloads` holds the synthetic
workloads.  Build with :func:`.build.build`.
"""

__all__ = ["psm", "workloads", "build"]
