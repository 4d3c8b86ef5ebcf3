"""GB300-native high-order gas-kinetic scheme with 3D WENO-AO reconstruction
(Pan & Xu, arXiv 1909.01580): CUDA kernels for sm_103a behind the C ABI of
include/hgks.h, with a thin ctypes binding (``hgks``) and seeded synthetic
workloads (``workloads``)."""
