"""GB300 (sm_103a) implementation of the D3Q19 pseudo-potential (Shan-Chen)
lattice Boltzmann step of arXiv:1905.09554.

Modules: `lbm` (ctypes binding of the C ABI in include/lbm_sc.h and the
`Lattice` / `Batch` wrappers), `autograd` (torch.autograd over the discrete
adjoint), `diagnostics` (neck radius, break-up time, growth rate, drops),
`calibration` (Laplace test, flat-interface coexistence, the Oh fixed point
of Sec. 3), `experiments` (the break-up run of Secs. 3-4), `inputs` (seeded
synthetic inputs), `build` (nvcc build of liblbm_sc.so).  The CUDA sources
are in `csrc/`.
"""
