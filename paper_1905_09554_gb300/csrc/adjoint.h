// Launchers of the discrete-adjoint kernels (adjoint_kernels.cu), used by the
// host API in lbm_sc.cu.
#pragma once
#include <cuda_runtime.h>

namespace lbm {

struct AdjointArgs {
    int nx, ny, nz;
    long long n;
    double G, tau, omega, rho0;
    int grid;  // blocks of adjoint_threads() threads (grid-stride loops)
};

int adjoint_threads();
// One reverse step: lam_out = (dS/df)^T lam_next at the forward state f, and
// acc[0] += dJ/dG, acc[1] += dJ/dtau of this step.  psi (n), gF (3n) and
// partials (2 * grid doubles) are scratch.
cudaError_t adjoint_step(const AdjointArgs& a, bool f64, const void* f, void* psi, const void* lam_next,
                         void* lam_out, void* gF, double* partials, double* acc, cudaStream_t st);
cudaError_t adjoint_seed(const AdjointArgs& a, bool f64, const double* dJdrho, void* lam, cudaStream_t st);
cudaError_t adjoint_rho0(const AdjointArgs& a, bool f64, const void* lam, double* out, cudaStream_t st);

}  // namespace lbm
