// Launchers of the discrete-adjoint kernels (adjoint_kernels.cu), used by the
// host API in lbm_sc.cu.
#pragma once
#include <cuda_runtime.h>

namespace lbm {

struct AdjointArgs {
    int nx, ny, nz;
    long long n;
    double G, tau, omega, rho0;
    float Gf, tauf, omegaf, rho0f;  // rounded on the host for the FP32 kernels
    int grid;  // blocks of adjoint_threads() threads (grid-stride loops)
};

int adjoint_threads();
int adjoint_rows_per_block();  // the step kernels walk x rows, this many per block
// The adjoint field is kept as lam_a(x) + gr(x): the force's contribution to
// dJ/drho is the same for every population, so it is stored once per cell
// (gr, n values) instead of being added to the 19 populations.
//
// One reverse step: (lam_out, gr_out) = (dS/df)^T (lam_next + gr_next) at the
// forward state f; this step's dJ/dG and dJ/dtau are added to the per-block
// running sums in `partials` (2 * grid doubles, zeroed before the first
// step), which adjoint_reduce adds into acc[0..1] once after the last step.
// psi (n) and gF (4n: psi gF and S.gF, see adj_collide_kernel) are scratch;
// acc is not touched here.  Needs nx*ny*nz < 2^32 (32-bit cell indices).
// psi_ready: psi already holds psi of f (the step kernel wrote it during the
// recomputation); otherwise it is computed first.
cudaError_t adjoint_step(const AdjointArgs& a, bool f64, const void* f, void* psi, bool psi_ready,
                         const void* lam_next, const void* gr_next, void* lam_out, void* gr_out, void* gF,
                         double* partials, double* acc, cudaStream_t st);
cudaError_t adjoint_reduce(const AdjointArgs& a, const double* partials, double* acc, cudaStream_t st);
// lam_a = dJ/drho (every a), gr = 0.
cudaError_t adjoint_seed(const AdjointArgs& a, bool f64, const double* dJdrho, void* lam, void* gr, cudaStream_t st);
// dJ/drho0 = sum_a w_a lam_a + gr.
cudaError_t adjoint_rho0(const AdjointArgs& a, bool f64, const void* lam, const void* gr, double* out,
                         cudaStream_t st);

}  // namespace lbm
