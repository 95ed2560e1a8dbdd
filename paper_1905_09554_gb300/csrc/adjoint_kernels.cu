// Discrete adjoint of the SRT Shan-Chen step (Sec. 2: Eqs. LBE, local_eq,
// momentum, SC_force, vel_shift), for FP32 or FP64 populations.
//
// Forward step at time t (state f = post-streaming populations):
//   rho = sum f, j = sum c f, psi = psi(rho), S(x) = sum_a w_a psi(x + c_a) c_a,
//   F = -G psi S, u' = (j + tau F)/rho, f* = f + omega (f_eq(rho, u') - f),
//   f_a(x + c_a, t + 1) = f*_a(x).
// Reverse step, given lam(t+1) = dJ/df(t+1):
//   1. streaming adjoint (pull): lam*_a(x) = lam_a(x + c_a, t+1);
//   2. collision adjoint (local, adj_collide_kernel): lam_loc = (df*/df)^T lam*,
//      gF = (df*/dF)^T lam*, and the tau and G terms of the parameter
//      gradients;
//   3. force adjoint (a gather over neighbours, adj_force_kernel):
//      g_psi(y) = -G [ S(y).gF(y) + sum_a w_a psi(y - c_a) c_a . gF(y - c_a) ],
//      g_rho = g_psi psi'(rho) with psi' = exp(-rho/rho0) = 1 - psi/rho0,
//      lam_a(y, t) = lam_loc_a(y) + g_rho(y) for every a.  Step 2 already
//      knows S(y) and psi(y), so it stores T = S.gF and V = psi gF per cell
//      and the gather reads only V of the 18 neighbours.
// Parameter gradients are summed in float64 per block and reduced in a fixed
// order (deterministic).
#include <cuda_runtime.h>

#include "adjoint.h"
#include "lattice.cuh"

namespace lbm {
namespace {

constexpr int kThreads = 256;
constexpr int kRowThreads = 32, kRows = kThreads / kRowThreads;  // (32, 8) blocks: 8 rows at a time

// The cells of one x row and the periodic neighbour offsets of the row and
// of its cells (32-bit: the adjoint needs nx*ny*nz < 2^32).  Blocks of
// (32, 8) threads walk the ny*nz rows (grid-stride); a warp covers 32
// consecutive x of a row, so the neighbour gathers stay coalesced and no
// cell index is ever divided.
struct Row {
    unsigned zo[3], yo[3];  // offsets of planes z-1, z, z+1 and rows y-1, y, y+1
};

__device__ __forceinline__ Row row_of(unsigned r, int nx, int ny, int nz) {
    const int y = int(r % unsigned(ny)), z = int(r / unsigned(ny));
    const int ym = y == 0 ? ny - 1 : y - 1, yp = y + 1 == ny ? 0 : y + 1;
    const int zm = z == 0 ? nz - 1 : z - 1, zp = z + 1 == nz ? 0 : z + 1;
    const unsigned plane = unsigned(nx) * unsigned(ny);
    Row w;
    w.zo[0] = unsigned(zm) * plane;
    w.zo[1] = unsigned(z) * plane;
    w.zo[2] = unsigned(zp) * plane;
    w.yo[0] = unsigned(ym) * unsigned(nx);
    w.yo[1] = unsigned(y) * unsigned(nx);
    w.yo[2] = unsigned(yp) * unsigned(nx);
    return w;
}

// Index of x + (dx, dy, dz), |d| <= 1, with xs = {x-1, x, x+1} wrapped.
__device__ __forceinline__ unsigned nb_of(const Row& w, const unsigned (&xs)[3], int dx, int dy, int dz) {
    return w.zo[dz + 1] + w.yo[dy + 1] + xs[dx + 1];
}

template <class F>
__device__ __forceinline__ void for_each_cell(int nx, int ny, int nz, F&& body) {
    const unsigned rows = unsigned(ny) * unsigned(nz);
    for (unsigned r = blockIdx.x * kRows + threadIdx.y; r < rows; r += gridDim.x * kRows) {
        const Row w = row_of(r, nx, ny, nz);
        for (int x = threadIdx.x; x < nx; x += kRowThreads) {
            const unsigned xs[3] = {unsigned(x == 0 ? nx - 1 : x - 1), unsigned(x), unsigned(x + 1 == nx ? 0 : x + 1)};
            body(w, xs, w.zo[1] + w.yo[1] + unsigned(x));
        }
    }
}

template <class R>
__device__ __forceinline__ R psi_fn(R rho, R rho0) {
    return rho0 * (R(1) - exp(-rho / rho0));
}

template <class R>
__global__ void __launch_bounds__(kThreads) adj_psi_kernel(const R* __restrict__ f, R* __restrict__ psi, unsigned n,
                                                           R rho0) {
    for (unsigned i = blockIdx.x * kThreads + threadIdx.y * kRowThreads + threadIdx.x; i < n; i += gridDim.x * kThreads) {
        R r = R(0);
        static_for<0, Q>([&](auto qc) {
            constexpr int q = decltype(qc)::value;
            r += f[size_t(q) * n + i];
        });
        psi[i] = psi_fn<R>(r, rho0);
    }
}

// Sum of (a, b) over the block, added to out2[0..1] (the block's running
// sums over the reverse steps); fixed order.
__device__ __forceinline__ void block_sum2(double a, double b, double* out2) {
    __shared__ double red[2][kThreads];
    const int tid = threadIdx.y * kRowThreads + threadIdx.x;
    red[0][tid] = a;
    red[1][tid] = b;
    __syncthreads();
    for (int s = kThreads / 2; s > 0; s >>= 1) {
        if (tid < s) {
            red[0][tid] += red[0][tid + s];
            red[1][tid] += red[1][tid + s];
        }
        __syncthreads();
    }
    if (tid == 0) {
        out2[0] += red[0][0];
        out2[1] += red[1][0];
    }
}

// Collision adjoint.  Besides lam_out it writes, per cell, the two pieces of
// the force adjoint that the gather of adj_force_kernel needs:
//   fa[0..2n) = V = psi gF (the cell's force sensitivity weighted by its psi)
//   fa[3n..4n) = T = S . gF (S = sum_a w_a psi(x + c_a) c_a, known here).
template <class R>
__global__ void __launch_bounds__(kThreads)
adj_collide_kernel(const R* __restrict__ f, const R* __restrict__ psi, const R* __restrict__ lam_next,
                   const R* __restrict__ gr_next, R* __restrict__ lam_out, R* __restrict__ fa,
                   double* __restrict__ partials, AdjointArgs a) {
    const unsigned n = unsigned(a.n);
    const R G = par<R>(a.G, a.Gf), tau = par<R>(a.tau, a.tauf), omega = par<R>(a.omega, a.omegaf);
    double accG = 0.0, accT = 0.0;
    for_each_cell(a.nx, a.ny, a.nz, [&](const Row& w, const unsigned (&xs)[3], unsigned i) {
        R fv[Q], ls[Q];
        R rho = R(0), jx = R(0), jy = R(0), jz = R(0), sx = R(0), sy = R(0), sz = R(0);
        static_for<0, Q>([&](auto qc) {
            constexpr int q = decltype(qc)::value;
            fv[q] = f[size_t(q) * n + i];
            rho += fv[q];
            jx += R(cx(q)) * fv[q];
            jy += R(cy(q)) * fv[q];
            jz += R(cz(q)) * fv[q];
            const unsigned nb = nb_of(w, xs, cx(q), cy(q), cz(q));
            ls[q] = lam_next[size_t(q) * n + nb] + gr_next[nb];  // streaming adjoint: pull from x + c_q
            if constexpr (q != 0) {
                const R pn = psi[nb];
                sx += R(wq(q) * cx(q)) * pn;
                sy += R(wq(q) * cy(q)) * pn;
                sz += R(wq(q) * cz(q)) * pn;
            }
        });
        const R ps = psi[i];
        const R Fx = -G * ps * sx, Fy = -G * ps * sy, Fz = -G * ps * sz;
        const R inv_rho = R(1) / rho;
        const R ux = (jx + tau * Fx) * inv_rho, uy = (jy + tau * Fy) * inv_rho, uz = (jz + tau * Fz) * inv_rho;
        const R u2 = ux * ux + uy * uy + uz * uz;
        // adjoint of f* = (1 - omega) f + omega f_eq(rho, u')
        R g_rho = R(0), gux = R(0), guy = R(0), guz = R(0), g_tau = R(0);
        static_for<0, Q>([&](auto qc) {
            constexpr int q = decltype(qc)::value;
            const R cu = R(cx(q)) * ux + R(cy(q)) * uy + R(cz(q)) * uz;
            const R wr = R(wq(q)) * rho;
            const R feq = wr * (R(1) + R(3) * cu + R(4.5) * cu * cu - R(1.5) * u2);
            const R mu = omega * ls[q];
            g_rho += mu * feq * inv_rho;
            // d f_eq / d u' = w rho (3 c + 9 (c.u') c - 3 u')
            const R k = R(3) + R(9) * cu;
            gux += mu * wr * (k * R(cx(q)) - R(3) * ux);
            guy += mu * wr * (k * R(cy(q)) - R(3) * uy);
            guz += mu * wr * (k * R(cz(q)) - R(3) * uz);
            g_tau -= ls[q] * (feq - fv[q]) * (omega * omega);  // d omega / d tau = -1/tau^2
        });
        // u' = (j + tau F)/rho
        const R gjx = gux * inv_rho, gjy = guy * inv_rho, gjz = guz * inv_rho;
        g_rho -= (gux * ux + guy * uy + guz * uz) * inv_rho;
        g_tau += (gux * Fx + guy * Fy + guz * Fz) * inv_rho;
        const R gFx = tau * gjx, gFy = tau * gjy, gFz = tau * gjz;
        static_for<0, Q>([&](auto qc) {
            constexpr int q = decltype(qc)::value;
            lam_out[size_t(q) * n + i] =
                (R(1) - omega) * ls[q] + g_rho + R(cx(q)) * gjx + R(cy(q)) * gjy + R(cz(q)) * gjz;
        });
        fa[i] = ps * gFx;
        fa[n + i] = ps * gFy;
        fa[2 * size_t(n) + i] = ps * gFz;
        fa[3 * size_t(n) + i] = sx * gFx + sy * gFy + sz * gFz;
        // dF/dG = -psi S
        accG += double(-(ps * sx) * gFx - (ps * sy) * gFy - (ps * sz) * gFz);
        accT += double(g_tau);
    });
    block_sum2(accG, accT, partials + 2 * blockIdx.x);
}

// Force adjoint: g_psi(y) = -G [ T(y) + sum_a w_a c_a . V(y - c_a) ] and the
// density term gr(y) = g_psi(y) psi'(rho(y)), psi' = 1 - psi/rho0.
template <class R>
__global__ void __launch_bounds__(kThreads)
adj_force_kernel(const R* __restrict__ psi, const R* __restrict__ fa, R* __restrict__ gr, AdjointArgs a) {
    const unsigned n = unsigned(a.n);
    const R G = par<R>(a.G, a.Gf), rho0 = par<R>(a.rho0, a.rho0f);
    const R* __restrict__ Vx = fa;
    const R* __restrict__ Vy = fa + n;
    const R* __restrict__ Vz = fa + 2 * size_t(n);
    const R* __restrict__ T = fa + 3 * size_t(n);
    for_each_cell(a.nx, a.ny, a.nz, [&](const Row& w, const unsigned (&xs)[3], unsigned i) {
        R term = T[i];
        static_for<1, Q>([&](auto qc) {
            constexpr int q = decltype(qc)::value;
            const unsigned dn = nb_of(w, xs, -cx(q), -cy(q), -cz(q));  // y - c_q
            R cv = R(0);
            if constexpr (cx(q) != 0) cv += R(cx(q)) * Vx[dn];
            if constexpr (cy(q) != 0) cv += R(cy(q)) * Vy[dn];
            if constexpr (cz(q) != 0) cv += R(cz(q)) * Vz[dn];
            term += R(wq(q)) * cv;
        });
        // the same for every population: stored once, added where it is read
        gr[i] = -G * term * (R(1) - psi[i] / rho0);
    });
}

// lam_a(x, T) = dJ/drho(x) for every a (rho = sum_a f_a); no force term yet.
template <class R>
__global__ void adj_seed_kernel(const double* __restrict__ g, R* __restrict__ lam, R* __restrict__ gr, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const R v = R(g[i]);
        gr[i] = R(0);
        static_for<0, Q>([&](auto qc) {
            constexpr int q = decltype(qc)::value;
            lam[q * n + i] = v;
        });
    }
}

// f_a(x, 0) = w_a rho0(x): dJ/drho0(x) = sum_a w_a lam_a(x, 0), with
// lam_a = stored part + force term gr (sum_a w_a = 1).
template <class R>
__global__ void adj_rho0_kernel(const R* __restrict__ lam, const R* __restrict__ gr, double* __restrict__ out,
                                long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double s = double(gr[i]);
        static_for<0, Q>([&](auto qc) {
            constexpr int q = decltype(qc)::value;
            s += wq(q) * double(lam[q * n + i]);
        });
        out[i] = s;
    }
}

// Fixed-order sum of the per-block partials into acc[0..1]: each of 256
// threads sums a strided subset in block order, then a fixed tree.
__global__ void __launch_bounds__(kThreads) adj_reduce_kernel(const double* __restrict__ partials, int nblocks,
                                                             double* __restrict__ acc) {
    __shared__ double red[2][kThreads];
    double g = 0.0, t = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += kThreads) {
        g += partials[2 * b];
        t += partials[2 * b + 1];
    }
    red[0][threadIdx.x] = g;
    red[1][threadIdx.x] = t;
    __syncthreads();
    for (int s = kThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            red[0][threadIdx.x] += red[0][threadIdx.x + s];
            red[1][threadIdx.x] += red[1][threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        acc[0] += red[0][0];
        acc[1] += red[1][0];
    }
}

template <class R>
cudaError_t run_adjoint_step(const AdjointArgs& a, const void* f, void* psi, bool psi_ready, const void* lam_next,
                             const void* gr_next, void* lam_out, void* gr_out, void* gF, double* partials,
                             double* acc, cudaStream_t st) {
    const int grid = a.grid;
    const dim3 block(kRowThreads, kRows);
    if (!psi_ready)
        adj_psi_kernel<R><<<grid, block, 0, st>>>(static_cast<const R*>(f), static_cast<R*>(psi), unsigned(a.n),
                                                  par<R>(a.rho0, a.rho0f));
    adj_collide_kernel<R><<<grid, block, 0, st>>>(static_cast<const R*>(f), static_cast<const R*>(psi),
                                                  static_cast<const R*>(lam_next), static_cast<const R*>(gr_next),
                                                  static_cast<R*>(lam_out), static_cast<R*>(gF), partials, a);
    adj_force_kernel<R><<<grid, block, 0, st>>>(static_cast<const R*>(psi), static_cast<const R*>(gF),
                                                static_cast<R*>(gr_out), a);
    (void)acc;  // the per-block sums stay in `partials` until adjoint_reduce
    return cudaGetLastError();
}

}  // namespace

cudaError_t adjoint_step(const AdjointArgs& a, bool f64, const void* f, void* psi, bool psi_ready,
                         const void* lam_next, const void* gr_next, void* lam_out, void* gr_out, void* gF,
                         double* partials, double* acc, cudaStream_t st) {
    return f64 ? run_adjoint_step<double>(a, f, psi, psi_ready, lam_next, gr_next, lam_out, gr_out, gF, partials,
                                          acc, st)
               : run_adjoint_step<float>(a, f, psi, psi_ready, lam_next, gr_next, lam_out, gr_out, gF, partials,
                                         acc, st);
}

cudaError_t adjoint_seed(const AdjointArgs& a, bool f64, const double* dJdrho, void* lam, void* gr, cudaStream_t st) {
    if (f64)
        adj_seed_kernel<double><<<a.grid, kThreads, 0, st>>>(dJdrho, static_cast<double*>(lam),
                                                             static_cast<double*>(gr), a.n);
    else
        adj_seed_kernel<float><<<a.grid, kThreads, 0, st>>>(dJdrho, static_cast<float*>(lam), static_cast<float*>(gr),
                                                            a.n);
    return cudaGetLastError();
}

cudaError_t adjoint_rho0(const AdjointArgs& a, bool f64, const void* lam, const void* gr, double* out,
                         cudaStream_t st) {
    if (f64)
        adj_rho0_kernel<double><<<a.grid, kThreads, 0, st>>>(static_cast<const double*>(lam),
                                                             static_cast<const double*>(gr), out, a.n);
    else
        adj_rho0_kernel<float><<<a.grid, kThreads, 0, st>>>(static_cast<const float*>(lam),
                                                            static_cast<const float*>(gr), out, a.n);
    return cudaGetLastError();
}

int adjoint_threads() { return kThreads; }
int adjoint_rows_per_block() { return kRows; }

cudaError_t adjoint_reduce(const AdjointArgs& a, const double* partials, double* acc, cudaStream_t st) {
    adj_reduce_kernel<<<1, kThreads, 0, st>>>(partials, a.grid, acc);
    return cudaGetLastError();
}

}  // namespace lbm
