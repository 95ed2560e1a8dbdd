// Step kernel with the two-belt (multirange) pseudo-potential force, the
// extension of Eq. SC_force that Sec. 2 of the paper names as the way to set
// the surface tension independently of the equation of state:
//
//   F(x) = -psi(x) [ G1 sum_{a in D3Q19} w_a psi(x + c_a) c_a
//                  + G2 sum_{b in E8} (p_b / 3) psi(x + e_b) e_b ]
//
// E8: the 92 vectors with components in {-2..2} and |e|^2 in
// {1, 2, 3, 4, 5, 6, 8}; p: per shell 4/45, 1/21, 2/105, 5/504, 1/315, 1/630,
// 1/5040, the weights with unit second moment whose moment tensors are
// isotropic to eighth order.  The factor 1/3 gives belt 2 the lattice's
// second moment cs2, so the bulk equation of state is
// P = rho cs2 + cs2 (G1 + G2) psi^2 / 2 whatever the split of G1 + G2.
//
// Register-staged like sc_step_kernel, with a two-cell psi halo: a ring of
// eight planes of (TX + 4) x (TY + 4) psi values in shared memory (TY = 8 or
// 16: both 17.6 GLUPS for FP32 at 256 x 256 x 575 on GB300; summing the
// neighbours per shell before the coefficients measured 16.2 / 13.6); each
// iteration fills plane z + 2 (every slot from its cell's 19 populations),
// loads the populations of plane z, and after one barrier computes the force
// from the 92 neighbours of planes z - 2 .. z + 2, collides and pushes (the
// streaming itself is the D3Q19 one).
#pragma once
#include "e8.cuh"
#include "step_kernel.cuh"

namespace lbm {

template <class Codec, int COLL, int TX, int TY>
__global__ void __launch_bounds__(TX * TY)
sc_step_mr_kernel(const typename Codec::S* __restrict__ src, typename Codec::S* __restrict__ dst, const StepArgs a) {
    using R = typename Codec::R;
    static_assert(!Codec::kLocal, "the multirange kernel stores populations directly");
    constexpr int NT = TX * TY, PX = TX + 4, PY = TY + 4, PLANE = PX * PY, NSLOT = 8;
    __shared__ R psi_s[NSLOT][PLANE];

    const int tid = threadIdx.x;
    const int lx = tid % TX, ly = tid / TX;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const long long n = a.n;
    const long long plane = (long long)nx * ny;
    const int zs = blockIdx.z * a.zchunk;
    if (zs >= nz) return;  // uniform over the block
    const int ze = min(zs + a.zchunk, nz);

    const int gx = wrap_index(x0 + lx, nx), gy = wrap_index(y0 + ly, ny);
    const bool active = (x0 + lx < nx) && (y0 + ly < ny);
    const int my_slot = (ly + 2) * PX + (lx + 2);
    const long long my_xy = (long long)gy * nx + gx;
    const int xp = (gx + 1 == nx) ? 0 : gx + 1, xm = (gx == 0) ? nx - 1 : gx - 1;
    const int yp = (gy + 1 == ny) ? 0 : gy + 1, ym = (gy == 0) ? ny - 1 : gy - 1;
    const long long yoff[3] = {(long long)ym * nx, (long long)gy * nx, (long long)yp * nx};
    const int xidx[3] = {xm, gx, xp};

    const R rho0 = par<R>(a.rho0, a.rho0f), inv_rho0 = par<R>(a.inv_rho0, a.inv_rho0f);
    const DevParams dev = a.dev;
    // G1 w(s) + G2 p(s) / 3 per shell s = |e|^2
    R coef[9];
#pragma unroll
    for (int s = 0; s < 9; ++s) coef[s] = R(a.G * mr::w_d3q19(s) + a.G2 * mr::p_e8(s) / 3.0);

    auto wrapz = [&](int z) { return wrap_index(z, nz); };
    auto slot_of = [&](int z) { return (z - zs + 2) & (NSLOT - 1); };
    // psi of every slot (tile and two-cell halo) of plane z
    auto fill = [&](int z) {
        const long long zo = (long long)wrapz(z) * plane;
        R* ps = psi_s[slot_of(z)];
        for (int s = tid; s < PLANE; s += NT) {
            const int sx = s % PX - 2, sy = s / PX - 2;
            const long long cell = (long long)wrap_index(y0 + sy, ny) * nx + wrap_index(x0 + sx, nx);
            ps[s] = psi_of<R>(cell_density<Codec>(src + zo + cell, n, dev), rho0, inv_rho0);
        }
    };

    for (int z = zs - 2; z <= zs + 1; ++z) fill(z);
    for (int z = zs; z < ze; ++z) {
        fill(z + 2);
        R fc[Q];
        const long long zo = (long long)z * plane;
        static_for<0, Q>([&](auto qc) {
            constexpr int q = decltype(qc)::value;
            fc[q] = Codec::template load<q>(src + q * n + zo + my_xy, dev);
        });
        __syncthreads();
        if (active) {
            const R* pl[5] = {psi_s[slot_of(z - 2)], psi_s[slot_of(z - 1)], psi_s[slot_of(z)],
                              psi_s[slot_of(z + 1)], psi_s[slot_of(z + 2)]};
            R sx = R(0), sy = R(0), sz = R(0);
            static_for<0, mr::kNE>([&](auto kc) {
                constexpr mr::Vec e = mr::e8(decltype(kc)::value);
                constexpr int s = e.x * e.x + e.y * e.y + e.z * e.z;
                const R v = coef[s] * pl[e.z + 2][my_slot + e.x + e.y * PX];
                if constexpr (e.x != 0) sx += R(e.x) * v;
                if constexpr (e.y != 0) sy += R(e.y) * v;
                if constexpr (e.z != 0) sz += R(e.z) * v;
            });
            const R mpsi = -pl[2][my_slot];
            const R Fx = mpsi * sx, Fy = mpsi * sy, Fz = mpsi * sz;
            if constexpr (COLL == COLL_SRT)
                collide_srt<R>(fc, Fx, Fy, Fz, par<R>(a.tau, a.tauf), par<R>(a.omega, a.omegaf));
            else if constexpr (COLL == COLL_MRT) collide_mrt<R>(fc, Fx, Fy, Fz, rates<R>(a));
            else if constexpr (COLL == COLL_MRT_SPARSE) collide_mrt_sparse<R, false>(fc, Fx, Fy, Fz, rates<R>(a));
            else if constexpr (COLL == COLL_MRT_SHEAR)
                collide_mrt_sparse<R, false, false>(fc, Fx, Fy, Fz, rates<R>(a));
            else collide_mrt_sparse<R, true>(fc, Fx, Fy, Fz, rates<R>(a));
            // Eq. LBE streaming: f_a(x + c_a, t + 1) = f*_a(x, t).
            const int zm = (z == 0) ? nz - 1 : z - 1, zn = (z + 1 == nz) ? 0 : z + 1;
            const long long zoff[3] = {(long long)zm * plane, zo, (long long)zn * plane};
            static_for<0, Q>([&](auto qc) {
                constexpr int q = decltype(qc)::value;
                const long long idx = zoff[cz(q) + 1] + yoff[cy(q) + 1] + xidx[cx(q) + 1];
                Codec::template store<q>(dst + (q * n + idx), fc[q], a.dev);
            });
        }
    }
}

}  // namespace lbm
