// The fused Shan-Chen D3Q19 time step (Sec. 2 of arXiv:1905.09554):
// pseudo-potential psi(rho), single-belt force (Eq. SC_force), SRT with the
// shifted equilibrium velocity (Eq. vel_shift) or MRT with Guo-like forcing at
// the barycentric velocity (Eq. barycentric), and periodic streaming
// (Eq. LBE), in ONE kernel launch per step.
//
// Design (push scheme, 2.5D z-march):
//  * The state holds post-streaming populations f_a(x, t), SoA
//    f[a][z][y][x].  A cell's density needs only its own 19 values, so every
//    population load is aligned and coalesced.
//  * A thread block owns a TX x TY column of cells and walks a chunk of z
//    planes.  For each plane it loads the 19 populations of its cells into
//    registers, turns rho into psi in shared memory, and also computes psi on
//    the one-cell ring around the tile (those loads are other blocks' cells
//    of the same plane and are normally served by L2).  A ring of four psi
//    planes lets the block collide plane z once plane z+1 is in, with one
//    barrier per plane.  psi never goes to HBM.
//  * After the collision each cell pushes f*_a to x + c_a in the other copy.
// HBM traffic per cell update is therefore one read and one write of the 19
// populations plus the halo/chunk re-reads that miss L2.
#pragma once
#include <cuda.h>

#include <cstdint>
#include <cstring>

#include "codec.cuh"
#include "lattice.cuh"
#include "step_args.h"

namespace lbm {

// psi = rho0 (1 - exp(-rho/rho0)).  Float arithmetic uses the hardware
// exponential (__expf, a few ulp for the densities of a two-phase state,
// |rho/rho0| < 4) instead of the correctly rounded expf, whose range
// reduction costs about eight more instructions per call.
template <class R>
__device__ __forceinline__ R psi_of(R rho, R rho0, R inv_rho0);
template <>
__device__ __forceinline__ double psi_of<double>(double rho, double rho0, double inv_rho0) {
    return rho0 * (1.0 - exp(-rho * inv_rho0));
}
template <>
__device__ __forceinline__ float psi_of<float>(float rho, float rho0, float inv_rho0) {
    return rho0 * (1.0f - __expf(-rho * inv_rho0));
}

// 1/rho.  Float arithmetic uses the hardware reciprocal with one rounding
// step (__fdividef, within 2 ulp) instead of the IEEE division, whose
// special-case check adds a branch per cell.
template <class R>
__device__ __forceinline__ R recip(R x) {
    if constexpr (sizeof(R) == sizeof(double)) return 1.0 / x;
    else return __fdividef(1.0f, x);
}

// Population q of the field starting at p (population stride n elements).
// The 64-bit product comes from kernel parameters only, so with 32-bit cell
// offsets (I = unsigned) an access costs the cell offset's 32-bit arithmetic
// and one widening add.
template <class S, class I>
__device__ __forceinline__ S* pop_at(S* p, int q, I n) {
    return p + (long long)q * (long long)n;
}

__device__ __forceinline__ int wrap_index(int i, int n) {
    i %= n;
    return i < 0 ? i + n : i;
}

// SRT with shifted equilibrium (Eq. vel_shift): u' = (j + tau F)/rho,
// f* = f + (f_eq(rho, u') - f)/tau.  Velocities come in +/- pairs (q, q+1),
// whose equilibria share the even part A and differ by the sign of the odd
// part B: f_eq = A +/- B.
template <class R>
__device__ __forceinline__ void collide_srt(R (&f)[Q], R Fx, R Fy, R Fz, R tau, R omega) {
    R rho = f[0], jx = R(0), jy = R(0), jz = R(0);
    static_for<0, 9>([&](auto pc) {
        constexpr int q = 2 * decltype(pc)::value + 1;
        const R sum = f[q] + f[q + 1], dif = f[q] - f[q + 1];
        rho += sum;
        if constexpr (cx(q) != 0) jx += R(cx(q)) * dif;
        if constexpr (cy(q) != 0) jy += R(cy(q)) * dif;
        if constexpr (cz(q) != 0) jz += R(cz(q)) * dif;
    });
    const R inv_rho = recip(rho);
    const R ux = (jx + tau * Fx) * inv_rho;
    const R uy = (jy + tau * Fy) * inv_rho;
    const R uz = (jz + tau * Fz) * inv_rho;
    const R usq = R(1.5) * (ux * ux + uy * uy + uz * uz);
    const R base = R(1) - usq;
    // w_a rho per speed shell, the rest one from sum_a w_a = 1: the rounded
    // weights float(1/3) + 6 float(1/18) + 12 float(1/36) sum to 1 + 3e-8,
    // which made FP32 runs gain ~3e-8 of their mass every step.
    const R r1 = R(wq(1)) * rho, r2 = R(wq(7)) * rho;
    const R r0 = rho - R(6) * r1 - R(12) * r2;
    // f* = (1 - omega) f + omega (A +/- B): omega w rho per shell once
    const R keep = R(1) - omega;
    const R o1 = omega * r1, o2 = omega * r2, o1b = R(3) * o1, o2b = R(3) * o2;
    f[0] = keep * f[0] + omega * (r0 * base);
    static_for<0, 9>([&](auto pc) {
        constexpr int q = 2 * decltype(pc)::value + 1;
        R cu = R(0);
        if constexpr (cx(q) != 0) cu += R(cx(q)) * ux;
        if constexpr (cy(q) != 0) cu += R(cy(q)) * uy;
        if constexpr (cz(q) != 0) cu += R(cz(q)) * uz;
        constexpr bool axis = wq(q) == wq(1);
        const R oA = (axis ? o1 : o2) * (base + R(4.5) * cu * cu);
        const R oB = (axis ? o1b : o2b) * cu;
        f[q] = keep * f[q] + (oA + oB);
        f[q + 1] = keep * f[q + 1] + (oA - oB);
    });
}

// MRT with Guo-like forcing (Eq. barycentric), d'Humieres D3Q19 basis:
// m = M f, u_b = (j + F/2)/rho,
// f* = f - M^-1 [ Lambda (m - m_eq(rho, u_b)) - (I - Lambda/2) M S ],
// with the closed forms of m_eq = M f_eq and of the Guo source moments M S.
// Conserved moments: the rho row vanishes and the j rows reduce to -F.
template <class R>
__device__ __forceinline__ void collide_mrt(R (&f)[Q], R Fx, R Fy, R Fz, const R (&s)[Q]) {
    // Pair sums feed the moments that are even in c, pair differences the
    // odd ones (M[k][q+1] = +/- M[k][q] for the opposite velocity q+1).
    R ps[9], pd[9];
    static_for<0, 9>([&](auto pc) {
        constexpr int p = decltype(pc)::value, q = 2 * p + 1;
        ps[p] = f[q] + f[q + 1];
        pd[p] = f[q] - f[q + 1];
    });
    R m[Q];
    static_for<0, Q>([&](auto kc) {
        constexpr int k = decltype(kc)::value;
        constexpr bool odd = mrt_moment_is_odd(k);
        R acc = R(0);
        if constexpr (!odd) {
            constexpr int c0 = mrt_coef(k, 0);
            if constexpr (c0 != 0) acc = R(c0) * f[0];
        }
        static_for<0, 9>([&](auto pc) {
            constexpr int p = decltype(pc)::value, q = 2 * p + 1;
            constexpr int c = mrt_coef(k, q);
            const R v = odd ? pd[p] : ps[p];
            if constexpr (c == 1) acc += v;
            else if constexpr (c == -1) acc -= v;
            else if constexpr (c != 0) acc += R(c) * v;
        });
        m[k] = acc;
    });
    const R rho = m[0];
    const R inv_rho = recip(rho);
    const R ux = (m[3] + R(0.5) * Fx) * inv_rho;
    const R uy = (m[5] + R(0.5) * Fy) * inv_rho;
    const R uz = (m[7] + R(0.5) * Fz) * inv_rho;
    const R ux2 = ux * ux, uy2 = uy * uy, uz2 = uz * uz;
    const R u2 = ux2 + uy2 + uz2;
    const R uF = ux * Fx + uy * Fy + uz * Fz;
    const R pxx = R(2) * ux2 - uy2 - uz2, pww = uy2 - uz2;
    const R gxx = R(2) * ux * Fx - uy * Fy - uz * Fz, gww = uy * Fy - uz * Fz;

    R meq[Q], sg[Q];
    meq[1] = rho * (R(-11) + R(19) * u2);         sg[1] = R(38) * uF;
    meq[2] = rho * (R(3) - R(5.5) * u2);          sg[2] = R(-11) * uF;
    meq[4] = R(-2.0 / 3.0) * rho * ux;            sg[4] = R(-2.0 / 3.0) * Fx;
    meq[6] = R(-2.0 / 3.0) * rho * uy;            sg[6] = R(-2.0 / 3.0) * Fy;
    meq[8] = R(-2.0 / 3.0) * rho * uz;            sg[8] = R(-2.0 / 3.0) * Fz;
    meq[9] = rho * pxx;                           sg[9] = R(2) * gxx;
    meq[10] = R(-0.5) * rho * pxx;                sg[10] = -gxx;
    meq[11] = rho * pww;                          sg[11] = R(2) * gww;
    meq[12] = R(-0.5) * rho * pww;                sg[12] = -gww;
    meq[13] = rho * ux * uy;                      sg[13] = ux * Fy + uy * Fx;
    meq[14] = rho * uy * uz;                      sg[14] = uy * Fz + uz * Fy;
    meq[15] = rho * ux * uz;                      sg[15] = ux * Fz + uz * Fx;
    meq[16] = R(0);                               sg[16] = R(0);
    meq[17] = R(0);                               sg[17] = R(0);
    meq[18] = R(0);                               sg[18] = R(0);

    // d[k] = (Lambda (m - m_eq) - (I - Lambda/2) S)_k / norm_k
    R d[Q];
    d[0] = R(0);
    d[3] = -Fx * R(1.0 / mrt_norm(3));
    d[5] = -Fy * R(1.0 / mrt_norm(5));
    d[7] = -Fz * R(1.0 / mrt_norm(7));
    static_for<0, Q>([&](auto kc) {
        constexpr int k = decltype(kc)::value;
        if constexpr (k != 0 && k != 3 && k != 5 && k != 7) {
            const R sk = s[k];
            d[k] = (sk * (m[k] - meq[k]) - (R(1) - R(0.5) * sk) * sg[k]) * R(1.0 / mrt_norm(k));
        }
    });
    // f* = f - M^T d: the even moments give the common part E of a velocity
    // pair, the odd ones the antisymmetric part O (f*_q = f_q - E - O,
    // f*_{q+1} = f_{q+1} - E + O).
    {
        R e0 = R(0);
        static_for<1, Q>([&](auto kc) {
            constexpr int k = decltype(kc)::value;
            constexpr int c = mrt_coef(k, 0);
            if constexpr (c != 0) e0 += R(c) * d[k];
        });
        f[0] -= e0;
    }
    static_for<0, 9>([&](auto pc) {
        constexpr int q = 2 * decltype(pc)::value + 1;
        R E = R(0), O = R(0);
        static_for<1, Q>([&](auto kc) {
            constexpr int k = decltype(kc)::value;
            constexpr int c = mrt_coef(k, q);
            constexpr bool odd = mrt_coef(k, q + 1) == -c && c != 0;
            if constexpr (c != 0) {
                if constexpr (odd) {
                    if constexpr (c == 1) O += d[k];
                    else if constexpr (c == -1) O -= d[k];
                    else O += R(c) * d[k];
                } else {
                    if constexpr (c == 1) E += d[k];
                    else if constexpr (c == -1) E -= d[k];
                    else E += R(c) * d[k];
                }
            }
        });
        f[q] -= E + O;
        f[q + 1] -= E - O;
    });
}

// MRT with Guo-like forcing when every rate outside K = {e, 3pxx, pww, pxy,
// pyz, pxz} equals 1 (the paper's rule, and the shear rule), or when every
// rate equals 1 (UNIT).  Writing m* = m_eq + S/2 + (1 - s)(m - m_eq + S/2),
// the conserved rows vanish (rho: m = m_eq, S = 0; j: m - m_eq = -F/2,
// S = F), rows with s = 1 vanish, and
//   f* = f_eq(rho, u_b) + S_pop/2 + sum_{k in K} M_k^T (1 - s_k)(m_k - m_eq_k + S_k/2)/norm_k.
// Algebraically identical to collide_mrt for such rates, with far fewer
// operations (only the even rows of K are transformed).  WITH_E = false is
// the shear rule's form: the energy row relaxes at 1 there, its correction
// is exactly zero and the row is left out (a separate instantiation, chosen
// on the host, so no kernel carries both forms).
template <class R, bool UNIT, bool WITH_E = true>
__device__ __forceinline__ void collide_mrt_sparse(R (&f)[Q], R Fx, R Fy, R Fz, const R (&s)[Q]) {
    constexpr int K0 = WITH_E ? 0 : 1;  // first row of K transformed
    R ps[9], rho = f[0], jx = R(0), jy = R(0), jz = R(0);
    static_for<0, 9>([&](auto pc) {
        constexpr int p = decltype(pc)::value, q = 2 * p + 1;
        ps[p] = f[q] + f[q + 1];
        const R dif = f[q] - f[q + 1];
        rho += ps[p];
        if constexpr (cx(q) != 0) jx += R(cx(q)) * dif;
        if constexpr (cy(q) != 0) jy += R(cy(q)) * dif;
        if constexpr (cz(q) != 0) jz += R(cz(q)) * dif;
    });
    const R inv_rho = recip(rho);
    const R ux = (jx + R(0.5) * Fx) * inv_rho;
    const R uy = (jy + R(0.5) * Fy) * inv_rho;
    const R uz = (jz + R(0.5) * Fz) * inv_rho;
    const R ux2 = ux * ux, uy2 = uy * uy, uz2 = uz * uz;
    const R u2 = ux2 + uy2 + uz2;
    const R uF = ux * Fx + uy * Fy + uz * Fz;

    // correction per even row of K, already divided by the row norm
    constexpr int KS[6] = {1, 9, 11, 13, 14, 15};
    R dk[6] = {R(0), R(0), R(0), R(0), R(0), R(0)};
    if constexpr (!UNIT) {
        const R pxx = R(2) * ux2 - uy2 - uz2, pww = uy2 - uz2;
        const R gxx = R(2) * ux * Fx - uy * Fy - uz * Fz, gww = uy * Fy - uz * Fz;
        const R meq[6] = {rho * (R(-11) + R(19) * u2), rho * pxx, rho * pww, rho * ux * uy, rho * uy * uz,
                          rho * ux * uz};
        const R sg[6] = {R(38) * uF, R(2) * gxx, R(2) * gww, ux * Fy + uy * Fx, uy * Fz + uz * Fy, ux * Fz + uz * Fx};
        static_for<K0, 6>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            constexpr int k = KS[i];
            R m = R(0);
            constexpr int c0 = mrt_coef(k, 0);
            if constexpr (c0 != 0) m = R(c0) * f[0];
            static_for<0, 9>([&](auto pc) {
                constexpr int p = decltype(pc)::value;
                constexpr int c = mrt_coef(k, 2 * p + 1);
                if constexpr (c == 1) m += ps[p];
                else if constexpr (c == -1) m -= ps[p];
                else if constexpr (c != 0) m += R(c) * ps[p];
            });
            dk[i] = (R(1) - s[k]) * (m - meq[i] + R(0.5) * sg[i]) * R(1.0 / mrt_norm(k));
        });
    }
    auto corr = [&](auto qc) {
        constexpr int q = decltype(qc)::value;
        R acc = R(0);
        if constexpr (!UNIT) {
            static_for<K0, 6>([&](auto ic) {
                constexpr int i = decltype(ic)::value;
                constexpr int c = mrt_coef(KS[i], q);
                if constexpr (c == 1) acc += dk[i];
                else if constexpr (c == -1) acc -= dk[i];
                else if constexpr (c != 0) acc += R(c) * dk[i];
            });
        }
        return acc;
    };
    const R base = R(1) - R(1.5) * u2;
    // w_a rho per speed shell, the rest one from sum_a w_a = 1 (as in
    // collide_srt: no systematic mass from the rounded weights)
    const R r1 = R(wq(1)) * rho, r2 = R(wq(7)) * rho;
    const R r0 = rho - R(6) * r1 - R(12) * r2;
    const R r1b = R(3) * r1, r2b = R(3) * r2, uF15 = R(1.5) * uF;
    f[0] = r0 * base - R(wq(0)) * uF15 + corr(std::integral_constant<int, 0>{});
    static_for<0, 9>([&](auto pc) {
        constexpr int q = 2 * decltype(pc)::value + 1;
        R cu = R(0), cF = R(0);
        if constexpr (cx(q) != 0) { cu += R(cx(q)) * ux; cF += R(cx(q)) * Fx; }
        if constexpr (cy(q) != 0) { cu += R(cy(q)) * uy; cF += R(cy(q)) * Fy; }
        if constexpr (cz(q) != 0) { cu += R(cz(q)) * uz; cF += R(cz(q)) * Fz; }
        constexpr bool axis = wq(q) == wq(1);
        // f_eq = A +/- B and the Guo source S/2 = E +/- O, as the even part
        // A + E = w rho (base + 4.5 cu^2) + w (4.5 cu cF - 1.5 u.F) and the
        // odd part B + O = 3 w rho cu + 1.5 w cF of the velocity pair
        const R cu45 = R(4.5) * cu;
        const R even = (axis ? r1 : r2) * (base + cu45 * cu) + R(wq(q)) * (cu45 * cF - uF15);
        const R odd = (axis ? r1b : r2b) * cu + R(1.5 * wq(q)) * cF;
        const R e = even + corr(std::integral_constant<int, q>{});  // even rows: equal on both members
        f[q] = e + odd;
        f[q + 1] = e - odd;
    });
}

template <class Codec>
__device__ __forceinline__ typename Codec::R cell_density(const typename Codec::S* __restrict__ p,
                                                          long long n, const DevParams& dev, float ref = 0.0f) {
    using R = typename Codec::R;
    R r = R(0);
    static_for<0, Q>([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        if constexpr (Codec::kLocal) r += Codec::template load_ref<q>(p + q * n, ref, dev);
        else r += Codec::template load<q>(p + q * n, dev);
    });
    return r;
}

// Force from the psi ring (planes z-1, z, z+1 of the tile + ring), collision
// of the cell's populations fc, and push to x + c_a in `dst`.
template <class Codec, int COLL, int PX, class I = long long>
__device__ __forceinline__ void update_cell(typename Codec::R (&fc)[Q], const typename Codec::R* pm,
                                            const typename Codec::R* p0, const typename Codec::R* pp,
                                            int slot, typename Codec::S* __restrict__ dst, I n,
                                            const I (&zoff)[3], const I (&yoff)[3],
                                            const int (&xidx)[3], const StepArgs& a,
                                            const float* const* rho_pl = nullptr) {
    using R = typename Codec::R;
    const R* pl[3] = {pm, p0, pp};
    // Eq. SC_force: F = -G psi(x) sum_a w_a psi(x + c_a) c_a.
    R sx = R(0), sy = R(0), sz = R(0);
    static_for<1, Q>([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        const R v = pl[cz(q) + 1][slot + cx(q) + cy(q) * PX];
        if constexpr (cx(q) != 0) sx += R(wq(q) * cx(q)) * v;
        if constexpr (cy(q) != 0) sy += R(wq(q) * cy(q)) * v;
        if constexpr (cz(q) != 0) sz += R(wq(q) * cz(q)) * v;
    });
    const R gpsi = -par<R>(a.G, a.Gf) * p0[slot];
    const R Fx = gpsi * sx, Fy = gpsi * sy, Fz = gpsi * sz;

    if constexpr (COLL == COLL_SRT) collide_srt<R>(fc, Fx, Fy, Fz, par<R>(a.tau, a.tauf), par<R>(a.omega, a.omegaf));
    else if constexpr (COLL == COLL_MRT) collide_mrt<R>(fc, Fx, Fy, Fz, rates<R>(a));
    else if constexpr (COLL == COLL_MRT_SPARSE) collide_mrt_sparse<R, false>(fc, Fx, Fy, Fz, rates<R>(a));
    else if constexpr (COLL == COLL_MRT_SHEAR) collide_mrt_sparse<R, false, false>(fc, Fx, Fy, Fz, rates<R>(a));
    else collide_mrt_sparse<R, true>(fc, Fx, Fy, Fz, rates<R>(a));

    // Eq. LBE streaming: f_a(x + c_a, t + 1) = f*_a(x, t).
    static_for<0, Q>([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        const I idx = zoff[cz(q) + 1] + yoff[cy(q) + 1] + xidx[cx(q) + 1];
        if constexpr (Codec::kLocal) {
            // deviation from the rest equilibrium at the destination's density
            const float ref = rho_pl[cz(q) + 1][slot + cx(q) + cy(q) * PX];
            Codec::template store_ref<q>(pop_at(dst, q, n) + idx, fc[q], ref, a.dev);
        } else {
            Codec::template store<q>(pop_at(dst, q, n) + idx, fc[q], a.dev);
        }
    });
}

template <class Codec, int COLL, int TX, int TY>
__global__ void __launch_bounds__(TX * TY)
sc_step_kernel(const typename Codec::S* __restrict__ src, typename Codec::S* __restrict__ dst,
               const StepArgs a) {
    using R = typename Codec::R;
    constexpr int PX = TX + 2, PY = TY + 2, PLANE = PX * PY, NSLOT = 4;
    constexpr int NHALO = 2 * PX + 2 * TY;
    static_assert(NHALO <= TX * TY, "tile too small for its halo ring");
    __shared__ R psi_s[NSLOT][PLANE];
    // local-reference storage: densities of the same planes (encode targets)
    constexpr bool LOCAL = Codec::kLocal;
    __shared__ float rho_s[LOCAL ? NSLOT : 1][LOCAL ? PLANE : 1];

    const int tid = threadIdx.x;
    const int lx = tid % TX, ly = tid / TX;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const long long n = a.n;
    const long long plane = (long long)nx * ny;
    const int zs = blockIdx.z * a.zchunk;
    if (zs >= nz) return;  // uniform over the block
    const int ze = min(zs + a.zchunk, nz);

    // Own cell (wrapped so that threads past a ragged edge still fill psi).
    const int gx = wrap_index(x0 + lx, nx), gy = wrap_index(y0 + ly, ny);
    const bool active = (x0 + lx < nx) && (y0 + ly < ny);
    const int my_slot = (ly + 1) * PX + (lx + 1);
    const long long my_xy = (long long)gy * nx + gx;

    // Ring cell handled by this thread, if any.
    int h_slot = -1;
    long long h_xy = 0;
    if (tid < NHALO) {
        int hx, hy;
        if (tid < PX) { hx = tid - 1; hy = -1; }
        else if (tid < 2 * PX) { hx = tid - PX - 1; hy = TY; }
        else { const int k = tid - 2 * PX; hx = (k < TY) ? -1 : TX; hy = (k < TY) ? k : k - TY; }
        h_slot = (hy + 1) * PX + (hx + 1);
        h_xy = (long long)wrap_index(y0 + hy, ny) * nx + wrap_index(x0 + hx, nx);
    }

    // Push targets in x and y (periodic).
    const int xp = (gx + 1 == nx) ? 0 : gx + 1, xm = (gx == 0) ? nx - 1 : gx - 1;
    const int yp = (gy + 1 == ny) ? 0 : gy + 1, ym = (gy == 0) ? ny - 1 : gy - 1;
    const long long yoff[3] = {(long long)ym * nx, (long long)gy * nx, (long long)yp * nx};
    const int xidx[3] = {xm, gx, xp};

    const R rho0 = par<R>(a.rho0, a.rho0f), inv_rho0 = par<R>(a.inv_rho0, a.inv_rho0f);
    const DevParams dev = a.dev;

    auto slot_of = [&](int z) { return (z - zs + 1) & (NSLOT - 1); };
    auto ref_at = [&](long long cell) -> float {
        if constexpr (LOCAL) return __ldg(a.ref_src + cell);
        else return 0.0f;
    };
    auto put_rho = [&](int slot, int idx, R r) {
        if constexpr (LOCAL) rho_s[slot][idx] = r;
    };
    auto load_q = [&](auto qc, const typename Codec::S* p, float ref) {
        constexpr int q = decltype(qc)::value;
        if constexpr (LOCAL) return Codec::template load_ref<q>(p, ref, dev);
        else return Codec::template load<q>(p, dev);
    };

    // Prologue: psi of plane zs-1, then populations and psi of plane zs.
    {
        const int zm = (zs == 0) ? nz - 1 : zs - 1;
        const long long zo = (long long)zm * plane;
        const R r = cell_density<Codec>(src + zo + my_xy, n, dev, ref_at(zo + my_xy));
        psi_s[slot_of(zs - 1)][my_slot] = psi_of<R>(r, rho0, inv_rho0);
        put_rho(slot_of(zs - 1), my_slot, r);
        if (h_slot >= 0) {
            const R rh = cell_density<Codec>(src + zo + h_xy, n, dev, ref_at(zo + h_xy));
            psi_s[slot_of(zs - 1)][h_slot] = psi_of<R>(rh, rho0, inv_rho0);
            put_rho(slot_of(zs - 1), h_slot, rh);
        }
    }
    R fc[Q];
    {
        const long long zo = (long long)zs * plane;
        const float ref = ref_at(zo + my_xy);
        R r = R(0);
        static_for<0, Q>([&](auto qc) {
            constexpr int q = decltype(qc)::value;
            fc[q] = load_q(qc, src + q * n + zo + my_xy, ref);
            r += fc[q];
        });
        psi_s[slot_of(zs)][my_slot] = psi_of<R>(r, rho0, inv_rho0);
        if (a.psi_out && active) static_cast<R*>(a.psi_out)[zo + my_xy] = psi_s[slot_of(zs)][my_slot];
        put_rho(slot_of(zs), my_slot, r);
        if (h_slot >= 0) {
            const R rh = cell_density<Codec>(src + zo + h_xy, n, dev, ref_at(zo + h_xy));
            psi_s[slot_of(zs)][h_slot] = psi_of<R>(rh, rho0, inv_rho0);
            put_rho(slot_of(zs), h_slot, rh);
        }
    }

    for (int z = zs; z < ze; ++z) {
        const int zn = (z + 1 == nz) ? 0 : z + 1;
        const int zp_slot = slot_of(z + 1);
        R fn[Q];
        {
            const long long zo = (long long)zn * plane;
            const float ref = ref_at(zo + my_xy);
            R r = R(0);
            static_for<0, Q>([&](auto qc) {
                constexpr int q = decltype(qc)::value;
                fn[q] = load_q(qc, src + q * n + zo + my_xy, ref);
                r += fn[q];
            });
            psi_s[zp_slot][my_slot] = psi_of<R>(r, rho0, inv_rho0);
            if (a.psi_out && active && z + 1 < ze) static_cast<R*>(a.psi_out)[zo + my_xy] = psi_s[zp_slot][my_slot];
            put_rho(zp_slot, my_slot, r);
            if (h_slot >= 0) {
                const R rh = cell_density<Codec>(src + zo + h_xy, n, dev, ref_at(zo + h_xy));
                psi_s[zp_slot][h_slot] = psi_of<R>(rh, rho0, inv_rho0);
                put_rho(zp_slot, h_slot, rh);
            }
        }
        __syncthreads();

        if (active) {
            const int zm = (z == 0) ? nz - 1 : z - 1;
            const long long zoff[3] = {(long long)zm * plane, (long long)z * plane, (long long)zn * plane};
            if constexpr (LOCAL) {
                const float* rp[3] = {rho_s[slot_of(z - 1)], rho_s[slot_of(z)], rho_s[zp_slot]};
                update_cell<Codec, COLL, PX>(fc, psi_s[slot_of(z - 1)], psi_s[slot_of(z)], psi_s[zp_slot], my_slot,
                                             dst, n, zoff, yoff, xidx, a, rp);
                a.ref_dst[zoff[1] + my_xy] = rho_s[slot_of(z)][my_slot];  // this cell's density now
            } else {
                update_cell<Codec, COLL, PX>(fc, psi_s[slot_of(z - 1)], psi_s[slot_of(z)], psi_s[zp_slot], my_slot,
                                             dst, n, zoff, yoff, xidx, a);
            }
        }
        static_for<0, Q>([&](auto qc) {
            constexpr int q = decltype(qc)::value;
            fc[q] = fn[q];
        });
    }
}


// ----------------------------------------------------------------------------
// Asynchronous-copy variant (FP32 / FP64 storage).
//
// Same arithmetic as sc_step_kernel, but the populations of each plane (the
// tile's cells and its one-cell ring) are fetched with cp.async into a
// three-stage shared-memory pipeline two planes ahead of the collision, so
// the loads in flight per SM no longer depend on registers.  Every thread
// reads back only the stage slots it copied itself, so the stages need no
// barrier; the psi ring keeps its single barrier per plane.  The grid is
// persistent: each block walks work items (xy tile, z chunk) in a fixed
// round-robin order.
// ----------------------------------------------------------------------------
namespace async_copy {
__device__ __forceinline__ void commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }
template <int BYTES>
__device__ __forceinline__ void copy(void* smem, const void* gmem) {
    static_assert(BYTES == 4 || BYTES == 8, "cp.async element size");
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(s), "l"(gmem), "n"(BYTES) : "memory");
}
}  // namespace async_copy

template <class Codec, int TX, int TY>
struct AsyncLayout {
    using S = typename Codec::S;
    using R = typename Codec::R;
    static constexpr int NT = TX * TY;
    static constexpr int NHALO = 2 * (TX + 2) + 2 * TY;
    static constexpr int PX = TX + 2;
    static constexpr int PLANE = PX * (TY + 2);
    static constexpr int NSTAGE = 3;
    static constexpr int NSLOT = 4;
    static constexpr int SLOTS = NT + NHALO;  // stage slots per population
    static constexpr size_t stage_bytes = sizeof(S) * Q * SLOTS;
    static constexpr size_t bytes = NSTAGE * stage_bytes + sizeof(R) * NSLOT * PLANE;
};

template <class Codec, int COLL, int TX, int TY>
__global__ void __launch_bounds__(TX * TY)
sc_step_async_kernel(const typename Codec::S* __restrict__ src, typename Codec::S* __restrict__ dst,
                     const StepArgs a) {
    using R = typename Codec::R;
    using S = typename Codec::S;
    using L = AsyncLayout<Codec, TX, TY>;
    constexpr int PX = L::PX, PLANE = L::PLANE, NT = L::NT, SLOTS = L::SLOTS;
    static_assert(L::NHALO <= NT, "tile too small for its halo ring");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    S* stage = reinterpret_cast<S*>(smem_raw);
    R* ring = reinterpret_cast<R*>(smem_raw + L::NSTAGE * L::stage_bytes);

    const int tid = threadIdx.x;
    const int lx = tid % TX, ly = tid / TX;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const long long n = a.n;
    const long long plane = (long long)nx * ny;
    const R rho0 = par<R>(a.rho0, a.rho0f), inv_rho0 = par<R>(a.inv_rho0, a.inv_rho0f);
    const DevParams dev = a.dev;
    const int my_slot = (ly + 1) * PX + (lx + 1);

    // Ring cell of this thread, as tile-relative coordinates (fixed per thread).
    int hx = 0, hy = 0, h_slot = -1;
    if (tid < L::NHALO) {
        if (tid < PX) { hx = tid - 1; hy = -1; }
        else if (tid < 2 * PX) { hx = tid - PX - 1; hy = TY; }
        else { const int k = tid - 2 * PX; hx = (k < TY) ? -1 : TX; hy = (k < TY) ? k : k - TY; }
        h_slot = (hy + 1) * PX + (hx + 1);
    }

    for (int item = blockIdx.x; item < a.n_items; item += gridDim.x) {
        const int tile = item % a.n_tiles, chunk = item / a.n_tiles;
        const int x0 = (tile % a.tiles_x) * TX, y0 = (tile / a.tiles_x) * TY;
        const int zs = chunk * a.zchunk;
        const int ze = min(zs + a.zchunk, nz);

        const int gx = wrap_index(x0 + lx, nx), gy = wrap_index(y0 + ly, ny);
        const bool active = (x0 + lx < nx) && (y0 + ly < ny);
        const long long my_xy = (long long)gy * nx + gx;
        const long long h_xy = (h_slot >= 0) ? (long long)wrap_index(y0 + hy, ny) * nx + wrap_index(x0 + hx, nx) : 0;
        const int xp = (gx + 1 == nx) ? 0 : gx + 1, xm = (gx == 0) ? nx - 1 : gx - 1;
        const int yp = (gy + 1 == ny) ? 0 : gy + 1, ym = (gy == 0) ? ny - 1 : gy - 1;
        const long long yoff[3] = {(long long)ym * nx, (long long)gy * nx, (long long)yp * nx};
        const int xidx[3] = {xm, gx, xp};

        auto stage_of = [&](int z) { return (z - zs + 1) % L::NSTAGE; };
        auto slot_of = [&](int z) { return (z - zs + 1) & (L::NSLOT - 1); };
        // Copy plane z (periodic) of this thread's cell and ring cell.
        auto issue = [&](int z) {
            const int zw = z < 0 ? z + nz : (z >= nz ? z - nz : z);
            const S* base = src + (long long)zw * plane;
            S* st = stage + stage_of(z) * (Q * SLOTS);
            static_for<0, Q>([&](auto qc) {
                constexpr int q = decltype(qc)::value;
                async_copy::copy<sizeof(S)>(st + q * SLOTS + tid, base + q * n + my_xy);
            });
            if (h_slot >= 0) {
                static_for<0, Q>([&](auto qc) {
                    constexpr int q = decltype(qc)::value;
                    async_copy::copy<sizeof(S)>(st + q * SLOTS + NT + tid, base + q * n + h_xy);
                });
            }
            async_copy::commit();
        };
        auto psi_from_stage = [&](int z) {
            const S* st = stage + stage_of(z) * (Q * SLOTS);
            R r = R(0);
            static_for<0, Q>([&](auto qc) {
                constexpr int q = decltype(qc)::value;
                r += Codec::template decode<q>(st[q * SLOTS + tid], dev);
            });
            ring[slot_of(z) * PLANE + my_slot] = psi_of<R>(r, rho0, inv_rho0);
            if (h_slot >= 0) {
                R rh = R(0);
                static_for<0, Q>([&](auto qc) {
                    constexpr int q = decltype(qc)::value;
                    rh += Codec::template decode<q>(st[q * SLOTS + NT + tid], dev);
                });
                ring[slot_of(z) * PLANE + h_slot] = psi_of<R>(rh, rho0, inv_rho0);
            }
        };

        __syncthreads();  // the previous item's readers of the psi ring are done
        issue(zs - 1);
        issue(zs);
        issue(zs + 1);
        async_copy::wait<2>();
        psi_from_stage(zs - 1);
        async_copy::wait<1>();
        psi_from_stage(zs);

        for (int z = zs; z < ze; ++z) {
            if (z + 2 <= ze) issue(z + 2);
            else async_copy::commit();
            async_copy::wait<1>();
            psi_from_stage(z + 1);
            __syncthreads();
            if (active) {
                const S* st = stage + stage_of(z) * (Q * SLOTS);
                R fc[Q];
                static_for<0, Q>([&](auto qc) {
                    constexpr int q = decltype(qc)::value;
                    fc[q] = Codec::template decode<q>(st[q * SLOTS + tid], dev);
                });
                const int zm = (z == 0) ? nz - 1 : z - 1;
                const int zn = (z + 1 == nz) ? 0 : z + 1;
                const long long zoff[3] = {(long long)zm * plane, (long long)z * plane, (long long)zn * plane};
                update_cell<Codec, COLL, PX>(fc, ring + slot_of(z - 1) * PLANE, ring + slot_of(z) * PLANE,
                                             ring + slot_of(z + 1) * PLANE, my_slot, dst, n, zoff, yoff, xidx, a);
            }
        }
    }
    async_copy::wait<0>();
}

// ----------------------------------------------------------------------------
// Pipelined variant (FP32 / FP64 storage, and the global-reference 16-bit
// formats with nx even).
//
// The register-staged kernel waits for each plane's loads right after issuing
// them.  Here the loads of plane z+2 are issued before the collision of
// plane z and consumed after it, so one plane of loads per thread is always
// in flight while the block computes.  The ring cells' populations (needed
// only for psi) go through a three-stage cp.async buffer two planes ahead,
// so ring loads never stall the block's barrier.  Persistent grid over
// (xy tile, z chunk) work items as in sc_step_async_kernel.
//
// 16-bit storage: cp.async moves at least 4 bytes, so each ring cell copies
// the aligned 4-byte word that holds it (with nx even a row never splits a
// word: the cell at even x is the low half, at odd x the high half), and the
// prefetched plane is kept as raw 16-bit values, decoded after the collision
// so that the decode does not wait for the loads.
// ----------------------------------------------------------------------------
template <class Codec, int TX, int TY>
struct PipeLayout {
    using S = typename Codec::S;
    using R = typename Codec::R;
    static constexpr bool kWord = sizeof(S) == 2;  // ring cells as aligned 4-byte words
    using HS = std::conditional_t<kWord, uint32_t, S>;
    static constexpr int NT = TX * TY;
    static constexpr int NHALO = 2 * (TX + 2) + 2 * TY;
    static constexpr int PX = TX + 2;
    static constexpr int PLANE = PX * (TY + 2);
    static constexpr int NSTAGE = 3;
    static constexpr int NSLOT = 4;
    static constexpr size_t stage_bytes = sizeof(HS) * Q * NHALO;
    // local-reference storage: the ring cells' reference densities (one
    // float per ring cell and stage) and the density planes (encode targets)
    static constexpr bool kLocal = Codec::kLocal;
    static constexpr size_t ref_stage_bytes = kLocal ? sizeof(float) * NHALO : 0;
    static constexpr size_t rho_ring_bytes = kLocal ? sizeof(float) * NSLOT * PLANE : 0;
    static constexpr size_t bytes =
        NSTAGE * (stage_bytes + ref_stage_bytes) + sizeof(R) * NSLOT * PLANE + rho_ring_bytes;
};

// The 16-bit value in the low (hi = 0) or high (hi = 1) half of a word.
template <class S>
__device__ __forceinline__ S half_of(uint32_t w, int hi) {
    const unsigned short b = hi ? (unsigned short)(w >> 16) : (unsigned short)(w & 0xffffu);
    S v;
    memcpy(&v, &b, sizeof(b));
    return v;
}

// Register budget: at most 65536 / (512 threads) = 128 registers per thread
// so that 512 threads per SM stay resident.  I is the element-offset type;
// both the single-lattice and the batch kernels use long long (with int
// offsets the kernel spills at its register budget: ~3.5% slower for one
// lattice, ~7% for a batch, measured on GB300).
//
// BATCH: the work items span several independent periodic boxes described by
// b.boxes (geometry and offset of each box's populations in src/dst); the
// physics parameters in `a` are shared.  Items are box-major, so a block
// finds its box by a binary search over the boxes' first items.
template <class Codec, int COLL, int TX, int TY, class I, bool BATCH = false>
__global__ void __launch_bounds__(TX * TY, (TX * TY >= 512) ? 1 : 512 / (TX * TY))
sc_step_pipe_kernel(const typename Codec::S* __restrict__ src_all, typename Codec::S* __restrict__ dst_all,
                    const StepArgs a, const BatchArgs b) {
    using R = typename Codec::R;
    using S = typename Codec::S;
    using L = PipeLayout<Codec, TX, TY>;
    using HS = typename L::HS;
    constexpr int PX = L::PX, PLANE = L::PLANE, NH = L::NHALO;
    static_assert(L::NHALO <= TX * TY, "tile too small for its halo ring");
    constexpr bool LOCAL = L::kLocal;
    static_assert(!LOCAL || (L::kWord && !BATCH), "local-reference storage: 16-bit, single lattice");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    HS* hstage = reinterpret_cast<HS*>(smem_raw);  // [NSTAGE][Q][NHALO]
    R* ring = reinterpret_cast<R*>(smem_raw + L::NSTAGE * L::stage_bytes);  // psi [NSLOT][PLANE]
    float* rstage = reinterpret_cast<float*>(ring + L::NSLOT * PLANE);        // ring refs [NSTAGE][NHALO]
    float* rring = rstage + L::NSTAGE * (LOCAL ? NH : 0);                     // rho [NSLOT][PLANE]

    const int tid = threadIdx.x;
    const int lx = tid % TX, ly = tid / TX;
    const R rho0 = par<R>(a.rho0, a.rho0f), inv_rho0 = par<R>(a.inv_rho0, a.inv_rho0f);
    const DevParams dev = a.dev;
    const int my_slot = (ly + 1) * PX + (lx + 1);

    // Ring cells go to the first NH threads, one each: the ring work then
    // fills a few whole warps (spreading it over every warp in short runs
    // measured 33% slower: all warps then issue the ring code with few lanes).
    int hx = 0, hy = 0, h_slot = -1;
    const int h = tid;
    if (h < NH) {
        if (h < PX) { hx = h - 1; hy = -1; }
        else if (h < 2 * PX) { hx = h - PX - 1; hy = TY; }
        else { const int k = h - 2 * PX; hx = (k < TY) ? -1 : TX; hy = (k < TY) ? k : k - TY; }
        h_slot = (hy + 1) * PX + (hx + 1);
    }

    const int n_items = BATCH ? b.n_items : a.n_items;
    for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
        int nx, ny, nz, tiles_x, n_tiles, zchunk, local;
        const S* __restrict__ src;
        S* __restrict__ dst;
        I n;
        if constexpr (BATCH) {
            int lo = 0, hi = b.nbox - 1;  // last box with item_begin <= item
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (b.boxes[mid].item_begin <= item) lo = mid;
                else hi = mid - 1;
            }
            const BatchBox& bx = b.boxes[lo];
            nx = bx.nx; ny = bx.ny; nz = bx.nz;
            tiles_x = bx.tiles_x; n_tiles = bx.n_tiles; zchunk = bx.zchunk;
            local = item - bx.item_begin;
            src = src_all + bx.base;
            dst = dst_all + bx.base;
            n = I(bx.n);
        } else {
            nx = a.nx; ny = a.ny; nz = a.nz;
            tiles_x = a.tiles_x; n_tiles = a.n_tiles; zchunk = a.zchunk;
            local = item;
            src = src_all;
            dst = dst_all;
            n = I(a.n);
        }
        const I plane = I(nx) * I(ny);
        const int tile = local % n_tiles, chunk = local / n_tiles;
        const int x0 = (tile % tiles_x) * TX, y0 = (tile / tiles_x) * TY;
        const int zs = chunk * zchunk;
        const int ze = min(zs + zchunk, nz);

        const int gx = wrap_index(x0 + lx, nx), gy = wrap_index(y0 + ly, ny);
        const bool active = (x0 + lx < nx) && (y0 + ly < ny);
        const I my_xy = I(gy) * I(nx) + I(gx);
        const I h_xy = (h_slot >= 0) ? I(wrap_index(y0 + hy, ny)) * I(nx) + I(wrap_index(x0 + hx, nx)) : I(0);
        const int hpar = L::kWord ? int(h_xy & 1) : 0;  // 16-bit: half of the ring cell's word
        const int xp = (gx + 1 == nx) ? 0 : gx + 1, xm = (gx == 0) ? nx - 1 : gx - 1;
        const int yp = (gy + 1 == ny) ? 0 : gy + 1, ym = (gy == 0) ? ny - 1 : gy - 1;
        const I yoff[3] = {I(ym) * I(nx), I(gy) * I(nx), I(yp) * I(nx)};
        const int xidx[3] = {xm, gx, xp};

        auto wrapz = [&](int z) { return z < 0 ? z + nz : (z >= nz ? z - nz : z); };
        auto stage_of = [&](int z) { return (z - zs + 1) % L::NSTAGE; };
        auto slot_of = [&](int z) { return (z - zs + 1) & (L::NSLOT - 1); };
        auto issue_halo = [&](int z) {
            if (h_slot >= 0) {
                const I off = I(wrapz(z)) * plane + h_xy - I(hpar);
                HS* st = hstage + stage_of(z) * (Q * NH);
                static_for<0, Q>([&](auto qc) {
                    constexpr int q = decltype(qc)::value;
                    async_copy::copy<sizeof(HS)>(st + q * NH + h, pop_at(src, q, n) + off);
                });
                if constexpr (LOCAL)
                    async_copy::copy<4>(rstage + stage_of(z) * NH + h, a.ref_src + (I(wrapz(z)) * plane + h_xy));
            }
            async_copy::commit();
        };
        auto halo_psi = [&](int z) {
            if (h_slot >= 0) {
                const HS* st = hstage + stage_of(z) * (Q * NH);
                R r = R(0);
                if constexpr (LOCAL) {
                    const float ref = rstage[stage_of(z) * NH + h];
                    static_for<0, Q>([&](auto qc) {
                        constexpr int q = decltype(qc)::value;
                        r += Codec::template decode_ref<q>(half_of<S>(st[q * NH + h], hpar), ref, dev);
                    });
                    rring[slot_of(z) * PLANE + h_slot] = r;
                } else {
                    static_for<0, Q>([&](auto qc) {
                        constexpr int q = decltype(qc)::value;
                        if constexpr (L::kWord)
                            r += Codec::template decode<q>(half_of<S>(st[q * NH + h], hpar), dev);
                        else
                            r += Codec::template decode<q>(st[q * NH + h], dev);
                    });
                }
                ring[slot_of(z) * PLANE + h_slot] = psi_of<R>(r, rho0, inv_rho0);
            }
        };
        auto load_plane = [&](R (&f)[Q], int z) {
            const I off = I(wrapz(z)) * plane + my_xy;
            if constexpr (LOCAL) {
                const float ref = __ldg(a.ref_src + off);
                static_for<0, Q>([&](auto qc) {
                    constexpr int q = decltype(qc)::value;
                    f[q] = Codec::template load_ref<q>(pop_at(src, q, n) + off, ref, dev);
                });
            } else {
                static_for<0, Q>([&](auto qc) {
                    constexpr int q = decltype(qc)::value;
                    f[q] = Codec::template load<q>(pop_at(src, q, n) + off, dev);
                });
            }
        };
        auto own_psi = [&](const R (&f)[Q], int z) {
            R r = R(0);
            static_for<0, Q>([&](auto qc) {
                constexpr int q = decltype(qc)::value;
                r += f[q];
            });
            const R p = psi_of<R>(r, rho0, inv_rho0);
            ring[slot_of(z) * PLANE + my_slot] = p;
            if constexpr (LOCAL) rring[slot_of(z) * PLANE + my_slot] = r;
            if constexpr (!BATCH) {  // the psi of the planes this item owns
                if (a.psi_out && active && z >= zs && z < ze) static_cast<R*>(a.psi_out)[I(z) * plane + my_xy] = p;
            }
        };
        // One plane: loads of z+2 go out before the collision of z and are
        // consumed after it.  fc holds plane z, fn plane z+1, fl receives z+2;
        // the caller rotates the three arrays instead of copying them.
        auto body = [&](R (&fc)[Q], R (&fn)[Q], R (&fl)[Q], int z) {
            const bool more = z + 2 <= ze;
            if (more) load_plane(fl, z + 2);
            if (more) issue_halo(z + 2);
            else async_copy::commit();
            async_copy::wait<1>();
            halo_psi(z + 1);
            __syncthreads();
            if (active) {
                const int zm = (z == 0) ? nz - 1 : z - 1;
                const int zn = (z + 1 == nz) ? 0 : z + 1;
                const I zoff[3] = {I(zm) * plane, I(z) * plane, I(zn) * plane};
                update_cell<Codec, COLL, PX, I>(fc, ring + slot_of(z - 1) * PLANE, ring + slot_of(z) * PLANE,
                                                ring + slot_of(z + 1) * PLANE, my_slot, dst, n, zoff, yoff, xidx,
                                                a);
            }
            if (more) own_psi(fl, z + 2);
            (void)fn;
        };

        __syncthreads();  // the previous item's readers of the psi ring are done
        issue_halo(zs - 1);
        issue_halo(zs);
        issue_halo(zs + 1);
        if constexpr (L::kWord) {
            // fc holds plane z (decoded), the other array plane z+1; the raw
            // loads of z+2 land in fr and are decoded into fc once plane z is
            // stored.  Two arrays alternate.
            S fr[Q];
            float fref = 0.0f;  // local-reference storage: the prefetched cell's reference
            auto body16 = [&](R (&fc)[Q], int z) {
                const bool more = z + 2 <= ze;
                if (more) {
                    const I off = I(wrapz(z + 2)) * plane + my_xy;
                    static_for<0, Q>([&](auto qc) {
                        constexpr int q = decltype(qc)::value;
                        fr[q] = __ldg(pop_at(src, q, n) + off);
                    });
                    if constexpr (LOCAL) fref = __ldg(a.ref_src + (I(wrapz(z + 2)) * plane + my_xy));
                    issue_halo(z + 2);
                } else {
                    async_copy::commit();
                }
                async_copy::wait<1>();
                halo_psi(z + 1);
                __syncthreads();
                if (active) {
                    const int zm = (z == 0) ? nz - 1 : z - 1;
                    const int zn = (z + 1 == nz) ? 0 : z + 1;
                    const I zoff[3] = {I(zm) * plane, I(z) * plane, I(zn) * plane};
                    if constexpr (LOCAL) {
                        const float* rp[3] = {rring + slot_of(z - 1) * PLANE, rring + slot_of(z) * PLANE,
                                              rring + slot_of(z + 1) * PLANE};
                        update_cell<Codec, COLL, PX, I>(fc, ring + slot_of(z - 1) * PLANE,
                                                        ring + slot_of(z) * PLANE, ring + slot_of(z + 1) * PLANE,
                                                        my_slot, dst, n, zoff, yoff, xidx, a, rp);
                        a.ref_dst[zoff[1] + my_xy] = rp[1][my_slot];  // this cell's density now
                    } else {
                        update_cell<Codec, COLL, PX, I>(fc, ring + slot_of(z - 1) * PLANE,
                                                        ring + slot_of(z) * PLANE, ring + slot_of(z + 1) * PLANE,
                                                        my_slot, dst, n, zoff, yoff, xidx, a);
                    }
                }
                if (more) {
                    static_for<0, Q>([&](auto qc) {
                        constexpr int q = decltype(qc)::value;
                        if constexpr (LOCAL) fc[q] = Codec::template decode_ref<q>(fr[q], fref, dev);
                        else fc[q] = Codec::template decode<q>(fr[q], dev);
                    });
                    own_psi(fc, z + 2);
                }
            };
            R fa[Q], fb[Q];
            load_plane(fa, zs - 1);
            own_psi(fa, zs - 1);
            load_plane(fa, zs);
            load_plane(fb, zs + 1);
            async_copy::wait<2>();
            halo_psi(zs - 1);
            async_copy::wait<1>();
            halo_psi(zs);
            own_psi(fa, zs);
            own_psi(fb, zs + 1);
            for (int z = zs; z < ze; z += 2) {
                body16(fa, z);
                if (z + 1 < ze) body16(fb, z + 1);
            }
        } else {
            R fa[Q], fb[Q], fcc[Q];
            load_plane(fa, zs - 1);
            own_psi(fa, zs - 1);
            load_plane(fa, zs);
            load_plane(fb, zs + 1);
            async_copy::wait<2>();
            halo_psi(zs - 1);
            async_copy::wait<1>();
            halo_psi(zs);
            own_psi(fa, zs);
            own_psi(fb, zs + 1);

            for (int z = zs; z < ze; z += 3) {
                body(fa, fb, fcc, z);
                if (z + 1 < ze) body(fb, fcc, fa, z + 1);
                if (z + 2 < ze) body(fcc, fa, fb, z + 2);
            }
        }
    }
    async_copy::wait<0>();
}

// ----------------------------------------------------------------------------
// Bulk-copy variant (FP32 storage, nx a multiple of 4).
//
// Warp-specialised: one producer warp fetches every plane of the tile plus a
// 4-column / 1-row halo (x0-4 .. x0+35, y0-1 .. y0+TY) with cp.async.bulk
// row copies (160 bytes each, split where the periodic wrap cuts a row) into
// a three-stage shared-memory buffer, completing on an mbarrier per stage;
// TX*TY consumer threads compute psi and collide from shared memory and
// release a stage through a second mbarrier.  Periodic wrap is applied in the
// copy addresses, so no fix-up is needed at box edges.  Every mbarrier wait is
// bounded: on timeout the thread sets *a.err and stops waiting, so the kernel
// always terminates (the host reports LBM_ETIMEOUT).
// ----------------------------------------------------------------------------
namespace bulk {
__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void bar_init(unsigned long long* b, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_init() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }
__device__ __forceinline__ void arrive(unsigned long long* b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ void arrive_expect_tx(unsigned long long* b, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(b)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool try_wait(unsigned long long* b, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: false (and *err set) if the phase did not complete within
// about one second (2^31 SM clocks).  `bad` short-circuits every later wait
// of the thread, so a stalled block finishes after one timeout per thread.
__device__ __forceinline__ bool wait(unsigned long long* b, unsigned parity, bool& bad, int* err) {
    if (bad) return false;
    if (try_wait(b, parity)) return true;
    const long long t0 = clock64();
    while (clock64() - t0 < (1LL << 31))
        if (try_wait(b, parity)) return true;
    bad = true;
    atomicOr(err, 1);
    return false;
}
__device__ __forceinline__ void copy(void* dst, const void* src, unsigned bytes, unsigned long long* b) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(b))
                 : "memory");
}
}  // namespace bulk

template <int TY>
struct BulkLayout {
    static constexpr int TX = 32;
    static constexpr int NT = TX * TY;                  // consumer threads
    static constexpr int NCW = NT / 32;                 // consumer warps
    static constexpr int ROWS = TY + 2;
    static constexpr int COLS = TX + 8;                 // x0-4 .. x0+TX+3
    static constexpr int NSTAGE = 3;
    static constexpr int PX = TX + 2;                   // psi ring pitch
    static constexpr int PLANE = PX * (TY + 2);
    static constexpr unsigned stage_floats = Q * ROWS * COLS;
    static constexpr unsigned stage_bytes = stage_floats * 4;
    static constexpr size_t bytes = NSTAGE * (size_t)stage_bytes + 4 * PLANE * 4 + 2 * NSTAGE * 8;
};

// Register budget: each of an SM's 4 sub-partitions holds 16384 registers
// for the warps placed on it, so w resident warps allow 16384 / (32 ceil(w/4))
// registers per thread: TY = 16, one block of 17 warps -> 96; TY = 8, two
// blocks of 9 warps -> 96; TY = 4, three blocks of 5 warps -> 128.
template <int COLL, int TY>
__global__ void __maxnreg__(TY >= 8 ? 96 : 128)
sc_step_bulk_kernel(const float* __restrict__ src, float* __restrict__ dst, const StepArgs a) {
    using L = BulkLayout<TY>;
    using R = float;
    constexpr int TX = L::TX, NT = L::NT, ROWS = L::ROWS, COLS = L::COLS, PX = L::PX, PLANE = L::PLANE;
    constexpr int NHALO = 2 * (TX + 2) + 2 * TY;
    static_assert(NHALO <= NT, "tile too small for its halo ring");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float* stage = reinterpret_cast<float*>(smem_raw);
    float* ring = stage + L::NSTAGE * L::stage_floats;
    unsigned long long* full = reinterpret_cast<unsigned long long*>(ring + 4 * PLANE);
    unsigned long long* empty = full + L::NSTAGE;

    const int tid = threadIdx.x;
    const bool producer = tid >= NT;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const long long n = a.n;
    const long long plane = (long long)nx * ny;
    bool bad = false;

    if (tid == 0) {
        for (int s = 0; s < L::NSTAGE; ++s) {
            bulk::bar_init(&full[s], 1);
            bulk::bar_init(&empty[s], L::NCW);
        }
        bulk::fence_init();
    }
    __syncthreads();

    unsigned g = 0;  // planes fetched so far by this block (same count on both sides)
    if (producer) {
        const int lane = tid - NT;
        for (int item = blockIdx.x; item < a.n_items; item += gridDim.x) {
            const int tile = item % a.n_tiles, chunk = item / a.n_tiles;
            const int x0 = (tile % a.tiles_x) * TX, y0 = (tile / a.tiles_x) * TY;
            const int zs = chunk * a.zchunk, ze = min(zs + a.zchunk, nz);
            const int xs = wrap_index(x0 - 4, nx);
            for (int p = zs - 1; p <= ze; ++p, ++g) {
                const int s = g % L::NSTAGE;
                if (a.test_stall) continue;  // failure test: the consumers' waits must time out
                if (g >= (unsigned)L::NSTAGE) bulk::wait(&empty[s], ((g / L::NSTAGE) - 1) & 1, bad, a.err);
                if (lane == 0) bulk::arrive_expect_tx(&full[s], L::stage_bytes);
                __syncwarp();
                if (!bad) {
                    const int zw = p < 0 ? p + nz : (p >= nz ? p - nz : p);
                    float* st = stage + s * L::stage_floats;
                    for (int u = lane; u < Q * ROWS; u += 32) {
                        const int q = u / ROWS, r = u % ROWS;
                        const int y = wrap_index(y0 - 1 + r, ny);
                        const float* row = src + (long long)q * n + (long long)zw * plane + (long long)y * nx;
                        float* d = st + (q * ROWS + r) * COLS;
                        int x = xs, left = COLS;
                        while (left > 0) {  // split where the periodic wrap cuts the row
                            const int piece = min(left, nx - x);
                            bulk::copy(d, row + x, piece * 4, &full[s]);
                            d += piece;
                            left -= piece;
                            x = 0;
                        }
                    }
                }
            }
        }
        // drain: the last planes' copies complete before the block exits
        if (!a.test_stall)
            for (unsigned k = (g > (unsigned)L::NSTAGE ? g - L::NSTAGE : 0); k < g; ++k)
            bulk::wait(&full[k % L::NSTAGE], (k / L::NSTAGE) & 1, bad, a.err);
        return;
    }

    // consumers
    const int lx = tid % TX, ly = tid / TX;
    const int warp = tid / 32, lane = tid % 32;
    const R rho0 = par<R>(a.rho0, a.rho0f), inv_rho0 = par<R>(a.inv_rho0, a.inv_rho0f);
    const int my_slot = (ly + 1) * PX + (lx + 1);
    const int my_st = (ly + 1) * COLS + (lx + 4);
    int h_slot = -1, h_st = 0;
    if (tid < NHALO) {
        int hx, hy;
        if (tid < PX) { hx = tid - 1; hy = -1; }
        else if (tid < 2 * PX) { hx = tid - PX - 1; hy = TY; }
        else { const int k = tid - 2 * PX; hx = (k < TY) ? -1 : TX; hy = (k < TY) ? k : k - TY; }
        h_slot = (hy + 1) * PX + (hx + 1);
        h_st = (hy + 1) * COLS + (hx + 4);
    }
    auto consumers_sync = [] { asm volatile("bar.sync 1, %0;\n" ::"n"(NT) : "memory"); };
    auto release = [&](unsigned gi) {
        __syncwarp();
        if (lane == 0) bulk::arrive(&empty[gi % L::NSTAGE]);
        (void)warp;
    };

    for (int item = blockIdx.x; item < a.n_items; item += gridDim.x) {
        const int tile = item % a.n_tiles, chunk = item / a.n_tiles;
        const int x0 = (tile % a.tiles_x) * TX, y0 = (tile / a.tiles_x) * TY;
        const int zs = chunk * a.zchunk, ze = min(zs + a.zchunk, nz);
        const int gx = wrap_index(x0 + lx, nx), gy = wrap_index(y0 + ly, ny);
        const bool active = (x0 + lx < nx) && (y0 + ly < ny);
        const int xp = (gx + 1 == nx) ? 0 : gx + 1, xm = (gx == 0) ? nx - 1 : gx - 1;
        const int yp = (gy + 1 == ny) ? 0 : gy + 1, ym = (gy == 0) ? ny - 1 : gy - 1;
        const long long yoff[3] = {(long long)ym * nx, (long long)gy * nx, (long long)yp * nx};
        const int xidx[3] = {xm, gx, xp};
        const unsigned g0 = g;
        auto st_of = [&](unsigned gi) { return stage + (gi % L::NSTAGE) * L::stage_floats; };
        auto slot_of = [&](int z) { return (z - zs + 1) & 3; };
        auto psi_from = [&](unsigned gi, int z) {
            const float* st = st_of(gi);
            R r = R(0);
            static_for<0, Q>([&](auto qc) {
                constexpr int q = decltype(qc)::value;
                r += st[q * ROWS * COLS + my_st];
            });
            ring[slot_of(z) * PLANE + my_slot] = psi_of<R>(r, rho0, inv_rho0);
            if (h_slot >= 0) {
                R rh = R(0);
                static_for<0, Q>([&](auto qc) {
                    constexpr int q = decltype(qc)::value;
                    rh += st[q * ROWS * COLS + h_st];
                });
                ring[slot_of(z) * PLANE + h_slot] = psi_of<R>(rh, rho0, inv_rho0);
            }
        };
        auto wait_plane = [&](unsigned gi) { bulk::wait(&full[gi % L::NSTAGE], (gi / L::NSTAGE) & 1, bad, a.err); };

        consumers_sync();  // the previous item's readers of the psi ring are done
        wait_plane(g0);
        psi_from(g0, zs - 1);
        release(g0);
        wait_plane(g0 + 1);
        psi_from(g0 + 1, zs);
        for (int z = zs; z < ze; ++z) {
            const unsigned gi = g0 + (z - zs) + 1;  // plane z
            wait_plane(gi + 1);
            psi_from(gi + 1, z + 1);
            consumers_sync();
            if (active) {
                const float* st = st_of(gi);
                R fc[Q];
                static_for<0, Q>([&](auto qc) {
                    constexpr int q = decltype(qc)::value;
                    fc[q] = st[q * ROWS * COLS + my_st];
                });
                const int zm = (z == 0) ? nz - 1 : z - 1;
                const int zn = (z + 1 == nz) ? 0 : z + 1;
                const long long zoff[3] = {(long long)zm * plane, (long long)z * plane, (long long)zn * plane};
                update_cell<CodecF32, COLL, PX>(fc, ring + slot_of(z - 1) * PLANE, ring + slot_of(z) * PLANE,
                                                ring + slot_of(z + 1) * PLANE, my_slot, dst, n, zoff, yoff, xidx,
                                                a);
            }
            release(gi);
        }
        release(g0 + (ze - zs) + 1);  // plane ze: psi only
        g = g0 + (ze - zs) + 2;
    }
}

// ----------------------------------------------------------------------------
// Tensor-copy variant (FP32 storage, nx a multiple of 32, ny a multiple of
// TY).
//
// The pipelined kernel's 19 loads per cell and plane become ONE
// cp.async.bulk.tensor.4d copy per plane of the tile's cells (box
// 32 x TY x 1 x 19 of the 4-D tensor map (x, y, z, population)), issued by a
// single thread into a four-stage shared-memory buffer three planes ahead
// and completing on an mbarrier per stage.  Tile boxes never leave the box of
// the lattice, so the tensor map's zero fill is never used; the one-cell ring
// (with its periodic wrap) keeps the four-stage 4/8-byte cp.async buffer of
// the pipelined kernel.  All threads compute; the per-plane barrier also
// marks the stage three planes back as free.  mbarrier waits are bounded as
// in the bulk-copy variant.
// ----------------------------------------------------------------------------
template <int TY>
struct TmaLayout {
    static constexpr int TX = 32;
    static constexpr int NT = TX * TY;
    static constexpr int NHALO = 2 * (TX + 2) + 2 * TY;
    static constexpr int PX = TX + 2;
    static constexpr int PLANE = PX * (TY + 2);
    static constexpr int NSTAGE = 4;
    static constexpr unsigned stage_floats = Q * NT;
    static constexpr unsigned stage_bytes = stage_floats * 4;
    static constexpr size_t bytes =
        NSTAGE * (size_t)stage_bytes + NSTAGE * (size_t)Q * NHALO * 4 + 4 * (size_t)PLANE * 4 + NSTAGE * 8;
};

namespace tma {
__device__ __forceinline__ void load_box(float* dst, const CUtensorMap* map, int x, int y, int z,
                                         unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];\n" ::"r"(bulk::smem_u32(dst)),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z), "r"(0), "r"(bulk::smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
}  // namespace tma

template <int COLL, int TY>
__global__ void __launch_bounds__(32 * TY, (TY >= 16) ? 1 : 2)
sc_step_tma_kernel(const __grid_constant__ CUtensorMap tmap, const float* __restrict__ src, float* __restrict__ dst,
                   const StepArgs a) {
    using L = TmaLayout<TY>;
    using R = float;
    constexpr int TX = L::TX, NT = L::NT, NH = L::NHALO, PX = L::PX, PLANE = L::PLANE, NS = L::NSTAGE;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float* istage = reinterpret_cast<float*>(smem_raw);             // [NS][Q][TY][TX]
    float* hstage = istage + NS * L::stage_floats;                 // [NS][Q][NH]
    float* ring = hstage + NS * Q * NH;                             // [4][PLANE]
    unsigned long long* full = reinterpret_cast<unsigned long long*>(ring + 4 * PLANE);

    const int tid = threadIdx.x;
    const int lx = tid % TX, ly = tid / TX;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const long long n = a.n;
    const long long plane = (long long)nx * ny;
    const R rho0 = par<R>(a.rho0, a.rho0f), inv_rho0 = par<R>(a.inv_rho0, a.inv_rho0f);
    const int my_slot = (ly + 1) * PX + (lx + 1);
    const int my_st = ly * TX + lx;
    bool bad = false;

    int hx = 0, hy = 0, h_slot = -1;
    const int h = tid;  // ring cells on the first NH threads, as in the pipelined kernel
    if (h < NH) {
        if (h < PX) { hx = h - 1; hy = -1; }
        else if (h < 2 * PX) { hx = h - PX - 1; hy = TY; }
        else { const int k = h - 2 * PX; hx = (k < TY) ? -1 : TX; hy = (k < TY) ? k : k - TY; }
        h_slot = (hy + 1) * PX + (hx + 1);
    }

    if (tid == 0) {
        for (int s = 0; s < NS; ++s) bulk::bar_init(&full[s], 1);
        bulk::fence_init();
    }
    __syncthreads();

    unsigned g = 0;  // planes issued so far by this block
    for (int item = blockIdx.x; item < a.n_items; item += gridDim.x) {
        const int tile = item % a.n_tiles, chunk = item / a.n_tiles;
        const int x0 = (tile % a.tiles_x) * TX, y0 = (tile / a.tiles_x) * TY;
        const int zs = chunk * a.zchunk, ze = min(zs + a.zchunk, nz);
        const int gx = x0 + lx, gy = y0 + ly;
        const long long h_xy =
            (h_slot >= 0) ? (long long)wrap_index(y0 + hy, ny) * nx + wrap_index(x0 + hx, nx) : 0;
        const int xp = (gx + 1 == nx) ? 0 : gx + 1, xm = (gx == 0) ? nx - 1 : gx - 1;
        const int yp = (gy + 1 == ny) ? 0 : gy + 1, ym = (gy == 0) ? ny - 1 : gy - 1;
        const long long yoff[3] = {(long long)ym * nx, (long long)gy * nx, (long long)yp * nx};
        const int xidx[3] = {xm, gx, xp};
        const unsigned g0 = g;  // plane p of this item has index g0 + (p - zs + 1)
        auto wrapz = [&](int z) { return z < 0 ? z + nz : (z >= nz ? z - nz : z); };
        auto gi_of = [&](int p) { return g0 + unsigned(p - zs + 1); };
        auto slot_of = [&](int z) { return (z - zs + 1) & 3; };
        auto issue = [&](int p) {  // plane p: tensor box (one thread) + ring copies; one cp.async group
            const unsigned gi = gi_of(p);
            const int s = gi % NS;
            const int zw = wrapz(p);
            if (tid == 0) {
                tma::fence_proxy_async();
                bulk::arrive_expect_tx(&full[s], L::stage_bytes);
                tma::load_box(istage + s * L::stage_floats, &tmap, x0, y0, zw, &full[s]);
            }
            if (h_slot >= 0) {
                const float* base = src + (long long)zw * plane + h_xy;
                float* st = hstage + s * (Q * NH);
                static_for<0, Q>([&](auto qc) {
                    constexpr int q = decltype(qc)::value;
                    async_copy::copy<4>(st + q * NH + h, base + q * n);
                });
            }
            async_copy::commit();
        };
        auto wait_box = [&](int p) {
            const unsigned gi = gi_of(p);
            bulk::wait(&full[gi % NS], (gi / NS) & 1, bad, a.err);
        };
        auto psi_from = [&](int p) {
            const int s = gi_of(p) % NS;
            const float* st = istage + s * L::stage_floats;
            R r = R(0);
            static_for<0, Q>([&](auto qc) {
                constexpr int q = decltype(qc)::value;
                r += st[q * NT + my_st];
            });
            ring[slot_of(p) * PLANE + my_slot] = psi_of<R>(r, rho0, inv_rho0);
            if (h_slot >= 0) {
                const float* hs = hstage + s * (Q * NH);
                R rh = R(0);
                static_for<0, Q>([&](auto qc) {
                    constexpr int q = decltype(qc)::value;
                    rh += hs[q * NH + h];
                });
                ring[slot_of(p) * PLANE + h_slot] = psi_of<R>(rh, rho0, inv_rho0);
            }
        };

        __syncthreads();  // the previous item is finished with every stage and the psi ring
        // prologue: planes zs-1 .. zs+2 (four cp.async groups, empty ones past ze)
        for (int p = zs - 1; p <= zs + 2; ++p) {
            if (p <= ze) issue(p);
            else async_copy::commit();
        }
        async_copy::wait<3>();
        wait_box(zs - 1);
        psi_from(zs - 1);
        async_copy::wait<2>();
        wait_box(zs);
        psi_from(zs);
        for (int z = zs; z < ze; ++z) {
            async_copy::wait<1>();
            wait_box(z + 1);
            psi_from(z + 1);
            __syncthreads();
            // every thread is past plane z-1: its stage takes plane z+3
            if (z + 3 <= ze) issue(z + 3);
            else async_copy::commit();
            const float* st = istage + (gi_of(z) % NS) * L::stage_floats;
            R fc[Q];
            static_for<0, Q>([&](auto qc) {
                constexpr int q = decltype(qc)::value;
                fc[q] = st[q * NT + my_st];
            });
            const int zm = (z == 0) ? nz - 1 : z - 1;
            const int zn = (z + 1 == nz) ? 0 : z + 1;
            const long long zoff[3] = {(long long)zm * plane, (long long)z * plane, (long long)zn * plane};
            update_cell<CodecF32, COLL, PX>(fc, ring + slot_of(z - 1) * PLANE, ring + slot_of(z) * PLANE,
                                            ring + slot_of(z + 1) * PLANE, my_slot, dst, n, zoff, yoff, xidx, a);
        }
        g = g0 + unsigned(ze - zs + 2);
    }
    async_copy::wait<0>();
}

}  // namespace lbm
