// D3Q19 lattice tables and the d'Humieres moment basis, as compile-time
// constants for the device code (Sec. 2 of arXiv:1905.09554: 19 velocities,
// "the set of weights for the D3Q19 lattice", cs^2 = 1/3).
//
// Every loop over populations or moments in the kernels is fully unrolled, so
// the integer coefficients below fold into adds and subtracts at compile time.
#pragma once
#include <type_traits>
#include <utility>

namespace lbm {

constexpr int Q = 19;

// Velocity order: rest, the six axis vectors in +/- pairs, then the twelve
// edge vectors in +/- pairs (xy, xz, yz planes).  Accessors are constexpr
// functions so that, with a compile-time index, they fold in device code.
__host__ __device__ constexpr int cx(int q) {
    constexpr int t[Q] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
    return t[q];
}
__host__ __device__ constexpr int cy(int q) {
    constexpr int t[Q] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
    return t[q];
}
__host__ __device__ constexpr int cz(int q) {
    constexpr int t[Q] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
    return t[q];
}
// Weight by speed shell: 1/3 rest, 1/18 axis, 1/36 edge.
__host__ __device__ constexpr double wq(int q) {
    return q == 0 ? 1.0 / 3.0 : (cx(q) * cx(q) + cy(q) * cy(q) + cz(q) * cz(q) == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
}

// A step parameter in the arithmetic type R: the double value for FP64, its
// float copy rounded once on the host otherwise (float(x) either way, so no
// result bit depends on where the rounding happened).
template <class R>
__host__ __device__ __forceinline__ R par(double d, float f) {
    if constexpr (sizeof(R) == sizeof(double)) return d;
    else return f;
}

// Compile-time loop: f(std::integral_constant<int, i>) for i in [B, E).
template <int B, int E, class F>
__host__ __device__ __forceinline__ void static_for(F&& f) {
    if constexpr (B < E) {
        f(std::integral_constant<int, B>{});
        static_for<B + 1, E>(f);
    }
}

// d'Humieres et al. (2002) D3Q19 moment basis, moment k evaluated at
// velocity q.  Order (0-based): rho, e, eps, jx, qx, jy, qy, jz, qz, 3pxx,
// 3pixx, pww, piww, pxy, pyz, pxz, mx, my, mz.
__host__ __device__ constexpr int mrt_coef(int k, int q) {
    const int x = cx(q), y = cy(q), z = cz(q);
    const int c2 = x * x + y * y + z * z;
    switch (k) {
        case 0: return 1;
        case 1: return 19 * c2 - 30;
        case 2: return (21 * c2 * c2 - 53 * c2 + 24) / 2;
        case 3: return x;
        case 4: return (5 * c2 - 9) * x;
        case 5: return y;
        case 6: return (5 * c2 - 9) * y;
        case 7: return z;
        case 8: return (5 * c2 - 9) * z;
        case 9: return 3 * x * x - c2;
        case 10: return (3 * c2 - 5) * (3 * x * x - c2);
        case 11: return y * y - z * z;
        case 12: return (3 * c2 - 5) * (y * y - z * z);
        case 13: return x * y;
        case 14: return y * z;
        case 15: return x * z;
        case 16: return (y * y - z * z) * x;
        case 17: return (z * z - x * x) * y;
        default: return (x * x - y * y) * z;
    }
}

// Squared norm of moment row k; the rows are mutually orthogonal, so
// M^-1 = M^T diag(1/norm).
__host__ __device__ constexpr int mrt_norm(int k) {
    int s = 0;
    for (int q = 0; q < Q; ++q) s += mrt_coef(k, q) * mrt_coef(k, q);
    return s;
}

// True when moment k is odd in c: opposite velocities (q, q+1) carry opposite
// coefficients (momentum, heat flux and the third-order m moments).
__host__ __device__ constexpr bool mrt_moment_is_odd(int k) {
    bool odd = true;
    for (int q = 1; q < Q; q += 2) odd = odd && (mrt_coef(k, q + 1) == -mrt_coef(k, q));
    return odd && mrt_coef(k, 0) == 0;
}

static_assert(mrt_moment_is_odd(3) && mrt_moment_is_odd(8) && mrt_moment_is_odd(16) && mrt_moment_is_odd(18),
              "odd moments");
static_assert(!mrt_moment_is_odd(0) && !mrt_moment_is_odd(11) && !mrt_moment_is_odd(12) && !mrt_moment_is_odd(15),
              "even moments");
static_assert(mrt_norm(0) == 19 && mrt_norm(1) == 2394 && mrt_norm(2) == 252, "basis");
static_assert(mrt_norm(4) == 40 && mrt_norm(10) == 72 && mrt_norm(16) == 8, "basis");

}  // namespace lbm
