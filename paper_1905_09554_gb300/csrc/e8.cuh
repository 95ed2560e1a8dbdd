// The E8 offset set and shell weights of the two-belt (multirange) force:
// the 92 vectors with components in {-2..2} and |e|^2 in {1,2,3,4,5,6,8}, and
// per shell the weights with unit second moment whose moment tensors are
// isotropic to eighth order; the D3Q19 lattice weights of the first belt.
// Used by the two-belt step kernel and by the velocity moments.
#pragma once

namespace lbm {
namespace mr {

constexpr int kNE = 92;  // E8 vectors

struct Vec {
    int x, y, z;
};

__host__ __device__ constexpr bool in_e8(int x, int y, int z) {
    const int s = x * x + y * y + z * z;
    return s == 1 || s == 2 || s == 3 || s == 4 || s == 5 || s == 6 || s == 8;
}

// k-th E8 vector in a fixed enumeration order (z, then y, then x ascending).
__host__ __device__ constexpr Vec e8(int k) {
    int c = 0;
    for (int z = -2; z <= 2; ++z)
        for (int y = -2; y <= 2; ++y)
            for (int x = -2; x <= 2; ++x)
                if (in_e8(x, y, z)) {
                    if (c == k) return Vec{x, y, z};
                    ++c;
                }
    return Vec{0, 0, 0};
}

// Belt-2 weight of a shell (unit second moment), 0 outside E8.
__host__ __device__ constexpr double p_e8(int s) {
    return s == 1 ? 4.0 / 45.0
         : s == 2 ? 1.0 / 21.0
         : s == 3 ? 2.0 / 105.0
         : s == 4 ? 5.0 / 504.0
         : s == 5 ? 1.0 / 315.0
         : s == 6 ? 1.0 / 630.0
         : s == 8 ? 1.0 / 5040.0
                  : 0.0;
}

// Belt-1 (D3Q19 lattice) weight of a shell.
__host__ __device__ constexpr double w_d3q19(int s) { return s == 1 ? 1.0 / 18.0 : (s == 2 ? 1.0 / 36.0 : 0.0); }

}  // namespace mr

}  // namespace lbm
