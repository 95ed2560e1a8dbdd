// Per-cell part of the ligament diagnostics, shared by lbm_diag and
// lbm_diag_noalloc: rho and j of one cell from its 19 populations in the
// codec's arithmetic type (float for 32- and 16-bit storage, double for FP64),
// returned as double for the float64 accumulation across cells.  `ref` is the
// cell's reference density for the local-reference codecs.
#pragma once
#include "codec.cuh"
#include "lattice.cuh"

namespace lbm {

template <class Codec>
__device__ __forceinline__ void diag_cell(const typename Codec::S* __restrict__ p, long long n,
                                          const DevParams& dev, double& rho, double& jx, double& jy,
                                          double& jz, float ref = 0.0f) {
    using R = typename Codec::R;
    R r = R(0), ax = R(0), ay = R(0), az = R(0);
    static_for<0, Q>([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        R fq;
        if constexpr (Codec::kLocal) fq = Codec::template load_ref<q>(p + q * n, ref, dev);
        else fq = Codec::template load<q>(p + q * n, dev);
        r += fq;
        if constexpr (cx(q) != 0) ax += R(cx(q)) * fq;
        if constexpr (cy(q) != 0) ay += R(cy(q)) * fq;
        if constexpr (cz(q) != 0) az += R(cz(q)) * fq;
    });
    rho = double(r);
    jx = double(ax);
    jy = double(ay);
    jz = double(az);
}

}  // namespace lbm
