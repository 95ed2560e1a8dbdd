// Per-thread part of the ligament diagnostics, shared by lbm_diag and
// lbm_diag_noalloc so that both give the same numbers.
//
// Each cell's rho and j come from its 19 populations in the codec's
// arithmetic type (float for 32- and 16-bit storage, double for FP64).  The
// thread sums its cells in that type over runs of kRun cells (the run is
// unrolled, so its loads are in flight together) and adds each run's
// partial sums to float64 accumulators.  With float storage this does one
// float64 add per quantity and run instead of per cell: the FP64 pipe of the
// GPU issues at a small fraction of the FP32 rate and bounded the per-cell
// form.  The order of all sums is fixed, so results are deterministic.
#pragma once
#include "codec.cuh"
#include "lattice.cuh"

namespace lbm {

template <class Codec>
__device__ __forceinline__ void diag_cell(const typename Codec::S* __restrict__ p, long long n,
                                          const DevParams& dev, float ref, typename Codec::R& rho,
                                          typename Codec::R& jx, typename Codec::R& jy,
                                          typename Codec::R& jz) {
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
    rho = r;
    jx = ax;
    jy = ay;
    jz = az;
}

// Cells first, first + stride, ... < count of the slice whose populations
// start at fz (population stride n; refz: the slice's reference densities for
// the local-reference codecs).  acc: mass, jx, jy, jz, liquid area, max rho,
// cells with rho <= 0 / NaN / Inf.
template <class Codec>
__device__ __forceinline__ void diag_accumulate(const typename Codec::S* __restrict__ fz, long long n,
                                                long long count, long long first, int stride, const DevParams& dev,
                                                double rho_v, double inv, const float* __restrict__ refz,
                                                double (&acc)[7]) {
    using R = typename Codec::R;
    constexpr int kRun = 8;
    for (int k = 0; k < 7; ++k) acc[k] = 0.0;
    const R rv = R(rho_v), iv = R(inv);
    for (long long i = first; i < count; i += (long long)kRun * stride) {
        R m = R(0), jx = R(0), jy = R(0), jz = R(0), area = R(0), mx = R(0);
        int bad = 0;
#pragma unroll
        for (int k = 0; k < kRun; ++k) {
            const long long c = i + (long long)k * stride;
            if (c < count) {
                R r, ax, ay, az;
                float rf = 0.0f;
                if constexpr (Codec::kLocal) rf = refz[c];
                diag_cell<Codec>(fz + c, n, dev, rf, r, ax, ay, az);
                m += r;
                jx += ax;
                jy += ay;
                jz += az;
                area += fmin(fmax((r - rv) * iv, R(0)), R(1));
                mx = fmax(mx, r);
                if (!(r > R(0)) || !isfinite(r)) ++bad;
            }
        }
        acc[0] += double(m);
        acc[1] += double(jx);
        acc[2] += double(jy);
        acc[3] += double(jz);
        acc[4] += double(area);
        acc[5] = fmax(acc[5], double(mx));
        acc[6] += double(bad);
    }
}

}  // namespace lbm
