// Storage codecs for the population arrays.  A codec names the stored type S,
// the arithmetic type R and how one population is read and written.
//
//  F64: double storage, double arithmetic.
//  F32: float storage, float arithmetic.
//  F16Dev / BF16Dev: 16-bit storage of the deviation from the rest
//     equilibrium at the reference density, d_a = (f_a - w_a rho_ref) * scale
//     with w_a rho_ref rounded to float once (DevParams::wrho), decoded to
//     float; arithmetic in float.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <type_traits>

#include "lattice.cuh"

namespace lbm {

struct DevParams {
    float rho_ref;
    float scale;
    float inv_scale;
    float wrho[Q];  // w_a rho_ref in float: the rest equilibrium the deviations are taken from
};

// The parameters of the deviation formats for a reference density and scale
// (filled the same way on the host and the device).
__host__ __device__ inline DevParams make_dev_params(double rho_ref, double scale) {
    DevParams d;
    d.rho_ref = float(rho_ref);
    d.scale = float(scale);
    d.inv_scale = float(1.0 / scale);
    for (int q = 0; q < Q; ++q) d.wrho[q] = float(wq(q)) * d.rho_ref;
    return d;
}

struct CodecF64 {
    static constexpr bool kLocal = false;
    using S = double;
    using R = double;
    static constexpr int kStorage = 0;
    template <int q>
    __device__ __forceinline__ static R decode(S v, const DevParams&) { return v; }
    template <int q>
    __device__ __forceinline__ static R load(const S* p, const DevParams&) { return __ldg(p); }
    template <int q>
    __device__ __forceinline__ static void store(S* p, R v, const DevParams&) { *p = v; }
};

struct CodecF32 {
    static constexpr bool kLocal = false;
    using S = float;
    using R = float;
    static constexpr int kStorage = 1;
    template <int q>
    __device__ __forceinline__ static R decode(S v, const DevParams&) { return v; }
    template <int q>
    __device__ __forceinline__ static R load(const S* p, const DevParams&) { return __ldg(p); }
    template <int q>
    __device__ __forceinline__ static void store(S* p, R v, const DevParams&) { *p = v; }
};

// Conversions of one 16-bit type.
template <class S16>
struct Half16 {
    __device__ __forceinline__ static float to_f(S16 v) {
        if constexpr (std::is_same<S16, __half>::value) return __half2float(v);
        else return __bfloat162float(v);
    }
    __device__ __forceinline__ static S16 from_f(float v) {
        if constexpr (std::is_same<S16, __half>::value) return __float2half_rn(v);
        else return __float2bfloat16_rn(v);
    }
};

// Deviations from the rest equilibrium at one global reference density:
// f_a = w_a rho_ref + d_a / scale, d_a rounded to S16.
template <class S16, int STORAGE>
struct CodecDev16 {
    static constexpr bool kLocal = false;
    using S = S16;
    using R = float;
    static constexpr int kStorage = STORAGE;
    __device__ __forceinline__ static float to_f(S v) { return Half16<S16>::to_f(v); }
    __device__ __forceinline__ static S from_f(float v) { return Half16<S16>::from_f(v); }
    // population from the stored deviation already widened to float
    template <int q>
    __device__ __forceinline__ static R decode_f(float h, const DevParams& d) {
        return fmaf(h, d.inv_scale, d.wrho[q]);
    }
    template <int q>
    __device__ __forceinline__ static R decode(S v, const DevParams& d) { return decode_f<q>(to_f(v), d); }
    template <int q>
    __device__ __forceinline__ static R load(const S* p, const DevParams& d) { return decode<q>(__ldg(p), d); }
    // the deviation before its rounding to S
    template <int q>
    __device__ __forceinline__ static float deviation(R v, const DevParams& d) {
        return (v - d.wrho[q]) * d.scale;
    }
    template <int q>
    __device__ __forceinline__ static S encode(R v, const DevParams& d) { return from_f(deviation<q>(v, d)); }
    template <int q>
    __device__ __forceinline__ static void store(S* p, R v, const DevParams& d) { *p = encode<q>(v, d); }
};
using CodecF16Dev = CodecDev16<__half, 2>;
using CodecBF16Dev = CodecDev16<__nv_bfloat16, 3>;


// Local-reference 16-bit storage: each cell also keeps, in a float field,
// the density it had at the previous step, and each stored population is the
// deviation from the rest equilibrium at that density,
// d_a = (f_a - w_a rho_ref(cell)) * scale.  The writer of a population knows
// the destination cell's current density (it is in the block's density
// planes), and the reader needs only its own cell's reference.
template <class S16>
struct CodecLocal16 {
    static constexpr bool kLocal = true;
    using S = S16;
    using R = float;
    static constexpr int kStorage = std::is_same<S16, __half>::value ? 4 : 5;
    __device__ __forceinline__ static float to_f(S v) { return Half16<S16>::to_f(v); }
    __device__ __forceinline__ static S from_f(float v) { return Half16<S16>::from_f(v); }
    template <int q>
    __device__ __forceinline__ static R decode_ref(S v, float ref, const DevParams& d) {
        return float(wq(q)) * ref + to_f(v) * d.inv_scale;
    }
    template <int q>
    __device__ __forceinline__ static R load_ref(const S* p, float ref, const DevParams& d) {
        return decode_ref<q>(__ldg(p), ref, d);
    }
    // the deviation before its rounding to S
    template <int q>
    __device__ __forceinline__ static float deviation_ref(R v, float ref, const DevParams& d) {
        return (v - float(wq(q)) * ref) * d.scale;
    }
    template <int q>
    __device__ __forceinline__ static S encode_ref(R v, float ref, const DevParams& d) {
        return from_f(deviation_ref<q>(v, ref, d));
    }
    template <int q>
    __device__ __forceinline__ static void store_ref(S* p, R v, float ref, const DevParams& d) {
        *p = encode_ref<q>(v, ref, d);
    }
    __device__ __forceinline__ static double decode_rt(const S* p, float w, float ref, const DevParams& d) {
        return double(w * ref + to_f(*p) * d.inv_scale);
    }
    __device__ __forceinline__ static void encode_rt(S* p, float w, double v, float ref, const DevParams& d) {
        *p = from_f((float(v) - w * ref) * d.scale);
    }
};
using CodecF16Local = CodecLocal16<__half>;
using CodecBF16Local = CodecLocal16<__nv_bfloat16>;

// Runtime (non-templated) decode/encode for the conversion kernels.
template <class Codec>
__device__ __forceinline__ double decode_rt(const typename Codec::S* p, float w, const DevParams& d);
template <>
__device__ __forceinline__ double decode_rt<CodecF64>(const double* p, float, const DevParams&) { return *p; }
template <>
__device__ __forceinline__ double decode_rt<CodecF32>(const float* p, float, const DevParams&) { return *p; }
// (w_a rho_ref rounded to float first, as in DevParams::wrho)
template <>
__device__ __forceinline__ double decode_rt<CodecF16Dev>(const __half* p, float w, const DevParams& d) {
    return double(fmaf(__half2float(*p), d.inv_scale, __fmul_rn(w, d.rho_ref)));
}
template <>
__device__ __forceinline__ double decode_rt<CodecBF16Dev>(const __nv_bfloat16* p, float w, const DevParams& d) {
    return double(fmaf(__bfloat162float(*p), d.inv_scale, __fmul_rn(w, d.rho_ref)));
}

template <class Codec>
__device__ __forceinline__ void encode_rt(typename Codec::S* p, float w, double v, const DevParams& d);
template <>
__device__ __forceinline__ void encode_rt<CodecF64>(double* p, float, double v, const DevParams&) { *p = v; }
template <>
__device__ __forceinline__ void encode_rt<CodecF32>(float* p, float, double v, const DevParams&) { *p = float(v); }
template <>
__device__ __forceinline__ void encode_rt<CodecF16Dev>(__half* p, float w, double v, const DevParams& d) {
    *p = __float2half_rn((float(v) - __fmul_rn(w, d.rho_ref)) * d.scale);
}
template <>
__device__ __forceinline__ void encode_rt<CodecBF16Dev>(__nv_bfloat16* p, float w, double v, const DevParams& d) {
    *p = __float2bfloat16_rn((float(v) - __fmul_rn(w, d.rho_ref)) * d.scale);
}

}  // namespace lbm
