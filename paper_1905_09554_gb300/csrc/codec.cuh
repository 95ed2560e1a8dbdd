// Storage codecs for the population arrays.  A codec names the stored type S,
// the arithmetic type R and how one population is read and written.
//
//  F64: double storage, double arithmetic.
//  F32: float storage, float arithmetic.
//  F16Dev / BF16Dev: 16-bit storage of the deviation from the rest
//     equilibrium at the reference density, d_a = (f_a - w_a rho_ref) * scale,
//     decoded to float; arithmetic in float.
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
};

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

struct CodecF16Dev {
    static constexpr bool kLocal = false;
    using S = __half;
    using R = float;
    static constexpr int kStorage = 2;
    template <int q>
    __device__ __forceinline__ static R decode(S v, const DevParams& d) {
        return float(wq(q)) * d.rho_ref + __half2float(v) * d.inv_scale;
    }
    template <int q>
    __device__ __forceinline__ static R load(const S* p, const DevParams& d) { return decode<q>(__ldg(p), d); }
    template <int q>
    __device__ __forceinline__ static S encode(R v, const DevParams& d) {
        return __float2half_rn((v - float(wq(q)) * d.rho_ref) * d.scale);
    }
    template <int q>
    __device__ __forceinline__ static void store(S* p, R v, const DevParams& d) { *p = encode<q>(v, d); }
};

struct CodecBF16Dev {
    static constexpr bool kLocal = false;
    using S = __nv_bfloat16;
    using R = float;
    static constexpr int kStorage = 3;
    template <int q>
    __device__ __forceinline__ static R decode(S v, const DevParams& d) {
        return float(wq(q)) * d.rho_ref + __bfloat162float(v) * d.inv_scale;
    }
    template <int q>
    __device__ __forceinline__ static R load(const S* p, const DevParams& d) { return decode<q>(__ldg(p), d); }
    template <int q>
    __device__ __forceinline__ static S encode(R v, const DevParams& d) {
        return __float2bfloat16_rn((v - float(wq(q)) * d.rho_ref) * d.scale);
    }
    template <int q>
    __device__ __forceinline__ static void store(S* p, R v, const DevParams& d) { *p = encode<q>(v, d); }
};


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
    __device__ __forceinline__ static float to_f(S v) {
        if constexpr (std::is_same<S16, __half>::value) return __half2float(v);
        else return __bfloat162float(v);
    }
    __device__ __forceinline__ static S from_f(float v) {
        if constexpr (std::is_same<S16, __half>::value) return __float2half_rn(v);
        else return __float2bfloat16_rn(v);
    }
    template <int q>
    __device__ __forceinline__ static R decode_ref(S v, float ref, const DevParams& d) {
        return float(wq(q)) * ref + to_f(v) * d.inv_scale;
    }
    template <int q>
    __device__ __forceinline__ static R load_ref(const S* p, float ref, const DevParams& d) {
        return decode_ref<q>(__ldg(p), ref, d);
    }
    template <int q>
    __device__ __forceinline__ static S encode_ref(R v, float ref, const DevParams& d) {
        return from_f((v - float(wq(q)) * ref) * d.scale);
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
template <>
__device__ __forceinline__ double decode_rt<CodecF16Dev>(const __half* p, float w, const DevParams& d) {
    return double(w * d.rho_ref + __half2float(*p) * d.inv_scale);
}
template <>
__device__ __forceinline__ double decode_rt<CodecBF16Dev>(const __nv_bfloat16* p, float w, const DevParams& d) {
    return double(w * d.rho_ref + __bfloat162float(*p) * d.inv_scale);
}

template <class Codec>
__device__ __forceinline__ void encode_rt(typename Codec::S* p, float w, double v, const DevParams& d);
template <>
__device__ __forceinline__ void encode_rt<CodecF64>(double* p, float, double v, const DevParams&) { *p = v; }
template <>
__device__ __forceinline__ void encode_rt<CodecF32>(float* p, float, double v, const DevParams&) { *p = float(v); }
template <>
__device__ __forceinline__ void encode_rt<CodecF16Dev>(__half* p, float w, double v, const DevParams& d) {
    *p = __float2half_rn((float(v) - w * d.rho_ref) * d.scale);
}
template <>
__device__ __forceinline__ void encode_rt<CodecBF16Dev>(__nv_bfloat16* p, float w, double v, const DevParams& d) {
    *p = __float2bfloat16_rn((float(v) - w * d.rho_ref) * d.scale);
}

}  // namespace lbm
