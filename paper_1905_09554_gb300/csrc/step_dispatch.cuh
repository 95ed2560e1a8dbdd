// Template dispatch from a StepLaunch to the step kernel instantiations of
// one (storage codec, collision) pair.  Each step_<storage>_<collision>.cu
// instantiates one pair, so the build compiles them in parallel.
#pragma once
#include "step_args.h"
#include "step_kernel.cuh"
#include "step_multirange.cuh"
#include "step_pair16.cuh"

namespace lbm {

template <class Codec, int COLL, int TY>
cudaError_t launch_step_t(const StepLaunch& c, const void* src, void* dst) {
    constexpr int TX = 32;
    const StepArgs& a = c.args;
    if constexpr ((std::is_same_v<Codec, CodecF32> || std::is_same_v<Codec, CodecF64>) && TY >= 8) {
        if (c.kernel == 6) {
            dim3 grid((a.nx + TX - 1) / TX, (a.ny + TY - 1) / TY, (a.nz + a.zchunk - 1) / a.zchunk);
            sc_step_mr_kernel<Codec, COLL, TX, TY><<<grid, TX * TY, 0, c.stream>>>(
                static_cast<const typename Codec::S*>(src), static_cast<typename Codec::S*>(dst), a);
            return cudaGetLastError();
        }
    }
    if (c.kernel == 6) return cudaErrorNotSupported;  // FP64 / FP32 on 32x8 or 32x16 tiles only
    if constexpr (std::is_same_v<Codec, CodecF32>) {
        if (c.kernel == 4) {
            sc_step_bulk_kernel<COLL, TY><<<c.grid, BulkLayout<TY>::NT + 32, BulkLayout<TY>::bytes, c.stream>>>(
                static_cast<const float*>(src), static_cast<float*>(dst), a);
            return cudaGetLastError();
        }
        if constexpr (TY >= 8) {
            if (c.kernel == 5) {
                sc_step_tma_kernel<COLL, TY><<<c.grid, 32 * TY, TmaLayout<TY>::bytes, c.stream>>>(
                    *c.tmap, static_cast<const float*>(src), static_cast<float*>(dst), a);
                return cudaGetLastError();
            }
        }
    }
    if constexpr (sizeof(typename Codec::S) == 2) {  // 16-bit formats, nx even (checked by the host)
        if (c.kernel == 7) {
            sc_step_pair16_kernel<Codec, COLL, TY, unsigned><<<c.grid, 32 * TY, Pair16Layout<Codec, TY>::bytes,
                                                               c.stream>>>(
                static_cast<const typename Codec::S*>(src), static_cast<typename Codec::S*>(dst), a);
            return cudaGetLastError();
        }
    }
    if (c.kernel == 7) return cudaErrorNotSupported;
    {  // every storage type (16-bit: nx even, checked by the host)
        if (c.kernel == 3) {
            const size_t sm = PipeLayout<Codec, TX, TY>::bytes;
            sc_step_pipe_kernel<Codec, COLL, TX, TY, unsigned><<<c.grid, TX * TY, sm, c.stream>>>(
                static_cast<const typename Codec::S*>(src), static_cast<typename Codec::S*>(dst), a, BatchArgs{});
            return cudaGetLastError();
        }
    }
    if constexpr (sizeof(typename Codec::S) >= 4 && (TY <= 8 || sizeof(typename Codec::S) == 4)) {
        if (c.kernel == 2) {
            sc_step_async_kernel<Codec, COLL, TX, TY><<<c.grid, TX * TY, AsyncLayout<Codec, TX, TY>::bytes, c.stream>>>(
                static_cast<const typename Codec::S*>(src), static_cast<typename Codec::S*>(dst), a);
            return cudaGetLastError();
        }
    }
    dim3 grid((a.nx + TX - 1) / TX, (a.ny + TY - 1) / TY, (a.nz + a.zchunk - 1) / a.zchunk);
    sc_step_kernel<Codec, COLL, TX, TY><<<grid, TX * TY, 0, c.stream>>>(
        static_cast<const typename Codec::S*>(src), static_cast<typename Codec::S*>(dst), a);
    return cudaGetLastError();
}

template <class Codec, int COLL, int TY>
int prepare_async_t(const StepLaunch& c) {
    constexpr int TX = 32;
    if constexpr (std::is_same_v<Codec, CodecF32> && TY >= 8) {
        if (c.kernel == 5) {
            auto kern = sc_step_tma_kernel<COLL, TY>;
            const int sm = (int)TmaLayout<TY>::bytes;
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
            int per_sm = 0;
            if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * TY, sm);
            return e == cudaSuccess ? per_sm : -int(e);
        }
    }
    if constexpr (std::is_same_v<Codec, CodecF32>) {
        if (c.kernel == 4) {
            auto kern = sc_step_bulk_kernel<COLL, TY>;
            const int sm = (int)BulkLayout<TY>::bytes;
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
            int per_sm = 0;
            if (e == cudaSuccess)
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, BulkLayout<TY>::NT + 32, sm);
            return e == cudaSuccess ? per_sm : -int(e);
        }
    }
    if constexpr (sizeof(typename Codec::S) == 2) {
        if (c.kernel == 7) {
            using Lay = Pair16Layout<Codec, TY>;
            auto kern = sc_step_pair16_kernel<Codec, COLL, TY, unsigned>;
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Lay::bytes);
            int per_sm = 0;
            if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, Lay::NT, Lay::bytes);
            return e == cudaSuccess ? per_sm : -int(e);
        }
    }
    if (c.kernel == 7) return 0;
    {  // every storage type (16-bit: nx even, checked by the host)
        if (c.kernel == 3) {
            using Lay = PipeLayout<Codec, TX, TY>;
            auto kern = sc_step_pipe_kernel<Codec, COLL, TX, TY, unsigned>;
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Lay::bytes);
            int per_sm = 0;
            if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, TX * TY, Lay::bytes);
            return e == cudaSuccess ? per_sm : -int(e);
        }
    }
    if constexpr (sizeof(typename Codec::S) >= 4 && (TY <= 8 || sizeof(typename Codec::S) == 4)) {
        using Lay = AsyncLayout<Codec, TX, TY>;
        auto kern = sc_step_async_kernel<Codec, COLL, TX, TY>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Lay::bytes);
        int per_sm = 0;
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, TX * TY, Lay::bytes);
        return e == cudaSuccess ? per_sm : -int(e);
    }
    return 0;
}

template <class Codec, int COLL, int TY>
cudaError_t launch_batch_t(const StepLaunch& c, const BatchArgs& b, const void* src, void* dst) {
    constexpr int TX = 32;
    const size_t sm = PipeLayout<Codec, TX, TY>::bytes;
    sc_step_pipe_kernel<Codec, COLL, TX, TY, unsigned, true><<<c.grid, TX * TY, sm, c.stream>>>(
        static_cast<const typename Codec::S*>(src), static_cast<typename Codec::S*>(dst), c.args, b);
    return cudaGetLastError();
}

template <class Codec, int COLL, int TY>
int prepare_batch_t(const StepLaunch&) {
    constexpr int TX = 32;
    using Lay = PipeLayout<Codec, TX, TY>;
    auto kern = sc_step_pipe_kernel<Codec, COLL, TX, TY, unsigned, true>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Lay::bytes);
    int per_sm = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, TX * TY, Lay::bytes);
    return e == cudaSuccess ? per_sm : -int(e);
}

template <class Codec, int COLL>
cudaError_t launch_step_cc(const StepLaunch& c, const void* src, void* dst) {
    switch (c.tile_y) {
        case 4: return launch_step_t<Codec, COLL, 4>(c, src, dst);
        case 16: return launch_step_t<Codec, COLL, 16>(c, src, dst);
        default: return launch_step_t<Codec, COLL, 8>(c, src, dst);
    }
}

template <class Codec, int COLL>
int prepare_step_cc(const StepLaunch& c) {
    switch (c.tile_y) {
        case 4: return prepare_async_t<Codec, COLL, 4>(c);
        case 16: return prepare_async_t<Codec, COLL, 16>(c);
        default: return prepare_async_t<Codec, COLL, 8>(c);
    }
}

template <class Codec, int COLL>
cudaError_t launch_batch_cc(const StepLaunch& c, const BatchArgs& b, const void* src, void* dst) {
    switch (c.tile_y) {
        case 4: return launch_batch_t<Codec, COLL, 4>(c, b, src, dst);
        case 16: return launch_batch_t<Codec, COLL, 16>(c, b, src, dst);
        default: return launch_batch_t<Codec, COLL, 8>(c, b, src, dst);
    }
}

template <class Codec, int COLL>
int prepare_batch_cc(const StepLaunch& c) {
    switch (c.tile_y) {
        case 4: return prepare_batch_t<Codec, COLL, 4>(c);
        case 16: return prepare_batch_t<Codec, COLL, 16>(c);
        default: return prepare_batch_t<Codec, COLL, 8>(c);
    }
}

}  // namespace lbm

// Defines the kernel table entry of one (storage, collision) pair.
#define LBM_STEP_INSTANCE(NAME, CODEC, COLL, WITH_BATCH)                                                \
    namespace lbm {                                                                                   \
    static cudaError_t launch_##NAME(const StepLaunch& l, const void* s, void* d) {                    \
        return launch_step_cc<CODEC, COLL>(l, s, d);                                                  \
    }                                                                                                 \
    static int prepare_##NAME(const StepLaunch& l) { return prepare_step_cc<CODEC, COLL>(l); }         \
    static cudaError_t batch_##NAME(const StepLaunch& l, const BatchArgs& b, const void* s, void* d) { \
        if constexpr (WITH_BATCH) return launch_batch_cc<CODEC, COLL>(l, b, s, d);                    \
        else return cudaErrorNotSupported;                                                            \
    }                                                                                                 \
    static int batch_prepare_##NAME(const StepLaunch& l) {                                            \
        if constexpr (WITH_BATCH) return prepare_batch_cc<CODEC, COLL>(l);                            \
        else return 0;                                                                                \
    }                                                                                                 \
    extern const StepKernels kStep_##NAME = {launch_##NAME, prepare_##NAME, batch_##NAME,             \
                                             batch_prepare_##NAME};                                   \
    }
