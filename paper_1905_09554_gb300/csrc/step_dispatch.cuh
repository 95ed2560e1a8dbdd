// Template dispatch from a StepLaunch to the step kernel instantiations of one
// storage codec; included by the per-storage translation units only.
#pragma once
#include "step_args.h"
#include "step_kernel.cuh"

namespace lbm {

template <class Codec, int COLL, int TY>
cudaError_t launch_step_t(const StepLaunch& c, const void* src, void* dst) {
    constexpr int TX = 32;
    const StepArgs& a = c.args;
    if constexpr (sizeof(typename Codec::S) >= 4) {
        if (c.kernel == 3) {
            const size_t sm = PipeLayout<Codec, TX, TY>::bytes;
            if (c.idx32)
                sc_step_pipe_kernel<Codec, COLL, TX, TY, int><<<c.grid, TX * TY, sm, c.stream>>>(
                    static_cast<const typename Codec::S*>(src), static_cast<typename Codec::S*>(dst), a, BatchArgs{});
            else
                sc_step_pipe_kernel<Codec, COLL, TX, TY, long long><<<c.grid, TX * TY, sm, c.stream>>>(
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

// Prepare the cp.async kernel: opt in to its shared memory and size the
// persistent grid from the occupancy calculator.  Returns 0 if the variant
// cannot run for this storage/tile.
template <class Codec, int COLL, int TY>
int prepare_async_t(const StepLaunch& c) {
    constexpr int TX = 32;
    if constexpr (sizeof(typename Codec::S) >= 4) {
        if (c.kernel == 3) {
            using Lay = PipeLayout<Codec, TX, TY>;
            auto kern = c.idx32 ? sc_step_pipe_kernel<Codec, COLL, TX, TY, int>
                                 : sc_step_pipe_kernel<Codec, COLL, TX, TY, long long>;
            if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Lay::bytes) !=
                cudaSuccess)
                return 0;
            int per_sm = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, TX * TY, Lay::bytes) != cudaSuccess)
                return 0;
            return per_sm;
        }
    }
    if constexpr (sizeof(typename Codec::S) >= 4 && (TY <= 8 || sizeof(typename Codec::S) == 4)) {
        using Lay = AsyncLayout<Codec, TX, TY>;
        auto kern = sc_step_async_kernel<Codec, COLL, TX, TY>;
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Lay::bytes) != cudaSuccess)
            return 0;
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, TX * TY, Lay::bytes) != cudaSuccess ||
            per_sm < 1)
            return 0;
        return per_sm;
    }
    return 0;
}

template <class Codec, int COLL>
int prepare_async_c(const StepLaunch& c) {
    switch (c.tile_y) {
        case 4: return prepare_async_t<Codec, COLL, 4>(c);
        case 16: return prepare_async_t<Codec, COLL, 16>(c);
        default: return prepare_async_t<Codec, COLL, 8>(c);
    }
}

template <class Codec, int COLL>
cudaError_t launch_step_c(const StepLaunch& c, const void* src, void* dst) {
    switch (c.tile_y) {
        case 4: return launch_step_t<Codec, COLL, 4>(c, src, dst);
        case 16: return launch_step_t<Codec, COLL, 16>(c, src, dst);
        default: return launch_step_t<Codec, COLL, 8>(c, src, dst);
    }
}

template <class Codec>
cudaError_t launch_step_s(const StepLaunch& c, const void* src, void* dst) {
    return c.coll == COLL_MRT ? launch_step_c<Codec, COLL_MRT>(c, src, dst)
                                         : launch_step_c<Codec, COLL_SRT>(c, src, dst);
}

template <class Codec>
int prepare_async_s(const StepLaunch& c) {
    return c.coll == COLL_MRT ? prepare_async_c<Codec, COLL_MRT>(c) : prepare_async_c<Codec, COLL_SRT>(c);
}

// Batched pipelined step: one launch advances every box of the batch.
template <class Codec, int COLL, int TY>
cudaError_t launch_batch_t(const StepLaunch& c, const BatchArgs& b, const void* src, void* dst) {
    constexpr int TX = 32;
    const size_t sm = PipeLayout<Codec, TX, TY>::bytes;
    sc_step_pipe_kernel<Codec, COLL, TX, TY, int, true><<<c.grid, TX * TY, sm, c.stream>>>(
        static_cast<const typename Codec::S*>(src), static_cast<typename Codec::S*>(dst), c.args, b);
    return cudaGetLastError();
}

template <class Codec, int COLL, int TY>
int prepare_batch_t(const StepLaunch&) {
    constexpr int TX = 32;
    using Lay = PipeLayout<Codec, TX, TY>;
    auto kern = sc_step_pipe_kernel<Codec, COLL, TX, TY, int, true>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Lay::bytes) != cudaSuccess)
        return 0;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, TX * TY, Lay::bytes) != cudaSuccess) return 0;
    return per_sm;
}

template <class Codec>
cudaError_t launch_batch_s(const StepLaunch& c, const BatchArgs& b, const void* src, void* dst) {
    const bool mrt = c.coll == COLL_MRT;
    switch (c.tile_y) {
        case 4: return mrt ? launch_batch_t<Codec, COLL_MRT, 4>(c, b, src, dst) : launch_batch_t<Codec, COLL_SRT, 4>(c, b, src, dst);
        case 16: return mrt ? launch_batch_t<Codec, COLL_MRT, 16>(c, b, src, dst) : launch_batch_t<Codec, COLL_SRT, 16>(c, b, src, dst);
        default: return mrt ? launch_batch_t<Codec, COLL_MRT, 8>(c, b, src, dst) : launch_batch_t<Codec, COLL_SRT, 8>(c, b, src, dst);
    }
}

template <class Codec>
int prepare_batch_s(const StepLaunch& c) {
    const bool mrt = c.coll == COLL_MRT;
    switch (c.tile_y) {
        case 4: return mrt ? prepare_batch_t<Codec, COLL_MRT, 4>(c) : prepare_batch_t<Codec, COLL_SRT, 4>(c);
        case 16: return mrt ? prepare_batch_t<Codec, COLL_MRT, 16>(c) : prepare_batch_t<Codec, COLL_SRT, 16>(c);
        default: return mrt ? prepare_batch_t<Codec, COLL_MRT, 8>(c) : prepare_batch_t<Codec, COLL_SRT, 8>(c);
    }
}

}  // namespace lbm
