// Allocation-free ligament diagnostics (lbm_diag_noalloc in include/lbm_sc.h).
//
// Who needs it: callers that may not allocate device memory while they run.
// Examples are a host application whose device memory is handed out entirely
// by its own pool allocator (so a raw cudaMalloc would fail or fragment the
// pool), or a tight time-stepping loop where cudaMalloc/cudaFree would
// implicitly synchronise the device.  Such a caller owns its population array
// and its output arrays and calls this entry point, which uses only the
// fixed scratch array below.
//
// The scratch is a file-scope __device__ array: every GPU that loads the
// library holds LBM_NOALLOC_MAX_NZ * 8 doubles of it (512 KiB) until the
// process exits.  In host code its name is only a host-side stand-in, so its
// device address is looked up once per device with cudaGetSymbolAddress.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "../../include/lbm_sc.h"
#include "codec.cuh"
#include "diag_cell.cuh"
#include "lattice.cuh"

using namespace lbm;

namespace {

constexpr int kMaxNz = LBM_NOALLOC_MAX_NZ;
constexpr int kThreads = 256;
constexpr int kMaxDevices = 64;

// Per-slice partials, quantity-major: slot k*kMaxNz + z with k = 0 mass,
// 1..3 momentum, 4 liquid area, 5 max rho, 6 bad cells; then the 4 totals
// (mass, momentum) and the total bad-cell count at 7*kMaxNz.
static __device__ __align__(256) double g_noalloc_scratch[8 * kMaxNz];

std::mutex g_setup_mutex;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

// One block per z slice, fixed-order tree reduction in float64 (the same
// per-slice arithmetic as the context-based diagnostics), written into the
// quantity-major scratch layout.
template <class Codec>
__global__ void __launch_bounds__(kThreads)
slice_diag_noalloc_kernel(double* __restrict__ scratch, const typename Codec::S* __restrict__ f, int nx, int ny,
                          long long n, double rho_l, double rho_v, DevParams dev) {
    __shared__ double red[7][kThreads];
    const int z = blockIdx.x;
    const long long plane = (long long)nx * ny;
    double acc[7];
    diag_accumulate<Codec>(f + z * plane, n, plane, threadIdx.x, kThreads, dev, rho_v, 1.0 / (rho_l - rho_v),
                           nullptr, acc);
    const double m = acc[0], jx = acc[1], jy = acc[2], jz = acc[3], area = acc[4], mx = acc[5], bad = acc[6];
    red[0][threadIdx.x] = m;
    red[1][threadIdx.x] = jx;
    red[2][threadIdx.x] = jy;
    red[3][threadIdx.x] = jz;
    red[4][threadIdx.x] = area;
    red[5][threadIdx.x] = mx;
    red[6][threadIdx.x] = bad;
    __syncthreads();
    for (int s = kThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            for (int k = 0; k < 7; ++k) {
                if (k == 5) red[k][threadIdx.x] = fmax(red[k][threadIdx.x], red[k][threadIdx.x + s]);
                else red[k][threadIdx.x] += red[k][threadIdx.x + s];
            }
        }
        __syncthreads();
    }
    if (threadIdx.x < 7) scratch[threadIdx.x * kMaxNz + z] = red[threadIdx.x][0];
}

// Totals over slices, summed in z order by one thread (deterministic), into
// scratch[7*kMaxNz + 0..4]; optionally copies the per-slice area / max rho and
// the totals to caller device arrays.
__global__ void totals_noalloc_kernel(double* __restrict__ scratch, int nz, double* mass, double* mom,
                                      double* area_z, double* maxrho_z) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        double m = 0, jx = 0, jy = 0, jz = 0, bad = 0;
        for (int z = 0; z < nz; ++z) {
            m += scratch[0 * kMaxNz + z];
            jx += scratch[1 * kMaxNz + z];
            jy += scratch[2 * kMaxNz + z];
            jz += scratch[3 * kMaxNz + z];
            bad += scratch[6 * kMaxNz + z];
        }
        double* tot = scratch + 7 * kMaxNz;
        tot[0] = m;
        tot[1] = jx;
        tot[2] = jy;
        tot[3] = jz;
        tot[4] = bad;
        if (mass) *mass = m;
        if (mom) {
            mom[0] = jx;
            mom[1] = jy;
            mom[2] = jz;
        }
    }
    for (int z = blockIdx.x * blockDim.x + threadIdx.x; z < nz; z += gridDim.x * blockDim.x) {
        if (area_z) area_z[z] = scratch[4 * kMaxNz + z];
        if (maxrho_z) maxrho_z[z] = scratch[5 * kMaxNz + z];
    }
}

// Device address of the scratch array on the current device, looked up once
// per device (the first call on each device does it).
cudaError_t scratch_address(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

template <class Codec>
cudaError_t launch_slices(double* scratch, const void* f, int nx, int ny, int nz, double rho_l, double rho_v,
                          const DevParams& dev, cudaStream_t st) {
    slice_diag_noalloc_kernel<Codec><<<nz, kThreads, 0, st>>>(scratch, static_cast<const typename Codec::S*>(f),
                                                              nx, ny, (long long)nx * ny * nz, rho_l, rho_v, dev);
    return cudaGetLastError();
}

}  // namespace

extern "C" lbm_status lbm_diag_noalloc(const void* f, int storage, int nx, int ny, int nz, double rho_ref,
                                       double dev_scale, double rho_l, double rho_v, double* mass, double mom[3],
                                       double* area_z, double* maxrho_z, int on_device, void* stream) {
    if (!f) return LBM_EINVAL;
    if (nx < 1 || ny < 1 || nz < 1) return LBM_EINVAL;
    if (nz > kMaxNz) return LBM_EUNSUPPORTED;  // beyond the static scratch capacity
    if (!(rho_l > rho_v)) return LBM_EINVAL;
    if (storage < LBM_F64 || storage > LBM_BF16_DEV) return LBM_EINVAL;
    if (storage >= LBM_F16_DEV && !(dev_scale > 0)) return LBM_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    double* scratch = nullptr;
    cudaError_t e = scratch_address(&scratch);
    if (e != cudaSuccess) return LBM_ECUDA;
    const DevParams dev = make_dev_params(rho_ref, dev_scale > 0 ? dev_scale : 1.0);
    switch (storage) {
        case LBM_F64: e = launch_slices<CodecF64>(scratch, f, nx, ny, nz, rho_l, rho_v, dev, st); break;
        case LBM_F32: e = launch_slices<CodecF32>(scratch, f, nx, ny, nz, rho_l, rho_v, dev, st); break;
        case LBM_F16_DEV: e = launch_slices<CodecF16Dev>(scratch, f, nx, ny, nz, rho_l, rho_v, dev, st); break;
        default: e = launch_slices<CodecBF16Dev>(scratch, f, nx, ny, nz, rho_l, rho_v, dev, st); break;
    }
    if (e != cudaSuccess) return LBM_ECUDA;
    const int tb = 256, tg = (nz + tb - 1) / tb;
    if (on_device) totals_noalloc_kernel<<<tg, tb, 0, st>>>(scratch, nz, mass, mom, area_z, maxrho_z);
    else totals_noalloc_kernel<<<tg, tb, 0, st>>>(scratch, nz, nullptr, nullptr, nullptr, nullptr);
    e = cudaGetLastError();
    if (e != cudaSuccess) return LBM_ECUDA;
    double tot[5];
    e = cudaMemcpyAsync(tot, scratch + 7 * kMaxNz, sizeof(tot), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && !on_device) {
        if (area_z) e = cudaMemcpyAsync(area_z, scratch + 4 * kMaxNz, sizeof(double) * nz, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && maxrho_z)
            e = cudaMemcpyAsync(maxrho_z, scratch + 5 * kMaxNz, sizeof(double) * nz, cudaMemcpyDeviceToHost, st);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return LBM_ECUDA;
    if (!on_device) {
        if (mass) *mass = tot[0];
        if (mom) {
            mom[0] = tot[1];
            mom[1] = tot[2];
            mom[2] = tot[3];
        }
    }
    if (tot[4] > 0 || !std::isfinite(tot[0]))
        return LBM_ENONFINITE;
    return LBM_OK;
}
