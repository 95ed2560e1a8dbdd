// C ABI of the D3Q19 Shan-Chen lattice Boltzmann library (include/lbm_sc.h):
// context management, initial states, the time-step driver, moments and
// diagnostics.  The fused step kernel lives in step_kernel.cuh.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/lbm_sc.h"
#include "codec.cuh"
#include "diag_cell.cuh"
#include "e8.cuh"
#include "lattice.cuh"
#include "step_args.h"
#include "adjoint.h"

using namespace lbm;

struct lbm_batch;

struct lbm_ctx {
    lbm_params p;
    cudaStream_t stream = nullptr;
    int device = 0;
    int num_sms = 0;
    void* f[2] = {nullptr, nullptr};  // population copies; f[cur] is the state
    bool own_f = false;
    float* ref[2] = {nullptr, nullptr};  // local-reference storage: density field paired with f[k]
    int cur = 0;
    long t = 0;
    long long n = 0;
    size_t elem = 0;                  // bytes per stored population
    double* scratch = nullptr;        // staging / moments scratch (lazily grown)
    size_t scratch_bytes = 0;
    double* diag = nullptr;           // per-slice diagnostic partials (8 * nz)
    int* dev_err = nullptr;           // device error word of the bounded waits
    std::vector<double> diag_host;
    long long own_bytes = 0;
    StepArgs args{};
    int zchunk = 0, tile_y = 8;
    int kernel = 1;                   // 1 register-staged, 2 cp.async, 3 pipelined, 4 bulk, 5 tensor
    CUtensorMap tmap[2];              // kernel 5: tensor maps of the two population copies
    int grid3 = 0;                    // kernel 5: grid of the pipelined kernel used for other buffers
    int coll = COLL_SRT;              // collision kernel (COLL_*)
    int grid = 0;                     // persistent grid size (kernels 2, 3)
    char err[512] = {0};
    lbm_batch* batch = nullptr;       // set when the context is a view of a batch box
    // discrete adjoint (allocated by lbm_adjoint_forward)
    struct Adjoint {
        void* cp = nullptr;           // checkpoints, ncp states
        void* seg = nullptr;          // recomputed states of one segment, `every` states
        void* lam[2] = {nullptr, nullptr};
        void* gr[2] = {nullptr, nullptr};  // the force term of lam, one value per cell
        void* psi = nullptr;          // psi of each state of a segment, `every` fields
        void* gF = nullptr;           // psi gF and S.gF of the reverse step, 4 fields
        double* partials = nullptr;   // 2 per block
        double* acc = nullptr;        // dJ/dG, dJ/dtau
        double* io = nullptr;         // host <-> device staging of one field
        size_t cp_bytes = 0, seg_bytes = 0, psi_bytes = 0;
        long T = -1;                  // steps of the recorded forward run
        int every = 0, ncp = 0;
    } adj;

    lbm_status fail(lbm_status s, const char* fmt, ...) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(err, sizeof(err), fmt, ap);
        va_end(ap);
        return s;
    }
};

static thread_local char g_create_err[512];

// A failed runtime call is reported through the returned status; its error
// is also taken out of the runtime's last-error slot (a non-sticky error such
// as an out-of-memory cudaMalloc would otherwise surface at the next launch
// check as a launch failure).
static lbm_status runtime_status(cudaError_t e) {
    if (e == cudaSuccess) return LBM_OK;
    (void)cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA;
}

#define LBM_CUDA(ctx, call)                                                                  \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return (ctx)->fail(runtime_status(e_), "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

#define LBM_LAUNCHED(ctx, what)                                                              \
    do {                                                                                     \
        cudaError_t e_ = cudaGetLastError();                                                 \
        if (e_ != cudaSuccess)                                                               \
            return (ctx)->fail(LBM_ECUDA, "%s launch failed: %s", what, cudaGetErrorString(e_)); \
    } while (0)

// ----------------------------------------------------------------------------
// Small kernels: initial states, conversions, moments, diagnostics.
// ----------------------------------------------------------------------------
namespace {

// Weight of population q in the library order (rest, 6 axis, 12 edge).
__device__ __forceinline__ float weight_rt(int q) {
    return q == 0 ? float(1.0 / 3.0) : (q < 7 ? float(1.0 / 18.0) : float(1.0 / 36.0));
}
__device__ __forceinline__ double weight_rt_d(int q) {
    return q == 0 ? 1.0 / 3.0 : (q < 7 ? 1.0 / 18.0 : 1.0 / 36.0);
}

// Runtime decode / encode of population q of `cell`; local-reference codecs
// use the cell's reference density ref[cell].
template <class Codec>
__device__ __forceinline__ double dec(const typename Codec::S* p, int q, const float* ref, long long cell,
                                      const DevParams& d) {
    if constexpr (Codec::kLocal) return Codec::decode_rt(p, weight_rt(q), ref[cell], d);
    else return decode_rt<Codec>(p, weight_rt(q), d);
}
template <class Codec>
__device__ __forceinline__ void enc(typename Codec::S* p, int q, double v, const float* ref, long long cell,
                                    const DevParams& d) {
    if constexpr (Codec::kLocal) Codec::encode_rt(p, weight_rt(q), v, ref[cell], d);
    else encode_rt<Codec>(p, weight_rt(q), v, d);
}

template <class Codec>
__global__ void rest_state_kernel(typename Codec::S* __restrict__ f, const double* __restrict__ rho,
                                  long long n, DevParams dev, float* ref) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const double r = rho[i];
        if constexpr (Codec::kLocal) ref[i] = float(r);
        for (int q = 0; q < Q; ++q) enc<Codec>(f + q * n + i, q, weight_rt_d(q) * r, ref, i, dev);
    }
}

template <class Codec>
__global__ void ligament_kernel(typename Codec::S* __restrict__ f, int nx, int ny, int nz, double R0,
                                double eps, int n_waves, double width, double rho_l, double rho_v,
                                DevParams dev, float* ref) {
    const long long n = (long long)nx * ny * nz;
    const double xc = 0.5 * (nx - 1), yc = 0.5 * (ny - 1);
    const double two_pi = 6.283185307179586476925286766559;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int x = int(i % nx);
        const int y = int((i / nx) % ny);
        const int z = int(i / ((long long)nx * ny));
        const double dx = x - xc, dy = y - yc;
        const double r = sqrt(dx * dx + dy * dy);
        const double R = R0 * (1.0 + eps * cos(two_pi * n_waves * z / nz));
        const double rho = rho_v + 0.5 * (rho_l - rho_v) * (1.0 - tanh((r - R) / width));
        if constexpr (Codec::kLocal) ref[i] = float(rho);
        for (int q = 0; q < Q; ++q) enc<Codec>(f + q * n + i, q, weight_rt_d(q) * rho, ref, i, dev);
    }
}

// Element i of `f` belongs to population q0 + i / n.
template <class Codec>
__global__ void decode_kernel(double* __restrict__ out, const typename Codec::S* __restrict__ f,
                              long long count, long long n, int q0, DevParams dev, const float* ref) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = dec<Codec>(f + i, q0 + int(i / n), ref, i % n, dev);
}

template <class Codec>
__global__ void encode_kernel(typename Codec::S* __restrict__ f, const double* __restrict__ in,
                              long long count, long long n, int q0, DevParams dev, const float* ref) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x)
        enc<Codec>(f + i, q0 + int(i / n), in[i], ref, i % n, dev);
}

// Local-reference codecs: the reference density of a cell given all its
// populations is their sum.  acc (float64) may be accumulated population by
// population (add = 1) before ref is set from it (add = 0, in = nullptr).
__global__ void ref_sum_kernel(float* __restrict__ ref, double* __restrict__ acc, const double* __restrict__ in,
                               long long n, int count_q, int mode) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        if (mode == 0) {  // all populations present in `in`
            double r = 0.0;
            for (int q = 0; q < count_q; ++q) r += in[q * n + i];
            ref[i] = float(r);
        } else if (mode == 1) {  // add one population into acc
            acc[i] = (count_q == 0 ? 0.0 : acc[i]) + in[i];
        } else {  // finish: ref from acc
            ref[i] = float(acc[i]);
        }
    }
}

template <class Codec>
__global__ void density_kernel(double* __restrict__ rho, const typename Codec::S* __restrict__ f,
                               long long n, DevParams dev, const float* ref) {
    // rho summed in the storage's arithmetic type, as the step kernel does
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        typename Codec::R r, jx, jy, jz;
        diag_cell<Codec>(f + i, n, dev, Codec::kLocal ? ref[i] : 0.0f, r, jx, jy, jz);
        rho[i] = double(r);
    }
}

// u_b = (j + F/2)/rho with F from Eq. SC_force evaluated on the density
// field `rho` (float64), j from the populations.
__device__ __forceinline__ int wrap_periodic(int i, int n) {  // periodic index, any offset
    i %= n;
    return i < 0 ? i + n : i;
}

template <class Codec>
__global__ void velocity_kernel(double* __restrict__ ux, double* __restrict__ uy, double* __restrict__ uz,
                                const double* __restrict__ rho, const typename Codec::S* __restrict__ f,
                                int nx, int ny, int nz, double G, double G2, double rho0, DevParams dev,
                                const float* ref) {
    const long long n = (long long)nx * ny * nz;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int x = int(i % nx);
        const int y = int((i / nx) % ny);
        const int z = int(i / ((long long)nx * ny));
        double jx = 0, jy = 0, jz = 0, sx = 0, sy = 0, sz = 0;
        static_for<0, Q>([&](auto qc) {
            constexpr int q = decltype(qc)::value;
            const double fq = dec<Codec>(f + q * n + i, q, ref, i, dev);
            jx += cx(q) * fq;
            jy += cy(q) * fq;
            jz += cz(q) * fq;
            if constexpr (q != 0) {
                int xx = x + cx(q), yy = y + cy(q), zz = z + cz(q);
                xx = xx < 0 ? nx - 1 : (xx == nx ? 0 : xx);
                yy = yy < 0 ? ny - 1 : (yy == ny ? 0 : yy);
                zz = zz < 0 ? nz - 1 : (zz == nz ? 0 : zz);
                const double rn = rho[((long long)zz * ny + yy) * nx + xx];
                const double psn = rho0 * (1.0 - exp(-rn / rho0));
                sx += wq(q) * cx(q) * psn;
                sy += wq(q) * cy(q) * psn;
                sz += wq(q) * cz(q) * psn;
            }
        });
        sx *= G;
        sy *= G;
        sz *= G;
        if (G2 != 0.0) {  // second belt of the two-belt force: E8 vectors, weights p/3
            static_for<0, mr::kNE>([&](auto kc) {
                constexpr mr::Vec e = mr::e8(decltype(kc)::value);
                constexpr double pw = mr::p_e8(e.x * e.x + e.y * e.y + e.z * e.z) / 3.0;
                const int xx = wrap_periodic(x + e.x, nx), yy = wrap_periodic(y + e.y, ny),
                          zz = wrap_periodic(z + e.z, nz);
                const double rn = rho[((long long)zz * ny + yy) * nx + xx];
                const double psn = G2 * pw * rho0 * (1.0 - exp(-rn / rho0));
                if constexpr (e.x != 0) sx += e.x * psn;
                if constexpr (e.y != 0) sy += e.y * psn;
                if constexpr (e.z != 0) sz += e.z * psn;
            });
        }
        const double r = rho[i];
        const double g = -rho0 * (1.0 - exp(-r / rho0));
        if (ux) ux[i] = (jx + 0.5 * g * sx) / r;
        if (uy) uy[i] = (jy + 0.5 * g * sy) / r;
        if (uz) uz[i] = (jz + 0.5 * g * sz) / r;
    }
}

// One block per z slice; fixed-order tree reduction in float64 (deterministic).
// out[8*z + k]: k = 0 mass, 1..3 momentum, 4 liquid area, 5 max rho,
// 6 count of cells with rho <= 0 or non-finite.
constexpr int DIAG_THREADS = 256;

template <class Codec>
__global__ void __launch_bounds__(DIAG_THREADS)
diag_kernel(double* __restrict__ out, const typename Codec::S* __restrict__ f, int nx, int ny,
            long long n, double rho_l, double rho_v, DevParams dev, const float* ref) {
    __shared__ double red[7][DIAG_THREADS];
    const int z = blockIdx.x;
    const long long plane = (long long)nx * ny;
    double acc[7];
    diag_accumulate<Codec>(f + z * plane, n, plane, threadIdx.x, DIAG_THREADS, dev, rho_v, 1.0 / (rho_l - rho_v),
                           Codec::kLocal ? ref + z * plane : nullptr, acc);
    const double m = acc[0], jx = acc[1], jy = acc[2], jz = acc[3], area = acc[4], mx = acc[5], bad = acc[6];
    red[0][threadIdx.x] = m;
    red[1][threadIdx.x] = jx;
    red[2][threadIdx.x] = jy;
    red[3][threadIdx.x] = jz;
    red[4][threadIdx.x] = area;
    red[5][threadIdx.x] = mx;
    red[6][threadIdx.x] = bad;
    __syncthreads();
    for (int s = DIAG_THREADS / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            for (int k = 0; k < 7; ++k) {
                if (k == 5) red[k][threadIdx.x] = fmax(red[k][threadIdx.x], red[k][threadIdx.x + s]);
                else red[k][threadIdx.x] += red[k][threadIdx.x + s];
            }
        }
        __syncthreads();
    }
    if (threadIdx.x < 7) out[8 * z + threadIdx.x] = red[threadIdx.x][0];
}

int grid_for(long long work, int threads, int num_sms) {
    long long b = (work + threads - 1) / threads;
    const long long cap = (long long)num_sms * 16;
    if (b > cap) b = cap;
    return int(b < 1 ? 1 : b);
}

// ----------------------------------------------------------------------------
// Typed dispatch
// ----------------------------------------------------------------------------
StepLaunch step_launch(const lbm_ctx* c) {
    StepLaunch l;
    l.args = c->args;
    l.kernel = c->kernel;
    l.tmap = nullptr;
    l.tile_y = c->tile_y;
    l.grid = c->grid;
    l.coll = c->coll;
    l.stream = c->stream;
    return l;
}

int prepare_async(lbm_ctx* c) {
    const int st = c->p.storage;
    // 16-bit storage: the pipelined kernel only, with nx even
    const bool word16 = st >= LBM_F16_DEV && (c->kernel == 3 || c->kernel == 7) && c->p.nx % 2 == 0;
    if (st != LBM_F64 && st != LBM_F32 && !word16) return 0;
    return step_kernels(st, c->coll).prepare(step_launch(c));
}

cudaError_t launch_step(const lbm_ctx* c, const void* src, void* dst, void* psi_out = nullptr) {
    StepLaunch l = step_launch(c);
    l.args.psi_out = psi_out;
    if (c->kernel == 5) {
        const int idx = src == c->f[0] ? 0 : (src == c->f[1] ? 1 : -1);
        if (idx >= 0) {
            l.tmap = &c->tmap[idx];
        } else {  // other buffers (adjoint segments): the pipelined kernel
            l.kernel = 3;
            l.grid = c->grid3;
        }
    }
    if (c->ref[0]) {  // local-reference storage: the density fields follow their population copies
        const int k = src == c->f[0] ? 0 : 1;
        l.args.ref_src = c->ref[k];
        l.args.ref_dst = c->ref[k ^ 1];
    }
    return step_kernels(c->p.storage, c->coll).launch(l, src, dst);
}

// Tensor maps of the two population copies for the tensor-copy kernel:
// 4-D (x, y, z, population), FP32, box 32 x tile_y x 1 x 19.
lbm_status encode_tensor_maps(lbm_ctx* c) {
    using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q{};
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || !fn || q != cudaDriverEntryPointSuccess)
        return c->fail(LBM_ECUDA, "cuTensorMapEncodeTiled is not available");
    const cuuint64_t nx = c->p.nx, ny = c->p.ny, nz = c->p.nz;
    const cuuint64_t dims[4] = {nx, ny, nz, (cuuint64_t)Q};
    const cuuint64_t strides[3] = {nx * 4, nx * ny * 4, nx * ny * nz * 4};
    const cuuint32_t box[4] = {32, (cuuint32_t)c->tile_y, 1, (cuuint32_t)Q};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    for (int k = 0; k < 2; ++k) {
        CUresult r = reinterpret_cast<EncodeFn>(fn)(&c->tmap[k], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, c->f[k], dims,
                                                    strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return c->fail(LBM_ECUDA, "cuTensorMapEncodeTiled failed (%d)", int(r));
    }
    return LBM_OK;
}

// Collision kernel for the operator and rates: the MRT specialisations are
// exact for rates equal to 1 outside the listed moments.
int collision_kernel(const lbm_params& p, const double (&s)[Q]) {
    if (p.collision != LBM_MRT_GUO) return COLL_SRT;
    bool unit = true, sparse = true;
    for (int k = 0; k < Q; ++k) {
        if (k == 0 || k == 3 || k == 5 || k == 7) continue;  // conserved: rate irrelevant
        const bool in_k = (k == 1 || k == 9 || k == 11 || k == 13 || k == 14 || k == 15);
        if (s[k] != 1.0) {
            unit = false;
            if (!in_k) sparse = false;
        }
    }
    if (unit) return COLL_MRT_UNIT;
    if (!sparse) return COLL_MRT;
    return s[1] == 1.0 ? COLL_MRT_SHEAR : COLL_MRT_SPARSE;  // e at 1: the shear rule
}

// Run `fn.template operator()<Codec>()` for the context's storage type.
template <class Fn>
auto with_codec(const lbm_ctx* c, Fn&& fn) {
    switch (c->p.storage) {
        case LBM_F64: return fn(CodecF64{});
        case LBM_F16_DEV: return fn(CodecF16Dev{});
        case LBM_BF16_DEV: return fn(CodecBF16Dev{});
        case LBM_F16_LOCAL: return fn(CodecF16Local{});
        case LBM_BF16_LOCAL: return fn(CodecBF16Local{});
        default: return fn(CodecF32{});
    }
}

lbm_status ensure_scratch(lbm_ctx* c, size_t bytes) {
    if (c->scratch_bytes >= bytes) return LBM_OK;
    if (c->scratch) {
        cudaStreamSynchronize(c->stream);
        cudaFree(c->scratch);
        c->own_bytes -= (long long)c->scratch_bytes;
        c->scratch = nullptr;
        c->scratch_bytes = 0;
    }
    LBM_CUDA(c, cudaMalloc(&c->scratch, bytes));
    c->scratch_bytes = bytes;
    c->own_bytes += (long long)bytes;
    return LBM_OK;
}

// Read and clear the device error word: a bounded device wait that timed out
// leaves the populations invalid.
lbm_status check_device_error(lbm_ctx* c) {
    int e = 0;
    LBM_CUDA(c, cudaMemcpyAsync(&e, c->dev_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    if (e) {
        LBM_CUDA(c, cudaMemsetAsync(c->dev_err, 0, sizeof(int), c->stream));
        return c->fail(LBM_ETIMEOUT, "a bounded device wait of the step kernel timed out; the populations are invalid");
    }
    return LBM_OK;
}

// Planes (plus one per work item for the two halo planes it reads first)
// on the busiest block when `grid` persistent blocks take the work items
// (tile, chunk of z planes), numbered chunk-major, round-robin.
long long busiest_block_planes(long long nz, long long tiles, long long grid, long long zc) {
    if (grid < 1 || tiles < 1 || zc < 1) return 0;
    const long long chunks = (nz + zc - 1) / zc, last = nz - (chunks - 1) * zc;
    const long long items = tiles * chunks;
    std::vector<long long> in_last(grid, 0);  // items of the last (shorter) chunk per block
    for (long long i = (chunks - 1) * tiles; i < items; ++i) ++in_last[i % grid];
    long long worst = 0;
    for (long long b = 0; b < grid; ++b) {
        const long long n = items / grid + (b < items % grid ? 1 : 0);
        const long long load = n * (zc + 1) - (zc - last) * in_last[b];
        if (load > worst) worst = load;
    }
    return worst;
}

int auto_zchunk(const lbm_ctx* c) {
    const long long xy_blocks = (long long)((c->p.nx + 31) / 32) * ((c->p.ny + c->tile_y - 1) / c->tile_y);
    // Aim at ~4 blocks per SM in total so that the tail of the grid is short,
    // with chunks no shorter than 16 planes (each chunk re-reads 2 planes).
    const long long want_blocks = 4LL * c->num_sms;
    long long chunks = (want_blocks + xy_blocks - 1) / xy_blocks;
    if (chunks < 1) chunks = 1;
    long long zc = (c->p.nz + chunks - 1) / chunks;
    if (zc < 16) zc = 16;
    if (zc > c->p.nz) zc = c->p.nz;
    return int(zc);
}

// Why a launch shape (step kernel variant, tile height, z chunk; 0 = auto)
// cannot serve a lattice with these parameters, or nullptr if it can.  The
// checks that need a device (occupancy, tensor maps) come later.
const char* launch_shape_error(const lbm_params& p, int kernel, int tile_y, int zchunk) {
    if (p.G2 != 0.0 && ((p.storage != LBM_F64 && p.storage != LBM_F32) || (kernel != 0 && kernel != 6) ||
                        (tile_y != 0 && tile_y != 8 && tile_y != 16)))
        return "the two-belt force (G2 != 0) runs kernel 6 on 32x8 or 32x16 tiles with FP64/FP32 storage";
    if (p.G2 == 0.0 && kernel == 6) return "kernel 6 is the two-belt force kernel (needs G2 != 0)";
    if (p.storage >= LBM_F16_LOCAL && (kernel == 2 || (kernel >= 4 && kernel != 7)))
        return "local-reference storage runs kernel 1, 3 or 7";
    if (kernel == 7 && (p.storage < LBM_F16_DEV || p.nx % 2 != 0)) return "kernel 7 needs 16-bit storage and nx even";
    if (kernel < 0 || kernel > 7) return "kernel must be 0 .. 7";
    if (tile_y != 0 && tile_y != 4 && tile_y != 8 && tile_y != 16) return "tile_y must be 0, 4, 8 or 16";
    if (zchunk < 0) return "zchunk must be >= 0";
    return nullptr;
}

// Choose and prepare the step kernel of a context: variant `kernel`, tile
// height `tile_y`, z planes per work item `zchunk` (0 = automatic for each),
// and derive the persistent grid and work items.  Used by lbm_create and by
// lbm_set_kernel_config / lbm_tune; on an error the message goes to msg.
lbm_status configure_step(lbm_ctx* c, int kernel, int tile_y, int zchunk, char* msg, size_t msg_len) {
    const lbm_params* p = &c->p;
    const long long n = c->n;
    StepArgs& a = c->args;
    c->grid = 0;
    c->grid3 = 0;
    // Auto launch shape (measured on GB300 at 256x256x575, GLUPS): FP32 runs
    // the pipelined kernel on 32x16 tiles (SRT 32.4; MRT tau = 0.8 30.2
    // against 28.8 on 32x8 and 26.9 on 32x4); the global-reference 16-bit
    // formats run the paired kernel on 64x8 tiles (FP16 SRT 35.6 against 32.7
    // for kernel 3 on 32x4), the local-reference ones kernel 3 on 32x8 tiles
    // (33.2 against 31.1 on 32x4, 29.8 on 32x16, 29.2 paired, 22.9
    // register-staged); 16-bit storage with nx odd and FP64 run the
    // register-staged kernel on 32x4 tiles (FP64 is bound by its FP64 pipe).
    const bool pipe_default = p->storage == LBM_F32 || (p->storage >= LBM_F16_DEV && p->nx % 2 == 0);
    const bool pair_default = (p->storage == LBM_F16_DEV || p->storage == LBM_BF16_DEV) && p->nx % 2 == 0;
    const bool pipe = kernel == 3 || (kernel == 0 && pipe_default && !pair_default);
    const bool pair = kernel == 7 || (kernel == 0 && pair_default);
    const int auto_ty = (kernel == 5 || (pipe && p->storage <= LBM_F32)) ? 16 : ((pipe || pair) ? 8 : 4);
    c->tile_y = tile_y ? tile_y : auto_ty;
    if (p->G2 != 0.0) c->tile_y = tile_y ? tile_y : 8;  // the two-belt kernel
    if (kernel == 4 && (p->storage != LBM_F32 || p->nx % 4 != 0)) {
        snprintf(msg, msg_len, "kernel 4 needs FP32 storage and nx %% 4 == 0");
        return LBM_EINVAL;
    }
    if (kernel == 5 && (p->storage != LBM_F32 || c->tile_y < 8 || p->nx % 32 != 0 || p->ny % c->tile_y != 0)) {
        snprintf(msg, msg_len,
                 "kernel 5 needs FP32 storage, tile_y 8 or 16, nx %% 32 == 0 and ny %% tile_y == 0");
        return LBM_EINVAL;
    }
    if (kernel < 0 || kernel > 7) {
        snprintf(msg, msg_len, "kernel must be 0 .. 7");
        return LBM_EINVAL;
    }
    // kernels 3 and 7 address cells with 32-bit offsets within a population
    const bool off32 = n <= 0xffffffffLL;
    if (!off32 && (kernel == 3 || kernel == 7)) {
        snprintf(msg, msg_len, "kernel %d needs nx*ny*nz < 2^32", kernel);
        return LBM_EINVAL;
    }
    c->kernel = p->G2 != 0.0 ? 6 : 1;
    if (p->G2 == 0.0 && kernel != 1 && !(kernel == 0 && (!pipe_default || !off32))) {
        c->kernel = kernel == 0 ? (pair_default ? 7 : 3) : kernel;
        const int per_sm = prepare_async(c);
        if (per_sm > 0) {
            c->grid = per_sm * c->num_sms;
        } else if (kernel >= 2) {
            if (per_sm < 0)
                snprintf(msg, msg_len, "kernel %d cannot be configured: %s",
                         kernel, cudaGetErrorString(cudaError_t(-per_sm)));
            else
                snprintf(msg, msg_len,
                         "kernel %d needs FP64/FP32 storage (kernel 2 with FP64: tile_y <= 8; "
                         "kernel 3 also takes the 16-bit formats with nx even) and must fit on an SM",
                         kernel);
            return LBM_EINVAL;
        } else {
            c->kernel = 1;
        }
    }
    if (c->kernel == 5) {
        c->kernel = 3;
        const int per3 = prepare_async(c);
        c->kernel = 5;
        if (per3 < 1 || encode_tensor_maps(c) != LBM_OK) {
            snprintf(msg, msg_len, "%s",
                     c->err[0] ? c->err : "the pipelined kernel cannot be configured");
            return LBM_ECUDA;
        }
        c->grid3 = per3 * c->num_sms;
    }
    const int tile_w = c->kernel == 7 ? 64 : 32;  // kernel 7: two cells per thread along x
    const int tiles_x = (p->nx + tile_w - 1) / tile_w, tiles_y = (p->ny + c->tile_y - 1) / c->tile_y;
    if (zchunk) {
        c->zchunk = zchunk < p->nz ? zchunk : p->nz;
    } else if (c->kernel >= 2 && c->kernel != 6) {
        // The longest chunk first: the address range that all blocks touch
        // at once grows with the chunk length times the plane size, so at
        // most 24 MiB of one population's planes (16..96 planes), and 8
        // planes for planes of 1.5 MiB and more.  Measured on GB300, FP32 SRT
        // on 32x16 tiles (GLUPS for chunks of 16 / 32 / 64 planes):
        // 576^2 x 1536 30.1 / 29.8 / 28.4, 640^2 x 1437 30.3 / 26.6 / 25.2,
        // 672^2 x 1792 28.7 / 22.9 / 21.7 (6 / 8 / 12 planes: 27.7 / 28.7 /
        // 20.0).
        const long long plane_bytes = (long long)p->nx * p->ny * (long long)c->elem;
        long long zmax = (24LL << 20) / (plane_bytes > 0 ? plane_bytes : 1);
        zmax = zmax < 16 ? 16 : (zmax > 96 ? 96 : zmax);
        if (c->tile_y >= 16 && plane_bytes >= (3LL << 19)) zmax = 8;
        if (zmax > p->nz) zmax = p->nz;
        // Within that bound, the chunk that spreads the planes most evenly
        // over the persistent blocks, which take the work items round-robin:
        // the least planes on the busiest block (busiest_block_planes).  On
        // 256^2 x 575 (128 tiles of 32x16, 152 blocks) chunks of 32 / 44 / 72
        // planes put 527 / 499 / 510 planes on the busiest block and ran at
        // 32.15 / 33.87 / 33.47 GLUPS (MRT at tau = 0.8: 30.72 / 32.42 /
        // 31.84).
        const long long tiles = (long long)tiles_x * tiles_y;
        const long long zlo = zmax < 8 ? zmax : 8;
        long long zc = zmax, best = -1;
        for (long long z = zmax; z >= zlo; --z) {  // ties: the longer chunk
            const long long load = busiest_block_planes(p->nz, tiles, c->grid, z);
            if (best < 0 || load < best) {
                best = load;
                zc = z;
            }
        }
        c->zchunk = int(zc < p->nz ? zc : p->nz);
    } else {
        c->zchunk = auto_zchunk(c);
    }
    a.zchunk = c->zchunk;
    a.tiles_x = tiles_x;
    a.n_tiles = tiles_x * tiles_y;
    a.n_items = a.n_tiles * ((p->nz + c->zchunk - 1) / c->zchunk);
    if (c->kernel >= 2 && c->grid > a.n_items) c->grid = a.n_items;
    if (c->grid3 > a.n_items) c->grid3 = a.n_items;

    return LBM_OK;
}

}  // namespace

// ----------------------------------------------------------------------------
// Public API
// ----------------------------------------------------------------------------
extern "C" {

void lbm_params_default(lbm_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->lattice = LBM_D3Q19;
    p->nx = p->ny = p->nz = 32;
    p->G = -5.5;
    p->collision = LBM_SRT_SHIFT;
    p->tau = 1.0;
    p->psi = LBM_PSI_EXP;
    p->rho0 = 1.0;
    p->storage = LBM_F32;
    p->rho_ref = 1.0;
    p->dev_scale = 1.0;
}

const char* lbm_last_error(const lbm_ctx* ctx) { return ctx ? ctx->err : g_create_err; }

lbm_status lbm_velocities(int c[57], double w[19]) {
    for (int q = 0; q < Q; ++q) {
        if (c) {
            c[3 * q + 0] = cx(q);
            c[3 * q + 1] = cy(q);
            c[3 * q + 2] = cz(q);
        }
        if (w) w[q] = wq(q);
    }
    return LBM_OK;
}

static lbm_status create_fail(lbm_status s, const char* msg) {
    snprintf(g_create_err, sizeof(g_create_err), "%s", msg);
    return s;
}

lbm_status lbm_create(const lbm_params* p, lbm_ctx** out) {
    g_create_err[0] = 0;
    if (!out) return create_fail(LBM_EINVAL, "lbm_create: out is NULL");
    *out = nullptr;
    if (!p) return create_fail(LBM_EINVAL, "lbm_create: params is NULL");
    if (p->lattice != LBM_D3Q19) return create_fail(LBM_EINVAL, "lbm_create: only D3Q19 is provided");
    if (p->nx < 1 || p->ny < 1 || p->nz < 1) return create_fail(LBM_EINVAL, "lbm_create: box sizes must be >= 1");
    const long long n = (long long)p->nx * p->ny * p->nz;
    if (n > (1LL << 40)) return create_fail(LBM_EINVAL, "lbm_create: box too large");
    if (p->collision != LBM_SRT_SHIFT && p->collision != LBM_MRT_GUO)
        return create_fail(LBM_EINVAL, "lbm_create: unknown collision operator");
    if (!(p->tau > 0.5) || !std::isfinite(p->tau)) return create_fail(LBM_EINVAL, "lbm_create: tau must be > 0.5");
    if (!std::isfinite(p->G)) return create_fail(LBM_EINVAL, "lbm_create: G must be finite");
    if (!std::isfinite(p->G2)) return create_fail(LBM_EINVAL, "lbm_create: G2 must be finite");
    if (const char* why = launch_shape_error(*p, p->kernel, p->tile_y, p->zchunk)) {
        snprintf(g_create_err, sizeof(g_create_err), "lbm_create: %s", why);
        return LBM_EINVAL;
    }
    if (p->psi != LBM_PSI_EXP) return create_fail(LBM_EINVAL, "lbm_create: unknown psi law");
    if (!(p->rho0 > 0) || !std::isfinite(p->rho0)) return create_fail(LBM_EINVAL, "lbm_create: rho0 must be > 0");
    if (p->storage < LBM_F64 || p->storage > LBM_BF16_LOCAL) return create_fail(LBM_EINVAL, "lbm_create: unknown storage");
    if (p->storage >= LBM_F16_DEV && (!(p->dev_scale > 0) || !std::isfinite(p->rho_ref)))
        return create_fail(LBM_EINVAL, "lbm_create: deviation storage needs dev_scale > 0 and finite rho_ref");
    if (p->collision == LBM_MRT_GUO && p->has_rates) {
        for (int k = 0; k < Q; ++k)
            if (!(p->s[k] > 0.0 && p->s[k] < 2.0))
                return create_fail(LBM_EINVAL, "lbm_create: MRT rates must lie in (0, 2)");
    }
    if ((p->f_a == nullptr) != (p->f_b == nullptr))
        return create_fail(LBM_EINVAL, "lbm_create: give both f_a and f_b or neither");
    if (p->f_a && ((reinterpret_cast<uintptr_t>(p->f_a) | reinterpret_cast<uintptr_t>(p->f_b)) & 15))
        return create_fail(LBM_EINVAL, "lbm_create: f_a/f_b must be 16-byte aligned");

    lbm_ctx* c = new (std::nothrow) lbm_ctx();
    if (!c) return create_fail(LBM_ENOMEM, "lbm_create: host allocation failed");
    c->p = *p;
    c->stream = static_cast<cudaStream_t>(p->stream);
    c->n = n;
    c->elem = p->storage == LBM_F64 ? 8 : (p->storage == LBM_F32 ? 4 : 2);
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
    if (e != cudaSuccess) {
        snprintf(g_create_err, sizeof(g_create_err), "lbm_create: no usable CUDA device: %s", cudaGetErrorString(e));
        delete c;
        return LBM_ECUDA;
    }
    const size_t fbytes = (size_t)Q * (size_t)n * c->elem;
    if (p->f_a) {
        c->f[0] = p->f_a;
        c->f[1] = p->f_b;
    } else {
        c->own_f = true;
        e = cudaMalloc(&c->f[0], fbytes);
        if (e == cudaSuccess) e = cudaMalloc(&c->f[1], fbytes);
        if (e != cudaSuccess) {
            snprintf(g_create_err, sizeof(g_create_err), "lbm_create: population allocation of 2 x %zu bytes failed: %s",
                     fbytes, cudaGetErrorString(e));
            cudaFree(c->f[0]);
            delete c;
            return runtime_status(e);
        }
        c->own_bytes += 2 * (long long)fbytes;
        cudaMemsetAsync(c->f[0], 0, fbytes, c->stream);
        cudaMemsetAsync(c->f[1], 0, fbytes, c->stream);
    }
    if (p->storage >= LBM_F16_LOCAL) {
        // the two density fields are the library's own even with caller-owned populations
        const size_t rbytes = sizeof(float) * (size_t)n;
        e = cudaMalloc(&c->ref[0], rbytes);
        if (e == cudaSuccess) e = cudaMalloc(&c->ref[1], rbytes);
        if (e == cudaSuccess) e = cudaMemsetAsync(c->ref[0], 0, rbytes, c->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(c->ref[1], 0, rbytes, c->stream);
        if (e != cudaSuccess) {
            snprintf(g_create_err, sizeof(g_create_err), "lbm_create: density-field allocation failed: %s",
                     cudaGetErrorString(e));
            cudaFree(c->ref[0]);
            cudaFree(c->ref[1]);
            if (c->own_f) { cudaFree(c->f[0]); cudaFree(c->f[1]); }
            delete c;
            return runtime_status(e);
        }
        c->own_bytes += 2 * (long long)rbytes;
    }
    e = cudaMalloc(&c->diag, sizeof(double) * 8 * (size_t)p->nz);
    if (e != cudaSuccess) {
        snprintf(g_create_err, sizeof(g_create_err), "lbm_create: diagnostics allocation failed: %s", cudaGetErrorString(e));
        cudaFree(c->ref[0]);
        cudaFree(c->ref[1]);
        if (c->own_f) { cudaFree(c->f[0]); cudaFree(c->f[1]); }
        delete c;
        return runtime_status(e);
    }
    c->own_bytes += (long long)(sizeof(double) * 8 * (size_t)p->nz);
    c->diag_host.resize(8 * (size_t)p->nz);
    e = cudaMalloc(&c->dev_err, 256);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->dev_err, 0, 256, c->stream);
    if (e != cudaSuccess) {
        snprintf(g_create_err, sizeof(g_create_err), "lbm_create: error-word allocation failed: %s",
                 cudaGetErrorString(e));
        cudaFree(c->diag);
        cudaFree(c->ref[0]);
        cudaFree(c->ref[1]);
        if (c->own_f) { cudaFree(c->f[0]); cudaFree(c->f[1]); }
        delete c;
        return runtime_status(e);
    }
    c->own_bytes += 256;

    // Kernel arguments.
    StepArgs& a = c->args;
    a.nx = p->nx;
    a.ny = p->ny;
    a.nz = p->nz;
    a.n = n;
    a.G = p->G;
    a.G2 = p->G2;
    a.tau = p->tau;
    a.omega = 1.0 / p->tau;
    a.rho0 = p->rho0;
    a.inv_rho0 = 1.0 / p->rho0;
    for (int k = 0; k < Q; ++k) a.s[k] = 1.0;
    if (p->collision == LBM_MRT_GUO) {
        if (p->has_rates) {
            for (int k = 0; k < Q; ++k) a.s[k] = p->s[k];
        } else {  // Sec. 2 rule: e, 3pxx, pww, pxy, pyz, pxz at 1/tau, others 1
            const int rel[6] = {1, 9, 11, 13, 14, 15};
            for (int k : rel) a.s[k] = 1.0 / p->tau;
        }
    }
    round_params(a);
    c->coll = collision_kernel(*p, a.s);
    a.err = c->dev_err;
    a.test_stall = p->test_stall ? 1 : 0;
    a.dev = make_dev_params(p->rho_ref, p->dev_scale);
    {
        char why[400] = {0};
        if (lbm_status st = configure_step(c, p->kernel, p->tile_y, p->zchunk, why, sizeof(why)); st != LBM_OK) {
            snprintf(g_create_err, sizeof(g_create_err), "lbm_create: %s", why);
            lbm_destroy(c);
            return st;
        }
    }

    e = cudaGetLastError();
    if (e != cudaSuccess) {
        snprintf(g_create_err, sizeof(g_create_err), "lbm_create: %s", cudaGetErrorString(e));
        lbm_destroy(c);
        return LBM_ECUDA;
    }
    *out = c;
    return LBM_OK;
}

void lbm_destroy(lbm_ctx* c) {
    if (!c || c->batch) return;  // batch boxes are destroyed with their batch
    cudaStreamSynchronize(c->stream);
    if (c->own_f) {
        cudaFree(c->f[0]);
        cudaFree(c->f[1]);
    }
    cudaFree(c->ref[0]);
    cudaFree(c->ref[1]);
    cudaFree(c->scratch);
    cudaFree(c->diag);
    cudaFree(c->dev_err);
    cudaFree(c->adj.cp);
    cudaFree(c->adj.seg);
    cudaFree(c->adj.lam[0]);
    cudaFree(c->adj.lam[1]);
    cudaFree(c->adj.gr[0]);
    cudaFree(c->adj.gr[1]);
    cudaFree(c->adj.psi);
    cudaFree(c->adj.gF);
    cudaFree(c->adj.partials);
    cudaFree(c->adj.acc);
    cudaFree(c->adj.io);
    delete c;
}

lbm_status lbm_set_stream(lbm_ctx* c, void* stream) {
    if (!c) return LBM_EINVAL;
    if (c->batch) return c->fail(LBM_EINVAL, "lbm_set_stream: the boxes of a batch run on the batch's stream");
    // work already enqueued on the old stream finishes before the new one is used
    LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    c->stream = static_cast<cudaStream_t>(stream);
    return LBM_OK;
}

long lbm_time(const lbm_ctx* c) { return c ? c->t : -1; }

int lbm_current_copy(const lbm_ctx* c) { return c ? c->cur : -1; }

long long lbm_device_bytes(const lbm_ctx* c) { return c ? c->own_bytes : 0; }

lbm_status lbm_kernel_config(const lbm_ctx* c, int* kernel, int* tile_y, int* zchunk, int* grid) {
    if (!c) return LBM_EINVAL;
    if (kernel) *kernel = c->kernel;
    if (tile_y) *tile_y = c->tile_y;
    if (zchunk) *zchunk = c->zchunk;
    if (grid) {
        if (c->kernel >= 2 && c->kernel != 6) {
            *grid = c->grid;
        } else {
            const StepArgs& a = c->args;
            *grid = ((a.nx + 31) / 32) * ((a.ny + c->tile_y - 1) / c->tile_y) * ((a.nz + a.zchunk - 1) / a.zchunk);
        }
    }
    return LBM_OK;
}

long long lbm_params_sizeof(void) { return (long long)sizeof(lbm_params); }

lbm_status lbm_set_kernel_config(lbm_ctx* c, int kernel, int tile_y, int zchunk) {
    if (!c) return LBM_EINVAL;
    if (c->batch) return c->fail(LBM_EINVAL, "lbm_set_kernel_config: this context is a box of a batch");
    if (const char* why = launch_shape_error(c->p, kernel, tile_y, zchunk))
        return c->fail(LBM_EINVAL, "lbm_set_kernel_config: %s", why);
    const int k0 = c->kernel, t0 = c->tile_y, z0 = c->zchunk;
    char why[400] = {0};
    const lbm_status st = configure_step(c, kernel, tile_y, zchunk, why, sizeof(why));
    if (st != LBM_OK) {
        char ignored[400];
        configure_step(c, k0, t0, z0, ignored, sizeof(ignored));  // the previous shape worked
        return c->fail(st, "lbm_set_kernel_config: %s", why);
    }
    return LBM_OK;
}

lbm_status lbm_tune(lbm_ctx* c, int trial_steps, int* kernel, int* tile_y, int* zchunk, double* ms_per_step) {
    if (!c) return LBM_EINVAL;
    if (c->batch) return c->fail(LBM_EINVAL, "lbm_tune: this context is a box of a batch (use lbm_batch_tune)");
    if (trial_steps < 1) return c->fail(LBM_EINVAL, "lbm_tune: trial_steps must be >= 1");
    struct Shape {
        int kernel, tile_y, zchunk;
    };
    std::vector<Shape> shapes;
    const lbm_params& p = c->p;
    const bool b16 = p.storage >= LBM_F16_DEV, even = p.nx % 2 == 0;
    for (int ty : {4, 8, 16}) {
        if (p.G2 != 0.0) {
            if (ty >= 8) shapes.push_back({6, ty, 0});
            continue;
        }
        shapes.push_back({1, ty, 0});                                          // register-staged ring
        if (!b16) shapes.push_back({2, ty, 0});                                // every population through cp.async
        if (!b16 || even)
            for (int zc : {0, 8, 16, 32}) shapes.push_back({3, ty, zc});       // register prefetch, cp.async ring
        if (p.storage == LBM_F32 && ty >= 8) shapes.push_back({5, ty, 0});     // tensor-copy boxes
        if (b16 && even)
            for (int zc : {0, 16}) shapes.push_back({7, ty, zc});              // paired words
    }
    const int k0 = c->kernel, t0 = c->tile_y, z0 = c->zchunk;
    cudaEvent_t e0, e1;
    LBM_CUDA(c, cudaEventCreate(&e0));
    LBM_CUDA(c, cudaEventCreate(&e1));
    float best = -1.0f;
    Shape pick{k0, t0, z0};
    const int steps = trial_steps + (trial_steps & 1);  // even: the state ends in the current copy
    for (const Shape& sh : shapes) {
        if (launch_shape_error(p, sh.kernel, sh.tile_y, sh.zchunk)) continue;
        char why[400];
        if (configure_step(c, sh.kernel, sh.tile_y, sh.zchunk, why, sizeof(why)) != LBM_OK) continue;
        const int cur = c->cur;
        bool ok = launch_step(c, c->f[cur], c->f[cur ^ 1]) == cudaSuccess &&
                  launch_step(c, c->f[cur ^ 1], c->f[cur]) == cudaSuccess;  // warm-up
        if (!ok) continue;
        cudaEventRecord(e0, c->stream);
        for (int k = 0; k < steps && ok; ++k)
            ok = launch_step(c, c->f[cur ^ (k & 1)], c->f[cur ^ (~k & 1)]) == cudaSuccess;
        cudaEventRecord(e1, c->stream);
        if (!ok || cudaEventSynchronize(e1) != cudaSuccess) continue;
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= steps;
        if (best < 0.0f || ms < best) {
            best = ms;
            pick = sh;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaGetLastError();  // a shape that failed to launch is skipped, not an error
    char why[400] = {0};
    lbm_status st = configure_step(c, pick.kernel, pick.tile_y, pick.zchunk, why, sizeof(why));
    if (st != LBM_OK) {
        char ignored[400];
        configure_step(c, k0, t0, z0, ignored, sizeof(ignored));
        return c->fail(st, "lbm_tune: %s", why);
    }
    if (best < 0.0f) return c->fail(LBM_ECUDA, "lbm_tune: no launch shape ran");
    if (kernel) *kernel = c->kernel;
    if (tile_y) *tile_y = c->tile_y;
    if (zchunk) *zchunk = c->zchunk;
    if (ms_per_step) *ms_per_step = best;
    return LBM_OK;
}

lbm_status lbm_init_ligament(lbm_ctx* c, double R0, double eps, int n_waves, double width, double rho_l,
                             double rho_v) {
    if (!c) return LBM_EINVAL;
    if (!(R0 > 0) || !(width > 0) || !(rho_l > 0) || !(rho_v > 0) || !std::isfinite(eps) || n_waves < 0)
        return c->fail(LBM_EINVAL, "lbm_init_ligament: need R0 > 0, width > 0, rho_l, rho_v > 0, n_waves >= 0");
    const int blocks = grid_for(c->n, 256, c->num_sms);
    const auto& p = c->p;
    with_codec(c, [&](auto codec) {
        using C = decltype(codec);
        ligament_kernel<C><<<blocks, 256, 0, c->stream>>>(static_cast<typename C::S*>(c->f[c->cur]), p.nx, p.ny,
                                                          p.nz, R0, eps, n_waves, width, rho_l, rho_v, c->args.dev,
                                                          c->ref[c->cur]);
        return 0;
    });
    LBM_LAUNCHED(c, "ligament_kernel");
    c->t = 0;
    return LBM_OK;
}

lbm_status lbm_set_density(lbm_ctx* c, const double* rho, int on_device) {
    if (!c) return LBM_EINVAL;
    if (!rho) return c->fail(LBM_EINVAL, "lbm_set_density: rho is NULL");
    const double* d_rho = rho;
    if (!on_device) {
        lbm_status s = ensure_scratch(c, sizeof(double) * (size_t)c->n);
        if (s != LBM_OK) return s;
        LBM_CUDA(c, cudaMemcpyAsync(c->scratch, rho, sizeof(double) * (size_t)c->n, cudaMemcpyHostToDevice, c->stream));
        d_rho = c->scratch;
    }
    const int blocks = grid_for(c->n, 256, c->num_sms);
    with_codec(c, [&](auto codec) {
        using C = decltype(codec);
        rest_state_kernel<C><<<blocks, 256, 0, c->stream>>>(static_cast<typename C::S*>(c->f[c->cur]), d_rho, c->n,
                                                            c->args.dev, c->ref[c->cur]);
        return 0;
    });
    LBM_LAUNCHED(c, "rest_state_kernel");
    if (!on_device) LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    c->t = 0;
    return LBM_OK;
}

lbm_status lbm_set_populations(lbm_ctx* c, const double* f, int on_device) {
    if (!c) return LBM_EINVAL;
    if (!f) return c->fail(LBM_EINVAL, "lbm_set_populations: f is NULL");
    float* ref = c->ref[c->cur];
    const int blocks = grid_for(c->n, 256, c->num_sms);
    if (on_device) {
        if (ref) ref_sum_kernel<<<blocks, 256, 0, c->stream>>>(ref, nullptr, f, c->n, Q, 0);
        with_codec(c, [&](auto codec) {
            using C = decltype(codec);
            encode_kernel<C><<<grid_for((long long)Q * c->n, 256, c->num_sms), 256, 0, c->stream>>>(
                static_cast<typename C::S*>(c->f[c->cur]), f, (long long)Q * c->n, c->n, 0, c->args.dev, ref);
            return 0;
        });
        LBM_LAUNCHED(c, "encode_kernel");
    } else {
        // One population at a time through an n-double staging buffer (plus
        // an n-double accumulator of the reference densities for the
        // local-reference storage, which needs them before the first encode).
        lbm_status s = ensure_scratch(c, sizeof(double) * (size_t)c->n * (ref ? 2 : 1));
        if (s != LBM_OK) return s;
        if (ref) {
            for (int q = 0; q < Q; ++q) {
                LBM_CUDA(c, cudaMemcpyAsync(c->scratch, f + (size_t)q * c->n, sizeof(double) * (size_t)c->n,
                                            cudaMemcpyHostToDevice, c->stream));
                ref_sum_kernel<<<blocks, 256, 0, c->stream>>>(ref, c->scratch + c->n, c->scratch, c->n, q, 1);
            }
            ref_sum_kernel<<<blocks, 256, 0, c->stream>>>(ref, c->scratch + c->n, nullptr, c->n, Q, 2);
            LBM_LAUNCHED(c, "ref_sum_kernel");
        }
        for (int q = 0; q < Q; ++q) {
            LBM_CUDA(c, cudaMemcpyAsync(c->scratch, f + (size_t)q * c->n, sizeof(double) * (size_t)c->n,
                                        cudaMemcpyHostToDevice, c->stream));
            with_codec(c, [&](auto codec) {
                using C = decltype(codec);
                encode_kernel<C><<<blocks, 256, 0, c->stream>>>(
                    static_cast<typename C::S*>(c->f[c->cur]) + (size_t)q * c->n, c->scratch, c->n, c->n, q,
                    c->args.dev, ref);
                return 0;
            });
            LBM_LAUNCHED(c, "encode_kernel");
        }
        LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    }
    c->t = 0;
    return LBM_OK;
}

lbm_status lbm_get_populations(lbm_ctx* c, double* f, int on_device) {
    if (!c) return LBM_EINVAL;
    if (lbm_status st = check_device_error(c); st != LBM_OK) return st;
    if (!f) return c->fail(LBM_EINVAL, "lbm_get_populations: f is NULL");
    if (on_device) {
        with_codec(c, [&](auto codec) {
            using C = decltype(codec);
            decode_kernel<C><<<grid_for((long long)Q * c->n, 256, c->num_sms), 256, 0, c->stream>>>(
                f, static_cast<const typename C::S*>(c->f[c->cur]), (long long)Q * c->n, c->n, 0, c->args.dev,
                c->ref[c->cur]);
            return 0;
        });
        LBM_LAUNCHED(c, "decode_kernel");
        return LBM_OK;
    }
    lbm_status s = ensure_scratch(c, sizeof(double) * (size_t)c->n);
    if (s != LBM_OK) return s;
    const int blocks = grid_for(c->n, 256, c->num_sms);
    for (int q = 0; q < Q; ++q) {
        with_codec(c, [&](auto codec) {
            using C = decltype(codec);
            decode_kernel<C><<<blocks, 256, 0, c->stream>>>(
                c->scratch, static_cast<const typename C::S*>(c->f[c->cur]) + (size_t)q * c->n, c->n, c->n, q,
                c->args.dev, c->ref[c->cur]);
            return 0;
        });
        LBM_LAUNCHED(c, "decode_kernel");
        LBM_CUDA(c, cudaMemcpyAsync(f + (size_t)q * c->n, c->scratch, sizeof(double) * (size_t)c->n,
                                    cudaMemcpyDeviceToHost, c->stream));
        LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    }
    return LBM_OK;
}

lbm_status lbm_step(lbm_ctx* c, long nsteps) {
    if (!c) return LBM_EINVAL;
    if (nsteps < 0) return c->fail(LBM_EINVAL, "lbm_step: n must be >= 0");
    if (c->batch) return c->fail(LBM_EINVAL, "lbm_step: this context is a box of a batch; use lbm_batch_step");
    for (long k = 0; k < nsteps; ++k) {
        cudaError_t e = launch_step(c, c->f[c->cur], c->f[c->cur ^ 1]);
        if (e != cudaSuccess) return c->fail(LBM_ECUDA, "step kernel launch failed: %s", cudaGetErrorString(e));
        c->cur ^= 1;
        ++c->t;
    }
    return LBM_OK;
}

lbm_status lbm_moments(lbm_ctx* c, double* rho, double* ux, double* uy, double* uz, int on_device) {
    if (!c) return LBM_EINVAL;
    if (lbm_status st = check_device_error(c); st != LBM_OK) return st;
    const size_t nb = sizeof(double) * (size_t)c->n;
    double *d_rho, *d_ux, *d_uy, *d_uz;
    if (on_device) {
        lbm_status s = rho ? LBM_OK : ensure_scratch(c, nb);
        if (s != LBM_OK) return s;
        d_rho = rho ? rho : c->scratch;
        d_ux = ux;
        d_uy = uy;
        d_uz = uz;
    } else {
        // staging for the requested fields only (rho always: u needs it)
        const int nf = 1 + (ux ? 1 : 0) + (uy ? 1 : 0) + (uz ? 1 : 0);
        lbm_status s = ensure_scratch(c, nf * nb);
        if (s != LBM_OK) return s;
        double* next = c->scratch;
        d_rho = next;
        next += c->n;
        d_ux = ux ? next : nullptr;
        next += ux ? c->n : 0;
        d_uy = uy ? next : nullptr;
        next += uy ? c->n : 0;
        d_uz = uz ? next : nullptr;
    }
    const int blocks = grid_for(c->n, 256, c->num_sms);
    const auto& p = c->p;
    with_codec(c, [&](auto codec) {
        using C = decltype(codec);
        const auto* f = static_cast<const typename C::S*>(c->f[c->cur]);
        density_kernel<C><<<blocks, 256, 0, c->stream>>>(d_rho, f, c->n, c->args.dev, c->ref[c->cur]);
        if (d_ux || d_uy || d_uz)
            velocity_kernel<C><<<blocks, 256, 0, c->stream>>>(d_ux, d_uy, d_uz, d_rho, f, p.nx, p.ny, p.nz, p.G, p.G2,
                                                              p.rho0, c->args.dev, c->ref[c->cur]);
        return 0;
    });
    LBM_LAUNCHED(c, "moments kernels");
    if (!on_device) {
        if (rho) LBM_CUDA(c, cudaMemcpyAsync(rho, d_rho, nb, cudaMemcpyDeviceToHost, c->stream));
        if (ux) LBM_CUDA(c, cudaMemcpyAsync(ux, d_ux, nb, cudaMemcpyDeviceToHost, c->stream));
        if (uy) LBM_CUDA(c, cudaMemcpyAsync(uy, d_uy, nb, cudaMemcpyDeviceToHost, c->stream));
        if (uz) LBM_CUDA(c, cudaMemcpyAsync(uz, d_uz, nb, cudaMemcpyDeviceToHost, c->stream));
        LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    }
    return LBM_OK;
}

lbm_status lbm_diag(lbm_ctx* c, double rho_l, double rho_v, double* mass, double mom[3], double* area_z,
                    double* maxrho_z) {
    if (!c) return LBM_EINVAL;
    if (lbm_status st = check_device_error(c); st != LBM_OK) return st;
    if (!(rho_l > rho_v)) return c->fail(LBM_EINVAL, "lbm_diag: need rho_l > rho_v");
    const auto& p = c->p;
    with_codec(c, [&](auto codec) {
        using C = decltype(codec);
        diag_kernel<C><<<p.nz, DIAG_THREADS, 0, c->stream>>>(
            c->diag, static_cast<const typename C::S*>(c->f[c->cur]), p.nx, p.ny, c->n, rho_l, rho_v, c->args.dev,
            c->ref[c->cur]);
        return 0;
    });
    LBM_LAUNCHED(c, "diag_kernel");
    LBM_CUDA(c, cudaMemcpyAsync(c->diag_host.data(), c->diag, sizeof(double) * 8 * (size_t)p.nz,
                                cudaMemcpyDeviceToHost, c->stream));
    LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    double m = 0, jx = 0, jy = 0, jz = 0, bad = 0;
    for (int z = 0; z < p.nz; ++z) {
        const double* d = &c->diag_host[8 * (size_t)z];
        m += d[0];
        jx += d[1];
        jy += d[2];
        jz += d[3];
        bad += d[6];
        if (area_z) area_z[z] = d[4];
        if (maxrho_z) maxrho_z[z] = d[5];
    }
    if (mass) *mass = m;
    if (mom) {
        mom[0] = jx;
        mom[1] = jy;
        mom[2] = jz;
    }
    if (bad > 0 || !std::isfinite(m))
        return c->fail(LBM_ENONFINITE, "lbm_diag: %.0f cells with rho <= 0 or non-finite at step %ld", bad, c->t);
    return LBM_OK;
}

}  // extern "C"

// ----------------------------------------------------------------------------
// Batches of independent boxes
// ----------------------------------------------------------------------------
struct lbm_batch {
    lbm_params p;                     // shared parameters (box sizes per box)
    int count = 0;
    std::vector<lbm_ctx*> box;        // per-box views over the shared copies
    std::vector<long long> base;      // element offset of each box
    void* f[2] = {nullptr, nullptr};
    size_t bytes = 0;                 // per copy
    int cur = 0;
    long t = 0;
    long long cells = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int num_sms = 0;
    int tile_y = 8, zchunk = 32, grid = 0;
    BatchArgs bargs{};
    BatchBox* boxes_dev = nullptr;
    StepArgs phys{};
    cudaGraphExec_t graph[2] = {nullptr, nullptr};  // two-step cycle starting from copy 0 / 1
    char err[512] = {0};

    lbm_status fail(lbm_status s, const char* fmt, ...) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(err, sizeof(err), fmt, ap);
        va_end(ap);
        return s;
    }
};

namespace {

StepLaunch batch_launch(const lbm_batch* b) {
    StepLaunch l;
    l.args = b->phys;
    l.kernel = 3;
    l.tile_y = b->tile_y;
    l.grid = b->grid;
    l.coll = b->box[0]->coll;
    l.stream = b->stream;
    return l;
}

cudaError_t batch_launch_step(const lbm_batch* b, int from) {
    const StepLaunch l = batch_launch(b);
    return step_kernels(b->p.storage, l.coll).batch(l, b->bargs, b->f[from], b->f[from ^ 1]);
}

void batch_drop_graphs(lbm_batch* b) {
    for (auto& g : b->graph) {
        if (g) cudaGraphExecDestroy(g);
        g = nullptr;
    }
}

// (Re)build the work-item table for tile height ty and chunk zc, upload it and
// size the persistent grid.
lbm_status batch_configure(lbm_batch* b, int ty, int zc) {
    const StepLaunch probe = [&] {
        StepLaunch l = batch_launch(b);
        l.tile_y = ty;
        return l;
    }();
    const int per_sm = step_kernels(b->p.storage, probe.coll).batch_prepare(probe);
    if (per_sm < 1)
        return b->fail(LBM_ECUDA, "batch kernel cannot be resident (tile_y %d): %s", ty,
                       per_sm < 0 ? cudaGetErrorString(cudaError_t(-per_sm)) : "no block fits on an SM");
    std::vector<BatchBox> boxes(b->count);
    int items = 0;
    for (int i = 0; i < b->count; ++i) {
        const lbm_params& q = b->box[i]->p;
        BatchBox& bx = boxes[i];
        bx.nx = q.nx;
        bx.ny = q.ny;
        bx.nz = q.nz;
        bx.tiles_x = (q.nx + 31) / 32;
        bx.n_tiles = bx.tiles_x * ((q.ny + ty - 1) / ty);
        bx.zchunk = zc < q.nz ? zc : q.nz;
        bx.item_begin = items;
        bx.base = b->base[i];
        bx.n = (long long)q.nx * q.ny * q.nz;
        items += bx.n_tiles * ((q.nz + bx.zchunk - 1) / bx.zchunk);
    }
    LBM_CUDA(b, cudaMemcpyAsync(b->boxes_dev, boxes.data(), sizeof(BatchBox) * b->count, cudaMemcpyHostToDevice,
                                b->stream));
    LBM_CUDA(b, cudaStreamSynchronize(b->stream));
    b->tile_y = ty;
    b->zchunk = zc;
    b->bargs.nbox = b->count;
    b->bargs.n_items = items;
    b->bargs.boxes = b->boxes_dev;
    b->grid = per_sm * b->num_sms < items ? per_sm * b->num_sms : items;
    batch_drop_graphs(b);
    return LBM_OK;
}

lbm_status batch_build_graph(lbm_batch* b, int from) {
    cudaGraph_t g = nullptr;
    LBM_CUDA(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e1 = batch_launch_step(b, from);
    cudaError_t e2 = batch_launch_step(b, from ^ 1);
    cudaError_t e3 = cudaStreamEndCapture(b->stream, &g);
    if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return b->fail(LBM_ECUDA, "capturing the batch step graph failed: %s",
                       cudaGetErrorString(e1 != cudaSuccess ? e1 : (e2 != cudaSuccess ? e2 : e3)));
    }
    cudaError_t e = cudaGraphInstantiate(&b->graph[from], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return b->fail(LBM_ECUDA, "cudaGraphInstantiate failed: %s", cudaGetErrorString(e));
    return LBM_OK;
}

}  // namespace

extern "C" {

lbm_status lbm_batch_create(const lbm_params* p, int count, const int* dims, lbm_batch** out) {
    g_create_err[0] = 0;
    if (!out) return create_fail(LBM_EINVAL, "lbm_batch_create: out is NULL");
    *out = nullptr;
    if (!p || !dims || count < 1) return create_fail(LBM_EINVAL, "lbm_batch_create: need params, dims and count >= 1");
    if (p->storage != LBM_F32 && p->storage != LBM_F64)
        return create_fail(LBM_EINVAL, "lbm_batch_create: batches support FP32 and FP64 storage");
    if (p->G2 != 0.0) return create_fail(LBM_EINVAL, "lbm_batch_create: batches use the single-belt force (G2 = 0)");
    if (p->f_a || p->f_b) return create_fail(LBM_EINVAL, "lbm_batch_create: the batch allocates its own copies");
    lbm_batch* b = new (std::nothrow) lbm_batch();
    if (!b) return create_fail(LBM_ENOMEM, "lbm_batch_create: host allocation failed");
    b->p = *p;
    b->count = count;
    const size_t elem = p->storage == LBM_F64 ? 8 : 4;
    b->base.resize(count);
    long long off = 0;
    for (int i = 0; i < count; ++i) {
        const int nx = dims[3 * i], ny = dims[3 * i + 1], nz = dims[3 * i + 2];
        if (nx < 1 || ny < 1 || nz < 1) {
            delete b;
            return create_fail(LBM_EINVAL, "lbm_batch_create: box sizes must be >= 1");
        }
        const long long n = (long long)nx * ny * nz;
        if ((long long)Q * n >= (1LL << 31)) {
            delete b;
            return create_fail(LBM_EINVAL, "lbm_batch_create: a box needs 19 * cells < 2^31");
        }
        b->base[i] = off;
        b->cells += n;
        // keep every box's copy 256-byte aligned
        const long long per = (long long)Q * n;
        const long long align = 256 / (long long)elem;
        off += (per + align - 1) / align * align;
    }
    b->bytes = (size_t)off * elem;
    cudaError_t e = cudaSuccess;
    int dev = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) {
        if (p->stream) {
            b->stream = static_cast<cudaStream_t>(p->stream);
        } else {  // graph capture needs a stream other than the legacy default
            e = cudaStreamCreate(&b->stream);
            b->own_stream = (e == cudaSuccess);
        }
    }
    if (e == cudaSuccess) e = cudaMalloc(&b->f[0], b->bytes);
    if (e == cudaSuccess) e = cudaMalloc(&b->f[1], b->bytes);
    if (e == cudaSuccess) e = cudaMalloc(&b->boxes_dev, sizeof(BatchBox) * count);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->f[0], 0, b->bytes, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->f[1], 0, b->bytes, b->stream);
    if (e != cudaSuccess) {
        snprintf(g_create_err, sizeof(g_create_err), "lbm_batch_create: %s", cudaGetErrorString(e));
        lbm_batch_destroy(b);
        return runtime_status(e);
    }
    b->box.assign(count, nullptr);
    for (int i = 0; i < count; ++i) {
        lbm_params q = *p;
        q.nx = dims[3 * i];
        q.ny = dims[3 * i + 1];
        q.nz = dims[3 * i + 2];
        q.stream = b->stream;
        q.f_a = static_cast<char*>(b->f[0]) + (size_t)b->base[i] * elem;
        q.f_b = static_cast<char*>(b->f[1]) + (size_t)b->base[i] * elem;
        q.kernel = 1;
        q.zchunk = 0;
        q.tile_y = 0;
        lbm_ctx* c = nullptr;
        lbm_status st = lbm_create(&q, &c);
        if (st != LBM_OK) {
            lbm_batch_destroy(b);
            return st;  // g_create_err holds the box's message
        }
        c->batch = b;
        b->box[i] = c;
    }
    b->phys = b->box[0]->args;
    const int ty = p->tile_y ? p->tile_y : (p->collision == LBM_MRT_GUO ? 4 : 8);
    const int zc = p->zchunk ? p->zchunk : 32;
    lbm_status st = batch_configure(b, ty, zc);
    if (st != LBM_OK) {
        snprintf(g_create_err, sizeof(g_create_err), "%s", b->err);
        lbm_batch_destroy(b);
        return st;
    }
    *out = b;
    return LBM_OK;
}

void lbm_batch_destroy(lbm_batch* b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    batch_drop_graphs(b);
    for (lbm_ctx* c : b->box) {
        if (c) {
            c->batch = nullptr;
            lbm_destroy(c);
        }
    }
    cudaFree(b->f[0]);
    cudaFree(b->f[1]);
    cudaFree(b->boxes_dev);
    if (b->own_stream) cudaStreamDestroy(b->stream);
    delete b;
}

const char* lbm_batch_last_error(const lbm_batch* b) { return b ? b->err : g_create_err; }

lbm_status lbm_batch_box(lbm_batch* b, int i, lbm_ctx** view) {
    if (!b || !view) return LBM_EINVAL;
    if (i < 0 || i >= b->count) return b->fail(LBM_EINVAL, "lbm_batch_box: index %d out of range", i);
    *view = b->box[i];
    return LBM_OK;
}

lbm_status lbm_batch_step(lbm_batch* b, long n) {
    if (!b) return LBM_EINVAL;
    if (n < 0) return b->fail(LBM_EINVAL, "lbm_batch_step: n must be >= 0");
    while (n >= 2) {
        if (!b->graph[b->cur]) {
            lbm_status st = batch_build_graph(b, b->cur);
            if (st != LBM_OK) return st;
        }
        LBM_CUDA(b, cudaGraphLaunch(b->graph[b->cur], b->stream));
        n -= 2;
        b->t += 2;
        for (lbm_ctx* c : b->box) c->t += 2;
    }
    if (n == 1) {
        cudaError_t e = batch_launch_step(b, b->cur);
        if (e != cudaSuccess) return b->fail(LBM_ECUDA, "batch step launch failed: %s", cudaGetErrorString(e));
        b->cur ^= 1;
        ++b->t;
        for (lbm_ctx* c : b->box) {
            c->cur ^= 1;
            ++c->t;
        }
    }
    return LBM_OK;
}

lbm_status lbm_batch_tune(lbm_batch* b, int trial_steps, int* tile_y, int* zchunk, double* ms_per_step) {
    if (!b) return LBM_EINVAL;
    if (trial_steps < 1) return b->fail(LBM_EINVAL, "lbm_batch_tune: trial_steps must be >= 1");
    const int tys[3] = {4, 8, 16};
    const int zcs[6] = {8, 16, 24, 32, 48, 64};
    cudaEvent_t e0, e1;
    LBM_CUDA(b, cudaEventCreate(&e0));
    LBM_CUDA(b, cudaEventCreate(&e1));
    float best = -1.0f;
    int best_ty = b->tile_y, best_zc = b->zchunk;
    for (int ty : tys) {
        for (int zc : zcs) {
            if (batch_configure(b, ty, zc) != LBM_OK) continue;
            if (batch_launch_step(b, 0) != cudaSuccess) continue;  // warm-up
            cudaEventRecord(e0, b->stream);
            for (int k = 0; k < trial_steps; ++k) batch_launch_step(b, k & 1);
            cudaEventRecord(e1, b->stream);
            if (cudaEventSynchronize(e1) != cudaSuccess) continue;
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            ms /= trial_steps;
            if (best < 0.0f || ms < best) {
                best = ms;
                best_ty = ty;
                best_zc = zc;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return b->fail(LBM_ECUDA, "lbm_batch_tune: %s", cudaGetErrorString(e));
    lbm_status st = batch_configure(b, best_ty, best_zc);
    if (st != LBM_OK) return st;
    if (tile_y) *tile_y = best_ty;
    if (zchunk) *zchunk = best_zc;
    if (ms_per_step) *ms_per_step = best;
    return best < 0.0f ? b->fail(LBM_ECUDA, "lbm_batch_tune: no launch shape ran") : LBM_OK;
}

lbm_status lbm_batch_config(const lbm_batch* b, int* tile_y, int* zchunk, int* grid, long long* cells) {
    if (!b) return LBM_EINVAL;
    if (tile_y) *tile_y = b->tile_y;
    if (zchunk) *zchunk = b->zchunk;
    if (grid) *grid = b->grid;
    if (cells) *cells = b->cells;
    return LBM_OK;
}

}  // extern "C"

// ----------------------------------------------------------------------------
// Discrete adjoint (SRT)
// ----------------------------------------------------------------------------
namespace {

AdjointArgs adjoint_args(const lbm_ctx* c) {
    AdjointArgs a;
    a.nx = c->p.nx;
    a.ny = c->p.ny;
    a.nz = c->p.nz;
    a.n = c->n;
    a.G = c->p.G;
    a.tau = c->p.tau;
    a.omega = 1.0 / c->p.tau;
    a.rho0 = c->p.rho0;
    a.Gf = float(a.G);
    a.tauf = float(a.tau);
    a.omegaf = float(a.omega);
    a.rho0f = float(a.rho0);
    const long long rows = (long long)c->p.ny * c->p.nz;
    const long long want = (rows + adjoint_rows_per_block() - 1) / adjoint_rows_per_block();
    const long long cap = 8LL * c->num_sms;
    a.grid = int(want < cap ? (want < 1 ? 1 : want) : cap);
    return a;
}

lbm_status adj_alloc(lbm_ctx* c, void** p, size_t bytes) {
    if (*p) return LBM_OK;
    LBM_CUDA(c, cudaMalloc(p, bytes));
    c->own_bytes += (long long)bytes;
    return LBM_OK;
}

}  // namespace

extern "C" {

lbm_status lbm_adjoint_forward(lbm_ctx* c, const double* rho0, int on_device, long nsteps, int every) {
    if (!c) return LBM_EINVAL;
    if (c->batch) return c->fail(LBM_EINVAL, "lbm_adjoint_forward: not available on a batch box");
    if (c->p.collision != LBM_SRT_SHIFT)
        return c->fail(LBM_EUNSUPPORTED, "lbm_adjoint_forward: the adjoint covers the SRT operator only");
    if (c->p.storage != LBM_F32 && c->p.storage != LBM_F64)
        return c->fail(LBM_EUNSUPPORTED, "lbm_adjoint_forward: FP32 or FP64 storage only");
    if (c->p.G2 != 0.0)
        return c->fail(LBM_EUNSUPPORTED, "lbm_adjoint_forward: the adjoint covers the single-belt force only");
    if (!rho0 || nsteps < 1 || every < 1) return c->fail(LBM_EINVAL, "lbm_adjoint_forward: need rho0, n >= 1, every >= 1");
    if (c->n > 0xffffffffLL) return c->fail(LBM_EUNSUPPORTED, "lbm_adjoint_forward: needs nx*ny*nz < 2^32");
    auto& A = c->adj;
    const size_t state = (size_t)Q * (size_t)c->n * c->elem;
    const int ncp = int((nsteps + every - 1) / every);
    if (A.cp && (A.cp_bytes < (size_t)ncp * state)) {
        cudaStreamSynchronize(c->stream);
        cudaFree(A.cp);
        c->own_bytes -= (long long)A.cp_bytes;
        A.cp = nullptr;
    }
    if (A.seg && (A.seg_bytes < (size_t)every * state)) {
        cudaStreamSynchronize(c->stream);
        cudaFree(A.seg);
        c->own_bytes -= (long long)A.seg_bytes;
        A.seg = nullptr;
    }
    if (!A.cp) {
        lbm_status st = adj_alloc(c, &A.cp, (size_t)ncp * state);
        if (st != LBM_OK) return st;
        A.cp_bytes = (size_t)ncp * state;
    }
    if (!A.seg) {
        lbm_status st = adj_alloc(c, &A.seg, (size_t)every * state);
        if (st != LBM_OK) return st;
        A.seg_bytes = (size_t)every * state;
    }
    lbm_status st = lbm_set_density(c, rho0, on_device);
    if (st != LBM_OK) return st;
    for (long t = 0; t < nsteps; ++t) {
        if (t % every == 0)
            LBM_CUDA(c, cudaMemcpyAsync(static_cast<char*>(A.cp) + (size_t)(t / every) * state, c->f[c->cur], state,
                                        cudaMemcpyDeviceToDevice, c->stream));
        st = lbm_step(c, 1);
        if (st != LBM_OK) return st;
    }
    A.T = nsteps;
    A.every = every;
    A.ncp = ncp;
    return LBM_OK;
}

lbm_status lbm_adjoint_backward(lbm_ctx* c, const double* dJdrho, int in_on_device, double* dJdrho0,
                                int out_on_device, double* dJdG, double* dJdtau) {
    if (!c) return LBM_EINVAL;
    auto& A = c->adj;
    if (A.T < 1) return c->fail(LBM_EINVAL, "lbm_adjoint_backward: call lbm_adjoint_forward first");
    if (!dJdrho) return c->fail(LBM_EINVAL, "lbm_adjoint_backward: dJdrho is NULL");
    const bool f64 = c->p.storage == LBM_F64;
    const size_t state = (size_t)Q * (size_t)c->n * c->elem;
    const AdjointArgs a = adjoint_args(c);
    lbm_status st;
    for (void** p : {&A.lam[0], &A.lam[1]}) {
        st = adj_alloc(c, p, state);
        if (st != LBM_OK) return st;
    }
    for (void** p : {&A.gr[0], &A.gr[1]}) {
        st = adj_alloc(c, p, (size_t)c->n * c->elem);
        if (st != LBM_OK) return st;
    }
    // psi of every state of a segment: written by the step kernel during the
    // recomputation where it supports that (kernels 1 and 3, and 5 whose
    // recomputation runs kernel 3), else computed by the reverse step
    const bool psi_fused = c->kernel == 1 || c->kernel == 3 || c->kernel == 5;
    const size_t psi_bytes = (size_t)c->n * c->elem;
    if (A.psi && A.psi_bytes < (size_t)A.every * psi_bytes) {
        cudaStreamSynchronize(c->stream);
        cudaFree(A.psi);
        c->own_bytes -= (long long)A.psi_bytes;
        A.psi = nullptr;
    }
    if (!A.psi) {
        if ((st = adj_alloc(c, &A.psi, (size_t)A.every * psi_bytes)) != LBM_OK) return st;
        A.psi_bytes = (size_t)A.every * psi_bytes;
    }
    if ((st = adj_alloc(c, &A.gF, 4 * (size_t)c->n * c->elem)) != LBM_OK) return st;
    if ((st = adj_alloc(c, reinterpret_cast<void**>(&A.partials), sizeof(double) * 2 * (size_t)a.grid)) != LBM_OK)
        return st;
    if ((st = adj_alloc(c, reinterpret_cast<void**>(&A.acc), sizeof(double) * 2)) != LBM_OK) return st;
    if ((!in_on_device || (dJdrho0 && !out_on_device)) &&
        (st = adj_alloc(c, reinterpret_cast<void**>(&A.io), sizeof(double) * (size_t)c->n)) != LBM_OK)
        return st;
    const double* g = dJdrho;
    if (!in_on_device) {
        LBM_CUDA(c, cudaMemcpyAsync(A.io, dJdrho, sizeof(double) * (size_t)c->n, cudaMemcpyHostToDevice, c->stream));
        g = A.io;
    }
    LBM_CUDA(c, cudaMemsetAsync(A.acc, 0, 2 * sizeof(double), c->stream));
    LBM_CUDA(c, cudaMemsetAsync(A.partials, 0, sizeof(double) * 2 * (size_t)a.grid, c->stream));
    LBM_CUDA(c, adjoint_seed(a, f64, g, A.lam[0], A.gr[0], c->stream));
    int cur = 0;  // lam[cur] holds dJ/df(t+1)
    for (int k = A.ncp - 1; k >= 0; --k) {
        const long t0 = (long)k * A.every;
        const long t1 = t0 + A.every < A.T ? t0 + A.every : A.T;
        // recompute the segment's states from its checkpoint
        char* seg = static_cast<char*>(A.seg);
        LBM_CUDA(c, cudaMemcpyAsync(seg, static_cast<char*>(A.cp) + (size_t)k * state, state,
                                    cudaMemcpyDeviceToDevice, c->stream));
        char* psi = static_cast<char*>(A.psi);
        for (long t = t0; t + 1 < t1; ++t) {
            cudaError_t e = launch_step(c, seg + (size_t)(t - t0) * state, seg + (size_t)(t - t0 + 1) * state,
                                        psi_fused ? psi + (size_t)(t - t0) * psi_bytes : nullptr);
            if (e != cudaSuccess) return c->fail(LBM_ECUDA, "adjoint recompute: %s", cudaGetErrorString(e));
        }
        for (long t = t1 - 1; t >= t0; --t) {
            // the segment's last state has no recomputed step after it
            const bool ready = psi_fused && t + 1 < t1;
            cudaError_t e = adjoint_step(a, f64, seg + (size_t)(t - t0) * state, psi + (size_t)(t - t0) * psi_bytes,
                                         ready, A.lam[cur], A.gr[cur], A.lam[cur ^ 1], A.gr[cur ^ 1], A.gF,
                                         A.partials, A.acc, c->stream);
            if (e != cudaSuccess) return c->fail(LBM_ECUDA, "adjoint step: %s", cudaGetErrorString(e));
            cur ^= 1;
        }
    }
    LBM_CUDA(c, adjoint_reduce(a, A.partials, A.acc, c->stream));
    if (dJdrho0) {
        double* out = out_on_device ? dJdrho0 : A.io;
        LBM_CUDA(c, adjoint_rho0(a, f64, A.lam[cur], A.gr[cur], out, c->stream));
        if (!out_on_device)
            LBM_CUDA(c, cudaMemcpyAsync(dJdrho0, A.io, sizeof(double) * (size_t)c->n, cudaMemcpyDeviceToHost, c->stream));
    }
    double acc[2] = {0.0, 0.0};
    LBM_CUDA(c, cudaMemcpyAsync(acc, A.acc, sizeof(acc), cudaMemcpyDeviceToHost, c->stream));
    LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    if (dJdG) *dJdG = acc[0];
    if (dJdtau) *dJdtau = acc[1];
    return LBM_OK;
}

// ----------------------------------------------------------------------------
// Checkpoint / resume (lbm_save, lbm_load)
// ----------------------------------------------------------------------------
// File layout (little-endian, as both supported hosts are): a 256-byte header
// (CkptHeader, zero padded), the stored populations of the current copy
// exactly as the device holds them (19 * n elements of the storage type), the
// float reference-density field for the local-reference formats, then a
// 64-bit checksum of everything before it: FNV-1a over 64-bit little-endian
// words (the offset basis and prime of 64-bit FNV-1a), the byte tail folded
// in one byte at a time.
struct CkptHeader {
    char magic[8];         // "LBMSCKP\0"
    uint32_t version;      // 1
    uint32_t header_bytes; // 256
    int32_t nx, ny, nz, storage, collision, pad0;
    int64_t t;
    double G, tau, rho0, rho_ref, dev_scale;
    double s[Q];
    uint64_t pop_bytes, ref_bytes;
};
static_assert(sizeof(CkptHeader) <= 256, "checkpoint header must fit in 256 bytes");

struct Fnv64 {
    uint64_t h = 0xcbf29ce484222325ULL;
    unsigned char tail[8];
    int ntail = 0;
    void word(uint64_t w) { h = (h ^ w) * 0x100000001b3ULL; }
    void add(const void* p, size_t len) {
        const unsigned char* b = static_cast<const unsigned char*>(p);
        while (len && ntail) {  // complete a pending word first
            tail[ntail++] = *b++;
            --len;
            if (ntail == 8) {
                uint64_t w;
                memcpy(&w, tail, 8);
                word(w);
                ntail = 0;
            }
        }
        for (; len >= 8; len -= 8, b += 8) {
            uint64_t w;
            memcpy(&w, b, 8);
            word(w);
        }
        while (len--) tail[ntail++] = *b++;
    }
    uint64_t finish() {
        for (int k = 0; k < ntail; ++k) h = (h ^ tail[k]) * 0x100000001b3ULL;
        ntail = 0;
        return h;
    }
};

static const size_t kCkptChunk = size_t(32) << 20;  // bytes per host staging buffer

// Device -> file through two pinned staging buffers (the copy of one chunk
// overlaps the write of the previous one).
static lbm_status ckpt_write_device(lbm_ctx* c, FILE* fp, const void* dev, size_t bytes, Fnv64& fnv,
                                    unsigned char* const (&buf)[2], cudaEvent_t const (&ev)[2]) {
    const char* src = static_cast<const char*>(dev);
    size_t issued = 0, written = 0;
    size_t len[2] = {0, 0};
    int k = 0;
    auto issue = [&](int slot) -> cudaError_t {
        len[slot] = bytes - issued < kCkptChunk ? bytes - issued : kCkptChunk;
        cudaError_t e = cudaMemcpyAsync(buf[slot], src + issued, len[slot], cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaEventRecord(ev[slot], c->stream);
        issued += len[slot];
        return e;
    };
    if (bytes) LBM_CUDA(c, issue(0));
    while (written < bytes) {
        if (issued < bytes) LBM_CUDA(c, issue(k ^ 1));
        LBM_CUDA(c, cudaEventSynchronize(ev[k]));
        fnv.add(buf[k], len[k]);
        if (fwrite(buf[k], 1, len[k], fp) != len[k]) return c->fail(LBM_EIO, "lbm_save: write failed");
        written += len[k];
        k ^= 1;
    }
    return LBM_OK;
}

// File -> device (into `dev`) through the pinned staging buffers.
static lbm_status ckpt_read_device(lbm_ctx* c, FILE* fp, void* dev, size_t bytes, Fnv64& fnv,
                                   unsigned char* const (&buf)[2], cudaEvent_t const (&ev)[2], const char* path) {
    char* dst = static_cast<char*>(dev);
    size_t done = 0;
    int k = 0;
    while (done < bytes) {
        const size_t len = bytes - done < kCkptChunk ? bytes - done : kCkptChunk;
        // the copy out of buf[k] (from this call or the previous one) has
        // finished; an event never recorded completes at once
        LBM_CUDA(c, cudaEventSynchronize(ev[k]));
        if (fread(buf[k], 1, len, fp) != len) return c->fail(LBM_EIO, "lbm_load: %s is truncated", path);
        fnv.add(buf[k], len);
        LBM_CUDA(c, cudaMemcpyAsync(dst + done, buf[k], len, cudaMemcpyHostToDevice, c->stream));
        LBM_CUDA(c, cudaEventRecord(ev[k], c->stream));
        done += len;
        k ^= 1;
    }
    return LBM_OK;
}

// Pinned staging buffers and their events for one save or load.
struct CkptStaging {
    unsigned char* buf[2] = {nullptr, nullptr};
    cudaEvent_t ev[2] = {nullptr, nullptr};
    ~CkptStaging() {
        for (int k = 0; k < 2; ++k) {
            if (ev[k]) cudaEventSynchronize(ev[k]);
            if (buf[k]) cudaFreeHost(buf[k]);
            if (ev[k]) cudaEventDestroy(ev[k]);
        }
    }
    cudaError_t init() {
        for (int k = 0; k < 2; ++k) {
            cudaError_t e = cudaMallocHost(reinterpret_cast<void**>(&buf[k]), kCkptChunk);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev[k], cudaEventDisableTiming);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
};

static void ckpt_fill_header(const lbm_ctx* c, CkptHeader& h) {
    memset(&h, 0, sizeof(h));
    memcpy(h.magic, "LBMSCKP", 8);
    h.version = 1;
    h.header_bytes = 256;
    h.nx = c->p.nx;
    h.ny = c->p.ny;
    h.nz = c->p.nz;
    h.storage = c->p.storage;
    h.collision = c->p.collision;
    h.t = c->t;
    h.G = c->p.G;
    h.tau = c->p.tau;
    h.rho0 = c->p.rho0;
    h.rho_ref = c->p.rho_ref;
    h.dev_scale = c->p.dev_scale;
    for (int k = 0; k < Q; ++k) h.s[k] = c->args.s[k];
    h.pop_bytes = (uint64_t)Q * (uint64_t)c->n * c->elem;
    h.ref_bytes = c->ref[0] ? sizeof(float) * (uint64_t)c->n : 0;
}

lbm_status lbm_save(lbm_ctx* c, const char* path) {
    if (!c) return LBM_EINVAL;
    if (!path || !path[0]) return c->fail(LBM_EINVAL, "lbm_save: empty path");
    if (c->batch) return c->fail(LBM_EINVAL, "lbm_save: this context is a box of a batch");
    if (lbm_status st = check_device_error(c); st != LBM_OK) return st;
    CkptStaging stg;
    LBM_CUDA(c, stg.init());
    unsigned char head[256] = {0};
    CkptHeader h;
    ckpt_fill_header(c, h);
    memcpy(head, &h, sizeof(h));
    // write to path.tmp and rename over path once complete, so an interrupted
    // save never replaces a good checkpoint with a partial one
    std::vector<char> tmp(strlen(path) + 5);
    snprintf(tmp.data(), tmp.size(), "%s.tmp", path);
    FILE* fp = fopen(tmp.data(), "wb");
    if (!fp) return c->fail(LBM_EIO, "lbm_save: cannot open %s for writing", tmp.data());
    Fnv64 fnv;
    fnv.add(head, sizeof(head));
    lbm_status st = fwrite(head, 1, sizeof(head), fp) == sizeof(head)
                        ? LBM_OK
                        : c->fail(LBM_EIO, "lbm_save: write failed");
    if (st == LBM_OK) st = ckpt_write_device(c, fp, c->f[c->cur], h.pop_bytes, fnv, stg.buf, stg.ev);
    if (st == LBM_OK && h.ref_bytes) st = ckpt_write_device(c, fp, c->ref[c->cur], h.ref_bytes, fnv, stg.buf, stg.ev);
    if (st == LBM_OK) {
        const uint64_t sum = fnv.finish();
        if (fwrite(&sum, 1, 8, fp) != 8) st = c->fail(LBM_EIO, "lbm_save: write failed");
    }
    if (fclose(fp) != 0 && st == LBM_OK) st = c->fail(LBM_EIO, "lbm_save: close failed");
    if (st == LBM_OK && rename(tmp.data(), path) != 0) st = c->fail(LBM_EIO, "lbm_save: cannot rename to %s", path);
    if (st != LBM_OK) remove(tmp.data());
    return st;
}

lbm_status lbm_load(lbm_ctx* c, const char* path) {
    if (!c) return LBM_EINVAL;
    if (!path || !path[0]) return c->fail(LBM_EINVAL, "lbm_load: empty path");
    if (c->batch) return c->fail(LBM_EINVAL, "lbm_load: this context is a box of a batch");
    if (lbm_status st = check_device_error(c); st != LBM_OK) return st;
    FILE* fp = fopen(path, "rb");
    if (!fp) return c->fail(LBM_EIO, "lbm_load: cannot open %s", path);
    struct Closer {
        FILE* f;
        ~Closer() { fclose(f); }
    } closer{fp};
    unsigned char head[256];
    if (fread(head, 1, sizeof(head), fp) != sizeof(head)) return c->fail(LBM_EIO, "lbm_load: %s is truncated", path);
    CkptHeader h;
    memcpy(&h, head, sizeof(h));
    if (memcmp(h.magic, "LBMSCKP", 8) != 0 || h.version != 1 || h.header_bytes != 256)
        return c->fail(LBM_EIO, "lbm_load: %s is not a version-1 checkpoint", path);
    CkptHeader mine;
    ckpt_fill_header(c, mine);
    if (h.nx != mine.nx || h.ny != mine.ny || h.nz != mine.nz || h.storage != mine.storage)
        return c->fail(LBM_EINVAL, "lbm_load: %s holds a %dx%dx%d box with storage %d; the context is %dx%dx%d, %d",
                       path, h.nx, h.ny, h.nz, h.storage, mine.nx, mine.ny, mine.nz, mine.storage);
    if (h.storage >= LBM_F16_DEV && (h.dev_scale != mine.dev_scale ||
                                     (h.storage < LBM_F16_LOCAL && h.rho_ref != mine.rho_ref)))
        return c->fail(LBM_EINVAL, "lbm_load: %s was written with another rho_ref / dev_scale", path);
    // the physics of the run: a state evolved under other parameters is not
    // the state of this context (a resumed run must equal an uninterrupted one)
    bool same_rates = true;
    for (int k = 0; k < Q; ++k) same_rates = same_rates && h.s[k] == mine.s[k];
    if (h.collision != mine.collision || h.G != mine.G || h.tau != mine.tau || h.rho0 != mine.rho0 || !same_rates)
        return c->fail(LBM_EINVAL,
                       "lbm_load: %s was written with other physics (collision %d, G %.17g, tau %.17g, rho0 %.17g%s); "
                       "the context has collision %d, G %.17g, tau %.17g, rho0 %.17g",
                       path, h.collision, h.G, h.tau, h.rho0, same_rates ? "" : ", other MRT rates", mine.collision,
                       mine.G, mine.tau, mine.rho0);
    if (h.pop_bytes != mine.pop_bytes || h.ref_bytes != mine.ref_bytes || h.t < 0)
        return c->fail(LBM_EIO, "lbm_load: %s has an inconsistent header", path);
    CkptStaging stg;
    LBM_CUDA(c, stg.init());
    // read into the other copy (the next step overwrites it anyway) and make
    // it current only once the checksum matches
    const int nxt = c->cur ^ 1;
    Fnv64 fnv;
    fnv.add(head, sizeof(head));
    lbm_status st = ckpt_read_device(c, fp, c->f[nxt], h.pop_bytes, fnv, stg.buf, stg.ev, path);
    if (st == LBM_OK && h.ref_bytes) st = ckpt_read_device(c, fp, c->ref[nxt], h.ref_bytes, fnv, stg.buf, stg.ev, path);
    if (st != LBM_OK) return st;
    uint64_t sum = 0;
    if (fread(&sum, 1, 8, fp) != 8) return c->fail(LBM_EIO, "lbm_load: %s is truncated", path);
    LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    if (sum != fnv.finish()) return c->fail(LBM_EIO, "lbm_load: checksum mismatch in %s", path);
    if (fgetc(fp) != EOF) return c->fail(LBM_EIO, "lbm_load: trailing bytes in %s", path);
    c->cur = nxt;
    c->t = (long)h.t;
    return LBM_OK;
}

lbm_status lbm_checkpoint_info(const char* path, int verify, int dims[3], int* storage, int* collision, long* t,
                               double* G, double* tau) {
    g_create_err[0] = 0;
    if (!path || !path[0]) return create_fail(LBM_EINVAL, "lbm_checkpoint_info: empty path");
    FILE* fp = fopen(path, "rb");
    if (!fp) return create_fail(LBM_EIO, "lbm_checkpoint_info: cannot open the file");
    struct Closer {
        FILE* f;
        ~Closer() { fclose(f); }
    } closer{fp};
    unsigned char head[256];
    if (fread(head, 1, sizeof(head), fp) != sizeof(head))
        return create_fail(LBM_EIO, "lbm_checkpoint_info: truncated header");
    CkptHeader h;
    memcpy(&h, head, sizeof(h));
    if (memcmp(h.magic, "LBMSCKP", 8) != 0 || h.version != 1 || h.header_bytes != 256)
        return create_fail(LBM_EIO, "lbm_checkpoint_info: not a version-1 checkpoint");
    const uint64_t n = (uint64_t)(h.nx > 0 ? h.nx : 0) * (uint64_t)(h.ny > 0 ? h.ny : 0) * (uint64_t)(h.nz > 0 ? h.nz : 0);
    const uint64_t elem = h.storage == LBM_F64 ? 8 : (h.storage == LBM_F32 ? 4 : 2);
    const bool local = h.storage >= LBM_F16_LOCAL;
    if (n == 0 || h.storage < LBM_F64 || h.storage > LBM_BF16_LOCAL || h.t < 0 ||
        h.pop_bytes != (uint64_t)Q * n * elem || h.ref_bytes != (local ? sizeof(float) * n : 0))
        return create_fail(LBM_EIO, "lbm_checkpoint_info: inconsistent header");
    if (verify) {
        Fnv64 fnv;
        fnv.add(head, sizeof(head));
        std::vector<unsigned char> buf(size_t(1) << 20);
        uint64_t left = h.pop_bytes + h.ref_bytes;
        while (left) {
            const size_t len = left < buf.size() ? (size_t)left : buf.size();
            if (fread(buf.data(), 1, len, fp) != len) return create_fail(LBM_EIO, "lbm_checkpoint_info: truncated file");
            fnv.add(buf.data(), len);
            left -= len;
        }
        uint64_t sum = 0;
        if (fread(&sum, 1, 8, fp) != 8) return create_fail(LBM_EIO, "lbm_checkpoint_info: truncated file");
        if (sum != fnv.finish()) return create_fail(LBM_EIO, "lbm_checkpoint_info: checksum mismatch");
        if (fgetc(fp) != EOF) return create_fail(LBM_EIO, "lbm_checkpoint_info: trailing bytes");
    }
    if (dims) {
        dims[0] = h.nx;
        dims[1] = h.ny;
        dims[2] = h.nz;
    }
    if (storage) *storage = h.storage;
    if (collision) *collision = h.collision;
    if (t) *t = (long)h.t;
    if (G) *G = h.G;
    if (tau) *tau = h.tau;
    return LBM_OK;
}

}  // extern "C"
