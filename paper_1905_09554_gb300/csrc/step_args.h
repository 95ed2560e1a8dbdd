// Arguments of the step kernels and the launch description shared between
// the host API (lbm_sc.cu) and the per-storage kernel translation units
// (step_f64.cu, step_f32.cu, step_f16.cu, step_bf16.cu).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include "codec.cuh"
#include "lattice.cuh"

namespace lbm {

// Collision kernels: SRT; MRT with general rates; MRT whose rates outside
// {e, 3pxx, pww, pxy, pyz, pxz} are 1; MRT with every rate 1; MRT whose
// rates outside {3pxx, pww, pxy, pyz, pxz} are 1 (the shear rule).
enum { COLL_SRT = 0, COLL_MRT = 1, COLL_MRT_SPARSE = 2, COLL_MRT_UNIT = 3, COLL_MRT_SHEAR = 4, COLL_COUNT = 5 };

struct StepArgs {
    int nx, ny, nz;
    int zchunk;           // planes per block (work item) along z
    int tiles_x, n_tiles; // xy tiles of the persistent kernel
    int n_items;          // n_tiles * number of z chunks
    long long n;          // cells = nx*ny*nz (population stride)
    double G;             // interaction strength G0 (first belt)
    double G2;            // second-belt strength of the two-belt force (kernel 6)
    double tau, omega;    // SRT relaxation time and 1/tau
    double rho0, inv_rho0;
    double s[Q];          // MRT rates, moment order
    // The same parameters rounded to float once on the host, for the float
    // arithmetic of the 32- and 16-bit formats: a double-to-float conversion
    // inside the cell loop would occupy the FP64 pipe (2 lanes per SM clock).
    float Gf, tauf, omegaf, rho0f, inv_rho0f;
    float sf[Q];
    DevParams dev;
    int* err;             // device error word (bit 0: a bounded wait timed out)
    const float* ref_src; // local-reference storage: density field of the source copy
    float* ref_dst;       // ... and of the destination copy
    int test_stall;       // failure test of the bounded waits (bulk kernel)
    // Optional (kernels 1 and 3): psi of the input state, one value per cell
    // in the arithmetic type (the adjoint's recomputation keeps it for the
    // reverse step); nullptr normally.
    void* psi_out;
};

// MRT rates in the arithmetic type R (see par() in lattice.cuh).
template <class R>
__host__ __device__ __forceinline__ const R (&rates(const StepArgs& a))[Q] {
    if constexpr (sizeof(R) == sizeof(double)) return a.s;
    else return a.sf;
}
// Fill the float copies from the double fields.
inline void round_params(StepArgs& a) {
    a.Gf = float(a.G);
    a.tauf = float(a.tau);
    a.omegaf = float(a.omega);
    a.rho0f = float(a.rho0);
    a.inv_rho0f = float(a.inv_rho0);
    for (int k = 0; k < Q; ++k) a.sf[k] = float(a.s[k]);
}

// One box of a batch: geometry, work items and where its populations start
// (element offset) in the batch's population copies.
struct BatchBox {
    int nx, ny, nz;
    int tiles_x, n_tiles, zchunk;
    int item_begin;       // first work item of the box (items are box-major)
    long long base;       // element offset of the box's 19 population fields
    long long n;          // cells of the box (population stride)
};

struct BatchArgs {
    int nbox;
    int n_items;
    const BatchBox* boxes;  // device array of nbox entries
};

// Launch description of one step.
struct StepLaunch {
    StepArgs args;
    int kernel;           // 1 register-staged, 2 cp.async-staged, 3 pipelined,
                          // 4 bulk-copy, 5 tensor-copy, 6 two-belt force
    const CUtensorMap* tmap;  // kernel 5: tensor map of the source copy
    int tile_y;           // 4, 8 or 16 (tile width is 32)
    int grid;             // persistent grid (kernels 2 and 3)
    int coll;             // COLL_SRT .. COLL_MRT_SHEAR
    cudaStream_t stream;
};

// Kernel entry points of one (storage, collision) pair, defined in
// step_<storage>_<collision>.cu.  launch enqueues one step src -> dst;
// prepare opts kernels 2/3 in to their shared memory and returns their
// resident blocks per SM (0 = cannot run); batch / batch_prepare do the same
// for the batched step (FP64/FP32 only).
struct StepKernels {
    cudaError_t (*launch)(const StepLaunch& l, const void* src, void* dst);
    int (*prepare)(const StepLaunch& l);
    cudaError_t (*batch)(const StepLaunch& l, const BatchArgs& b, const void* src, void* dst);
    int (*batch_prepare)(const StepLaunch& l);
};

// storage: LBM_F64 .. LBM_BF16_LOCAL (0..5); coll: COLL_SRT .. COLL_MRT_SHEAR.
const StepKernels& step_kernels(int storage, int coll);

}  // namespace lbm
