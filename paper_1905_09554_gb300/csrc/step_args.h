// Arguments of the step kernels and the launch description shared between
// the host API (lbm_sc.cu) and the per-storage kernel translation units
// (step_f64.cu, step_f32.cu, step_f16.cu, step_bf16.cu).
#pragma once
#include <cuda_runtime.h>

#include "codec.cuh"
#include "lattice.cuh"

namespace lbm {

enum { COLL_SRT = 0, COLL_MRT = 1 };

struct StepArgs {
    int nx, ny, nz;
    int zchunk;           // planes per block (work item) along z
    int tiles_x, n_tiles; // xy tiles of the persistent kernel
    int n_items;          // n_tiles * number of z chunks
    long long n;          // cells = nx*ny*nz (population stride)
    double G;             // interaction strength G0
    double tau, omega;    // SRT relaxation time and 1/tau
    double rho0, inv_rho0;
    double s[Q];          // MRT rates, moment order
    DevParams dev;
};

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
    int kernel;           // 1 register-staged, 2 cp.async-staged, 3 pipelined
    int tile_y;           // 4, 8 or 16 (tile width is 32)
    int grid;             // persistent grid (kernels 2 and 3)
    bool idx32;           // 32-bit element offsets (pipelined kernel)
    int coll;             // COLL_SRT or COLL_MRT
    cudaStream_t stream;
};

// Per storage type (defined in step_<type>.cu).  launch_step_* enqueues one
// step src -> dst; prepare_step_* opts kernels 2/3 in to their shared memory
// and returns their resident blocks per SM (0 = the variant cannot run).
cudaError_t launch_step_f64(const StepLaunch& l, const void* src, void* dst);
cudaError_t launch_step_f32(const StepLaunch& l, const void* src, void* dst);
cudaError_t launch_step_f16(const StepLaunch& l, const void* src, void* dst);
cudaError_t launch_step_bf16(const StepLaunch& l, const void* src, void* dst);
int prepare_step_f64(const StepLaunch& l);
int prepare_step_f32(const StepLaunch& l);
int prepare_step_f16(const StepLaunch& l);
int prepare_step_bf16(const StepLaunch& l);

// Batched step (pipelined kernel over many boxes; FP32 and FP64 storage).
cudaError_t launch_batch_step_f64(const StepLaunch& l, const BatchArgs& b, const void* src, void* dst);
cudaError_t launch_batch_step_f32(const StepLaunch& l, const BatchArgs& b, const void* src, void* dst);
int prepare_batch_step_f64(const StepLaunch& l);
int prepare_batch_step_f32(const StepLaunch& l);

}  // namespace lbm
