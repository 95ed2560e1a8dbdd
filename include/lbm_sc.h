/*
 * lbm_sc.h -- C ABI of the D3Q19 pseudo-potential (Shan-Chen) lattice
 * Boltzmann step for one NVIDIA GB300 (sm_103a).
 *
 * Method: Chiappini, Xue, Falcucci, Sbragaglia, "Hydrodynamic behavior of the
 * Pseudo-Potential lattice Boltzmann method for interfacial flows"
 * (arXiv:1905.09554), Sec. 2 (Eqs. LBE, local_eq, momentum, SC_force,
 * vel_shift, barycentric) and the ligament set-up of Sec. 3.
 *
 * Conventions shared by every call
 * --------------------------------
 *  - A field is nx*ny*nz values, x fastest: cell (x, y, z) sits at
 *    index (z*ny + y)*nx + x.  Populations are 19 such fields, population a
 *    at offset a*nx*ny*nz, in the order returned by lbm_velocities().
 *  - The box is periodic in all three directions.
 *  - The state at time t holds the post-streaming, pre-collision populations
 *    f_a(x, t).  One step = Shan-Chen force, collision, streaming.
 *  - Every call returns an lbm_status; none aborts or exits.  On failure the
 *    context keeps a message (lbm_last_error).
 *  - Pointers marked "host or device" are read/written on the host when
 *    `on_device` is 0 and dereferenced by kernels when it is 1 (then they must
 *    be device memory of the context's GPU, 8-byte aligned).  The caller owns
 *    every array it passes; the library keeps no pointer to it after return.
 *  - All work is ordered on the context's CUDA stream.  Calls that return
 *    data to host memory synchronise that stream before returning; calls
 *    that only enqueue work (lbm_step, device-side set/get) do not.
 *  - A context is not thread-safe: one host thread at a time.
 */
#ifndef LBM_SC_H
#define LBM_SC_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx;

typedef enum {
    LBM_OK = 0,
    LBM_EINVAL = 1,        /* bad argument or parameter                      */
    LBM_ENOMEM = 2,        /* device allocation failed                        */
    LBM_ECUDA = 3,         /* a CUDA call or launch failed                    */
    LBM_ENONFINITE = 4,    /* the diagnostics found rho <= 0, NaN or Inf      */
    LBM_ETIMEOUT = 5,      /* a bounded device wait gave up                   */
    LBM_EIO = 6,           /* file read/write or checksum failure             */
    LBM_EUNSUPPORTED = 7   /* valid request this build does not provide       */
} lbm_status;

enum { LBM_D3Q19 = 0 };                        /* the only lattice (Sec. 2)   */
enum { LBM_SRT_SHIFT = 0,                      /* SRT, velocity shift, Eq. vel_shift */
       LBM_MRT_GUO = 1 };                      /* MRT, Guo-like forcing, Eq. barycentric */
enum { LBM_PSI_EXP = 0 };                      /* psi = rho0 (1 - exp(-rho/rho0)), Sec. 2 */
enum { LBM_F64 = 0,                            /* populations stored as double      */
       LBM_F32 = 1,                            /* stored as float, float arithmetic */
       LBM_F16_DEV = 2,                        /* half  deviations, float arithmetic */
       LBM_BF16_DEV = 3,                       /* bf16 deviations, float arithmetic  */
       LBM_F16_LOCAL = 4,                      /* half  deviations from a per-cell
                                                  reference density, float arithmetic */
       LBM_BF16_LOCAL = 5 };                   /* bf16 deviations from a per-cell
                                                  reference density, float arithmetic */

typedef struct {
    int lattice;          /* LBM_D3Q19                                              */
    int nx, ny, nz;       /* periodic box, each >= 1                                */
    double G;             /* interaction strength G0 of Eq. SC_force (< 0 attracts) */
    int collision;        /* LBM_SRT_SHIFT or LBM_MRT_GUO                           */
    double tau;           /* SRT relaxation time (> 0.5); MRT: shear rate = 1/tau   */
    int has_rates;        /* MRT only: 1 = use s[] below, 0 = Sec. 2 rule           */
    double s[19];         /* MRT rates in d'Humieres moment order (0-based):
                             rho e eps jx qx jy qy jz qz 3pxx 3pixx pww piww pxy
                             pyz pxz mx my mz.  Sec. 2 rule: e, 3pxx, pww, pxy,
                             pyz, pxz relax at 1/tau, the rest at 1.              */
    int psi;              /* LBM_PSI_EXP                                            */
    double rho0;          /* reference density of psi (the paper fixes 1.0)        */
    int storage;          /* LBM_F64 / LBM_F32 / LBM_F16_DEV / LBM_BF16_DEV /
                             LBM_F16_LOCAL / LBM_BF16_LOCAL                          */
    double rho_ref;       /* deviation storage: f_a = w_a rho_ref + d_a / dev_scale,
                             in float arithmetic with w_a rho_ref rounded to float
                             once per velocity (decode: fma(d_a, 1/dev_scale,
                             w_a rho_ref); encode: (f_a - w_a rho_ref) * dev_scale
                             rounded to nearest).
                             Local-reference storage ignores it: there rho_ref is
                             a float field R(x) the library allocates (2 x 4 bytes
                             per cell beside the populations), set from each cell's
                             density whenever the populations are set or
                             initialised, and by every step to the density of the
                             cell before the step (so f(t+1) is stored relative to
                             rho(t), which differs from rho(t+1) by O(|div j|)).
                             Local-reference storage runs step kernel 1, 3 or 7 and
                             is not accepted by batches, the adjoint or
                             lbm_diag_noalloc.                                        */
    double dev_scale;     /* deviation storage scale (> 0)                          */
    void *stream;         /* cudaStream_t for all work; NULL = legacy default       */
    void *f_a, *f_b;      /* optional caller-owned device buffers for the two
                             population copies (each 19*nx*ny*nz elements of the
                             storage type, 16-byte aligned); NULL = the library
                             allocates (and frees them in lbm_destroy).            */
    int zchunk;           /* step kernel: z planes per work item; 0 = auto (at most
                             32, and at most 24 MiB of one population's planes
                             on 32x16 tiles; 8 when one population's plane is
                             1.5 MiB or more)                                       */
    int tile_y;           /* step kernel: tile height (4, 8 or 16); 0 = auto: 16
                             for FP32 SRT and unit-rate MRT, 8 for other FP32
                             MRT and for kernel 7, 4 otherwise                      */
    int kernel;           /* step kernel variant: 0 = auto (3 for FP32 and the
                             local-reference formats, 7 for the global-reference
                             16-bit formats, when nx is even for 16-bit storage;
                             else 1),
                             1 = register-staged,
                             2 = cp.async-staged persistent, 3 = pipelined
                             persistent (2: FP64/FP32 storage; 3: also the
                             16-bit formats when nx is even),
                             4 = warp-specialised bulk-copy (FP32, nx % 4 == 0),
                             5 = tensor-copy pipeline (FP32, tile_y 8 or 16,
                             nx % 32 == 0, ny % tile_y == 0; steps on buffers
                             other than the two copies, e.g. the adjoint's
                             recomputation, run kernel 3),
                             6 = two-belt force (chosen when G2 != 0),
                             7 = paired 16-bit pipeline: two cells per thread
                             along x, 64-cell tile rows, shifted pushes as
                             aligned 32-bit words through warp shuffles (16-bit
                             formats, nx even; the auto choice for the
                             global-reference ones).  Kernels 3 and 7 need
                             nx*ny*nz < 2^32 (auto then falls back to 1).    */
    int test_stall;       /* test only: with kernel 4 the copy warp issues nothing,
                             so every bounded wait times out (about 1 s) and the
                             next lbm_diag / lbm_moments / lbm_get_populations
                             returns LBM_ETIMEOUT.  0 in normal use.               */
    double G2;            /* second belt of the two-belt (multirange) force that
                             Sec. 2 names (0 = Eq. SC_force alone):
                             F = -psi(x) [G sum_{D3Q19} w_a psi(x + c_a) c_a
                               + G2 sum_{E8} (p_b / 3) psi(x + e_b) e_b],
                             E8 = the 92 vectors with components in {-2..2} and
                             |e|^2 in {1,2,3,4,5,6,8}, p per shell 4/45, 1/21,
                             2/105, 5/504, 1/315, 1/630, 1/5040 (isotropic to 8th
                             order).  Bulk EoS P = rho cs2 + cs2 (G + G2) psi^2/2;
                             the split of G + G2 sets the surface tension.  Runs
                             kernel 6 (register-staged, two-cell psi halo, 32x8
                             tiles, or 32x16 when tile_y = 16) with FP64/FP32
                             storage; not available to batches or the adjoint.     */
} lbm_params;

/* Fill *p with defaults: D3Q19, 32^3, G = -5.5, SRT tau = 1, psi exp, rho0 = 1,
 * FP32 storage, rho_ref = 1, dev_scale = 1, default stream. */
void lbm_params_default(lbm_params *p);

/* Create a context on the current CUDA device.  Validates *p, allocates the
 * population copies (unless given) and small diagnostic buffers, and leaves the
 * populations zero.  On failure *out is NULL and lbm_last_error(NULL) returns
 * the message. */
lbm_status lbm_create(const lbm_params *p, lbm_ctx **out);

/* Free everything the context allocated; NULL-safe. */
void lbm_destroy(lbm_ctx *ctx);

/* Message of the last failure on ctx (or of the last failed lbm_create on
 * this thread when ctx is NULL); "" if none.  Owned by the library. */
const char *lbm_last_error(const lbm_ctx *ctx);

/* The library's velocity order: c[3*a + i] is component i (x, y, z) of
 * velocity a, w[a] its weight (D3Q19, Sec. 2).  Either pointer may be NULL. */
lbm_status lbm_velocities(int c[57], double w[19]);

/* Perturbed-ligament initial state (Sec. 3): a liquid cylinder along z
 * through ((nx-1)/2, (ny-1)/2) with surface radius
 * R(z) = R0 (1 + eps cos(2 pi n_waves z / nz)) and density
 * rho = rho_v + (rho_l - rho_v)/2 (1 - tanh((r - R(z)) / width)); velocity
 * zero, so f_a = w_a rho.  Resets the step counter. */
lbm_status lbm_init_ligament(lbm_ctx *ctx, double R0, double eps, int n_waves,
                             double width, double rho_l, double rho_v);

/* State at rest with the given density field (host or device, float64,
 * nx*ny*nz): f_a = w_a rho.  Resets the step counter. */
lbm_status lbm_set_density(lbm_ctx *ctx, const double *rho, int on_device);

/* Set / read all populations as float64 (host or device, 19*nx*ny*nz, library
 * velocity order).  Storage conversion happens on the device. */
lbm_status lbm_set_populations(lbm_ctx *ctx, const double *f, int on_device);
lbm_status lbm_get_populations(lbm_ctx *ctx, double *f, int on_device);

/* Advance n >= 0 time steps (Eq. LBE): Shan-Chen force (Eq. SC_force with the
 * psi law, plus the second belt when G2 != 0), SRT with the shifted equilibrium velocity u' = u + tau F / rho
 * (Eq. vel_shift) or MRT with Guo-like forcing at u_b = u + F/(2 rho)
 * (Eq. barycentric), then periodic streaming.  Enqueues n kernel launches. */
lbm_status lbm_step(lbm_ctx *ctx, long n);

/* Steps taken since the last initialisation. */
long lbm_time(const lbm_ctx *ctx);

/* Which of the two population copies holds the current state: 0 for f_a,
 * 1 for f_b of lbm_params (or the first / second copy the context allocated
 * itself); -1 for a NULL context.  Lets a caller that owns the copies read
 * the stored populations directly (e.g. for lbm_diag_noalloc). */
int lbm_current_copy(const lbm_ctx *ctx);

/* Macroscopic fields of the current state (Eq. momentum): rho and the
 * barycentric velocity u_b = (sum_a c_a f_a + F/2) / rho (Eq. barycentric),
 * reported for both operators (F includes the second belt when G2 != 0).
 * Each output (host or device, float64, nx*ny*nz) may be NULL to skip it. */
lbm_status lbm_moments(lbm_ctx *ctx, double *rho, double *ux, double *uy,
                       double *uz, int on_device);

/* Ligament diagnostics of the current state, accumulated in float64 on the
 * device, one thread block per z slice, deterministic:
 *   mass     = sum rho                          (host, 1 value)
 *   mom      = sum_a c_a f_a over the box        (host, 3 values)
 *   area_z   = sum_xy clamp((rho - rho_v)/(rho_l - rho_v), 0, 1) per slice
 *   maxrho_z = max_xy rho per slice              (host, nz values each)
 * area_z/maxrho_z may be NULL.  rho_l/rho_v define the liquid fraction used
 * for the neck radius R(z) = sqrt(area_z / pi) (Sec. 4).  Returns
 * LBM_ENONFINITE if any cell has rho <= 0, NaN or Inf. */
lbm_status lbm_diag(lbm_ctx *ctx, double rho_l, double rho_v, double *mass,
                    double mom[3], double *area_z, double *maxrho_z);

/* Select the CUDA stream (cudaStream_t, NULL = legacy default) for later
 * calls.  The previous stream is synchronised first, so work enqueued on it
 * is complete before the new stream sees the buffers.  LBM_EINVAL for a box
 * of a batch (it runs on the batch's stream). */
lbm_status lbm_set_stream(lbm_ctx *ctx, void *stream);

/* Checkpoint / resume.  lbm_save writes the current state (the stored
 * populations exactly as held on the device, the reference-density field of
 * the local-reference formats, the step count t and the parameters) to
 * `path` (written to path.tmp, then renamed, so an interrupted save leaves
 * an existing file intact).  lbm_load restores a state saved from a context
 * with the same box, storage (and, for the deviation formats, the same
 * rho_ref / dev_scale) and physics (collision operator, G, tau, rho0 and the
 * MRT rates, compared bit for bit): stepping on from the loaded state gives
 * bit-identical results to never having stopped.  The second-belt strength
 * G2 is not recorded in the file and not checked.  File layout: a
 * 256-byte header, the populations, the reference field, a 64-bit FNV-1a
 * checksum over 64-bit words of everything before it.  Both synchronise the
 * context's stream; both stage through 2 x 32 MiB of pinned host memory
 * allocated for the call.
 * Returns LBM_EIO if the file cannot be opened, written or read, is
 * truncated, has trailing bytes or fails the checksum (the context's state is
 * then unchanged: the file is read into the spare copy and made current only
 * after the checksum matches), LBM_EINVAL for a box, storage or physics
 * mismatch (state unchanged), a batch box, or an empty path. */
lbm_status lbm_save(lbm_ctx *ctx, const char *path);
lbm_status lbm_load(lbm_ctx *ctx, const char *path);

/* Header of a checkpoint written by lbm_save, read on the host alone (no
 * context, no CUDA call): dims = (nx, ny, nz), storage (lbm_storage),
 * collision (lbm_collision), the step count t, G and tau.  With verify != 0
 * the whole file is read and its checksum checked as lbm_load does.  Any
 * output pointer may be NULL.  Returns LBM_EINVAL for a NULL or empty path,
 * LBM_EIO if the file cannot be read, is not a version-1 checkpoint, has an
 * inconsistent header, or (verify) is truncated, has trailing bytes or fails
 * the checksum; the message is then in lbm_last_error(NULL). */
lbm_status lbm_checkpoint_info(const char *path, int verify, int dims[3],
                               int *storage, int *collision, long *t,
                               double *G, double *tau);

/* Bytes of device memory the context allocated itself. */
long long lbm_device_bytes(const lbm_ctx *ctx);

/* Launch configuration the context chose for the step kernel: variant
 * (1 register-staged, 2 cp.async-staged, 3 pipelined, 4 bulk-copy, 5 tensor
 * copy, 6 two-belt force, 7 paired 16-bit), tile height, z planes per work
 * item and grid size
 * (blocks).  Any pointer may be NULL. */
lbm_status lbm_kernel_config(const lbm_ctx *ctx, int *kernel, int *tile_y,
                             int *zchunk, int *grid);

/* sizeof(lbm_params) in this build, so that bindings can check their layout. */
long long lbm_params_sizeof(void);

/* Change the step kernel's launch shape: variant, tile height and z planes
 * per work item (0 = automatic for each), with the same rules as the
 * lbm_params fields of those names.  Returns LBM_EINVAL (launch shape
 * unchanged) for a shape that cannot serve this lattice, LBM_ECUDA if it
 * cannot be configured on this device.  Not for a box of a batch. */
lbm_status lbm_set_kernel_config(lbm_ctx *ctx, int kernel, int tile_y,
                                 int zchunk);

/* Autotuner of the step's launch shape: times trial_steps (rounded up to even)
 * steps of each candidate on this lattice and keeps the fastest.  The
 * candidates differ in how the psi halo and the populations are staged:
 * kernel 1 (ring cells loaded into registers), 2 (every population through
 * cp.async), 3 (register prefetch one plane ahead, ring through cp.async;
 * with z chunks of 8, 16, 32 planes or automatic), 5 (tensor-copy boxes,
 * FP32), 7 (paired 16-bit words), each on 32x4, 32x8 and 32x16 tiles
 * (64-wide for kernel 7); kernel 6 on 32x8 / 32x16 when G2 != 0.  The trial
 * steps advance whatever state the context holds (its step counter does not
 * change): tune before setting the initial state.  Outputs (any may be NULL):
 * the chosen kernel, tile height, z chunk and its time per step in ms.
 * Returns LBM_ECUDA if no candidate ran. */
lbm_status lbm_tune(lbm_ctx *ctx, int trial_steps, int *kernel, int *tile_y,
                    int *zchunk, double *ms_per_step);

/* ---------------------------------------------------------------------------
 * Discrete adjoint of the SRT step (Sec. 2: Eqs. LBE, local_eq, momentum,
 * SC_force, vel_shift), for gradients of an objective J(rho(T)) with respect
 * to the initial density, G and tau.  Not in the paper: a GPU service built on
 * its step.  FP32 or FP64 storage (the adjoint field uses the storage type,
 * the G and tau gradients are summed in float64).
 * ------------------------------------------------------------------------- */

/* Start from rest with density rho0 (host or device, float64, nx*ny*nz), run
 * n >= 1 steps and keep every `every`-th state (t = 0, every, 2 every, ...) as
 * a checkpoint in device memory owned by the context; the state ends at
 * t = n.  Checkpoint memory: ceil(n/every) + every states.  Collision must be
 * LBM_SRT_SHIFT, G2 zero and nx*ny*nz < 2^32 (else LBM_EUNSUPPORTED). */
lbm_status lbm_adjoint_forward(lbm_ctx *ctx, const double *rho0, int on_device,
                               long n, int every);

/* Given dJdrho = dJ/drho(x, T) (float64 field, host or device), run the
 * discrete adjoint back to t = 0, recomputing each segment's states from its
 * checkpoint, and return dJ/drho0 (float64 field, host or device; may be
 * NULL), dJ/dG and dJ/dtau (host doubles; may be NULL).  Synchronises the
 * context's stream.  Working memory besides the checkpoints: two adjoint
 * states, `every` psi fields (the recomputation stores psi of each state it
 * steps from, with step kernels 1, 3 and 5) and six more fields. */
lbm_status lbm_adjoint_backward(lbm_ctx *ctx, const double *dJdrho,
                                int in_on_device, double *dJdrho0,
                                int out_on_device, double *dJdG,
                                double *dJdtau);

/* ---------------------------------------------------------------------------
 * Batches: many independent periodic boxes (uneven sizes) advanced together.
 * The method is the paper's step (Sec. 2) applied to each box; batching is a
 * GPU execution form, not in the paper.
 * ------------------------------------------------------------------------- */
typedef struct lbm_batch lbm_batch;

/* Create `count` boxes sharing the physics of *p (G, collision, tau, rates,
 * psi, storage: FP32 or FP64; p->nx/ny/nz are ignored; p->tile_y / zchunk
 * choose the initial launch shape, 0 = default).  dims[3*i + 0..2] are box
 * i's nx, ny, nz (each box needs 19 * cells < 2^31).  One allocation per
 * population copy holds every box (256-byte aligned per box).  If p->stream
 * is NULL the batch creates its own stream (needed to capture the step graph).
 * On failure *out is NULL and lbm_batch_last_error(NULL) has the message. */
lbm_status lbm_batch_create(const lbm_params *p, int count, const int *dims,
                            lbm_batch **out);
void lbm_batch_destroy(lbm_batch *b);                  /* NULL-safe */
const char *lbm_batch_last_error(const lbm_batch *b);

/* Context view of box i, owned by the batch: use it with lbm_init_ligament,
 * lbm_set_density, lbm_set/get_populations, lbm_moments, lbm_diag.  Stepping
 * it alone (lbm_step) returns LBM_EINVAL; lbm_destroy ignores it. */
lbm_status lbm_batch_box(lbm_batch *b, int i, lbm_ctx **view);

/* Advance every box n >= 0 steps with one kernel launch per step over the
 * work items (xy tile, z chunk) of all boxes; pairs of steps are replayed
 * from a captured CUDA graph. */
lbm_status lbm_batch_step(lbm_batch *b, long n);

/* Autotune the launch shape: times trial_steps steps for each tile height in
 * {4, 8, 16} and z chunk in {8, 16, 24, 32, 48, 64}, keeps the fastest and reports it
 * (any pointer may be NULL).  The trial steps overwrite the populations:
 * tune first, then initialise the boxes. */
lbm_status lbm_batch_tune(lbm_batch *b, int trial_steps, int *tile_y,
                          int *zchunk, double *ms_per_step);

/* Current launch shape, grid size and total cells. */
lbm_status lbm_batch_config(const lbm_batch *b, int *tile_y, int *zchunk,
                            int *grid, long long *cells);

/* ---------------------------------------------------------------------------
 * Allocation-free diagnostics.  The paper has no counterpart: this is a
 * service of the library, not part of the method.
 *
 * For callers that may not allocate device memory while they run: a program
 * whose device memory is all handed out by its own pool allocator (where a
 * raw cudaMalloc fails or fragments the pool), or a tight time-stepping loop
 * in which cudaMalloc/cudaFree would implicitly synchronise the device.
 * lbm_create allocates; this call does not.  It needs no context: the caller
 * passes its own population array f (device memory, 19*nx*ny*nz elements of
 * `storage` in the library's velocity order and field layout, LBM_F64 ..
 * LBM_BF16_DEV; rho_ref and dev_scale as in lbm_params for the deviation
 * formats; the local-reference formats also need a context's density field
 * and get LBM_EINVAL) and its own outputs,
 * and gets the same quantities as lbm_diag (mass, mom[3], area_z[nz],
 * maxrho_z[nz]; area_z/maxrho_z may be NULL).  Outputs are host memory when
 * on_device is 0, device memory when it is 1.  Work runs on `stream`
 * (cudaStream_t, NULL = legacy default), which the call synchronises before
 * it returns.
 *
 * Scratch: a fixed array in the library's device memory, LBM_NOALLOC_MAX_NZ
 * slices (8 doubles per slice, 512 KiB), which every GPU that loads the
 * library holds until the process exits.  The first call on each device looks
 * up that array's device address; make that first call before any stream
 * capture.  All calls share the one array and each overwrites what it reads,
 * so calls that overlap on the GPU (other host threads, other streams) race:
 * serialise them.  The call never calls cudaMalloc/cudaFree or any allocating
 * library routine.
 *
 * Returns LBM_EUNSUPPORTED (and does nothing) when nz > LBM_NOALLOC_MAX_NZ,
 * LBM_EINVAL for other bad arguments, LBM_ECUDA if a launch or copy fails,
 * LBM_ENONFINITE (outputs still written) if any cell has rho <= 0, NaN or Inf.
 * ------------------------------------------------------------------------- */
#define LBM_NOALLOC_MAX_NZ 8192
lbm_status lbm_diag_noalloc(const void *f, int storage, int nx, int ny, int nz,
                            double rho_ref, double dev_scale, double rho_l,
                            double rho_v, double *mass, double mom[3],
                            double *area_z, double *maxrho_z, int on_device,
                            void *stream);

#ifdef __cplusplus
}
#endif
#endif /* LBM_SC_H */
