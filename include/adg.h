/*
 * adg.h -- C ABI of the GB300 (sm_103a) asynchronous discontinuous Galerkin operator.
 *
 * The library advances the compressible Euler equations (Section 2, Eq. 1-3, no source
 * term) discretised by a nodal DG method on a periodic, uniform Cartesian quad/hex mesh
 * (Section 2.1, Eq. 4-7) with the Rusanov flux of Eq. 8-9 and low-storage explicit
 * Runge-Kutta time stepping (Section 2.3, Eq. 10, Table 2).  The asynchronous variants of
 * Section 3 are emulated on one GPU: the mesh is cut into P[0] x P[1] (x P[2]) logical
 * subdomains ("processing elements"); fluxes on faces between two subdomains use delayed
 * data held in a device ring buffer of past time levels, refreshed on the schedule of
 * Algorithm 2 (standard flux), Algorithm 3 (AT flux, Eq. 14-15) or a seeded random-delay
 * schedule.  Interior faces always use current data.
 *
 * Discretisation details fixed by this library:
 *   - nodes and quadrature: (degree+1)^dim Gauss-Legendre points per element, collocated;
 *   - state layout (host and device): FP64, structure of arrays [var][element][node],
 *       var     = rho, rho*u_x, rho*u_y, (rho*u_z), E               (dim+2 variables)
 *       element = ex + n_elem[0] * (ey + n_elem[1] * ez)           (x fastest)
 *       node    = a + (degree+1) * (b + (degree+1) * c)            (xi_x fastest),
 *     node a in direction d sits at lo[d] + (ex + (xi_a + 1)/2) * h[d] with xi_a the a-th
 *     Gauss-Legendre point on [-1, 1] in increasing order;
 *   - the time step is constant for a run (the AT weights assume equally spaced levels).
 *
 * Conventions for every entry point:
 *   - returns ADG_OK or an error status; no exception or abort crosses the ABI;
 *     adg_last_error() gives a message for the last failing call on a handle (or, with a
 *     NULL handle, for the last failing adg_create / host helper on this thread);
 *   - caller buffers are read or written only during the call; the library keeps no
 *     pointer to them.  "on_device" arguments say whether a pointer is a CUDA device
 *     address (1) or host memory (0);
 *   - a handle owns all device memory it allocates; handles are not thread-safe (use one
 *     per thread); all device work is ordered on the handle's CUDA stream.
 */
#ifndef ADG_H
#define ADG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct adg_solver adg_solver;

typedef enum {
  ADG_OK = 0,
  ADG_ERR_INVALID = 1,     /* bad argument (size, range, NULL where not allowed)        */
  ADG_ERR_UNSUPPORTED = 2, /* valid but not built (e.g. degree above the compiled range) */
  ADG_ERR_CUDA = 3,        /* a CUDA runtime call failed; see adg_last_error             */
  ADG_ERR_OOM = 4,         /* device allocation failed                                   */
  ADG_ERR_NONFINITE = 5,   /* the state holds NaN or Inf (adg_check_finite)              */
  ADG_ERR_TIMEOUT = 6,     /* a bounded device-side wait gave up (fused / element path)  */
  ADG_ERR_STATE = 7        /* call out of order (e.g. adg_step before adg_set_state)      */
} adg_status;

/* How faces between two subdomains get their flux (Section 3). */
typedef enum {
  ADG_FLUX_SYNC = 0,        /* Algorithm 1: every face uses current data; P ignored       */
  ADG_FLUX_STD_DELAYED = 1, /* Algorithm 2 / Eq. 13: reuse the stored flux of level n-k   */
  ADG_FLUX_AT = 2,          /* Algorithm 3 / Eq. 14: AT combination of stored fluxes      */
  ADG_FLUX_AT_TRACE = 3,    /* AT extrapolation of both stored traces, then Eq. 8         */
  ADG_FLUX_LEARNED = 4      /* as AT_TRACE, each extrapolated trace corrected by the learned
                               predictor (adg_set_learned_model); needs at_np = 2       */
} adg_flux;

typedef enum {
  ADG_DELAY_CAA = 0,   /* Algorithm 2 (n % L == 0) or Algorithm 3 (n % (L+Np+1) < Np+1)   */
  ADG_DELAY_RANDOM = 1 /* per step and subdomain interface: delay = splitmix64(seed ^
                          (n * n_iface + iface)) % (random_delay_max + 1), reduced to 0
                          while the history is shorter than the delay needs             */
} adg_delay_mode;

typedef enum {
  ADG_RK_2R_22 = 0,  /* LSERK(2,2), Table 2, two-register form of Eq. 10              */
  ADG_RK_2R_33 = 1,  /* LSERK(3,3), Table 2                                            */
  ADG_RK_2N_CK45 = 2 /* Carpenter & Kennedy (1994) five-stage fourth-order 2N scheme
                        (not printed in the paper)                                     */
} adg_rk;

typedef enum {
  ADG_PREC_FP64 = 0,  /* operator in native FP64                                         */
  ADG_PREC_FP32 = 1,  /* operator (traces, fluxes, volume terms) in FP32; the solution is
                         still accumulated in FP64                                      */
  ADG_PREC_DF64 = 2   /* operator in FP32-pair ("double-float") arithmetic, about 48
                         significant bits; solution accumulated in FP64                 */
} adg_precision;

typedef enum {
  ADG_PATH_AUTO = 0,   /* the faster path on GB300 for the arithmetic: ADG_PATH_ELEMENT
                          for FP32, ADG_PATH_SPLIT for FP64 and FP32 pairs               */
  ADG_PATH_SPLIT = 1,  /* per RK stage a face-flux launch, then a volume/update launch    */
  ADG_PATH_FUSED = 2,  /* per RK stage one launch per tile of elements: face fluxes and
                          volume/update work together, tiles staged by TMA copies        */
  ADG_PATH_ELEMENT = 3 /* per RK stage one volume/update launch in which every element
                          evaluates the numerical flux on each of its own faces from the
                          stored traces (no face-flux launch, no face-flux array)        */
} adg_kernel_path;

typedef struct {
  int dim;          /* 2 or 3                                                          */
  int n_elem[3];    /* elements per direction; entries beyond dim are ignored          */
  double lo[3];     /* periodic box [lo, hi] per direction                             */
  double hi[3];
} adg_mesh;

typedef struct {
  adg_rk rk;                 /* default ADG_RK_2N_CK45                                  */
  double dt;                 /* > 0: fixed time step; <= 0: from cfl at adg_set_state  */
  double cfl;                /* dt = cfl h_min / ((2 degree + 1) max(|u| + c)), default 0.1 */
  double t_end;              /* > 0: dt shortened so that a whole number of steps ends at t_end */
  double gamma;              /* ratio of specific heats, default 1.4                   */
  adg_delay_mode delay_mode; /* default ADG_DELAY_CAA                                  */
  uint64_t seed;             /* random-delay seed                                      */
  int random_delay_max;      /* 0..15, random mode only                                */
  int at_np;                 /* AT stencil uses at_np+1 stored levels; <= 0: = degree  */
  adg_precision precision;   /* default ADG_PREC_FP64                                  */
  void* cuda_stream;         /* cudaStream_t to order work on; NULL: the legacy default
                                stream (the stream torch uses unless told otherwise)     */
  adg_kernel_path kernel_path; /* kernels of adg_step, default ADG_PATH_AUTO; the paths
                                give the same results up to rounding (the learned flux
                                always takes the split path, trace logging the split or
                                element path)                                            */
} adg_options;

/* Fills *opt with the defaults listed above. */
adg_status adg_default_options(adg_options* opt);

/* Creates a solver (allocates every device buffer it will use).
 *   mesh:      periodic uniform mesh; n_elem[d] >= 1 and divisible by P[d].
 *   degree:    polynomial degree N_p, 1..7 in 2D and 1..5 in 3D.
 *   P:         logical subdomains per direction (entries beyond dim ignored); P[d] = 1
 *              gives no subdomain boundary across direction d (the periodic wrap face is
 *              then interior).
 *   max_delay: L of Algorithms 2/3: >= 1 for ADG_FLUX_STD_DELAYED, >= 0 for the AT modes;
 *              ignored by ADG_FLUX_SYNC and by the random mode.
 *   flux:      face rule on subdomain boundaries.
 *   opt:       NULL for defaults.
 * Errors: ADG_ERR_INVALID, ADG_ERR_UNSUPPORTED, ADG_ERR_OOM, ADG_ERR_CUDA.  *out is set
 * to NULL on error. */
adg_status adg_create(const adg_mesh* mesh, int degree, const int P[3], int max_delay,
                      adg_flux flux, const adg_options* opt, adg_solver** out);

/* Copies a state in (count must equal adg_info's n_dof) and restarts the schedule: the
 * step counter and time go to 0, the delay history is emptied, and dt is derived from
 * this state when options.dt <= 0.  Errors: ADG_ERR_INVALID (count, NULL), ADG_ERR_CUDA. */
adg_status adg_set_state(adg_solver* s, const double* u, int64_t count, int on_device);

/* Evaluates the initial condition at the nodes and sets it as the state (like
 * adg_set_state).  Isentropic vortex (Section 5.1): strength beta, centre (x0, y0),
 * background velocity (1, 0), nearest periodic image; in 3D it is extruded along z.   */
adg_status adg_init_vortex(adg_solver* s, double t, double beta, double x0, double y0);
/* Taylor-Green vortex on the box (rho0 = V0 = 1, p0 = 1/(gamma mach^2)); 3D only.      */
adg_status adg_init_tgv(adg_solver* s, double mach);

/* Advances n_steps time steps (each: all Runge-Kutta stages).  Work is enqueued on the
 * handle's stream; the call returns without waiting for the GPU.
 * Errors: ADG_ERR_STATE (no state set), ADG_ERR_INVALID (n_steps < 0), ADG_ERR_CUDA. */
adg_status adg_step(adg_solver* s, int n_steps);

/* Copies the current state out (waits for the stream).  count must equal n_dof.
 * ADG_ERR_TIMEOUT if a fused-path or element-path kernel gave up waiting for the TMA
 * copies of its tile (each wait is limited to about one second; the state is then not
 * valid). */
adg_status adg_get_state(adg_solver* s, double* u, int64_t count, int on_device);

/* Synchronous DG operator k = M^{-1} L_h(u) (Eq. 7; every face with current data) for an
 * arbitrary state u of n_dof values, written to k (same layout).  Does not touch the
 * solver's state or schedule.  Waits for the stream. */
adg_status adg_rhs(adg_solver* s, const double* u, double* k, int64_t count, int on_device);

/* Schedule of steps n0 .. n0+n-1 (integer data, computed on the host):
 *   comm[i]: 1 when every subdomain face uses current data in step n0+i;
 *   k[i]:    the delay counter of Algorithms 2/3 (random mode: the largest delay);
 *   iface_delay (nullable) [n][n_iface]: the delay of each subdomain interface.
 * Interface numbering: for each direction d with P[d] > 1 (in increasing d) one block of
 * P[0]*P[1]*P[2] interfaces, indexed by the subdomain on the low side of the face. */
adg_status adg_get_schedule(const adg_solver* s, int64_t n0, int n, int32_t* comm, int32_t* k,
                            int32_t* iface_delay);

/* Current time, step count, time step and number of degrees of freedom
 * (n_dof = (dim+2) * n_elements * (degree+1)^dim).  Any pointer may be NULL. */
adg_status adg_info(const adg_solver* s, double* t, int64_t* step, double* dt, int64_t* n_dof);

/* Conserved totals sum_e sum_q omega_q |J| w_q for each variable (dim+2 values) of the
 * current state; a deterministic reduction.  Waits for the stream. */
adg_status adg_conservation(adg_solver* s, double* sums);

/* Absolute L2 errors (density, momentum vector, energy) of the current state against the
 * exact isentropic vortex at time t, with (degree+2)^dim Gauss points per element.      */
adg_status adg_l2_error_vortex(adg_solver* s, double t, double beta, double x0, double y0,
                               double* err3);

/* ADG_OK if every state value is finite, ADG_ERR_NONFINITE otherwise. */
adg_status adg_check_finite(adg_solver* s);

/* ---- checkpoint / resume ---------------------------------------------------------- */
/* A checkpoint holds everything later steps depend on: the solution, the stored traces,
 * the ring of stored subdomain-face levels with its head, the step index, time and time
 * step.  Restoring it into a handle created with the same mesh, degree, subdomains,
 * maximum delay, flux, RK scheme, delay mode and seed, and precision continues the run
 * bit for bit (the delay schedule depends only on the step index and the seed).  Setting
 * a state with adg_set_state instead restarts the schedule at step 0, with the warm-up
 * communication steps of Algorithm 3.
 * adg_checkpoint_bytes: size of the checkpoint of this handle.
 * adg_checkpoint_save: waits for the stream and writes the checkpoint to the host buffer
 *   buf (bytes >= adg_checkpoint_bytes).  ADG_ERR_STATE without a state.
 * adg_checkpoint_restore: reads a checkpoint from host memory; ADG_ERR_INVALID if it is
 *   truncated, not a checkpoint, or from an incompatible handle (adg_last_error says which
 *   field differs).  The buffer is owned by the caller and not kept. */
adg_status adg_checkpoint_bytes(const adg_solver* s, int64_t* bytes);
adg_status adg_checkpoint_save(adg_solver* s, void* buf, int64_t bytes);
adg_status adg_checkpoint_restore(adg_solver* s, const void* buf, int64_t bytes);

/* Kernel timing.  While enabled, adg_step records a CUDA event pair on the handle's stream
 * around every kernel it launches.  adg_get_profile waits for the stream and returns, per
 * kernel kind (0: face-flux kernel, 1: volume/update kernel), the summed device time in ms
 * and the launch count since profiling was enabled or last read; it then resets them.
 * At most 2048 events are kept: when they are used up, adg_step waits for the stream once
 * and folds the recorded pairs into the running totals (profiling is a diagnostic mode;
 * with it off, adg_step never waits). */
adg_status adg_set_profiling(adg_solver* s, int enable);
adg_status adg_get_profile(adg_solver* s, double* ms, int64_t* launches);

/* ---- operator without device allocation ------------------------------------------ */

/* Size of the built-in device scratch array used by adg_rhs_noalloc (32 MiB). */
#define ADG_NOALLOC_SCRATCH_BYTES (32u << 20)

/* The synchronous FP64 operator k = M^{-1} L_h(u) of adg_rhs, for callers that cannot
 * allocate device memory: a host application that owns the whole device memory budget
 * (a fixed arena or pool that forbids outside allocations), or a loop where the implicit
 * device synchronisation and unbounded latency of cudaMalloc are not acceptable.  The
 * paper has no counterpart; this is a library convenience.
 *
 * Needs no handle and allocates nothing: no cudaMalloc, no cudaFree, no allocating
 * library routine.  Its scratch (operator tables, face traces, face fluxes) sits in one
 * file-scope device array of ADG_NOALLOC_SCRATCH_BYTES that every GPU loading the library
 * holds until the process exits.  The first call on a device looks up that array's
 * device address (cudaGetSymbolAddress, with the device current); make that first call
 * before any stream capture.  Every call overwrites all the scratch it later reads, so
 * nothing carries over between calls; calls that overlap on the GPU (two streams, two
 * host threads) share the one array and race.
 *   mesh, degree: as in adg_create (periodic uniform mesh; degree 1..7 in 2D, 1..5 in 3D);
 *   gamma:        ratio of specific heats (> 1);
 *   u, k:         DEVICE pointers, n_dof = (dim+2) * n_elements * (degree+1)^dim values each,
 *                 layout as for adg_set_state; u is read, k written;
 *   count:        must equal n_dof;
 *   cuda_stream:  cudaStream_t the work is ordered on (NULL = legacy default stream).
 * The call enqueues the work and returns without waiting: the operator tables travel as
 * a kernel argument and a kernel stores them into the scratch array, so no host memory is
 * read after the call returns and no copy from pageable memory stalls the host.  A mesh
 * whose scratch
 * (2 d + d) (d+2) n_elements (degree+1)^(d-1) doubles plus the tables exceeds
 * ADG_NOALLOC_SCRATCH_BYTES is rejected with ADG_ERR_INVALID; adg_last_error(NULL) says
 * how many bytes it needed.  Other errors: ADG_ERR_INVALID (arguments), ADG_ERR_CUDA. */
adg_status adg_rhs_noalloc(const adg_mesh* mesh, int degree, double gamma, const double* u,
                           double* k, int64_t count, void* cuda_stream);

/* Arithmetic peak probe (no counterpart in the paper; it supplies the denominators of the
 * roofline fractions the library reports).  Measures, on the current device, the rate of
 * one instruction kind with every warp slot busy on independent dependency chains:
 *   kind 0: FP64 FMA; 1: FP32 FMA; 2: FP64 tensor MMA (mma.sync m8n8k4 f64);
 *   3: FP64 FMA and FP64 MMA in alternate warps (shows whether the two paths add up);
 *   4: packed FP32x2 FMA; 5: FP64 add; 6: FP64 multiply (one flop per operation).
 * tflops receives the best of three timed launches (about 50 ms each at the nominal
 * rates) in TFLOP/s (an FMA counts as 2 flops, an m8n8k4 MMA as 512 per warp); ms
 * (nullable) that launch's duration; sm_mhz (nullable) the SM clock during it (clock64
 * cycles of one thread over the global nanosecond timer).  Allocates and frees a small
 * device buffer and a private stream; waits for its own launches.  Errors:
 * ADG_ERR_INVALID, ADG_ERR_CUDA (adg_last_error(NULL) has the text). */
adg_status adg_measure_peak(int kind, double* tflops, double* ms, double* sm_mhz);

/* Check of the bounded device-side wait (no counterpart in the paper).  The fused and
 * element-path kernels wait for their tiles' TMA copies on an mbarrier for at most about
 * one second and then set an error flag (ADG_ERR_TIMEOUT from adg_get_state) instead of
 * hanging.  This probe runs the same wait, with limit_cycles SM clock cycles
 * (0 < limit_cycles <= 4e9), in one block of 128 threads on a barrier that nothing arrives
 * at: *threads_gave_up receives the number of threads that gave up (128 when the limit
 * works), *cycles (nullable) the cycles thread 0 waited.  Uses a private stream and a
 * 16-byte device buffer; waits for its launch.  Errors: ADG_ERR_INVALID, ADG_ERR_CUDA
 * (adg_last_error(NULL) has the text). */
adg_status adg_probe_wait(int64_t limit_cycles, int* threads_gave_up, int64_t* cycles);

/* Message for the last failing call on s (NULL: on this thread, for calls without a
 * handle).  Valid until the next call on the same handle/thread. */
const char* adg_last_error(const adg_solver* s);

/* Frees the handle and its device memory.  NULL-safe. */
void adg_destroy(adg_solver* s);

/* ---- batched solver ------------------------------------------------------------------ */
/* Many independent instances (own mesh, degree, subdomains and max_delay; shared flux
 * rule and options) advanced together.  Instances with the same dimension and degree form
 * a group: every RK stage runs one persistent face-flux launch and one persistent volume
 * launch per group (with the FP32 operator, unless options.kernel_path is ADG_PATH_SPLIT:
 * one persistent element-path launch, every element evaluating its own faces' fluxes;
 * instances the autotuner leaves to separate stepping take options.kernel_path, with
 * ADG_PATH_FUSED read as ADG_PATH_SPLIT), and one whole step of all groups is captured once into a CUDA graph
 * and replayed by adg_batch_step.  The schedule of Algorithms 2/3 advances on the device,
 * per instance.  Results equal those of separate adg_solver handles bit for bit. */
typedef struct adg_batch adg_batch;

/* meshes[n], degrees[n], P[3n], max_delay[n]; all meshes of one dimension.  Each
 * instance's time step comes from options.cfl (or options.dt) at its own state. */
adg_status adg_batch_create(int n, const adg_mesh* meshes, const int* degrees, const int* P,
                            const int* max_delay, adg_flux flux, const adg_options* opt,
                            adg_batch** out);
/* State of instance i: the isentropic vortex (beta, centre), or a given state. */
adg_status adg_batch_init_vortex(adg_batch* b, int i, double beta, double x0, double y0);
adg_status adg_batch_set_state(adg_batch* b, int i, const double* u, int64_t count, int on_device);
/* Advances every instance by n_steps steps (graph replays; enqueued, does not wait).
 * Errors: ADG_ERR_STATE if an instance has no state. */
adg_status adg_batch_step(adg_batch* b, int n_steps);
/* Autotuner: for every degree group, times on the real buffers the volume launch with
 * tiles of about 64, 128 and 256 threads, each launched as one resident wave of persistent
 * blocks and as one block per tile, and with the instances that fill the GPU four times,
 * once, or never given the single-handle volume launch of their own; then the face-flux
 * launch in both shapes; and keeps the fastest; finally it times whole steps with the
 * instances that fill the GPU once over kept in the graph or stepped as separate handles
 * (single-handle launches, host-side schedule, after the graph's work on the same stream)
 * and keeps the faster.  tile_threads (nullable) receives the tile chosen per group in
 * increasing degree.  It overwrites every instance's state (set states afterwards). */
adg_status adg_batch_autotune(adg_batch* b, int trials, int* tile_threads);
adg_status adg_batch_get_state(adg_batch* b, int i, double* u, int64_t count, int on_device);
adg_status adg_batch_info(const adg_batch* b, int i, double* t, int64_t* step, double* dt,
                          int64_t* n_dof, int* degree);
adg_status adg_batch_l2_error_vortex(adg_batch* b, int i, double t, double beta, double x0,
                                     double y0, double* err3);
int adg_batch_num_groups(const adg_batch* b);
const char* adg_batch_last_error(const adg_batch* b);
void adg_batch_destroy(adg_batch* b);

/* ---- learned ghost-trace predictor ------------------------------------------------- */
/* A small MLP (4 -> 64 -> 64 -> 1, tanh hidden layers) with BF16 weights and FP32
 * accumulation, used by ADG_FLUX_LEARNED to correct the AT extrapolation of subdomain
 * traces.  Not part of the paper's method: an add-on whose error is measured against, and
 * which falls back to, the plain AT extrapolation.  Parameters: adg_mlp_num_params()
 * values laid out W1[64][4] | b1[64] | W2[64][64] | b2[64] | w3[64] | b3.
 * All pointers below are DEVICE pointers; work is enqueued on cuda_stream. */
int adg_mlp_num_params(void);
/* Mean squared error over n samples (x[n][4], target[n]): ADDS d(loss)/d(params) to grad
 * (FP32, one value per parameter) and the loss to *loss (one float).  Forward and backward
 * pass in FP32 arithmetic with the BF16 weights. */
adg_status adg_mlp_grad(const uint16_t* params_bf16, const float* x, const float* target,
                        int64_t n, float* grad, float* loss, void* cuda_stream);
/* y[n] = MLP(x[n][4]).  The hidden 64 x 64 layer runs on the tensor cores (BF16 MMA with
 * FP32 accumulation; the FP32 activations enter as three BF16 terms, so the result has
 * FP32 accuracy); the solver's learned flux uses the same kernel. */
adg_status adg_mlp_forward(const uint16_t* params_bf16, const float* x, int64_t n, float* y,
                           void* cuda_stream);
/* One Adam step (step counter t >= 1) on FP32 master params with moments m, v; writes the
 * BF16 copy and zeroes grad. */
adg_status adg_mlp_adam(float* params, uint16_t* params_bf16, float* grad, float* m, float* v,
                        float lr, float beta1, float beta2, float eps, int t, void* cuda_stream);
/* BF16 copy (round to nearest even) of FP32 params. */
adg_status adg_mlp_to_bf16(const float* params, uint16_t* params_bf16, void* cuda_stream);

/* Model of ADG_FLUX_LEARNED: params_bf16 (HOST, adg_mlp_num_params() BF16 values) and the
 * trust bound.  Per trace value the AT extrapolation E3 (three levels) and the linear one
 * E2 (two levels) give the error estimate e = E3 - E2; the network output y is applied as
 * E3 + e y only when |y| <= trust, so a correction never exceeds trust times AT's own
 * error estimate; otherwise (and where e is at rounding level) E3 stands. */
adg_status adg_set_learned_model(adg_solver* s, const uint16_t* params_bf16, float trust);
/* Trace log for training data: while set, every RK stage of adg_step first appends one
 * record with the traces of the current stage input on all subdomain faces (both sides),
 * FP64, to the DEVICE buffer dev_log (capacity n_records records; later stages are not
 * logged once it is full).  *record_len (nullable) = values per record
 * = 2 (sides) x (dim+2) x n_subdomain_faces x (degree+1)^(dim-1), ordered
 * [side][var][face][face node].  dev_log = NULL switches logging off. */
adg_status adg_set_trace_log(adg_solver* s, double* dev_log, int64_t n_records,
                             int64_t* record_len);
/* Training samples from a trace log of a synchronous run (records step*stages + stage):
 * dev_picks[n][4] = (channel within a record, step, stage, delay k >= 1) with
 * step - k - 2 >= 0.  Writes the network inputs dev_x[n][4], the targets dev_target[n]
 * (truth minus AT extrapolation, in units of the AT error estimate E3 - E2) and dev_ok[n]
 * (0 where that estimate is at rounding level, below 1e-9 of the levels: no sample).  Uses the solver's RK stage offsets. */
adg_status adg_learned_samples(adg_solver* s, const double* dev_log, int64_t n_records,
                               const int32_t* dev_picks, int64_t n, float* dev_x,
                               float* dev_target, int32_t* dev_ok);

/* ---- host-only helpers (no GPU needed) ---------------------------------------------- */

/* Gauss-Legendre nodes x[n] (increasing) and weights w[n] on [-1, 1], 1 <= n <= 8. */
adg_status adg_host_gauss(int n, double* x, double* w);
/* AT weights of Eq. 14 for delay k_m (fractional allowed): c[0..np] on levels
 * n-k_m, ..., n-k_m-np, from the moment conditions of Eq. 15 with r = 1. */
adg_status adg_host_at_coeffs(int np, double km, double* c);
/* Low-storage coefficients of a scheme: a[s], b[s], stage abscissae c[s]; returns the
 * stage count in *stages.  2R: a = (a_1..a_{s-1}, 0), b as in Table 2.  2N: A_i, B_i.  */
adg_status adg_host_rk(adg_rk scheme, int* stages, double* a, double* b, double* c);
/* Same schedule as adg_get_schedule without a solver (dim, P[3] as in adg_create). */
adg_status adg_host_schedule(adg_flux flux, adg_delay_mode mode, int max_delay, int np, int dim,
                             const int P[3], uint64_t seed, int random_delay_max, int64_t n0,
                             int n, int32_t* comm, int32_t* k, int32_t* iface_delay);
/* Number of subdomain interfaces (see adg_get_schedule). */
int adg_host_num_interfaces(int dim, const int P[3]);

#ifdef __cplusplus
}
#endif
#endif /* ADG_H */
