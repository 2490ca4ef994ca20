/*
 * pic.h -- C ABI of the GB300 electrostatic particle-in-cell hot path.
 *
 * The library advances electrons in a periodic box [0,Lx) x [0,Ly) x [0,Lz)
 * under their own space-charge field plus optional uniform external B and a
 * quadrupole external E (the Vlasov-Poisson model of Section 3.1 of
 * arXiv 2205.11052, Eq. Vlasov and Eq. potential, in the normalised units of
 * Section 3.2: eps0 = 1).  One step is the PIC cycle of Section 3.1:
 *   scatter (CIC deposit) -> FFT Poisson solve -> gather (CIC) -> push,
 * with a cell-centred grid, periodic boundaries and the synchronised Boris
 * integrator of Section 3.2 (read here as drift-kick-drift).
 *
 * Conventions shared by every call
 *  - Status: every int-returning call returns PIC_OK (0) or a negative
 *    PIC_ERR_* code; pic_last_error() then describes the failure.  No C++
 *    exception crosses this boundary.
 *  - Threads: a handle must not be used from two host threads at once.
 *  - Memory: the library allocates no device memory of its own for the
 *    simulation state.  pic_buffer_sizes() reports one arena size; the caller
 *    allocates it (for instance as a torch tensor) and binds it with
 *    pic_bind_workspace().  The caller owns the arena and the stream and must
 *    keep both alive until pic_destroy().  cuFFT plans are created inside
 *    pic_bind_workspace() with automatic work-area allocation disabled (their
 *    work area lives in the arena; cuFFT may still keep small internal tables).
 *  - Ordering: all device work is enqueued on the bound stream, asynchronously
 *    with respect to the host, except where a call says it synchronises.
 *    Calls that take host buffers synchronise before returning.
 *  - Layouts: particle positions and velocities cross the boundary as FP64
 *    arrays of shape (n, 3), row-major (x0 y0 z0 x1 y1 z1 ...).  Grid fields
 *    are row-major (Nz, Ny, Nx) with x fastest: node (i, j, k) sits at
 *    ((i + 1/2) hx, (j + 1/2) hy, (k + 1/2) hz), h_d = L_d / N_d
 *    (cell-centred grid, Section 3.2).
 */
#ifndef PIC_GB300_PIC_H
#define PIC_GB300_PIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
#define PIC_OK               0
#define PIC_ERR_ARG         -1  /* invalid argument or configuration           */
#define PIC_ERR_CAPACITY    -2  /* more particles or larger buffers than bound  */
#define PIC_ERR_CUDA        -3  /* a CUDA runtime call or kernel launch failed  */
#define PIC_ERR_CUFFT       -4  /* a cuFFT call failed                          */
#define PIC_ERR_DEVICE_FLAG -5  /* a kernel raised an error flag (NaN, bad cell) */
#define PIC_ERR_TIMEOUT     -6  /* a bounded device-side wait ran out           */
#define PIC_ERR_STATE       -7  /* call out of order (e.g. no workspace bound)  */

/* device error flag bits reported by pic_device_flags() */
#define PIC_FLAG_NONFINITE   1  /* a non-finite position, velocity or field value */
#define PIC_FLAG_BAD_CELL    2  /* a particle cell index outside the grid          */
#define PIC_FLAG_TIMEOUT     4  /* a bounded wait inside a kernel gave up           */

typedef struct pic_ctx *pic_handle_t;

/* Periodic cell-centred grid: n[d] nodes (1..1024; n[0] >= 2) on [0, L[d]). */
typedef struct {
    int32_t n[3];
    double  L[3];
} pic_grid_t;

/* One electron species with uniform macro-particle charge (Section 3.1). */
typedef struct {
    double  q_over_m;      /* charge-to-mass ratio; -1 in normalised units      */
    double  total_charge;  /* Q_e; each loaded particle carries Q_e / n_loaded  */
    int64_t n_particles;   /* particle capacity, 0 .. 2^31 - 1                  */
} pic_species_t;

/* Time step, external fields and tuning knobs (0 selects the default). */
typedef struct {
    double  dt;            /* time step (> 0)                                    */
    double  B_ext[3];      /* uniform external magnetic field                    */
    double  wz2;           /* quadrupole external field (Section 4.3):
                              E_ext = wz2 * (-(x-cx)/2, -(y-cy)/2, (z-cz)),
                              c = box centre; wz2 is the axial frequency squared */
    int32_t tile[3];       /* deposit tile, in cells per axis (default 8)        */
    int32_t guard;         /* tile guard layers, in cells (default 2)            */
    int32_t sort_period;   /* re-bin particles every K steps (default 1;
                              negative = only when loaded)                      */
    int32_t diag_every;    /* record diagnostics every K steps (0 = never)       */
    int32_t diag_capacity; /* diagnostic records kept on the device (default 1024) */
    int32_t mode[3];       /* Fourier mode tracked by the diagnostics            */
    int32_t mode_comp;     /* component of E for that mode: 0 = x, 1 = y, 2 = z  */
    int32_t block;         /* threads per block of the particle kernels (256);
                              ensembles: of the batched push + deposit, a
                              multiple of 32 in 64..256 (autotuned)          */
    int32_t chunk;         /* max particles per deposit work item, 32..4095
                              (default 4095)                                     */
    int32_t options;       /* PIC_OPT_* bits (default 0)                         */
    uint64_t seed;         /* random stream of PIC_OPT_UNIFORM_MOVE              */
    double  stray_rebin;   /* stray-triggered re-binning in pic_step (default 0 =
                              off): > 0 makes the device decide before every
                              step whether to re-bin, doing so when the last
                              push left more than stray_rebin x n_particles
                              particles outside their tile's guard (any small
                              positive value re-bins on the first stray), or
                              when sort_period (> 0) pushes have passed       */
} pic_params_t;

/* options: accumulate the deposit in 2^-20 fixed point (u32 shared-memory
 * tile, u64 grid) instead of FP32.  Integer sums are order independent, so
 * the deposit is then deterministic and conserves charge exactly; weights are
 * rounded to 2^-20 (relative error below 1e-6 of a node's charge). */
#define PIC_OPT_FIXED_DEPOSIT 1
/* The uniform plasma test (Section 4.4): each step moves every particle by an
 * independent uniform displacement in [-h_d, h_d) per axis instead of the
 * gather and push; deposit, field solve and diagnostics run as usual and the
 * velocities are left unchanged.  The displacement of axis d of the particle
 * loaded as number pid in step n is (2u - 1) h_d with u = (r >> 40) 2^-24,
 * r = the c-th output of the SplitMix64 generator (Steele, Lea and Flood,
 * 2014) seeded with params.seed, c = ((n 2^32) + pid) 4 + d + 1.  Not
 * available with the adjoint or in ensembles. */
#define PIC_OPT_UNIFORM_MOVE 2
/* The adjoint also yields the gradient of J with respect to the field
 * parameters: B_ext (Eq. momentum_eqn through the Boris rotation) and the
 * quadrupole strength wz2 = omega_z^2 (Section 4.3), read with
 * pic_adjoint_param_gradient.  The forward sweep then also stores each step's
 * velocities before the kick (12 more bytes per particle and stored step in
 * the adjoint buffer). */
#define PIC_OPT_ADJOINT_PARAMS 4

/* Sizes the caller must provide before any device work. */
typedef struct {
    size_t  workspace_bytes;     /* one device arena, 256-byte aligned start   */
    size_t  workspace_align;     /* required alignment of the arena (bytes)    */
    int64_t particle_capacity;   /* = species n_particles                       */
    int64_t grid_nodes;          /* Nx * Ny * Nz                                */
    int64_t staging_particles;   /* particles per host<->device transfer chunk  */
} pic_bufsizes_t;

/* One diagnostic record (FP64).  Field quantities refer to the field of
 * step `step`, computed at the half step t_field = (step + 1/2) dt of the
 * drift-kick-drift cycle; particle quantities use the synchronised
 * velocities v_{step+1} at t = (step + 1) dt. */
typedef struct {
    int64_t step;
    double  t_field;
    double  Wx, Wy, Wz;      /* int E_d^2 dV = h^3 sum_g E_d,g^2 (Figs. of Section 4) */
    double  Q;               /* h^3 sum_g rho_g: electron charge on the grid    */
    double  mode_re, mode_im;/* (1/N_g) sum_g E_c,g exp(-2 pi i m.g/N)           */
    double  t;
    double  Px, Py, Pz;      /* m_p sum_p v_p                                    */
    double  K;               /* (1/2) m_p sum_p |v_p|^2                           */
} pic_diag_t;

/* ------------------------------------------------------------ lifecycle */

/* Validate the configuration and create a handle.  Host-only: no CUDA call
 * is made, so this also works where no GPU is present.
 * Errors: PIC_ERR_ARG for null pointers, grid sizes outside 1..1024 (or
 * n[0] < 2), non-positive or non-finite lengths or dt, capacity outside
 * 0..2^31-1, tiles < 1, negative guard, diag mode out of range. */
int pic_create(const pic_grid_t *grid, const pic_species_t *species,
               const pic_params_t *params, pic_handle_t *out);

/* Report the device arena size (and derived sizes) for this handle. Host-only. */
int pic_buffer_sizes(pic_handle_t h, pic_bufsizes_t *out);

/* Bind the caller-allocated device arena (at least workspace_bytes, aligned
 * to workspace_align) and a CUDA stream (cudaStream_t as void*, NULL = legacy
 * default stream) on the current device; creates the cuFFT plans and clears
 * the diagnostics and flags.  May be called again to rebind.
 * Errors: PIC_ERR_ARG (null or misaligned pointer), PIC_ERR_CAPACITY
 * (arena too small), PIC_ERR_CUDA, PIC_ERR_CUFFT. */
int pic_bind_workspace(pic_handle_t h, void *dev_arena, size_t bytes, void *stream);

/* Change the stream later work is enqueued on. */
int pic_set_stream(pic_handle_t h, void *stream);

/* Release host-side state and cuFFT plans (not the caller's arena). */
void pic_destroy(pic_handle_t h);

/* Thread-local text of the most recent failure on this host thread. */
const char *pic_last_error(void);

/* ------------------------------------------------------------ state I/O */

/* Load n synchronised particles (x_0, v_0), FP64 arrays of shape (n, 3),
 * from host memory (src_is_device = 0) or device memory (src_is_device = 1).
 * Page-locked host arrays are read in place by the load kernel (above 2^22
 * particles in ranges, each binned on a library-owned side stream while the
 * next one is read); pageable host arrays are copied in chunks through the
 * arena.  Positions may lie outside [0, L) and are wrapped periodically.
 * Resets the step counter and diagnostics, half-drifts to
 * x_{1/2} = x_0 + dt/2 v_0 (the drift-kick-drift state kept on the device),
 * stores each particle as (cell, FP32 offset, FP32 velocity) and bins it
 * (Section 3.2; particle storage as in Section 2's SoA layout); particles in
 * arbitrary order go through coarse binning passes first.  Host sources
 * synchronise; device sources are enqueued.
 * Errors: PIC_ERR_CAPACITY (n > capacity), PIC_ERR_ARG, PIC_ERR_CUDA. */
int pic_load_particles(pic_handle_t h, const double *x, const double *v,
                       int64_t n, int src_is_device);

/* Write the synchronised state (x_n, v_n) of all loaded particles, in load
 * order, as FP64 (n, 3) arrays to host (dst_is_device = 0) or device memory.
 * Positions are wrapped into [0, L).  Synchronises for host destinations. */
int pic_get_particles(pic_handle_t h, double *x, double *v, int dst_is_device);

/* Copy the current grid fields: rho (N_g FP32, electron charge density of
 * the last deposit) and E (N_g x 4 FP32: Ex, Ey, Ez, 0 of the last solve).
 * Either pointer may be NULL.  Synchronises for host destinations. */
int pic_get_field(pic_handle_t h, float *rho, float *E, int dst_is_device);

/* Overwrite rho (N_g FP32 values, layout as above, electron charge density)
 * from host (src_is_device = 0; synchronises) or device memory, e.g. to
 * solve for the field of a given density with pic_field_solve(). */
int pic_set_rho(pic_handle_t h, const float *rho, int src_is_device);

/* Number of particles currently loaded and steps taken since the load. */
int pic_get_counts(pic_handle_t h, int64_t *n_particles, int64_t *step);

/* ------------------------------------------------------------ the cycle */

/* Re-bin the particles: periodic counting sort by tile-major cell index and
 * rebuild the deposit work list.  (Not in the paper; keeps particles
 * cell-ordered so the deposit can accumulate in shared-memory tiles.) */
int pic_sort(pic_handle_t h);

/* Scatter (Section 3.1 step 1): rho_g = sum_p q_p W(x_g - x_p) / h^3 with the
 * CIC shape on the cell-centred grid (Section 3.2), from the current
 * half-step positions x_{n+1/2}.  Overwrites rho. */
int pic_deposit(pic_handle_t h);

/* Field solve (Section 3.1 step 2, Eq. potential; Section 3.2): the uniform
 * ion background cancels the mean of rho; E^_d = -i k_d rho^ / |k|^2 with
 * k_d = 2 pi m_d / L_d, the k = 0 mode and each axis' Nyquist gradient set to
 * zero, then E = IFFT.  Overwrites E. */
int pic_field_solve(pic_handle_t h);

/* Gather + push (Section 3.1 steps 3-4, Eq. momentum_eqn; Section 3.2):
 * interpolate E (+ E_ext) to x_{n+1/2} with the CIC weights, Boris-rotate
 * v_n -> v_{n+1} about B_ext, drift x_{n+1/2} -> x_{n+3/2} = x_{n+1/2} + dt v_{n+1},
 * apply the periodic boundary, and advance the step counter. */
int pic_gather_push(pic_handle_t h);

/* n full steps: [re-bin when due] deposit, solve, gather+push, and the FP64
 * diagnostic reductions every diag_every steps.  Only kernel launches, cuFFT
 * executions and memsets are enqueued (no host synchronisation), so the
 * sequence can be captured in a CUDA graph by the caller.
 * Re-binning is due every sort_period steps, counted on the host; with
 * params.stray_rebin > 0 the decision is taken on the device instead, before
 * each step, from the stray count of the previous push and the pushes since
 * the last re-binning: the sort kernels are launched every step and return at
 * once unless a re-binning is due, so a captured graph re-bins exactly when
 * the run needs it. */
int pic_step(pic_handle_t h, int n);

/* Re-binning statistics since the last load (synchronising): re-binnings
 * performed (the load's own binning included), and the "strays": particles
 * deposited outside their tile's guard by the pushes since the last
 * re-binning (with stray_rebin on: by the last push alone, as each decision
 * clears the count).  Either pointer may be NULL.  (Not in the paper: the
 * binning is this library's.) */
int pic_rebin_stats(pic_handle_t h, int64_t *rebins, int64_t *strays);

/* ------------------------------------------------------------ diagnostics */

/* Copy up to max_records diagnostic records (oldest first; at most the last
 * diag_capacity are kept) to host memory and report how many were written.
 * Synchronises, then returns PIC_ERR_TIMEOUT if a kernel's bounded wait gave
 * up, or PIC_ERR_DEVICE_FLAG if a kernel raised another flag. */
int pic_diagnostics(pic_handle_t h, pic_diag_t *out, int max_records, int *n_out);

/* Read (synchronising) and optionally clear the device error flag word. */
int pic_device_flags(pic_handle_t h, int32_t *flags, int clear);

/* Exercise the failure path of the kernels' bounded waits without a fault
 * (not in the paper; failure detection of this library).  The staged sort
 * waits on mbarriers for its bulk copies with a time limit; this call runs one
 * kernel whose wait has nothing to wait for (an mbarrier no thread arrives on,
 * no copy in flight), so the wait gives up after that limit (two seconds of
 * the GPU's clock), the kernel raises PIC_FLAG_TIMEOUT in the flag word and returns, and
 * the context stays usable.  Synchronises; returns PIC_ERR_TIMEOUT when the
 * flag was raised (the expected result) and leaves the flag set, so that
 * pic_diagnostics and pic_device_flags report it until it is cleared. */
int pic_selftest_timeout(pic_handle_t h);

/* ------------------------------------------------------------ timers */

/* Per-phase device timers, in the spirit of the per-kernel timers the paper
 * reports (Section 5.1, Table parallel_comm_kernels: scatter, solve, gather +
 * push ...).  When enabled, every phase call records a CUDA event pair on the
 * bound stream around its kernels; the library also counts its own kernel
 * launches (cuFFT's kernels excluded).  Do not enable timers while the
 * stream is being captured into a CUDA graph. */
#define PIC_PHASE_SORT     0   /* binning: histogram, scan, scatter, work list   */
#define PIC_PHASE_DEPOSIT  1   /* the deposit kernel                              */
#define PIC_PHASE_SOLVE    2   /* R2C FFT, Green kernel, C2R FFT                  */
#define PIC_PHASE_PUSH     3   /* the fused gather + push kernel                  */
#define PIC_PHASE_DIAG     4   /* FP64 diagnostic reductions                      */
#define PIC_PHASE_COUNT    5

/* Enable (1) or disable (0) the timers; either way the accumulators and the
 * launch counter are reset.  Errors: PIC_ERR_STATE before binding. */
int pic_enable_timers(pic_handle_t h, int enable);

/* Synchronise and report, per phase, the summed device time (ms) and the
 * number of timed calls, plus the library kernels launched since enabling.
 * Any pointer may be NULL. */
int pic_read_timers(pic_handle_t h, double ms[PIC_PHASE_COUNT],
                    int64_t calls[PIC_PHASE_COUNT], int64_t *kernel_launches);

/* ------------------------------------------------------------ adjoint */

/* Gradient of the final field energy (not in the paper).
 *
 * Objective: J = sum_d w_d h^3 sum_g E_d,g^2, the weighted field energy of
 * the field used by the last of n_steps steps (the W_d of pic_diag_t for that
 * step), as a function of the synchronised state (x_0, v_0) loaded last.
 * The gradient is the exact discrete adjoint of the drift-kick-drift step of
 * pic_step, external fields included: the gather and the deposit appear as
 * each other's transposes, the spectral operator as its conjugate symbol and
 * the Boris rotation R (v' = R v + (dt q/m / 2)(R + I) e) as R^T.
 * Memory: the forward pass stores a checkpoint of the particle state every
 * `checkpoint_every` steps; the reverse sweep recomputes one segment at a
 * time from its checkpoint, keeping that segment's positions and fields (the
 * last segment is kept by the forward pass itself; with checkpoint_every >=
 * n_steps - 1 nothing is recomputed).  Both sweeps re-bin the particles at
 * every checkpoint and every sort_period steps and record each order, and
 * the multipliers are permuted back across each re-binning.  The reverse
 * deposit of the 3-vector G^T le accumulates in int32 shared tiles whose
 * scale comes from a bound on |le| carried from step to step.  FP32 particle
 * and grid arithmetic; J and the final reductions in FP64. */

/* Bytes of the caller-owned device buffer for pic_adjoint_forward/backward. */
int pic_adjoint_buffer_bytes(pic_handle_t h, int n_steps, int checkpoint_every, size_t *bytes);

/* Run n_steps >= 1 steps from the loaded state, storing checkpoints in `buf`
 * (device, >= pic_adjoint_buffer_bytes, 256-byte aligned), and write J to
 * host memory (synchronises).  weights: 3 non-negative finite doubles.
 * Leaves the particles at the state after n_steps - 1 steps.
 * Errors: PIC_ERR_ARG (bad counts or weights, null or misaligned buffer),
 * PIC_ERR_CAPACITY (buffer too small), PIC_ERR_STATE (nothing loaded). */
int pic_adjoint_forward(pic_handle_t h, int n_steps, int checkpoint_every,
                        const double weights[3], void *buf, size_t bytes, double *J);

/* Reverse sweep of the last pic_adjoint_forward (which must be the last call
 * that changed the particles): writes scale * dJ/dx_0 and scale * dJ/dv_0 as
 * FP64 (n, 3) arrays in load order to host (dst_is_device = 0, synchronises)
 * or device memory, then restores the initial state x_0, v_0 (as loaded, up
 * to its FP32 storage) and the step counter. */
int pic_adjoint_backward(pic_handle_t h, double scale, double *dJdx, double *dJdv,
                         int dst_is_device);

/* After pic_adjoint_backward on a run created with PIC_OPT_ADJOINT_PARAMS:
 * grad = scale * (dJ/dB_x, dJ/dB_y, dJ/dB_z, dJ/d(wz2)) on the host.  Each
 * reverse step adds sum_p lv_tot^T (dR/dB_k) vm (R the Boris rotation, vm the
 * velocity after the first half kick, lv_tot the adjoint of the step's new
 * velocity) and sum_p le . Q(y_p) (Q the quadrupole's direction field, le the
 * adjoint of the particle's field); the per-step sums are FP64 over FP32
 * per-thread partials.  Errors: PIC_ERR_STATE (option not set, or no
 * backward pass since the last forward), PIC_ERR_ARG (null grad). */
int pic_adjoint_param_gradient(pic_handle_t h, double grad[4]);

/* sum_i a_i b_i over n FP64 device values, accumulated in FP64 in a fixed
 * order (e.g. dJ/dalpha = <dJ/dx_0, dx_0/dalpha>); result to host memory. */
int pic_dot_f64(pic_handle_t h, const double *a, const double *b, int64_t n, double *out);

/* ------------------------------------------------------------ batched ensembles */

/* Many independent runs of uneven size (not in the paper): every instance is
 * the scheme above on its own periodic grid with its own particles and total
 * charge; all share q/m, dt, external fields and the tuning knobs of
 * pic_params_t.  Each phase of a step (binning, deposit, field solve per
 * grid size, fused gather + push + deposit, diagnostics) is one launch over
 * all instances -- a persistent kernel walks the work items of every
 * instance -- so a whole step of the ensemble can be captured in one CUDA
 * graph.  Memory follows the single-run rules: one caller-owned arena. */
typedef struct pic_batch *pic_batch_t;

typedef struct {
    int32_t n[3];          /* grid nodes per axis (1..1024; n[0] >= 2) */
    double  L[3];          /* box lengths */
    int64_t n_particles;   /* particles of this instance */
    double  total_charge;  /* Q_e of this instance */
} pic_instance_t;

/* Validate and lay out the ensemble (host-only).  Errors: PIC_ERR_ARG. */
int pic_batch_create(const pic_instance_t *inst, int n_inst, double q_over_m,
                     const pic_params_t *params, pic_batch_t *out);
int pic_batch_buffer_sizes(pic_batch_t b, pic_bufsizes_t *out);
int pic_batch_bind_workspace(pic_batch_t b, void *dev_arena, size_t bytes, void *stream);
int pic_batch_set_stream(pic_batch_t b, void *stream);
void pic_batch_destroy(pic_batch_t b);

/* x, v: FP64 (N_total, 3), the instances' particles concatenated in the order
 * of the pic_instance_t array; host (synchronises) or device memory. */
int pic_batch_load_particles(pic_batch_t b, const double *x, const double *v, int src_is_device);

/* n steps of every instance (enqueue only, capturable). */
int pic_batch_step(pic_batch_t b, int n);

/* Up to max_records diagnostic records per instance, oldest first, written
 * as out[record * n_inst + instance]; synchronises. */
int pic_batch_diagnostics(pic_batch_t b, pic_diag_t *out, int max_records, int *n_out);

/* Synchronised (x_n, v_n) of every instance, in the load layout. */
int pic_batch_get_particles(pic_batch_t b, double *x, double *v, int dst_is_device);

/* ------------------------------------------------------------ no allocation */

/* Largest grid accepted by pic_field_energy_noalloc (512^3 nodes). */
#define PIC_NOALLOC_MAX_NODES 134217728LL

/* Field energies and grid charge without any device allocation.
 *
 * The paper has no counterpart: this entry point exists for callers that may
 * not allocate device memory while they run -- e.g. a host application that
 * hands this code a fixed memory budget it manages itself, or a time-critical
 * loop where cudaMalloc (which can synchronise the device, or fail once memory
 * is fragmented) is forbidden.  Such callers cannot bind a workspace arena, so
 * the reduction keeps its scratch (per-block FP64 partials, 256 KiB) in a
 * statically sized __device__ array of the library that every GPU loading the
 * library holds until the process exits.
 *
 * Computes, on the stream (async), into out[0..3] on the device:
 *   Wx, Wy, Wz = cell_volume * sum_g E_d,g^2   and   Q = cell_volume * sum_g rho_g,
 * the same quantities as the diagnostics of pic_step (FP64 sums of FP32 data).
 *   rho    device pointer, n_nodes FP32 values
 *   E      device pointer, n_nodes x 4 FP32 (Ex, Ey, Ez, unused), 16-byte aligned
 *          (the layout pic_get_field returns)
 *   out    device pointer to 4 doubles; the caller owns inputs and outputs
 *   stream cudaStream_t as void*, NULL = legacy default stream
 * Every call looks up the scratch array's device address
 * (cudaGetSymbolAddress, which allocates nothing) on the device that is
 * current, so a device reset between calls is harmless; the first call on
 * each device also loads the library's device code there and does that
 * set-up, so make it before any stream capture.  All calls share the one
 * scratch array, which keeps the last call's partials (every partial a call
 * reads is written by that same call, so nothing needs clearing); calls whose
 * kernels overlap on the GPU race on it and must be ordered by the caller.
 * Allocates nothing: no cudaMalloc, cudaFree or allocating library routine.
 * Errors: PIC_ERR_ARG (null pointer, n_nodes < 1, cell_volume <= 0, E
 * misaligned), PIC_ERR_CAPACITY (n_nodes > PIC_NOALLOC_MAX_NODES),
 * PIC_ERR_CUDA (launch failure); pic_last_error() describes it. */
int pic_field_energy_noalloc(const float *rho, const float *E, int64_t n_nodes,
                             double cell_volume, double *out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* PIC_GB300_PIC_H */
