/*
 * fullwave_gb.h -- C ABI of the GB300 (sm_103a) heterogeneous power-law
 * attenuation FDTD library.
 *
 * Method: Sode & Pinton, "Spatially heterogeneous power-law attenuation with
 * multiple relaxation mechanisms for ultrasound modeling".  The library
 * calibrates N Debye relaxation mechanisms per tissue class on the host
 * (Sec. 3.1-3.2), builds a device-resident medium (Sec. 2.1, Sec. 4.6), and
 * advances the stretched pressure-velocity system on the GPU (Sec. 2.1,
 * Sec. 3.3).
 *
 * Conventions shared by every call
 * --------------------------------
 * - Return value: FW_OK (0) or a negative FW_ERR_* code; no call throws,
 *   aborts or exits.  fw_strerror() names a code.  Errors raised by work
 *   already queued on a stream (non-finite pressure) are sticky on the
 *   medium and reported by fw_status().
 * - Units are SI (m, s, kg/m^3, Pa, m/s); alpha0 is in dB/(MHz^y cm).
 * - Maps are C-order: 3D [nz][ny][nx], 2D [ny][nx]; x is the fastest axis
 *   and the slowest axis is depth.  In 2D the physical directions are x and
 *   the depth axis y.
 * - Pointer arguments documented as "host or device" may point to pageable
 *   or pinned host memory or to device memory of the current device; the
 *   library copies what it needs and never keeps the caller's pointer.
 *   The caller owns every buffer it passes in.
 * - "stream" arguments are cudaStream_t values passed as void* (NULL = the
 *   legacy default stream).  Calls that take a stream are asynchronous with
 *   respect to the host unless stated otherwise.
 * - Device memory of a medium comes from the allocator installed with
 *   fw_set_allocator() (cudaMalloc by default) and is released by
 *   fw_destroy_medium().
 */
#ifndef FULLWAVE_GB_H
#define FULLWAVE_GB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FW_MAX_MECH 4
#define FW_MAX_W 8

/* error codes */
#define FW_OK 0
#define FW_ERR_ARG (-1)         /* invalid argument (sizes, ranges, CFL)      */
#define FW_ERR_CUDA (-2)        /* a CUDA runtime call failed                 */
#define FW_ERR_NOMEM (-3)       /* device or host allocation failed           */
#define FW_ERR_UNSTABLE (-4)    /* non-finite pressure seen by the monitor    */
#define FW_ERR_STATE (-5)       /* call not valid in the medium's state       */
#define FW_ERR_UNSUPPORTED (-6) /* combination not compiled into the library  */
#define FW_ERR_SIZE (-7)        /* size above a fixed limit of the call       */

/* storage of the memory variables psi (fields p, v are FP32 unless F64) */
#define FW_STORE_F32 0   /* FP32 everything                                   */
#define FW_STORE_BF16 1  /* psi in bfloat16, FP32 arithmetic                  */
#define FW_STORE_F16 2   /* psi in binary16, scaled units (see fw_set_sources), FP32 arithmetic */
#define FW_STORE_F64 3   /* FP64 everything: verification build of the kernels */

/* fields for fw_read_field */
#define FW_FIELD_P 0     /* pressure p at integer points                        */
#define FW_FIELD_V 1     /* velocity v_d, idx = d, at i + 1/2 along d           */
#define FW_FIELD_PSI1 2  /* gradient-side memory variable, idx = nu*ndim + d    */
#define FW_FIELD_PSI2 3  /* divergence-side memory variable summed over d, idx = nu */
#define FW_FIELD_PSI1P 4 /* absorbing-layer mechanism, gradient side, idx = d   */
#define FW_FIELD_PSI2P 5 /* absorbing-layer mechanism, divergence side, idx = d */

/* Grid and time step (Sec. 3.3).  The absorbing layer (transition L_T plus
 * absorbing L_B cells) lines every side inside the nx*ny*nz grid; its maps
 * are replaced by the nearest interior values (adaptive PML, Sec. 4.6). */
typedef struct fw_grid {
    int ndim;          /* 2 or 3                                               */
    int nx, ny, nz;    /* points; 2D uses nz = 1                               */
    double dx;         /* grid step [m], > 0                                   */
    double dt;         /* time step [s]; <= 0 selects dt from cfl              */
    double cfl;        /* dt = cfl*dx/max(c/sqrt(kappa1 kappa2)) when dt <= 0  */
    int pml;           /* L_B cells (0: no absorbing layer)                    */
    int transition;    /* L_T cells                                            */
    double f0;         /* centre frequency [Hz] of the absorbing profile       */
    double pml_r0;     /* design reflection of the profile, <= 0 means 1e-5    */
    int layer_relax;   /* 0: the relaxation classes of the absorbing layer are
                        * inherited from the nearest interior cell (the adaptive
                        * layer of Sec. 4.6, the default); 1: the caller's own
                        * class map (or alpha0, y maps) is kept inside the
                        * layer, e.g. one fixed class everywhere in it (the
                        * homogeneous layers of Sec. 4.6).  c, rho and beta
                        * are inherited either way; other values: FW_ERR_ARG */
    int time_order;    /* 2 (or 0): second-order leapfrog with the 8th-order
                        * Taylor staggered weights.  4: the time-space stencil
                        * of Sec. 3.3 (2M = 8th order in space, fourth order
                        * in time, after Tan & Huang, J. Comput. Phys. 276
                        * (2014)): every first derivative along d adds to its
                        * on-axis differences the two-point difference along
                        * d at the +-1 neighbours across each other axis,
                        * with per-cell weights a_m(r), b(r) = r^2/24 from the
                        * cell's Courant number r = c dt / dx, so that the
                        * scheme's plane-wave relation matches omega = c |k|
                        * to those orders.  Stability limit of c_eff dt / dx
                        * about 0.647 (2D), 0.516 (3D), checked at creation.
                        * Other values: FW_ERR_ARG */
} fw_grid;

/* Relaxation parameters of one class (Sec. 2.1): kappa_x1, kappa_x2 and for
 * each mechanism nu d^nu and alpha^nu of both stretches.  2 + 4N values. */
typedef struct fw_relax_params {
    int n_mech;                    /* N, 1..FW_MAX_MECH                        */
    double kappa1, kappa2;
    double d1[FW_MAX_MECH], alpha1[FW_MAX_MECH];
    double d2[FW_MAX_MECH], alpha2[FW_MAX_MECH];
} fw_relax_params;

/* Options of the calibration (Sec. 3.2); fw_fit_default_opts fills the
 * paper's values: 1-20 MHz, 200 log-spaced samples, w in {.1,.3,.5,.7,.9},
 * 5e4 iterations, tolerance 1e-25, reference frequency 1 MHz, c0 1540 m/s. */
typedef struct fw_fit_opts {
    double f_min, f_max;   /* band [Hz]                                        */
    int n_freq;            /* log-spaced samples                               */
    int n_w;               /* number of weights in w[]                         */
    double w[FW_MAX_W];    /* real/imaginary balance weights                   */
    int maxiter;           /* Nelder-Mead iterations                           */
    double xatol, fatol;   /* simplex spread tolerances                        */
    double f_ref;          /* omega_0 / 2 pi of the Kramers-Kronig relation    */
    double c0;             /* phase velocity at f_ref [m/s]                    */
    int n_threads;         /* host threads for the weight sweep, <= 0: all     */
} fw_fit_opts;

typedef struct fw_fit_report {
    double J;          /* objective at the selected weight                     */
    double w;          /* selected weight                                      */
    double nrmse;      /* attenuation NRMSE of the model vs alpha0 f^y         */
    double disp_rmse;  /* phase-velocity RMSE vs Kramers-Kronig [m/s]          */
    int failed;        /* NRMSE > 10 % or dispersion error > 5 m/s (Sec. 3.2)  */
    int n_iter, n_eval;
} fw_fit_report;

typedef struct fw_medium fw_medium;

typedef struct fw_medium_info {
    int ndim, nx, ny, nz, n_mech, storage, n_classes, nonlinear;
    double dx, dt, c_max, ceff_max;
    size_t device_bytes;
    long long step;    /* completed time steps                               */
    int n_src, n_rcv, n_rec;
    int time_order;    /* 2 or 4 (fw_grid.time_order)                       */
} fw_medium_info;

/* ---- calibration (host, FP64) ------------------------------------------- */

/* Fill *opts with the paper's defaults (see fw_fit_opts). */
void fw_fit_default_opts(fw_fit_opts *opts);

/* Calibrate N mechanisms to alpha(f) = alpha0 f^y and its Kramers-Kronig
 * dispersion (Sec. 3.1-3.2, Table 2): adaptive Nelder-Mead on the
 * normalised complex-wavenumber objective for every weight of opts->w, the
 * weight with the lowest attenuation NRMSE kept (dispersion error breaks
 * ties).  alpha0 = 0 returns the lossless set (d = 0, kappa = 1) without
 * fitting.  opts may be NULL (defaults).  Errors: FW_ERR_ARG for n_mech
 * outside 1..4, alpha0 < 0, y outside the paper's valid range [0.4, 2.0]
 * (abstract, Sec. 3.1) when alpha0 > 0, or bad opts.  A poor fit is
 * not an error: rep->failed is set.  rep may be NULL.  Blocking; thread-safe. */
int fw_fit_relaxation(double alpha0, double y, int n_mech, const fw_fit_opts *opts,
                      fw_relax_params *out, fw_fit_report *rep);

/* The objective J(theta) of Sec. 3.2 for one weight w, theta in the Table 2
 * layout [kappa1, kappa2, then per mechanism log10 d1, log10 d2, log10 a1,
 * log10 a2] (2 + 4N doubles).  For inspection and tests. */
int fw_fit_objective(double alpha0, double y, double w, const fw_fit_opts *opts,
                     const double *theta, int n_mech, double *J);

/* The calibration's targets at n frequencies f_hz (host arrays): the
 * power-law attenuation alpha0 f^y in Np/m (Eq. power_law_attenuation,
 * alpha0 in dB/(MHz^y cm)) into alpha, and the phase velocity of its
 * Kramers-Kronig pair (Eq. kk_relation) with c(f_ref) = c0 into c_phase
 * (m/s); |y - 1| < 1e-6 takes the logarithmic limit of the relation.  The
 * same arithmetic as the fit's objective.  Errors: FW_ERR_ARG (alpha0 < 0,
 * c0 or f_ref not positive, a frequency not positive, y outside [0.4, 2.0]
 * when alpha0 > 0, NULL arrays). */
int fw_fit_targets(double alpha0, double y, double c0, double f_ref, const double *f_hz, int n,
                   double *alpha, double *c_phase);

/* Model complex wavenumber of Eq. dispersion_relations for a parameter set
 * and medium speed c at n frequencies f_hz: writes Re k and Im k (attenuation
 * is -Im k).  Host arrays of n doubles. */
int fw_model_wavenumber(const fw_relax_params *p, double c, const double *f_hz, int n,
                        double *k_re, double *k_im);

/* Adaptive bounded Nelder-Mead used by the calibration (Gao & Han
 * coefficients, bounds by clipping), exposed for reuse: minimises f over n
 * variables starting from x (overwritten with the minimiser).  lo/hi may be
 * NULL (unbounded).  fmin, n_iter, n_eval may be NULL. */
int fw_nelder_mead(int n, double *x, const double *lo, const double *hi,
                   double (*f)(const double *x, void *ctx), void *ctx,
                   int maxiter, double xatol, double fatol,
                   double *fmin, int *n_iter, int *n_eval);

/* ---- media ------------------------------------------------------------- */

/* Install the device allocator used for every later medium (NULL, NULL
 * restores cudaMalloc/cudaFree).  alloc returns NULL on failure. */
void fw_set_allocator(void *(*alloc)(size_t bytes, void *ctx),
                      void (*release)(void *ptr, void *ctx), void *ctx);

/* Device bytes a medium of this grid needs (state, maps, tables; not the
 * source/receiver buffers): the fields and memory variables of Sec. 2.1
 * (Eqs. wave1, wave2, relaxation4), the absorbing-layer memory of Sec. 4.6
 * and the per-voxel maps.  For admission control.  Errors: FW_ERR_ARG. */
int fw_medium_bytes(const fw_grid *g, int n_mech, int storage, int nonlinear, size_t *bytes);

/* Build a medium from per-voxel maps (Sec. 2.1, Sec. 4.6): every distinct
 * (alpha0, y) pair becomes a class calibrated with fw_fit_relaxation (on
 * host threads, one job per class and weight); the class's reference speed
 * c0 is opts->c0 when opts is given with c0 > 0, else the mean c of the
 * class's voxels.  c, rho, alpha0, y: host or device float arrays of
 * nx*ny*nz values; beta may be NULL (linear).  The rest is as in
 * fw_create_medium_classes.
 * Errors: FW_ERR_ARG (non-positive c or rho, y outside the valid range
 * [0.4, 2.0] (abstract, Sec. 3.1) where alpha0 > 0, more than 65535 classes, CFL above the stability limit),
 * FW_ERR_NOMEM, FW_ERR_CUDA.  Blocking (returns when the medium is ready). */
int fw_create_medium(const fw_grid *g, const float *c, const float *rho, const float *beta,
                     const float *alpha0, const float *y, int n_mech, int storage,
                     const fw_fit_opts *opts, void *stream, fw_medium **out);

/* Build a medium from a class map and a class table: class_idx (uint16,
 * host or device, nx*ny*nz) indexes classes[0..n_classes-1], all with the
 * same n_mech.  Per-voxel c, rho, beta as above.  A velocity point v_d[i]
 * (at i+1/2 along d) uses the class of cell i.  The stability limit on
 * c_eff*dt/dx is 1/(sqrt(D) sum|c_m|) = 0.5497 (2D), 0.4488 (3D) for the
 * leapfrog; for the time-space stencil (time_order 4) creation requires
 * (c_eff,max dt/dx) max_theta |K(theta; r)| dx/2 <= 1 for the weights of the
 * smallest and of the largest r = c dt/dx of the map.  Blocking. */
int fw_create_medium_classes(const fw_grid *g, const float *c, const float *rho,
                             const float *beta, const uint16_t *class_idx,
                             const fw_relax_params *classes, int n_classes, int storage,
                             void *stream, fw_medium **out);

/* Sources (the volume source of the simulation protocol, Sec. 4.1: an
 * additive source on p, one step of the pressure update's K dt per unit
 * volume rate, Eq. wave2): mask (host, uint8, nx*ny*nz)
 * selects cells in C order; waveforms (host, n_wave x n_steps floats, volume
 * rate [m^D/s]); wave_of_src (host, one int per source in mask order) picks
 * a waveform row, or NULL: one shared row (n_wave = 1) or one row per source
 * (n_wave = n_src).  Time step `it` adds dt*K/dx^D * waveform[it] after the
 * pressure update (nothing once it >= n_steps).  Replaces earlier sources.
 * FW_STORE_F16 media keep the memory variables in scaled units, psi1 dx /
 * p_ref and psi2 dx Z / p_ref (Z = 1.54e6 kg/(m^2 s)), so that those of
 * fields within about 1e-4..1e4 times p_ref stay in the normal range of
 * binary16; this call sets p_ref to 1/100 of the largest pressure increment
 * one step of the sources adds (10 Pa before any source) and rescales what
 * the memory variables already hold. */
int fw_set_sources(fw_medium *m, const uint8_t *mask, const float *waveforms, int n_wave,
                   int n_steps, const int32_t *wave_of_src);

/* Receivers (the pressure traces the measurements of Sec. 4.1-4.3 are
 * taken from): mask (host, uint8) selects cells in C order; time step `it`
 * records p after the source into column it/decim when it % decim == 0, for
 * it < n_steps.  Traces are [n_rcv][ceil(n_steps/decim)] and are zeroed. */
int fw_set_receivers(fw_medium *m, const uint8_t *mask, int decim, int n_steps);

/* Advance n_steps time steps on stream with plain kernel launches: one step
 * is the velocity half step (Eqs. wave1, relaxation4, relaxation_psi on the
 * gradient side), the pressure half step (Eqs. wave2, relaxation4,
 * relaxation_psi on the divergence side; absorbing mechanism of Sec. 2.1 /
 * Sec. 4.6), then sources and receivers, on the staggered grid of Sec. 3.3.
 * Errors: FW_ERR_ARG, FW_ERR_CUDA, or the medium's sticky error. */
int fw_step(fw_medium *m, int n_steps, void *stream);

/* Advance n_steps time steps (the same step as fw_step, Sec. 2.1 / 3.3) on
 * stream through cached CUDA graphs of fixed step chunks (the fast path;
 * bitwise the same results as fw_step).  Errors as fw_step. */
int fw_run(fw_medium *m, int n_steps, void *stream);

/* fw_step with a CUDA event around each sweep: advances n_steps on stream
 * (plain launches), waits for them, and returns the summed device time [ms]
 * of the velocity sweeps, the pressure sweeps and the source/receiver
 * kernels, the device time from the first launch to the last, and the number
 * of kernels launched.  Output pointers may be NULL.  For measurement;
 * results equal fw_step's. */
int fw_step_timed(fw_medium *m, int n_steps, void *stream, double *ms_velocity, double *ms_pressure,
                  double *ms_io, double *ms_total, int *n_launches);

/* Replace waveform samples [it0, it0+n) of every waveform row from samples
 * (n_wave x n floats, host or device; pinned host memory keeps the copy
 * asynchronous).  Ordered on stream.  FP32 and 16-bit media only
 * (FW_ERR_UNSUPPORTED for FW_STORE_F64).  For streaming inputs step by step. */
int fw_set_waveform_samples(fw_medium *m, int it0, int n, const float *samples, void *stream);

/* Copy trace columns [col0, col0+ncol) of every receiver to dst
 * (n_rcv x ncol, host or device, in the medium's field type: float, double
 * for FW_STORE_F64).  Ordered on stream; asynchronous for pinned or device
 * dst.  For streaming results step by step. */
int fw_read_receivers_range(fw_medium *m, int col0, int ncol, void *dst, void *stream);

/* Copy a field of the state of Sec. 2.1 (p, v_d, the memory variables psi of
 * Eq. relaxation4, the absorbing-layer memory) to dst (host or device),
 * unpadded C order, as float (as_f64 = 0) or double (as_f64 = 1); 16-bit
 * memory variables come back in the units of the FP32 ones.  Ordered on
 * stream; blocking.  Device memory: one staging buffer of the field's size
 * from the installed allocator.  Errors: FW_ERR_ARG (field, idx, pointer),
 * FW_ERR_NOMEM, FW_ERR_CUDA. */
int fw_read_field(fw_medium *m, int which, int idx, void *dst, int as_f64, void *stream);

/* fw_read_field without any device allocation.  No counterpart in the
 * paper: this is a service of the library for callers that cannot allocate
 * device memory when they read results, e.g. a process whose device memory
 * is all handed out by another framework's caching allocator, a real-time
 * loop with a memory budget fixed at start-up, or code that must not let
 * cudaMalloc/cudaFree synchronise the device.
 * Same arguments, layout and result as fw_read_field, but the copy is staged
 * in one device array of FW_NOALLOC_MAX_BYTES bytes that the library defines
 * at file scope, and no call allocates or frees device memory.  CUDA loads
 * device code lazily, so the array takes its device memory when the library
 * first looks up its address on a device: every fw_create_medium* does that
 * for the medium's device before it returns, so the array is resident from
 * the first medium on (before the caller hands the rest of the device to a
 * pool) and stays until the process exits.
 * - Limit: nx*ny*nz*(as_f64 ? 8 : 4) <= FW_NOALLOC_MAX_BYTES (64 MiB, e.g.
 *   a 256^3 float field), else FW_ERR_SIZE and nothing is copied.
 * - The address lookup happens outside any stream capture (at medium
 *   creation); should it have failed there, the first call on the device
 *   repeats it, so make that call before any capture.  The medium's device
 *   must be current.
 * - All calls share the one array and it keeps the last call's contents:
 *   calls whose work overlaps on the GPU (other streams, other host threads)
 *   race on it and must be ordered by the caller.  Blocking, like
 *   fw_read_field.
 * Errors: FW_ERR_ARG (bad field or pointer), FW_ERR_SIZE, FW_ERR_CUDA. */
#define FW_NOALLOC_MAX_BYTES (64u << 20)
int fw_read_field_noalloc(fw_medium *m, int which, int idx, void *dst, int as_f64, void *stream);

/* Write a field from src (host or device, same layout/type rules).  For
 * initial conditions and tests.  Blocking. */
int fw_write_field(fw_medium *m, int which, int idx, const void *src, int as_f64, void *stream);

/* Copy the receiver traces [n_rcv][n_rec] to dst (host or device) as float
 * or double.  Blocking. */
int fw_read_receivers(fw_medium *m, void *dst, int as_f64, void *stream);

/* Full state (every field, memory variable, step counter) as an opaque
 * byte image for checkpoint/resume: fw_state_bytes gives its size,
 * fw_save_state copies it to dst, fw_load_state restores it (host or
 * device buffers).  Blocking.  Resuming is bit-exact. */
int fw_state_bytes(fw_medium *m, size_t *bytes);
int fw_save_state(fw_medium *m, void *dst, void *stream);
int fw_load_state(fw_medium *m, const void *src, void *stream);

/* Gradient of a receiver functional with respect to the sound-speed map
 * c(x) and the attenuation map alpha0(x), by the discrete adjoint of the
 * time step (the transpose of the velocity and pressure sweeps of Sec. 2.1
 * with the discretisation of Sec. 3.3); the paper names inverse problems as
 * the use of the forward model but prints no gradient method.
 * Runs n_steps forward from the medium's current state exactly as fw_run
 * (traces recorded, the medium ends n_steps later), keeping a state image
 * every checkpoint_every steps (<= 0: sqrt(n_steps)), then runs the adjoint
 * backwards, recomputing each segment's states from its checkpoint, and
 * returns dL/dc and dL/dalpha0 for
 *     L = sum_{r, col} G[r][col] * trace[r][col],
 * G = dL/dtraces, [n_rcv][n_rec] (e.g. trace - d_obs for the misfit
 * 1/2 |trace - d_obs|^2); columns not recorded in this window do not count.
 * Readings: c enters through K dt = rho c^2 dt (update and source gain);
 * dt, the absorbing profile and the class relaxation sets stay fixed;
 * alpha0 scales the d of the voxel's class, d^nu(x) = d^nu_class alpha0(x) /
 * alpha0_class, kappa and alpha^nu fixed, so dL/dalpha0 = dL/ds / alpha0
 * with s that factor; the absorbing layer's inherited maps fold back onto
 * the cells they copy.  The state at the start of the window is held fixed.
 * alpha0: the medium's alpha0 map [nx*ny*nz] (host or device), or NULL: then
 * grad_alpha0 receives dL/ds.  G, alpha0, grad_c, grad_alpha0 are float
 * (as_f64 = 0) or double (as_f64 = 1), C order, host or device; grad_c or
 * grad_alpha0 may be NULL.  Device memory: ceil(n_steps/K) + 2(K - 1) + 3
 * state images (about fw_state_bytes each; 2D), or ceil(n_steps/K) +
 * 2(K - 1) + 2 state images and 6 fields (3D), plus 4 FP64 maps and the two
 * output maps, from the installed allocator, released before return.  The
 * recomputation of one segment runs on a stream of its own beside the
 * adjoint of the next.  Blocking.
 * Errors: FW_ERR_ARG, FW_ERR_UNSUPPORTED (nonlinear media, 16-bit storage, the
 * time-space stencil (time_order 4), more than 65535 points along either of
 * the two slower axes),
 * FW_ERR_NOMEM, FW_ERR_CUDA, or the medium's sticky error. */
int fw_gradient(fw_medium *m, int n_steps, int checkpoint_every, const void *G, const void *alpha0,
                void *grad_c, void *grad_alpha0, int as_f64, void *stream);

/* Stability monitor (the divergence of long runs counted in Sec. 4.6 and
 * Sec. 5.5: non-finite pressure): synchronises the
 * medium's last stream and returns FW_OK or FW_ERR_UNSTABLE (sticky);
 * max_abs_p (may be NULL) receives max |p| seen since creation. */
int fw_status(fw_medium *m, float *max_abs_p);

int fw_medium_get_info(fw_medium *m, fw_medium_info *info);

/* Release the medium and all its device memory (NULL is ignored). */
void fw_destroy_medium(fw_medium *m);

/* ---- serving: continuous batching of simulation requests ---------------
 * No counterpart in the paper (it runs one simulation at a time).  A server
 * owns one device arena of opts.hbm_budget bytes and a scheduler thread.
 * Requests queue in arrival order; one is admitted as soon as a slot is free
 * and its footprint (fw_medium_bytes plus source/receiver buffers and the
 * upload staging) fits in what the arena has left (first fit in the order of
 * opts.policy; a queued request skipped FW_SERVER_MAX_SKIPS times blocks the
 * ones of its class behind it until it fits).  Admitted media are built by a
 * worker thread from the request's maps, stay resident on the device, and
 * advance in chunks of opts.chunk_steps steps through their cached CUDA
 * graphs (fw_run), each request on a stream of a pool, at most two chunks in
 * flight per request, so the work of all admitted requests overlaps on the
 * GPU: each chunk enqueues the request's tiles (the CTAs of its sweeps) and
 * the block scheduler serves the tiles of higher-priority streams first
 * (opts.policy).  A finished request's traces are copied to its traces_out, its
 * medium is released into the arena, and the next request is admitted.
 * Kernels are deterministic: a request's result does not depend on what
 * else is admitted.  Times are seconds on the server's clock (fw_server_now).
 * FWGB_SERVER_DEBUG=1 in the environment logs builds and failed chunks to
 * stderr. */
#define FW_SERVER_MAX_SKIPS 8
#define FW_CANCELLED (-8)        /* completion status of a cancelled request */

typedef struct fw_server fw_server;

typedef struct fw_server_opts {
    size_t hbm_budget;   /* device arena [bytes]; requests larger are refused (FW_ERR_NOMEM) */
    int max_active;      /* admitted requests at once (slots), >= 1                           */
    int chunk_steps;     /* time steps per scheduling quantum, >= 1 (32 = one cached graph)   */
    int n_streams;       /* device streams per priority level, >= 1                           */
    int policy;          /* 0: size classes (default): requests with voxels x steps <=
                          * short_work are admitted ahead of the others and run on the
                          * highest-priority streams; long requests are admitted in
                          * arrival order, keep two slots free for short ones (when
                          * max_active >= 4), and the oldest running one runs at a middle
                          * priority above the other long ones.  1: arrival order, one
                          * priority for all.  Other values: FW_ERR_ARG                      */
    double short_work;   /* voxel-steps bound of a short request; <= 0: 5e9                   */
} fw_server_opts;

/* One simulation request.  Every pointer must stay valid until the request
 * completes (its completion record has been returned by fw_server_poll).
 * Maps and masks as for fw_create_medium_classes / fw_set_sources /
 * fw_set_receivers; traces_out (host or device, float, [n_rcv][n_rec],
 * n_rec = ceil(n_steps / decim)) receives the traces at completion. */
typedef struct fw_request {
    fw_grid grid;
    const float *c, *rho, *beta;
    const uint16_t *class_idx;
    const fw_relax_params *classes;
    int n_classes;
    int storage;                 /* FW_STORE_F32, BF16 or F16                      */
    const uint8_t *src_mask;
    const float *waveforms;
    int n_wave;
    const int32_t *wave_of;
    const uint8_t *rcv_mask;
    int decim;
    int n_steps;
    float *traces_out;
    long long tag;               /* caller's label, returned in the completion      */
} fw_request;

typedef struct fw_completion {
    long long id, tag;
    int status;                  /* FW_OK, FW_ERR_UNSTABLE, FW_CANCELLED, or the error of
                                    building the medium (FW_ERR_ARG, FW_ERR_NOMEM, ...)  */
    double t_submit, t_admit, t_done;   /* server clock [s]; t_admit < 0 if never admitted */
    long long voxel_steps;       /* voxels x steps advanced                               */
    float max_abs_p;
} fw_completion;

typedef struct fw_server_stats {
    int queued, building, active, done;
    size_t bytes_reserved, bytes_budget, bytes_largest_free;
} fw_server_stats;

/* Create a server on the current device (its arena is allocated here with
 * cudaMalloc).  Errors: FW_ERR_ARG, FW_ERR_NOMEM, FW_ERR_CUDA. */
int fw_server_create(const fw_server_opts *opts, fw_server **out);

/* Queue a request; *id (may be NULL) receives its id.  Never blocks on the
 * GPU.  A request whose footprint exceeds the whole budget completes at once
 * with FW_ERR_NOMEM.  Errors: FW_ERR_ARG (bad request fields). */
int fw_server_submit(fw_server *s, const fw_request *req, long long *id);

/* Wait up to timeout_s seconds (0: do not wait) for completions and copy up
 * to max of them into out; *n receives how many.  Each completion is
 * returned once. */
int fw_server_poll(fw_server *s, fw_completion *out, int max, int *n, double timeout_s);

/* Cancel a queued or running request (it completes with FW_CANCELLED after
 * its in-flight chunks end).  FW_ERR_ARG if the id is unknown or done. */
int fw_server_cancel(fw_server *s, long long id);

int fw_server_stats_get(fw_server *s, fw_server_stats *st);

/* Seconds on the server's clock (zero at creation). */
double fw_server_now(fw_server *s);

/* Cancel what is queued, let running requests end their in-flight chunks,
 * release everything.  NULL is ignored. */
void fw_server_destroy(fw_server *s);

const char *fw_strerror(int code);

/* Library version: major*10000 + minor*100 + patch. */
int fw_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FULLWAVE_GB_H */
