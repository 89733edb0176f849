/*
 * ch_flow.h - C ABI of the GB300 pseudo-spectral channel solver.
 *
 * The library advances the coupled incompressible Navier-Stokes + Cahn-Hilliard (phase-field)
 * equations in a plane channel, x, y periodic, walls at z = +-1, exactly as stated in Roccon,
 * "A GPU-ready pseudo-spectral method for direct numerical simulations of multiphase turbulence"
 * (arXiv:2406.01322):
 *   - Sec. 2.1.1, Eq. (CHE) and the chemical potential: Cahn-Hilliard with mobility 1/Pe;
 *   - Sec. 2.1.2, Eqs. (cont), (NSE), (kort): NS with the Korteweg capillary stress;
 *   - Sec. 2.2, Eqs. (omegaz), (ww), (omegadef), (phisplit): wall-normal velocity-vorticity
 *     formulation, split CH operator, Fourier x Fourier x Chebyshev discretisation (3/2 rule in
 *     x and y), AB2 on non-linear terms, Crank-Nicolson on NS linear terms, implicit Euler on CH
 *     linear terms, step sequence i)-v);
 *   - Sec. 3.2.1: Chebyshev transform as a DCT-I; Sec. 3.2.2: batched tridiagonal (tau)
 *     Helmholtz solves per (kx, ky).
 * Every step of the time step runs in this library's own sm_103a CUDA kernels.
 *
 * Conventions
 *   Physical fields: float64, C order (nz, ny, nx), x_i = i lx/nx, y_j = j ly/ny,
 *     z_k = cos(pi k/(nz-1)) (k = 0 is the top wall z = +1).
 *   Spectral fields: complex float64 stored as interleaved (re, im) pairs, layout
 *     [mx][j][n] (n fastest): mx = 0..nx/2-1, j = 0..ny-1 in FFT order (my = j for j < ny/2,
 *     my = j - ny for j > ny/2; j = ny/2 is the y Nyquist row and is kept zero),
 *     n = 0..nz-1 the Chebyshev index.  Coefficient of T_n(z) exp(i(kx x + ky y)) with
 *     kx = 2 pi mx / lx, ky = 2 pi my / ly; forward transforms are normalised by 1/(nx ny).
 *   Pointers: every field pointer passed to a ch_* call is DEVICE memory of the current CUDA
 *     device unless the function name ends in _host (then it is host memory, pinned or not).
 *     The caller owns every buffer it passes; the library owns its internal buffers, obtained
 *     through the allocator callbacks given to ch_init_grid (cudaMalloc when they are NULL).
 *   Streams: all work is enqueued on the stream given to ch_init_grid (or ch_set_stream);
 *     calls return once the work is enqueued unless stated otherwise.
 *   Errors: every call returns CH_OK (0) or a negative CH_ERR_* code; no exception or abort
 *     crosses the ABI.  A handle is not thread-safe; use one handle per stream.
 */
#ifndef CH_FLOW_H
#define CH_FLOW_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CH_OK 0
#define CH_ERR_ARG (-1)      /* null pointer, non-positive dt, bad enum value            */
#define CH_ERR_SIZE (-2)     /* nx, ny not even and {2,3}-smooth, nz-1 not {2,3}-smooth   */
#define CH_ERR_ALLOC (-3)    /* allocator callback or cudaMalloc returned NULL / failed   */
#define CH_ERR_CUDA (-4)     /* a CUDA runtime call or kernel launch failed               */
#define CH_ERR_DIVERGED (-5) /* diagnostics found NaN/Inf                                 */
#define CH_ERR_TIMEOUT (-6)  /* a bounded device-side wait gave up                        */
#define CH_ERR_STATE (-7)    /* call out of order, e.g. ch_step before ch_set_fields      */

#define CH_PREC_FP64 0  /* every stage in float64                                         */
#define CH_PREC_MIXED 1 /* x/y transforms and physical-space products in float32; the
                           Chebyshev transform, tau solves, state and mass stay float64      */
#define CH_PREC_DFLOAT 2 /* x/y transforms and physical-space products in double-float (the
                           unevaluated sum of two floats, ~48-bit significand, on the float32
                           pipe); the rest as in CH_PREC_FP64.  Not a precision of the paper:
                           an FP64-accurate variant for GPUs whose float64 rate is low       */

typedef struct ch_grid ch_grid; /* opaque, owned by the library */

typedef struct {
  int nx, ny, nz;     /* collocation points; nx, ny even with nx/2, ny/2 and 3nx/2, 3ny/2
                         {2,3}-smooth (radix 2, 3, 4 FFTs); nz - 1 even, {2,3}-smooth, >= 4 */
  double lx, ly;      /* box lengths in x, y (walls at z = +-1, half height h = 1)           */
  double re_tau;      /* friction Reynolds number, Eq. (Re)                                */
  double we;          /* Weber number, Eq. (We)                                            */
  double ch;          /* Cahn number (interface thickness)                                 */
  double pe;          /* Peclet number                                                     */
  double dt;          /* time step (> 0)                                                   */
  double gx, gy;      /* mean pressure gradient -dp/dx, -dp/dy driving the mean flow       */
  int precision;      /* CH_PREC_FP64, CH_PREC_MIXED or CH_PREC_DFLOAT                      */
  int dealias_z;      /* must be 0: no padding of the Chebyshev direction                  */
  int bc;             /* walls (Sec. 2.1: no-slip, free-slip or a combination): 0 no-slip
                         (u = v = w = dw/dz = 0) at both walls, 1 free-slip (du/dz = dv/dz = 0,
                         w = 0, d2w/dz2 = 0) at both, 2 no-slip at z = -1 and free-slip at
                         z = +1, 3 free-slip at z = -1 and no-slip at z = +1; phi no-flux at
                         both.  Other values: CH_ERR_ARG                                  */
} ch_params;

typedef void* (*ch_alloc_fn)(size_t bytes, void* ctx);
typedef void (*ch_free_fn)(void* ptr, void* ctx);

typedef struct {
  double t;           /* simulated time                                                    */
  long long step;     /* number of steps taken since ch_set_fields / ch_set_state          */
  double mass;        /* integral of phi, exact Clenshaw-Curtis sum of its (0,0) line      */
  double kinetic;     /* 1/2 integral |u|^2 (uniform x,y weights, Clenshaw-Curtis in z)    */
  double grad2;       /* integral |grad phi|^2 (interfacial area measure)                  */
  double free_energy; /* integral 1/4 (phi^2-1)^2 + Ch^2/2 |grad phi|^2, Sec. 2.1.1         */
  double cfl;         /* dt max(|u|/dx + |v|/dy + |w|/dz_k)                                */
  double max_phi;     /* max |phi| on the grid                                             */
  int nan;            /* 1 if any u, v, w, phi sample is NaN or Inf                        */
} ch_diag;

/* Create a solver for one channel.  Validates sizes (CH_ERR_SIZE) and parameters (CH_ERR_ARG),
 * allocates every internal buffer through alloc/free (or cudaMalloc/cudaFree when alloc is
 * NULL), builds FFT plans and twiddle tables.  stream is a cudaStream_t (NULL = default
 * stream).  On success *out receives the handle.  Synchronous. */
int ch_init_grid(const ch_params* p, ch_alloc_fn alloc, ch_free_fn free_fn, void* alloc_ctx,
                 void* stream, ch_grid** out);

/* Replace the stream used by every later call. */
int ch_set_stream(ch_grid* g, void* stream);

/* Step i) of Sec. 2.2: physical u, v, w, phi (device, (nz,ny,nx) float64) -> spectral state
 * (omega_z = dv/dx - du/dy, w, mean flow, phi; Eq. (omegadef)).  Modes that the grid cannot hold
 * (x and y Nyquist) are dropped and a non-solenoidal velocity is projected.  Resets the
 * Adams-Bashforth history (the next step is forward Euler on the non-linear terms), t and step,
 * and evaluates the non-linear terms of the new state. */
int ch_set_fields(ch_grid* g, const double* u, const double* v, const double* w, const double* phi);

/* As ch_set_fields with HOST input arrays (copied to the device on the handle's stream). */
int ch_set_fields_host(ch_grid* g, const double* u, const double* v, const double* w,
                       const double* phi);

/* Advance nsteps full time steps (Sec. 2.2 steps i)-v)), asynchronously on the stream.  After
 * the first step the per-step launch sequence is replayed from a captured CUDA graph. */
int ch_step(ch_grid* g, int nsteps);

/* The kernels of one time step in the order ch_step_timed reports them in: zrhs (DCT,
 * assembly, AB2, right-hand sides), zsolve (tau solves), zbwd (update, velocity, backward DCT),
 * y backward, x line, y forward, then the two Chebyshev transforms on the tensor cores
 * (forward of the nine products before zrhs, backward of the five fields after zbwd), which run
 * only under CH_CHEB_TC (zero time otherwise; zrhs and zbwd then skip their DCTs). */
#define CH_STEP_KERNELS 8

/* Method of the Chebyshev transforms (Sec. 3.2.1) inside the step:
 * CH_CHEB_FFT: DCT-I through one N-point complex FFT per line, in float64, fused into zrhs/zbwd
 *   (the default);
 * CH_CHEB_TC: the transform as a product with the fixed Nz x Nz Chebyshev matrix on the tensor
 *   cores, float64-accurate by an exact split of both operands into eight signed 7-bit digits
 *   (bf16, Ozaki scheme; fp32 accumulation is exact for these integers) and a recombination in
 *   64-bit integers; error a few units of 2^-53 of max|row| x max_n sum_k |B_nk| per line, the
 *   accuracy of a float64 transform.  Two extra launches per step and a 9-field float64 coefficient buffer.
 *   Single grids (any precision) with nz <= 496; not with the adjoint. */
#define CH_CHEB_FFT 0
#define CH_CHEB_TC 1

/* Select the step's Chebyshev method; allocates the tensor-core tables and buffer on the first
 * CH_CHEB_TC (synchronous).  CH_ERR_ARG: bad method; CH_ERR_STATE: a reverse sweep is open;
 * CH_ERR_SIZE: nz > 496.
 * The captured step graph is rebuilt at the next ch_step. */
int ch_set_chebyshev(ch_grid* g, int method);
int ch_get_chebyshev(const ch_grid* g);

/* Pruned transforms of the 3/2-rule padding (Sec. 3.2.1; the NEXT item "pruned padded FFTs"):
 * on = 1 gives the x and y transforms of the step a schedule that starts with radix 3, so the
 * backward (zero-padded) transforms skip the zero middle third of their input in their first
 * pass and the forward (truncated) ones skip the unused middle third of their output in their
 * last pass; on = 0 restores the default schedules.  The result equals the unpruned step to
 * rounding.  Synchronous; takes effect at the next step (the step graph is rebuilt).
 * CH_ERR_ARG: on not 0 or 1; CH_ERR_STATE: a reverse sweep is open. */
int ch_set_fft_pruning(ch_grid* g, int on);
int ch_get_fft_pruning(const ch_grid* g);

/* Chebyshev transform along z of nf fields of complex lines (device, float64 (re, im) pairs,
 * layout [field][mx * ny + j][n], field stride (nx/2) ny nz, the layout of ch_get_spectral) with
 * the selected method: dir 0 samples at z_k = cos(pi k / N) -> coefficients a_n, dir 1 the
 * inverse.  in and out must not overlap.  Asynchronous on the handle's stream. */
int ch_chebyshev_lines(ch_grid* g, int dir, const double* in, double* out, int nf);

/* Synchronise the handle's stream; CH_ERR_TIMEOUT (and the flag cleared) if a bounded device
 * wait of the tensor-core kernels gave up since the last check (its outputs are then invalid),
 * else CH_OK.  ch_diagnostics reports the same condition. */
int ch_device_status(ch_grid* g);

/* Test of the failure path of the bounded device waits (not in the paper; library
 * infrastructure): one thread runs a loop of nwaits (>= 1) waits, with the tensor-core
 * transform's wait helper, on mbarrier phases that nothing completes.  The first wait gives up
 * after its bound (about one second); every later wait of the loop returns at once (the helper
 * short-circuits after a failure), so the kernel ends after about one bound whatever nwaits is.
 * The failure is recorded in device memory and the kernel returns: expected result
 * CH_ERR_TIMEOUT, with the CUDA context still usable (no fault, trap or hang), and *spun (if not
 * NULL) = the number of waits that actually waited, 1.  Synchronous, on the legacy default
 * stream; CH_ERR_ARG for nwaits < 1, CH_ERR_ALLOC / CH_ERR_CUDA if the test itself cannot run,
 * CH_OK if the waits completed. */
int ch_selftest_bounded_wait(int nwaits, int* spun);

/* Measured float64 FMA rate of the current device (not in the paper; the denominator behind
 * the float64 kernels' ALU roofline): a kernel of independent fused multiply-add chains (eight
 * per thread; 16 CTAs of 8 warps per SM, two waves) timed with CUDA events after one warm-up
 * launch;
 * *tflops = 2 flops per FMA / time.  Synchronous, on the legacy default stream; allocates a
 * small device buffer (the chains' results, so the compiler keeps them).  CH_ERR_ARG for a NULL
 * pointer, CH_ERR_ALLOC / CH_ERR_CUDA if it cannot run. */
int ch_fp64_fma_rate(double* tflops);

/* As ch_step, but launched without the graph and bracketed by CUDA events on the stream: on
 * return (the stream is synchronised) kernel_ms[0..CH_STEP_KERNELS-1] hold the summed device
 * time of each of the step's kernels and *total_ms the time from the first launch to the end of
 * the last.  kernel_ms may be NULL.  Used by the benchmark to attribute step time. */
int ch_step_timed(ch_grid* g, int nsteps, double* kernel_ms, double* total_ms);

/* Number of kernel launches one ch_step makes per time step. */
int ch_launches_per_step(const ch_grid* g);

/* Spectral state -> physical u, v, w, phi (device, (nz,ny,nx) float64) on the unpadded grid. */
int ch_get_fields(ch_grid* g, double* u, double* v, double* w, double* phi);

/* As ch_get_fields into HOST arrays; synchronises the stream before returning. */
int ch_get_fields_host(ch_grid* g, double* u, double* v, double* w, double* phi);

/* Diagnostics of the current state (fills *out, synchronises the stream).  Returns
 * CH_ERR_DIVERGED when NaN/Inf is found (out->nan = 1). */
int ch_diagnostics(ch_grid* g, ch_diag* out);

/* Bytes of the checkpoint written by ch_get_state: spectral state, Adams-Bashforth history,
 * time, step count and start flag.  Restoring it with ch_set_state resumes bit-for-bit. */
size_t ch_state_bytes(const ch_grid* g);
int ch_get_state(ch_grid* g, void* dev_buf);
int ch_set_state(ch_grid* g, const void* dev_buf);

/* Spectral state (device, complex float64, layout above): omega_z (its (0,0) line holds
 * ubar + i vbar), w, phi.  Any pointer may be NULL to skip that field. */
int ch_get_spectral(ch_grid* g, double* omega, double* w, double* phi);
int ch_set_spectral(ch_grid* g, const double* omega, const double* w, const double* phi);

/* Stage-level entry points (used by the parity tests; each runs the same kernels as ch_step).
 *
 * ch_transform_forward: physical (nz,ny,nx) float64 -> spectral coefficients (layout above),
 *   Fourier in x and y (1/(nx ny)) then the Chebyshev DCT-I (Sec. 3.2.1).
 * ch_transform_backward: the inverse, evaluated on the unpadded grid.
 * ch_nonlinear: the nine non-linear coefficient arrays of the current state the step uses, in
 *   the order Sxx - Szz, Syy - Szz, Sxy, Sxz, Syz (Sigma_ij = -u_i u_j + kappa T_ij, Eq. (kort);
 *   the isotropic part Szz delta_ij is a gradient and does not enter Eqs. (omegaz), (ww)), phi^3,
 *   u phi, v phi, w phi, formed on the 3/2-padded grid and returned as complex float64
 *   coefficients (9 consecutive spectral fields) - steps ii) and vi) of Sec. 2.2. */
int ch_transform_forward(ch_grid* g, const double* phys, double* spec);
int ch_transform_backward(ch_grid* g, const double* spec, double* phys);
int ch_nonlinear(ch_grid* g, double* out9);

/* ---- Discrete adjoint (float64 grids) ---------------------------------------------------------
 * Reverse-mode derivative of the discrete step map (Sec. 2.2, steps i)-v); not in the paper: a
 * service of this library for optimisation / sensitivity studies) for the objective of the
 * final state
 *   J = 1/2 int |u|^2 dV + int |grad phi|^2 dV   (exact integrals of the interpolants)
 * with respect to the physical initial fields u, v, w, phi given to ch_set_fields.
 * ch_objective: J of the current state (host double; synchronises the stream).
 * ch_adjoint_begin: allocates the reverse-sweep workspace (24 spectral fields plus six y-padded
 *   fields, with the grid's allocator) and seeds the sweep with dJ/ds of the CURRENT state (the
 *   final state of the forward run); *J receives J (may be NULL).
 * ch_adjoint_step: reverses ONE forward step.  `state` is a device buffer written by
 *   ch_get_state just before that forward step; steps are reversed last to first.  The handle's
 *   state becomes the saved one but its non-linear terms are not recomputed: ch_step,
 *   ch_step_timed and ch_nonlinear answer CH_ERR_STATE until ch_set_state / ch_set_fields /
 *   ch_set_spectral.
 * ch_adjoint_gradient: after the step reversed last (the first forward step), writes
 *   dJ/du0, dJ/dv0, dJ/dw0, dJ/dphi0 into four device (nz,ny,nx) float64 arrays.
 * ch_adjoint_end: frees the workspace (ch_destroy does too).
 * Mixed-precision, double-float, free-slip and CH_CHEB_TC grids: CH_ERR_ARG.  Grids whose padded
 * x length Px = 3 nx / 2 exceeds 602 (the transposed x line keeps 24 lines of Px complex
 * float64, 384 Px bytes, in the 226 KiB of shared memory a block may use): CH_ERR_SIZE
 * (nx <= 384 among the supported sizes).
 * Calls out of order (step/gradient before begin; J of an unset grid): CH_ERR_STATE. */
int ch_objective(ch_grid* g, double* J);
int ch_adjoint_begin(ch_grid* g, double* J);
int ch_adjoint_step(ch_grid* g, const void* state);
/* as ch_adjoint_step with events around its launches (synchronises the stream):
 * kernel_ms[0..CH_ADJ_KERNELS-1] = field recomputation (z backward, y backward), transposed
 * tau solves, transposed right-hand sides, transposed y forward pass, transposed x line,
 * transposed y backward pass, i ky fold, transposed z backward. */
#define CH_ADJ_KERNELS 9
int ch_adjoint_step_timed(ch_grid* g, const void* state, double* kernel_ms);
/* ch_adjoint_segment: reverses the `nsteps` forward steps that follow `checkpoint` (a
 * ch_get_state buffer) in one call: restores the checkpoint, recomputes nsteps - 1 steps while
 * keeping each state's y-padded forward fields (the only values of a state the reverse step
 * uses: the linearisation point of the x line), then reverses the steps last to first.  Needs
 * nsteps x 6 y-padded fields of device memory (6 * 16 * nx/2 * 3ny/2 * nz bytes per step, from
 * the grid's allocator, kept until ch_adjoint_end).  Afterwards the handle holds the last
 * recomputed state with its non-linear terms (it may step on).  Same reverse arithmetic as
 * ch_adjoint_step: the gradient is bitwise the same. */
int ch_adjoint_segment(ch_grid* g, const void* checkpoint, int nsteps);
int ch_adjoint_gradient(ch_grid* g, double* gu, double* gv, double* gw, double* gphi);
int ch_adjoint_end(ch_grid* g);

/* ---- Interface rendering (headless) ----------------------------------------------------------
 * ch_render_interface: an image of the interface phi = 0 of the current state (the surface shown
 * for the drop simulation in Sec. 4) for visual checks, without any graphics API.  camera =
 * {eye x, y, z, target x, y, z, up x, y, z} in box coordinates (x in [0, lx], y in [0, ly],
 * z in [-1, 1]); fov_deg = vertical field of view in (0, 180); step = ray-march step (<= 0: half
 * the smallest of dx, dy and pi/N).  Per pixel: a perspective ray through the box, phi sampled
 * trilinearly on the collocation grid (periodic in x, y; between Gauss-Lobatto nodes in z) every
 * `step`, the first sign change refined by 40 bisections, a headlight shade from the spectral
 * gradient of phi.  rgb: device array height x width x 3 (row-major, top row first); depth
 * (device, height x width doubles, may be NULL): ray parameter of the hit, -1 for no hit.
 * Enqueued on the handle's stream.  CH_ERR_ARG for null pointers, sizes < 1, a degenerate camera;
 * CH_ERR_STATE before the fields are set. */
int ch_render_interface(ch_grid* g, unsigned char* rgb, double* depth, int width, int height,
                        const double* camera, double fov_deg, double step);

/* ---- Ensemble of independent channels (uneven sizes) ---------------------------------------
 * Not in the paper: a batching service of this library.  Each member is an ordinary ch_grid
 * (created here with the given allocator and stream; all members share one `precision`, any of
 * the three; CH_ERR_ARG if they differ).  One ensemble step advances every member by one time
 * step with six grouped persistent launches (one per stage; their CTAs walk a work list spanning
 * all members; with CH_CHEB_TC two more per member), captured once into a CUDA graph and
 * replayed.  Members are set, read and diagnosed through their ch_grid handles
 * (ch_ensemble_member); ch_ensemble_step needs every member set.  ch_ensemble_autotune times the
 * transforms' radix schedules and the persistent CTAs per SM of each stage on the live members
 * (their states are saved and restored bit for bit) and keeps the fastest; the choice is cached
 * per size signature for the process.  ch_ensemble_tuning writes the choice as a JSON object. */
typedef struct ch_ensemble ch_ensemble;
int ch_ensemble_init(const ch_params* members, int n, ch_alloc_fn alloc, ch_free_fn free_fn,
                     void* alloc_ctx, void* stream, ch_ensemble** out);
int ch_ensemble_size(const ch_ensemble* e);
int ch_ensemble_member(ch_ensemble* e, int i, ch_grid** out);
int ch_ensemble_step(ch_ensemble* e, int nsteps);
/* as ch_ensemble_step with events between the six grouped launches (stream synchronised):
 * stage_ms[0..CH_ENSEMBLE_STAGES-1] summed per stage (zrhs zsolve zbwd y backward x line
 * y forward), *total_ms over all steps */
#define CH_ENSEMBLE_STAGES 6
int ch_ensemble_step_timed(ch_ensemble* e, int nsteps, double* stage_ms, double* total_ms);
int ch_ensemble_autotune(ch_ensemble* e, int reps);
/* Chebyshev method of the ensemble step (CH_CHEB_FFT default, CH_CHEB_TC): with CH_CHEB_TC the
 * grouped zrhs and zbwd stages read and write float64 Chebyshev coefficients and each member's
 * z transforms (Sec. 3.2.1) run on the tensor cores as in ch_set_chebyshev, one launch per
 * member before zrhs and one after zbwd, inside the step's graph and timed with stages 0 and 2
 * of ch_ensemble_step_timed.  Sets every member's own method too (a later ch_set_chebyshev on a
 * member does not change the ensemble's).  The tuning is kept per method: switching takes the
 * cached choice for the new method or the defaults; the graph is rebuilt at the next step.
 * Errors: CH_ERR_ARG for an unknown method or a null handle, and the errors of
 * ch_set_chebyshev (CH_ERR_SIZE for nz > 496, CH_ERR_ALLOC); the method is unchanged then. */
int ch_ensemble_set_chebyshev(ch_ensemble* e, int method);
int ch_ensemble_get_chebyshev(const ch_ensemble* e);
int ch_ensemble_tuning(const ch_ensemble* e, char* buf, size_t n);
void ch_ensemble_destroy(ch_ensemble* e);

/* Allocation-free variant of ch_transform_forward, for callers that must not allocate device
 * memory when they call it: plug-ins whose host application's memory pool already owns the GPU's
 * memory, or fixed-latency loops that must stay out of the allocator.  (The paper has no
 * counterpart; it is a service of this library.)
 * The same transform as ch_transform_forward for a grid of nx, ny, nz (same size rules and the
 * same radix schedules), equal to it to rounding (its twiddles are computed on the device
 * instead of in extended precision on the host: about 1e-15 relative): phys is a device
 * (nz,ny,nx) float64 field, spec receives device complex float64 coefficients in the layout
 * above.  No handle, no cudaMalloc/cudaFree: the working memory is one static device array of
 * ch_noalloc_scratch_bytes() (64 MiB) that every GPU loading this library keeps until the
 * process exits; grids whose two (nx/2, ny, nz) complex work fields plus twiddles do not fit in
 * it are rejected with CH_ERR_SIZE.  Set-up done by the calls themselves: the first call on a
 * device (with that device current) looks up the array's address, and the first call for a
 * grid larger than any before it may raise a kernel's shared-memory limit; make those calls
 * before any stream capture.  All calls share the array and leave their data in it; calls that
 * overlap on the GPU (other streams or host threads) race.  Enqueued on `stream` (a cudaStream_t
 * of the current device, NULL = default stream); returns once enqueued. */
int ch_transform_forward_noalloc(int nx, int ny, int nz, const double* phys, double* spec,
                                 void* stream);
size_t ch_noalloc_scratch_bytes(void);

/* Release every buffer owned by the handle (synchronises its stream). */
void ch_destroy(ch_grid* g);

/* Static string for a status code. */
const char* ch_status_string(int status);
/* Text of the CUDA error behind the calling thread's last CH_ERR_CUDA ("no error" if none). */
const char* ch_last_cuda_error(void);

#ifdef __cplusplus
}
#endif

#endif /* CH_FLOW_H */
