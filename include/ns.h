/*
 * ns.h -- C ABI of libns_gb300.so: the pseudo-spectral Navier-Stokes hot path
 * of the FluidSim paper (arXiv 1807.01769) on one GB300 GPU (sm_103a).
 *
 * What the library computes.  The paper's solvers advance a spectral state on
 * a periodic box with "FFT, IFFT, dealiasing, divergence, curl" operators and
 * Runge-Kutta 4 ("Implementation and architecture / The simulation object";
 * "CFD pseudo-spectral code comparisons / Tri-dimensional simulations": FFTs,
 * Runge-Kutta 4, curl, vector product, projection).  Concretely, on the box
 * [0, 2 pi)^d with N points per axis:
 *   3D (velocity u_hat, 3 components):
 *     N(u) = P(k) [ dealias( FFT( u x omega ) ) ] + F,  omega_hat = i k x u_hat,
 *     P(k) = I - k k^T / |k|^2,  N(0) = 0.
 *   2D (vorticity w_hat):
 *     N(w) = dealias( FFT( -(u . grad w) ) ) + F,  u = (d_y psi, -d_x psi),
 *     psi_hat = w_hat / |k|^2,  N(0) = 0.
 *   Dealiasing keeps a mode iff every |k_i| <= kc = floor((N-1)/3).
 *   Time step: Lawson integrating-factor RK4 with E = exp(-nu |k|^2 dt),
 *   E2 = exp(-nu |k|^2 dt / 2):
 *     a = E2 (u + dt/2 k1), b = E2 u + dt/2 k2, c = E u + dt E2 k3,
 *     u' = E u + dt/6 (E k1 + 2 E2 k2 + 2 E2 k3 + k4),  k_i = N(stage input).
 *   FFT normalisation: forward divided by N^d, inverse unnormalised.
 *
 * Canonical host layouts (all FP64, C order):
 *   physical   3D: [3][N][N][N] = (comp, z, y, x);  2D: [N][N] = (y, x);
 *              point j on an axis sits at x_j = 2 pi j / N.
 *   spectral   truncated half spectrum, complex as (re, im) double pairs:
 *              3D: [3][c][c][h] = (comp, kz, ky, kx);  2D: [c][h] = (ky, kx);
 *              c = 2 kc + 1, h = kc + 1; index i on a full axis holds the
 *              wavenumber i (i <= kc) or i - c (i > kc); index i on the x axis
 *              holds kx = i.  Modes outside this set are zero by definition.
 *
 * Conventions for every entry point:
 *   - return NS_OK (0) or a negative NS_E* code; nothing throws across the ABI;
 *     ns_last_error() describes the last failure of a state.
 *   - host pointers are read or written only during the call; the library
 *     never keeps them.  All device memory is owned by the ns_state and freed
 *     by ns_destroy.
 *   - work is enqueued on the state's stream (ns_set_stream; by default a
 *     stream the library creates).  Calls that return host data synchronise
 *     that stream; ns_step only enqueues.
 *   - the state is bound to the CUDA device that was current at ns_init;
 *     every call switches to it and restores the caller's device.
 *   - one ns_state must not be used from two threads at the same time.
 */
#ifndef NS_GB300_H
#define NS_GB300_H

#ifdef __cplusplus
extern "C" {
#endif

#define NS_OK 0
#define NS_EINVAL (-1)       /* bad argument: null pointer, bad grid, nu < 0, dt <= 0, ... */
#define NS_ENOMEM (-2)       /* device allocation failed */
#define NS_ECUDA (-3)        /* a CUDA runtime call or kernel launch failed */
#define NS_EUNSUPPORTED (-4) /* grid size or precision this build does not handle */
#define NS_ENONFINITE (-5)   /* diagnostics found a NaN or Inf in the state */
#define NS_ETIMEOUT (-6)     /* a bounded device wait (TMA tile load) gave up; reported by
                                ns_sync and the diagnostics, the affected steps are invalid */

#define NS_FP64 0 /* state, FFTs and products in double precision */
#define NS_FP32 1 /* state, FFTs and products in single precision; integrating
                     factors computed in FP64 (on the host, or on the device
                     under CFL stepping) and rounded, reductions in FP64 */
#define NS_FP32_TC 2 /* as NS_FP32, except that the x-line transforms and the
                        product (3D, n = 64 .. 512) run on the tensor cores:
                        each transform is a pair of BF16 GEMMs on hi + lo
                        splits of the FP32 values (three products, FP32
                        accumulation), about 1e-5 relative error per
                        transform instead of 1e-7 */

typedef struct ns_state ns_state;

/* Grid description.  dim = 2 or 3; n = points per axis, a power of two with
 * 16 <= n <= 2048 (2D) or 16 <= n <= 1024 (3D); precision = NS_FP64|NS_FP32, or
 * NS_FP32_TC for 3D grids with n in {64, 128, 256, 512} (NS_EUNSUPPORTED otherwise). */
typedef struct {
  int dim;
  int n;
  int precision;
} ns_grid;

/* Sizes implied by a grid (host only, no GPU needed).  Any output pointer may
 * be null.  kc, c, h as above; state_doubles = doubles in the canonical
 * spectral layout (2 per complex); phys_doubles = doubles in the physical
 * layout; nbins = length of the energy spectrum (shells 0 .. round(sqrt(d) kc)).
 * Returns NS_EINVAL / NS_EUNSUPPORTED for a bad grid. */
int ns_sizes(const ns_grid *grid, int *kc, int *c, int *h, long long *state_doubles, long long *phys_doubles,
             int *nbins);

/* Create a solver state on the current CUDA device.
 *   nu >= 0 kinematic viscosity (the nu_2 parameter of the paper's solvers);
 *   dt > 0 constant time step (the paper's benchmarks use RK4 with a constant
 *   time step: "Performance / 2D benchmarks");
 *   forcing_phys: nullable host field in the physical layout (3 components in
 *   3D, one vorticity forcing field in 2D); it is transformed, dealiased,
 *   projected (3D) and held constant in time.  Copied, not kept.
 * The initial state is zero.  On failure *out is set to null. */
int ns_init(ns_state **out, const ns_grid *grid, double nu, double dt, const double *forcing_phys);

/* Set the state from a host physical field (velocity in 3D, vorticity in 2D):
 * FFT, dealias, project (3D), zero mean.  Synchronises.  The buffer holds
 * phys_doubles (ns_sizes); a page-locked one the device can address is read
 * in place by the first transform, a pageable one through device staging. */
int ns_set_state(ns_state *s, const double *phys_host);

/* Write the state to a host physical field (inverse FFT).  Synchronises.  A
 * page-locked buffer is written in place by the last transform. */
int ns_get_state(ns_state *s, double *phys_host);

/* Set / get the state in the canonical truncated spectral layout (host
 * complex128 as double pairs).  Set rounds to the state precision.  The caller
 * supplies a Hermitian-consistent kx = 0 plane (u(0,-ky,-kz) = conj u(0,ky,kz));
 * the inverse transforms use the real part of self-conjugate sums.  Synchronise.
 * The buffer holds the whole state (state_doubles of ns_sizes).  A page-locked
 * buffer the device can address (cudaHostAlloc, cudaHostRegister) is read or
 * written in place by the conversion kernel over the host link; a pageable one
 * goes through a device staging buffer.  Either way the same values. */
int ns_set_state_spectral(ns_state *s, const double *spec_host);
int ns_get_state_spectral(ns_state *s, double *spec_host);

/* Advance nsteps >= 0 Lawson IF-RK steps (RK4 unless ns_set_scheme chose
 * RK2; dt constant unless ns_set_cfl).  Asynchronous: returns after the
 * work is enqueued on the state's stream (a captured CUDA graph per step).
 * While the caller captures that stream into a graph of its own, the step's
 * kernels are enqueued one by one instead, so the caller's graph holds them;
 * the constant-dt time counter of ns_get_time then counts the capture, not
 * its replays. */
int ns_step(ns_state *s, int nsteps);

/* Time-stepping scheme ("sim.time_stepping": Runge-Kutta of order 2 or 4 with
 * the exact integrating factor for viscosity): order 4 (default) is the
 * Lawson IF-RK4 step above; order 2 the Lawson IF-RK2 midpoint step
 *   a = E2 (u + dt/2 N(u)),  u <- E u + dt E2 N(a).
 * NS_EINVAL for any other order.  Synchronises; the next ns_step captures a
 * new step graph. */
int ns_set_scheme(ns_state *s, int order);

/* CFL-adaptive time step ("sim.time_stepping" determines dt from the CFL
 * criterion): with cfl > 0 every step first takes
 *   dt = min(dt_init, cfl * (2 pi / N) / max_i max_x |u_i(x)|)
 * over the velocity components with a non-zero maximum (dt_init = the dt of
 * ns_init), the maxima taken on the grid points by the first x pass of the
 * step, and integrates with it; dt and the integrating factors are updated on
 * the device inside the step graph, so stepping stays asynchronous.  cfl = 0
 * returns to the constant dt_init.  NS_EINVAL for cfl < 0 or not finite,
 * NS_EUNSUPPORTED for cfl > 0 on a state with hyper-viscosity.  Synchronises. */
int ns_set_cfl(ns_state *s, double cfl);

/* Hyper-viscosity beside nu (the paper's viscosity parameter nu_2 is named for
 * the power of the Laplacian; its higher orders are read as nu4 and nu8): the
 * linear operator becomes -(nu |k|^2 + nu4 |k|^4 + nu8 |k|^8),
 * integrated exactly by the integrating factor (which no longer factors over
 * the axes, so E and E2 come from |k|^2-indexed tables).  nu4 = nu8 = 0
 * returns to plain viscosity.  NS_EINVAL for negative or non-finite values,
 * NS_EUNSUPPORTED together with CFL stepping.  Synchronises. */
int ns_set_hyperviscosity(ns_state *s, double nu4, double nu8);

/* Simulated time (sum of the steps taken since ns_init) and the dt of the
 * last step (the constant dt without CFL).  Synchronises when CFL is on. */
int ns_get_time(ns_state *s, double *t, double *dt);

/* One evaluation of the nonlinear term N(state) (forcing included), written
 * to a host buffer in the canonical spectral layout.  Synchronises. */
int ns_eval_rhs(ns_state *s, double *rhs_host);

/* Mean energy and enstrophy of the state, accumulated in FP64
 * ("sim.output.spatial_means"):
 *   3D: E = sum w |u_hat|^2 / 2,          Omega = sum w |i k x u_hat|^2 / 2;
 *   2D: E = sum w |w_hat|^2 / (2 |k|^2),  Omega = sum w |w_hat|^2 / 2;
 * w = 1 on the kx = 0 plane, 2 elsewhere.  Synchronises.  Returns
 * NS_ENONFINITE (values still written) if either is NaN or Inf. */
int ns_diagnostics(ns_state *s, double *energy, double *enstrophy);

/* Energy and enstrophy budget terms of the state ("sim.output.spatial_means":
 * forcing power and dissipation), FP64, w as above, with the damping rate of
 * a mode d(k) = nu |k|^2 + nu4 |k|^4 + nu8 |k|^8 (nu4 = nu8 = 0 unless set by
 * ns_set_hyperviscosity):
 *   3D: out[0] P_E = sum w Re(u_hat* . F_hat)         (energy injection),
 *       out[1] D_E = sum w d(k) |u_hat|^2             (energy dissipation),
 *       out[2] P_Z = sum w |k|^2 Re(u_hat* . F_hat)   (enstrophy injection),
 *       out[3] D_Z = sum w |k|^2 d(k) |u_hat|^2       (enstrophy dissipation);
 *   2D: out[0] P_E = sum w Re(w_hat* F_hat) / |k|^2,  out[1] D_E = sum w d(k) |w_hat|^2 / |k|^2,
 *       out[2] P_Z = sum w Re(w_hat* F_hat),          out[3] D_Z = sum w d(k) |w_hat|^2.
 * F_hat is the stored (dealiased, projected) forcing; zero without one.  The
 * Galerkin system gives dE/dt = P_E - D_E, and in 2D dOmega/dt = P_Z - D_Z.
 * Synchronises; NS_ENONFINITE (values still written) on NaN or Inf. */
int ns_budget(ns_state *s, double *out);

/* Shell energy spectrum ("sim.output.spectra", versus the modulus of the
 * wavenumber): out[m] = sum over modes with round(|k|) = m of the energy
 * density above, m = 0 .. *nbins-1.  *nbins: in = capacity of out, out = bins
 * used; NS_EINVAL if the capacity is too small.  FP64.  Synchronises. */
int ns_energy_spectrum(ns_state *s, double *out, int *nbins);

/* Bind the state to a CUDA stream (a cudaStream_t passed as void*, e.g.
 * torch.cuda.current_stream().cuda_stream); null restores the library's own
 * stream.  The caller keeps the stream alive while it is bound. */
int ns_set_stream(ns_state *s, void *cuda_stream);

/* Wait for all work enqueued for this state.  Reports asynchronous kernel
 * failures as NS_ECUDA. */
int ns_sync(ns_state *s);

/* Instrumented stepping for measurement: advances nsteps like ns_step but
 * launches kernel by kernel with CUDA events around every launch on the
 * state's stream, then synchronises.  kernel_ms[i] (total milliseconds) and
 * kernel_launches[i] are filled for kernel class i < capacity (see
 * ns_kernel_name / ns_num_kernels). */
int ns_profile_step(ns_state *s, int nsteps, double *kernel_ms, int *kernel_launches, int capacity);

/* Number of kernel classes and their names (static strings). */
int ns_num_kernels(void);
const char *ns_kernel_name(int id);

/* Algorithmic (compulsory) DRAM bytes one launch of kernel class id moves for
 * this state's grid: bytes read from inputs + bytes written to outputs, no
 * re-reads.  -1 for an unknown id. */
long long ns_kernel_bytes(const ns_state *s, int id);

/* Device bytes held by the state. */
long long ns_device_bytes(const ns_state *s);

/* ------------------------------------------------------------------------
 * Ensembles of independent 2D runs (vorticity form, same nu and dt, grid
 * sizes n[m] in {64, 128, 256, 512}, one precision).  Each RK stage is two
 * persistent launches over the work units of all members (x pass over line
 * groups; fused y pass = forward, dealias, RK stage, next inverse over kx
 * tiles), captured in one CUDA graph per step.  Every member follows exactly
 * the arithmetic of ns_step on its own grid (bitwise the same result).  The
 * paper runs one problem per process set ("Performance / Scalability"); small
 * problems are batched here because one alone cannot fill the GPU.
 * ------------------------------------------------------------------------ */
typedef struct ns_ensemble ns_ensemble;

/* Create an ensemble on the current device; all states start at zero.
 * autotune != 0 times the schedule candidates on the zero state and keeps
 * the fastest: the tile shapes (fused y pass in blocks of 256 or 512 threads,
 * i.e. kx tiles of 2048/N or 4096/N columns; x pass in blocks of 4 or 8
 * warps), blocks per SM of each pass (x in {1, 2, 4, 8}, y in {1, 2, 4},
 * at most 2048 resident threads) and the task order (member-major or round
 * robin); otherwise 256-thread y tiles, 4-warp x blocks, x = 4, y = 2,
 * member-major.  Every schedule gives the same result bit for bit (the
 * transforms' radix plan is fixed, as in ns_step).  NS_EUNSUPPORTED for a
 * grid size outside the set above. */
int ns_ensemble_init(ns_ensemble **out, int count, const int *n, int precision, double nu, double dt, int autotune);

/* Current schedule / set a schedule (task_order 0 = member by member,
 * 1 = round robin over members).  Set synchronises the ensemble's stream. */
int ns_ensemble_schedule(const ns_ensemble *e, int *x_blocks_per_sm, int *y_blocks_per_sm, int *task_order);
int ns_ensemble_set_schedule(ns_ensemble *e, int x_blocks_per_sm, int y_blocks_per_sm, int task_order);
/* Current tile shapes / set them (y_threads 256 or 512, x_warps 4 or 8;
 * else NS_EINVAL).  Set synchronises the ensemble's stream. */
int ns_ensemble_tiles(const ns_ensemble *e, int *y_threads, int *x_warps);
int ns_ensemble_set_tiles(ns_ensemble *e, int y_threads, int x_warps);
/* Fused form: every RK stage as ONE cooperative launch (the x pass over all
 * members, a grid-wide barrier, the fused y pass) instead of two launches.
 * Query the blocks per SM of that launch (0 = the two-launch form) and the
 * most that can be resident; set 0 (two launches) or 1..max (else
 * NS_EUNSUPPORTED).  A nonzero setting also selects the tile shapes it runs
 * (256-thread y blocks, 8-warp x blocks); ns_ensemble_set_tiles returns to the
 * two-launch form.  The barrier's wait is bounded: a wait that gives up is
 * reported as NS_ETIMEOUT by ns_ensemble_sync.  Set synchronises the
 * ensemble's stream.  Results are those of the two-launch form, bit for bit. */
int ns_ensemble_fused(const ns_ensemble *e, int *blocks_per_sm, int *max_blocks_per_sm);
int ns_ensemble_set_fused(ns_ensemble *e, int blocks_per_sm);

/* Member state in the canonical 2D truncated spectral layout (host complex128
 * as double pairs, [c][h] of that member's grid).  Synchronise. */
int ns_ensemble_set_state_spectral(ns_ensemble *e, int member, const double *spec_host);
int ns_ensemble_get_state_spectral(ns_ensemble *e, int member, double *spec_host);

/* Advance every member nsteps Lawson IF-RK4 steps (asynchronous). */
int ns_ensemble_step(ns_ensemble *e, int nsteps);

/* Per-member energy and enstrophy (arrays of count doubles), FP64.
 * Synchronises; NS_ENONFINITE if a member holds NaN or Inf. */
int ns_ensemble_diagnostics(ns_ensemble *e, double *energy, double *enstrophy);

int ns_ensemble_set_stream(ns_ensemble *e, void *cuda_stream);
int ns_ensemble_sync(ns_ensemble *e);
void ns_ensemble_destroy(ns_ensemble *e);
const char *ns_ensemble_last_error(const ns_ensemble *e);

/* Device-side state and forcing exchange (used by the learned closure):
 *   ns_state_to_phys_device  : the state in physical space (layout as
 *     ns_get_state, FP64) written to a DEVICE buffer, enqueued on the state's
 *     stream (no synchronisation);
 *   ns_set_forcing_phys_device: the forcing replaced by the FFT, dealiasing
 *     and (3D) projection of a DEVICE physical field (FP64); enqueued.  A state
 *     created without forcing gets one here. */
int ns_state_to_phys_device(ns_state *s, double *phys_dev);
int ns_set_forcing_phys_device(ns_state *s, const double *phys_dev);

/* ------------------------------------------------------------------------
 * Learned closure network (no counterpart in the paper): four 3x3
 * convolutions on a periodic height x width grid, channels 1 -> 32 -> 32 ->
 * 32 -> 1, exact GELU after the first three, BF16 activations and weights with
 * FP32 accumulation and an FP32 Adam master copy.  Data [batch][y][x], FP32,
 * device pointers.  Parameters flat: W0 b0 W1 b1 W2 b2 W3 b3, W as
 * [Cout][Cin][3][3].  Weight gradients are accumulated with atomics (their
 * last bits depend on the order).
 * ------------------------------------------------------------------------ */
typedef struct ns_cnn ns_cnn;
int ns_cnn_init(ns_cnn **out, int height, int width, int max_batch, unsigned long long seed);
int ns_cnn_num_params(const ns_cnn *c);
int ns_cnn_get_params(ns_cnn *c, float *host);
int ns_cnn_set_params(ns_cnn *c, const float *host);
/* y = net(x), enqueued on stream (null = legacy default stream). */
int ns_cnn_forward(ns_cnn *c, const float *x_dev, float *y_dev, int batch, void *stream);
/* Gradient of mean((net(x) - t)^2) into grad_host (num_params floats) and the
 * loss; no update; synchronous. */
int ns_cnn_gradients(ns_cnn *c, const float *x_dev, const float *t_dev, int batch, float *grad_host, float *loss);
/* One Adam step (beta 0.9 / 0.999, eps 1e-8) on mean((net(x) - t)^2);
 * loss_out (nullable, host) receives the loss before the update. */
int ns_cnn_train_step(ns_cnn *c, const float *x_dev, const float *t_dev, int batch, float lr, float *loss_out,
                      void *stream);
void ns_cnn_destroy(ns_cnn *c);
const char *ns_cnn_last_error(const ns_cnn *c);
/* Elementwise helpers on device arrays: dst = (float)(scale src);
 * dst = base + scale src (base nullable). */
int ns_f64_to_f32(const double *src_dev, float *dst_dev, long long n, double scale, void *stream);
int ns_f32_axpy_f64(const float *src_dev, const double *base_dev, double *dst_dev, long long n, double scale,
                    void *stream);

/* Diagnostics for callers that cannot allocate device memory.
 * The FluidSim paper has no counterpart: this entry point exists for ordinary
 * host code that must not call cudaMalloc -- an allocator hook, code under a
 * memory pool that must not grow, a process whose device memory is owned and
 * budgeted by another framework -- but holds a spectrum on the device.  It
 * makes CUDA runtime calls and launches kernels, so it must not be called from
 * a stream callback or a host function enqueued with cudaLaunchHostFunc.  It computes what ns_diagnostics and
 * ns_energy_spectrum compute, with the same kernels and summation order, and
 * allocates nothing: its partial sums live in a static device array of
 * NS_NOALLOC_SCRATCH_DOUBLES doubles (2 MiB) that every GPU loading the
 * library holds until the process exits.
 *   grid     : dim, n, precision of the data;
 *   spec_dev : DEVICE pointer to the state in the canonical truncated spectral
 *              layout (rows of h complex numbers, no padding), complex128 for
 *              NS_FP64 or complex64 for NS_FP32; read only;
 *   out_dev  : DEVICE pointer to nbins + 2 doubles: out[0] energy, out[1]
 *              enstrophy, out[2 + m] the shell spectrum (see ns_sizes);
 *   cuda_stream: cudaStream_t as void* (null = the legacy default stream).
 * Asynchronous: returns once the work is enqueued; synchronise the stream
 * before reading out_dev.  Returns NS_OK, NS_EINVAL (null pointer, bad grid),
 * NS_EUNSUPPORTED (the grid needs more scratch than the static array holds:
 * every 2D grid fits, 3D up to n = 256), or NS_ECUDA.  Every call looks up
 * the array's device address (cudaGetSymbolAddress) on the current device.
 * The first call on a device loads the library module that holds the array
 * (CUDA loads modules lazily) and so commits its 2 MiB then: make one warm-up
 * call per device outside any region where allocation is forbidden and
 * before any stream capture; later calls allocate nothing.  All calls
 * share the array, so calls whose kernels may overlap on the GPU (unordered
 * streams) race on it; calls on one stream are ordered and safe.  Each call
 * rewrites the scratch it reads, so nothing needs clearing in between. */
#define NS_NOALLOC_SCRATCH_DOUBLES 262144
int ns_diagnostics_noalloc(const ns_grid *grid, const void *spec_dev, double *out_dev, void *cuda_stream);

/* Measured FP32 fused-multiply-add rate of a device, in TFLOP/s (2 flops per
 * FMA): every SM runs warps of eight independent FMA chains per thread, timed
 * with CUDA events after one untimed launch.  It is the denominator of the
 * flop efficiency reported beside the HBM roofline, since the FFT passes sit
 * close to the FP32 ALU bound too (the paper's per-task profile, "CFD
 * pseudo-spectral code comparisons / Tri-dimensional simulations", puts most
 * of a step in the FFTs).  Runs on its own stream and synchronises; allocates
 * 4 bytes per launched thread for the chains' results and frees them. */
int ns_fp32_fma_peak(int device, double *tflops);

/* Release everything the state owns.  Null is ignored. */
void ns_destroy(ns_state *s);

/* Description of the last failure of s (or of the last failed ns_init when s
 * is null).  Static storage owned by the library. */
const char *ns_last_error(const ns_state *s);

#ifdef __cplusplus
}
#endif

#endif /* NS_GB300_H */
