/*
 * flups.h - C ABI of the GB300 (sm_103a) FFT pressure-projection library.
 *
 * The library computes the pressure-projection step of FluTAS (arXiv 2204.08834,
 * Sec. 3.3 "Pressure correction algorithm", Eqs. us_predic, poisson, corr, p_upt) with
 * the FFT/tridiagonal direct Poisson solver of Sec. 3.3.1:
 *
 *   f       = (rho0/dt) D u** + D[(1 - rho0/rho_f) G p_hat],   p_hat = c1 p^n - c2 p^{n-1}
 *   L p     = f - <f>_V,   <p>_V = 0                            (L = D G, 7-point MAC operator)
 *   u^{n+1} = u** - (dt/rho0) [G p - (1 - rho0/rho_f) G p_hat]
 *
 * with rho0 the minimum density (Sec. 3.3), rho_f the arithmetic mean of the two cell
 * densities beside a face, and <.>_V the volume-weighted mean.  x and y are periodic;
 * z is periodic (uniform spacing, third Fourier transform) or bounded by walls
 * (homogeneous Neumann for p, w = 0 on the wall faces, possibly stretched spacing,
 * Gauss elimination along z per (kx, ky) wavenumber).
 *
 * Layout of every field: float64, C-contiguous [nz][ny][nx] (x fastest), DEVICE memory
 * owned by the caller unless a function says HOST.  u[k][j][i] is the x-face i+1/2,
 * v[k][j][i] the y-face j+1/2, w[k][j][i] the z-face k+1/2 (top face of cell k; with
 * walls w[nz-1] is the top wall face).  Field pointers must be 16-byte aligned.
 *
 * Streams: every call is stream-ordered on the plan's CUDA stream and returns without
 * waiting for the GPU, except where a function says it synchronises.
 *
 * Errors: no call throws.  Argument errors are returned at once; CUDA errors are
 * returned as FLUPS_ECUDA by the call that observes them.  A call that fails leaves
 * the output buffers in an unspecified state.
 */
#ifndef FLUPS_H
#define FLUPS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct flups_plan_s* flups_plan;

typedef enum {
    FLUPS_OK = 0,
    FLUPS_EINVAL = 1,        /* bad argument: null pointer, size, spacing, alignment       */
    FLUPS_EUNSUPPORTED = 2,  /* size outside what the kernels support (see plan_create)     */
    FLUPS_ENOMEM = 3,        /* device allocation failed                                   */
    FLUPS_ECUDA = 4,         /* a CUDA runtime call or kernel launch failed                */
    FLUPS_ENONFINITE = 5,    /* a non-finite or non-positive density, or a NaN residual    */
    FLUPS_ENOCONV = 6,       /* refinement did not reach rtol within max_iter              */
    FLUPS_ESTATE = 7,        /* call order violated (rhs/correct before set_density)       */
    FLUPS_ETIMEOUT = 8       /* a bounded device-side wait gave up; outputs are invalid    */
} flups_status;

typedef enum { FLUPS_BC_PERIODIC = 0, FLUPS_BC_WALLS = 1 } flups_bc;

/* Ends of the x and y directions (flups_plan_create_bc): periodic, or homogeneous Neumann
 * (dp/dn = 0) / homogeneous Dirichlet (p = 0) on the low (index -1/2) and high (n-1/2) boundary
 * faces of the direction. */
typedef enum {
    FLUPS_XY_PERIODIC = 0,
    FLUPS_XY_NEUMANN = 1,     /* Neumann at both faces   */
    FLUPS_XY_DIRICHLET = 2,   /* Dirichlet at both faces */
    FLUPS_XY_NEU_DIR = 3,     /* Neumann low, Dirichlet high */
    FLUPS_XY_DIR_NEU = 4      /* Dirichlet low, Neumann high */
} flups_xy_bc;

typedef enum {
    FLUPS_FP64 = 0,          /* FFTs and z solve in FP64, one direct pass                  */
    FLUPS_FP32_REFINE = 1    /* FFTs and z solve in FP32; FP64 residual f - L p, FP64
                                defect-correction update p += delta, repeated to rtol      */
} flups_prec;

#define FLUPS_HIST 16

typedef struct {
    int iters;                          /* FP32 solves performed (FP64: 1)                   */
    double rel_res;                     /* ||f - <f> - L p||_2 / ||f - <f>||_2 last computed;
                                           -1 when not computed (FP64 with rtol <= 0)        */
    double rel_res_hist[FLUPS_HIST];    /* rel_res after each FP32 solve                     */
} flups_info;

/*
 * flups_plan_create - plan a projection on an nx x ny x nz grid (Sec. 3, MAC grid).
 *   nx, ny : 2^a >= 8, or 3 * 2^a >= 24 and a multiple of 8 (radix-2/4/8 and radix-3
 *            transforms), at most 4096 (x, y periodic).
 *   nz     : the same rule when bc = FLUPS_BC_PERIODIC; any value in [2, 8192] with
 *            bc = FLUPS_BC_WALLS.  nx ny nz < 2^31.
 *            With prec = FLUPS_FP64, ny and a periodic nz are at most 2048.
 *   dx, dy : uniform spacings (> 0).
 *   dzf    : HOST array of nz cell widths along z (> 0), copied; must be uniform when
 *            bc = FLUPS_BC_PERIODIC.  Cell centres lie midway between faces.
 *   prec   : flups_prec.
 *   stream : cudaStream_t (NULL = legacy default stream).
 * The plan allocates its own device workspace (spectrum, face coefficients, tables);
 * flups_workspace_bytes reports its size.  The current CUDA device is recorded and
 * made current by every later call on the plan.
 */
flups_status flups_plan_create(flups_plan* out, int nx, int ny, int nz, double dx, double dy,
                               const double* dzf, int bc, int prec, void* stream);
/*
 * flups_plan_create_bc - as flups_plan_create, with Neumann or Dirichlet ends in x and/or y
 * (Sec. 3.3.1: the eigen-expansion along x and y holds for any homogeneous boundary
 * conditions; cosine and sine series by FFTs with pre/post-processing).
 *   bcx, bcy : flups_xy_bc.  Neumann at both ends: cosine series (DCT-II/III), modes
 *              cos(pi k (2i+1)/(2n)), eigenvalues -4 sin^2(pi k/(2n))/h^2; Dirichlet at both
 *              ends (p = 0 on the boundary face): sine series (DST-II/III), modes
 *              sin(pi (k+1)(2i+1)/(2n)), eigenvalues -4 sin^2(pi (k+1)/(2n))/h^2; mixed ends:
 *              modes cos (Neumann low) or sin (Dirichlet low) of pi (2k+1)(2i+1)/(4n) (DCT-IV,
 *              DST-IV), eigenvalues -4 sin^2(pi (2k+1)/(4n))/h^2.
 *   bc       : the z treatment, as in flups_plan_create.
 * A plan with any non-periodic x/y end takes only flups_solve (set_density, rhs, correct and
 * the host-buffer projection return FLUPS_EUNSUPPORTED).  Its solve is L p = f when an end is
 * Dirichlet (L is then nonsingular and the mean of f is kept), and L p = f - <f>_V with
 * <p>_V = 0 otherwise.  FLUPS_FP64: one direct pass, residual not evaluated (info->rel_res
 * stays -1).  FLUPS_FP32_REFINE: FP32 transforms, the FP64 defect f - <f> - L p with the ends'
 * ghost rules, repeated to rtol by a host-driven loop (synchronises; not graph capturable).
 */
flups_status flups_plan_create_bc(flups_plan* out, int nx, int ny, int nz, double dx, double dy,
                                  const double* dzf, int bcx, int bcy, int bc, int prec, void* stream);
flups_status flups_plan_destroy(flups_plan plan);
flups_status flups_set_stream(flups_plan plan, void* stream);
size_t       flups_workspace_bytes(flups_plan plan);
/* flups_launch_count - number of CUDA kernels this plan has launched so far (host counter). */
unsigned long long flups_launch_count(flups_plan plan);

/*
 * Per-kernel timing (tracing aid; no counterpart in the paper, which reports only a
 * breakdown of the whole time step, Sec. 6.2).  flups_set_profiling(plan, 1) makes every
 * later launch bracket its kernel(s) with CUDA events on the plan's stream (up to 1024
 * regions between reads; later ones are not recorded); 0 stops it.  flups_profile_read
 * synchronises the stream and writes, for every kernel id 0 <= k < FLUPS_NKERNELS, the
 * total milliseconds ms[k] and the number of timed regions n[k] (HOST arrays) recorded
 * since the previous read.  flups_kernel_name(k) names kernel id k (static string).
 */
#define FLUPS_NKERNELS 26
flups_status flups_set_profiling(flups_plan plan, int on);
flups_status flups_profile_read(flups_plan plan, double* ms, long long* n);
const char*  flups_kernel_name(int id);

/*
 * flups_set_density - register the density field for the next rhs/correct calls (Sec. 3.3).
 *   rho  : DEVICE [nz][ny][nx], read once here; not retained.
 *   rho0 : > 0 uses this value as rho0; <= 0 computes rho0 = min(rho) on the device
 *          (Sec. 3.3: "the minimum value of the density field").
 * Stores the face coefficients (1 - rho0/rho_f)/h per face in the plan workspace.
 * Non-finite or non-positive densities are reported as FLUPS_ENONFINITE by the next
 * synchronising call (flups_get_rho0 or flups_solve with info != NULL).
 */
flups_status flups_set_density(flups_plan plan, const double* rho, double rho0);

/* flups_get_rho0 - copy rho0 to *rho0_host (HOST); synchronises the plan's stream. */
flups_status flups_get_rho0(flups_plan plan, double* rho0_host);

/*
 * flups_plan_sync - wait for every call queued on the plan's stream and return the errors
 * the device latched meanwhile (no counterpart in the paper; the library's error exit):
 * FLUPS_ETIMEOUT when a bounded device-side wait gave up (the time-out is cleared once
 * reported), FLUPS_ENONFINITE when the density registered by flups_set_density holds a
 * non-finite or non-positive value, FLUPS_ECUDA when the stream reports a CUDA error
 * (flups_last_cuda_error names it), FLUPS_OK otherwise.
 */
flups_status flups_plan_sync(flups_plan plan);

/* flups_last_cuda_error - name of the last CUDA error a call of this thread observed
 * ("cudaSuccess" if none); a static string. */
const char* flups_last_cuda_error(void);

/*
 * flups_rhs - right-hand side of the split Poisson equation (Eqs. us_predic + poisson):
 *   f = (rho0/dt) D u** + D[(1 - rho0/rho_f) G p_hat],  p_hat = c1 p_n - c2 p_nm1.
 *   u, v, w   : DEVICE, the predicted velocity u** (read only).
 *   p_n, p_nm1: DEVICE pressures at t^n and t^{n-1}; p_nm1 may be NULL (then p_hat = c1 p_n).
 *   c1, c2    : extrapolation weights (1 + r, r with r = dt^{n+1}/dt^n; 2 and 1 at constant dt).
 *   dt        : > 0.
 *   f         : DEVICE output [nz][ny][nx]; must not alias an input.
 */
flups_status flups_rhs(flups_plan plan, const double* u, const double* v, const double* w,
                       const double* p_n, const double* p_nm1, double c1, double c2, double dt,
                       double* f);

/*
 * flups_solve - p with L p = f - <f>_V and <p>_V = 0 (Sec. 3.3.1: forward FFT along x and
 * y, Gauss elimination along z or a z FFT, inverse y and x).
 *   f        : DEVICE input (read only); p : DEVICE output, may not alias f.
 *   rtol     : FLUPS_FP32_REFINE: stop when the FP64 relative residual <= rtol (1e-10 for
 *              the throughput metric); FLUPS_FP64: if > 0 and info != NULL the residual is
 *              evaluated after the direct solve and reported (not needed otherwise).
 *   max_iter : maximum number of FP32 solves (refine mode), 1..64.
 *   info     : HOST, may be NULL.  Refine mode synchronises once per FP32 solve to read
 *              the residual norm; FP64 mode synchronises only when info != NULL.
 * Returns FLUPS_ENOCONV if rtol was not reached (p holds the last iterate),
 * FLUPS_ENONFINITE if a residual norm is not finite.
 */
flups_status flups_solve(flups_plan plan, const double* f, double* p, double rtol, int max_iter,
                         flups_info* info);

/*
 * flups_solve_graphable - the FP32-refine solve of flups_solve as a fixed sequence of
 * stream-ordered kernels with no host synchronisation, so that it can be captured into a
 * CUDA graph (the refinement of Sec. 3.3.1's solver is not in the paper; this form serves
 * batched ensembles).  At most max_iter FP32 solves run; after each FP64 defect norm a
 * device-side flag ends the sequence early (the remaining kernels return at once) once
 * ||f - <f> - L p|| <= rtol ||f - <f>||, so p equals what flups_solve returns.
 * Plan must be FLUPS_FP32_REFINE.  Read the outcome with flups_solve_result.
 */
flups_status flups_solve_graphable(flups_plan plan, const double* f, double* p, double rtol, int max_iter);

/* flups_solve_result - synchronises the plan's stream and reports the last defect norm of
 * the previous flups_solve_graphable (info->rel_res; info->iters = its max_iter);
 * FLUPS_ENOCONV if it is above rtol. */
flups_status flups_solve_result(flups_plan plan, double rtol, flups_info* info);

/*
 * flups_correct - velocity correction (Eqs. us_predic + corr):
 *   u^{n+1} = u** - (dt/rho0) [G p - (1 - rho0/rho_f) G p_hat], in place on u, v, w.
 *   p        : DEVICE solution of flups_solve; p_n, p_nm1, c1, c2 as in flups_rhs.
 * With walls the top wall face w[nz-1] is set to 0.
 */
flups_status flups_correct(flups_plan plan, const double* p, const double* p_n,
                           const double* p_nm1, double c1, double c2, double dt,
                           double* u, double* v, double* w);

/*
 * flups_project_host - one whole projection with HOST buffers (end-to-end form):
 * copies u, v, w, rho, p_n, p_nm1 to plan-owned device buffers, runs set_density(rho,
 * rho0 = min), rhs, solve and correct, and copies u, v, w (in place) and p back.
 * The inputs travel on a plan-owned copy stream, rho first, so the density pass overlaps
 * the other copies; p travels back on it while the correction runs.  Host buffers should
 * be page-locked for full copy bandwidth.  Synchronises both streams before returning
 * (also on error), so no copy touches the caller's buffers afterwards.
 */
flups_status flups_project_host(flups_plan plan, double* u, double* v, double* w,
                                const double* rho, const double* p_n, const double* p_nm1,
                                double c1, double c2, double dt, double rtol, int max_iter,
                                double* p_out, flups_info* info);

/*
 * flups_solve_host - flups_solve with HOST buffers (end-to-end form of the solve): copies f
 * (nz*ny*nx float64) to a plan-owned device buffer (allocated on the first call), solves as
 * flups_solve, copies p back to p_out.  Host buffers should be page-locked for full copy
 * bandwidth.  Synchronises the plan's stream before returning (also on error), so no copy
 * touches the caller's buffers afterwards.  With FLUPS_ENOCONV p_out holds the last iterate.
 */
flups_status flups_solve_host(flups_plan plan, const double* f, double* p_out, double rtol, int max_iter,
                              flups_info* info);

/*
 * flups_solve_fp64_noalloc - the FP64 direct solve of flups_solve (FLUPS_FP64 mode) for
 * callers that cannot allocate device memory, for example a solver plug-in inside a host
 * application that owns and pre-reserves the whole device memory budget, or code running
 * under a memory manager that forbids allocations once a run has started.  The paper has
 * no counterpart to this entry point.
 *   nx, ny   : powers of two, 8 <= nx <= 4096, 8 <= ny <= 2048 (the 3 * 2^a lengths that
 *              flups_plan_create also takes are not supported here: FLUPS_EUNSUPPORTED).
 *   nz       : bc = FLUPS_BC_PERIODIC: a power of two in [8, 2048]; FLUPS_BC_WALLS: any
 *              value in [2, 8192].
 *   dx, dy, bc: as in flups_plan_create.
 *   dzf      : HOST array of nz cell widths as in flups_plan_create; read during the call
 *              only, so it need not outlive it.
 *   f, p     : DEVICE input and output, as in flups_solve (p may not alias f).
 *   stream   : cudaStream_t (NULL = legacy default stream).
 * No plan is needed and nothing is allocated: the workspace (spectrum, z multipliers,
 * tables) lives in one static device array of FLUPS_NOALLOC_MAX_BYTES that every GPU
 * loading the library holds until exit.  A grid whose workspace does not fit (about
 * 16 MiB: e.g. 64^3 or 128x128x32 periodic fit, 128^3 does not) returns
 * FLUPS_EUNSUPPORTED before any GPU work.  The first call on a device (and the first call
 * after that device's context was replaced, e.g. by cudaDeviceReset) looks up the array's
 * device address (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  Every call reuses the same array, so calls that overlap on
 * the GPU race: serialise them.  Stream-ordered; does not synchronise.
 */
#define FLUPS_NOALLOC_MAX_BYTES (16u << 20)
flups_status flups_solve_fp64_noalloc(int nx, int ny, int nz, double dx, double dy, const double* dzf,
                                      int bc, const double* f, double* p, void* stream);

/*
 * Batched ensembles of independent FP32-refine solves of mixed sizes in one CUDA graph
 * launch (no counterpart in the paper, which solves one field per time step; the solver
 * of every member is the Sec. 3.3.1 method of flups_solve).
 *
 * flups_batch_create - n members, member m with grid nx[m] x ny[m] x nz[m], spacings dx[m],
 *   dy[m], HOST cell widths dzf[m] (nz[m] values) and boundary condition bc[m], each with its
 *   own plan (as flups_plan_create with FLUPS_FP32_REFINE).  nstreams (1..32) worker streams
 *   run members concurrently; stream is the origin stream the graph launches on.  With
 *   autotune != 0, every distinct member size is timed once for the transform CTA thread cap
 *   (256/512/1024) and the radix sequence of its power-of-two transforms, and the fastest
 *   pair is kept (flups_batch_member_tuning reports it).
 * flups_batch_solve - solves L p[m] = f[m] - <f[m]> for every member (DEVICE pointers) with
 *   at most max_iter FP32 solves each and early exit at rtol (flups_solve_graphable).  The
 *   first call, and any call whose pointers, rtol or max_iter differ from the previous one,
 *   captures the members' kernels into a CUDA graph; later calls replay it.  With info !=
 *   NULL (HOST array of n) it synchronises and reports each member's last defect norm;
 *   FLUPS_ENOCONV if some member is above rtol.  Without info it does not synchronise.
 */
typedef struct flups_batch_s* flups_batch;
flups_status flups_batch_create(flups_batch* out, int n, const int* nx, const int* ny, const int* nz,
                                const double* dx, const double* dy, const double* const* dzf, const int* bc,
                                int nstreams, int autotune, void* stream);
flups_status flups_batch_solve(flups_batch batch, const double* const* f, double* const* p, double rtol,
                               int max_iter, flups_info* info);
flups_status flups_batch_destroy(flups_batch batch);
/* flups_batch_graph_kernels - kernels in the captured graph (one flups_batch_solve replay). */
unsigned long long flups_batch_graph_kernels(flups_batch batch);
/* flups_batch_member_tuning - CTA thread cap and radix variant (0: radix 8 first, 1: radix 4)
 * chosen for member m. */
flups_status flups_batch_member_tuning(flups_batch batch, int m, int* cta_threads, int* radix_variant);

/*
 * flups_varcoef_solve - the exact variable-coefficient pressure that the split of Sec. 3.3
 * approximates (the split replaces 1/rho by the constant 1/rho0 in the Poisson operator and
 * carries the difference through p_hat, Eqs. us_predic and poisson):
 *     D((rho0/rho_f) G p) = f - <f>_V,   <p>_V = 0,
 * rho_f the arithmetic mean of the two cell densities beside a face, rho0 the plan's minimum
 * density from flups_set_density.  Solved by conjugate gradients in the volume-weighted inner
 * product, preconditioned with the plan's own constant-coefficient solve (FP64 plans: one
 * direct pass; FP32-refine plans: three FP32 passes with FP64 defect correction).  Not in the
 * paper: these pressures are the training targets of the learned p_hat (flups_pnet_*) and the
 * reference its splitting error is measured against.  With p_hat = p, flups_rhs/solve/correct
 * return p again and the velocity u** - (dt/rho_f) G p.
 *   rho  : DEVICE density, the field given to flups_set_density
 *   f    : DEVICE right-hand side, e.g. flups_rhs with c1 = c2 = 0, i.e. (rho0/dt) D u**
 *   p    : DEVICE output (may not alias f or rho)
 *   rtol : stop when ||r||_V <= rtol ||f - <f>_V||_V (volume-weighted 2-norms)
 *   info : HOST, may be NULL: iterations, final relative residual, first 16 residuals
 * Returns FLUPS_ESTATE before set_density, FLUPS_ENOCONV after max_iter iterations (p holds
 * the last iterate).  Allocates 7 fields of plan-owned workspace on the first call.
 * Synchronises once per iteration.
 */
flups_status flups_varcoef_solve(flups_plan plan, const double* rho, const double* f, double* p, double rtol,
                                 int max_iter, flups_info* info);

/*
 * Learned splitting pressure (not in the paper, which extrapolates p_hat = 2 p^n - p^{n-1} for
 * a constant time step, Sec. 3.3).  A periodic 3-D convolutional net predicts a correction to
 * the extrapolation:
 *     p_hat = 2 p^n - p^{n-1} + s y(1 - rho0/rho, p^n/s, p^{n-1}/s),   s = rms(p^n),
 * y = four 3x3x3 convolutions 3 -> 16 -> 16 -> 16 -> 1 with ReLU between layers.  Convolutions
 * run on the tensor cores with bfloat16 weights and FP32 accumulation; activations and
 * gradients are stored as bfloat16, master weights and Adam moments as FP32.
 *
 * Parameters (FLUPS_PNET_NPARAMS floats, HOST arrays): for each layer l = 1..4 its weights
 * W_l[out][in][27] followed by its biases b_l[out]; tap t = 9 (dz+1) + 3 (dy+1) + (dx+1)
 * multiplies the input at cell (k+dz, j+dy, i+dx), indices periodic.
 *
 * flups_pnet_create  - a net for one grid nx x ny x nz (all periodic) with nx a multiple of
 *                      32, ny of 8, nz of 4, at most 2^28 cells (FLUPS_EUNSUPPORTED
 *                      otherwise); params must be finite.  Allocates 224 bytes a cell plus
 *                      the weight-gradient partials.  Synchronises.
 * flups_pnet_predict - p_hat (DEVICE, may not alias the inputs) from DEVICE rho, p_n, p_nm1
 *                      and rho0 > 0 (HOST, normally the plan's flups_get_rho0).
 * flups_pnet_train_step - one Adam step (beta1 0.9, beta2 0.999, eps 1e-8, learning rate lr)
 *                      on loss = mean over cells of (y - (p_next - 2 p_n + p_nm1)/s)^2;
 *                      loss (HOST, may be NULL) receives the loss before the step, and then
 *                      the call synchronises; without it the call is stream-ordered only.
 * flups_pnet_eval_loss - the same loss without a step (synchronises).
 * flups_pnet_set_params / get_params - HOST copies of the FP32 master parameters; set resets
 *                      the Adam state; both synchronise.
 * flups_pnet_get_grads - the parameter gradient of the last train step (HOST); synchronises.
 * flups_pnet_get_adam / set_adam - HOST copies of the Adam moments m, v (FLUPS_PNET_NPARAMS
 *                      floats each, v >= 0) and the number of Adam steps taken (0 .. 2^31-1);
 *                      with the master parameters they are the whole training state, so
 *                      set_params followed by set_adam resumes training exactly (set_params
 *                      resets them, so set_adam comes second).  Both synchronise; set_adam
 *                      returns FLUPS_EINVAL for non-finite or negative entries.
 * flups_pnet_launch_count - kernels this net has launched so far.
 * flups_pnet_set_profiling / profile_read / kernel_name - optional CUDA-event timing of the
 *                      net's kernel groups (FLUPS_PNET_NKERNELS entries: features, hidden
 *                      convolutions, output convolution, backward-data convolutions, weight
 *                      gradients, update), as flups_set_profiling for plans.
 * Every call runs on the stream given at create.
 */
#define FLUPS_PNET_NPARAMS 15601
typedef struct flups_pnet_s* flups_pnet;
flups_status flups_pnet_create(flups_pnet* out, int nx, int ny, int nz, const float* params, void* stream);
flups_status flups_pnet_destroy(flups_pnet net);
flups_status flups_pnet_set_params(flups_pnet net, const float* params);
flups_status flups_pnet_get_params(flups_pnet net, float* params);
flups_status flups_pnet_get_grads(flups_pnet net, float* grads);
flups_status flups_pnet_get_adam(flups_pnet net, float* m, float* v, long long* step);
flups_status flups_pnet_set_adam(flups_pnet net, const float* m, const float* v, long long step);
flups_status flups_pnet_predict(flups_pnet net, const double* rho, double rho0, const double* p_n,
                                const double* p_nm1, double* p_hat);
flups_status flups_pnet_train_step(flups_pnet net, const double* rho, double rho0, const double* p_n,
                                   const double* p_nm1, const double* p_next, float lr, double* loss);
flups_status flups_pnet_eval_loss(flups_pnet net, const double* rho, double rho0, const double* p_n,
                                  const double* p_nm1, const double* p_next, double* loss);
unsigned long long flups_pnet_launch_count(flups_pnet net);
#define FLUPS_PNET_NKERNELS 6
flups_status flups_pnet_set_profiling(flups_pnet net, int on);
flups_status flups_pnet_profile_read(flups_pnet net, double* ms, long long* n);
const char* flups_pnet_kernel_name(int id);

/*
 * flups_momentum_predict - the momentum predictor of one phase (Sec. 3.3, Eq. uss_predic),
 * the step before flups_rhs, on the plan's grid (z must be periodic):
 *   M^n = -D(u^n u^n) + nu L u^n,   u** = u^n + dt (f1 M^n - f2 M^{n-1} + g),
 *   f1 = 1 + dt/(2 dt_prev), f2 = dt/(2 dt_prev)  (second-order Adams-Bashforth, Sec. 3.2/3.3).
 * The convective flux is in divergence form from two-point averages (u u at cell centres,
 * u v, u w, v w on cell edges), L the 7-point Laplacian; constant density and viscosity,
 * so surface tension vanishes and the body force is the constant acceleration g.
 *   u, v, w    : u^n, DEVICE, read only (layout above).
 *   us, vs, ws : u**, DEVICE, written.  No output may overlap another argument.
 *   m_state    : DEVICE, 3 x nz*ny*nx pairs of float32 (hi, lo) = 24 bytes per cell, 16-byte
 *                aligned, [component][nz][ny][nx]: M^{n-1} on entry (read only when
 *                dt_prev > 0), M^n on return (hi + lo carries 48 significant bits).
 *   nu         : kinematic viscosity >= 0;  gx, gy, gz : body acceleration.
 *   dt > 0; dt_prev <= 0 marks the first step (forward Euler, M^{n-1} not read).
 *   arith      : FLUPS_MOM_PAIR - M in pairs of float32 on a fixed-point grid set by
 *                max(|u|,|v|,|w|) (an extra pass over u, v, w), error ~2^-38 max|u|^2/h in M;
 *                needs dx = dy = dz; velocities whose maximum lies outside the range the
 *                pair arithmetic covers are computed in float64 by the same launch.
 *                FLUPS_MOM_FP64 - float64 throughout, any spacings.
 * Returns FLUPS_EUNSUPPORTED for z walls or FLUPS_MOM_PAIR on unequal spacings,
 * FLUPS_EINVAL for bad arguments.  Stream-ordered, no synchronisation, graph capturable.
 */
#define FLUPS_MOM_PAIR 0
#define FLUPS_MOM_FP64 1
flups_status flups_momentum_predict(flups_plan plan, const double* u, const double* v, const double* w,
                                    double* us, double* vs, double* ws, void* m_state, double nu,
                                    double gx, double gy, double gz, double dt, double dt_prev, int arith);

/*
 * flups_vof_step - one step of the volume fraction (Sec. 3.1, Eqs. phi_split and vof_corr_step;
 * Appendix A): MTHINC reconstruction of the interface in every cell,
 *     H = (1 + tanh(beta (T(x~) + d_th))) / 2,  x~ in [0, 1]^3 the cell's local coordinates,
 * T the quadratic built from the Youngs normal n and K = grad n (linear along the direction of
 * the largest normal component, where the cell integral of H is taken exactly; two-point
 * Gauss-Legendre along the other two), d_th such that the cell integral of H is phi; then the
 * split updates x, y, z, each with fluxes that integrate H of the upwind cell over the volume
 * swept through the face in dt, phi^p = (phi^s - (F_{i+1/2} - F_{i-1/2})) /
 * (1 - dt/h (u_{i+1/2} - u_{i-1/2})), and the divergence correction
 * phi^{n+1} = phi^z - sum_p dt/h_p phi^p (u_{i+1/2} - u_{i-1/2})_p, which conserves sum(phi).
 *   plan   : the grid (triply periodic, uniform z spacing, nx, ny, nz multiples of 8)
 *   phi    : DEVICE [nz][ny][nx] float64, phi^n on entry, phi^{n+1} on return (in place)
 *   u, v, w: DEVICE face velocities at t^n (layout as for flups_rhs), read only
 *   dt > 0 with |u| dt / dx <= 1 (likewise v, w); beta > 0 the sharpness beta_th
 *   stages : DEVICE 3 nz ny nx float64 for phi^x, phi^y, phi^z (or NULL: plan workspace)
 * Reconstruction and fluxes run in FP32, the updates in FP64 (sum(phi) is conserved to FP64
 * rounding).  A
 * face with |u| dt / h > 1 (or a non-finite velocity) is latched and reported by the next
 * flups_plan_sync as FLUPS_EINVAL (its flux is taken as 0).  Allocates 56 bytes per cell of
 * plan workspace on the first call.  Stream-ordered, no synchronisation.  Returns
 * FLUPS_EUNSUPPORTED for walls, ends in x or y, or sizes that are not multiples of 8.
 */
flups_status flups_vof_step(flups_plan plan, double* phi, const double* u, const double* v, const double* w,
                            double dt, double beta, double* stages);

/* flups_selftest_wait_timeout - diagnostic of the library's failure detection (no paper
 * counterpart): launches one kernel whose thread waits, through the same bounded wait the
 * pipelined transform passes use, on an mbarrier that nothing ever arrives at, with `limit`
 * polls (1 .. 2^20).  The wait gives up, the kernel records the time-out in a device error
 * word and returns, and the call returns FLUPS_ETIMEOUT with the context still usable
 * (FLUPS_OK would mean the wait did not time out).  Synchronises `stream`. */
flups_status flups_selftest_wait_timeout(void* stream, int limit);

/* flups_status_string - static, human-readable name of a status code. */
const char* flups_status_string(int status);

/* flups_last_cuda_error - name of the last CUDA error that made a call of this thread
 * return FLUPS_ECUDA or FLUPS_ENOMEM ("cudaSuccess" if none); static string. */
const char* flups_last_cuda_error(void);

#ifdef __cplusplus
}
#endif

#endif /* FLUPS_H */
