/*
 * rklpcg.h -- C ABI of the GB300 (sm_103a) library that advances frozen-coefficient
 * parabolic operators u_t = F(u) on a logically rectangular spherical (r, theta, phi)
 * grid by RKL2 super-time-stepping or by backward Euler + preconditioned CG, after
 * Caplan, Mikic, Linker & Lionello, arXiv:1610.01265.
 *
 * Operators (Sec. 4.1, boxed blue terms):
 *   conduction  F(T) = (1/(3 k n)) div(kappa0 T^{5/2} bhat bhat . grad T)
 *   viscosity   F(v) = (1/rho) div(nu rho grad v), per Cartesian component of v
 * discretised with coefficients frozen at the start of a large step (lagged
 * diffusivity, Sec. 1) so that F(u) = M u, M = -W^{-1} S, with S symmetric positive
 * semi-definite (19-point anisotropic stencil for conduction, App. B p = 19;
 * 7-point for viscosity) and W the cell heat capacity (3 k n V) or mass (rho V).
 *
 * Grid and layout.  nr x nth x nph cells; radial faces given by the caller (any
 * strictly increasing positive radii, in units of rkl_grid.rsun_cm, by default
 * R_sun = 6.96e10 cm); theta faces
 * j pi / nth (cell-centred, zero-area pole faces); phi faces k 2 pi / nph, periodic.
 * Zero-flux boundaries at the first and last radial face.  Every field is a
 * contiguous float64 array indexed ((k * nth) + j) * nr + i, r fastest; a field of
 * ncomp components is ncomp such arrays back to back.
 *
 * Memory.  Array arguments may be CUDA device pointers (the fast path) or host
 * pointers (pageable or pinned); host arrays are copied through device buffers owned
 * by the context on the context's stream inside the call, which then returns only
 * after the result is back in host memory.  The library never frees, and never
 * keeps after the call returns, any caller pointer.  With device pointers every
 * call is asynchronous on the context's stream except for the scalar outputs
 * (*_out), which are valid when the call returns.
 *
 * Errors.  Every entry point returns RKL_OK (0) or a negative RKL_E* code; nothing
 * aborts or throws across the ABI.  rkl_strerror() names a code and
 * rkl_last_error() gives the context's last detailed message.  Device-side failures
 * (non-finite inputs, CG breakdown, non-convergence) are reported through a status
 * word written by the kernels, never by trapping the GPU.  The FP32 kernels that stream
 * planes through bulk asynchronous copies wait for them with a time limit (about two
 * seconds); a wait that runs out (a device fault, never an ordinary outcome) writes NaN
 * over the outputs of that kernel and sets an error word, and the next call that
 * synchronises with the device (a PCG state read, or the end of a call on host arrays)
 * returns RKL_ECUDA and clears it.  A context is not thread-safe: one host thread at a
 * time.
 */
#ifndef RKLPCG_H
#define RKLPCG_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rkl_ctx rkl_ctx;

typedef struct {
  int nr, nth, nph;       /* cells along r, theta, phi: nr >= 1, 1 <= nth, 3 <= nph, both <= 65535 */
  const double *r_faces;  /* HOST array of nr+1 radial faces in units of rsun_cm, copied at create */
  double rsun_cm;         /* length unit of r_faces in cm; 0 selects R_sun = 6.96e10 cm
                             (negative or non-finite: RKL_EINVAL) */
} rkl_grid;

enum {
  RKL_OK = 0,
  RKL_EINVAL = -1,     /* bad argument (null pointer, size, dt, s, block ...) */
  RKL_ENOMEM = -2,     /* device allocation failed */
  RKL_ECUDA = -3,      /* a CUDA runtime call failed (see rkl_last_error) */
  RKL_ENONFINITE = -4, /* NaN/Inf or non-positive T, n, rho, nu found in the inputs */
  RKL_ENOTCONV = -5,   /* PCG reached maxit without meeting rtol (u holds x_maxit) */
  RKL_EBREAKDOWN = -6, /* PCG breakdown: p.Ap <= 0 or not finite (u holds the last x) */
  RKL_ESTATE = -7      /* call out of order (e.g. a solver before set_coeffs) */
};

enum { RKL_OP_CONDUCTION = 0, RKL_OP_VISCOSITY = 1 };
enum { RKL_PC_JACOBI = 1, RKL_PC_BILU0 = 2 };
enum { RKL_F64 = 0, RKL_F32MIX = 1 };

#define RKL_BETA_TCUT 1 /* set_coeffs: kappa times (T / 5e5 K)^{5/2} below 5e5 K (Sec. 4.1 beta_Tcut) */
#define RKL_FLUX_FORM 2 /* set_coeffs (conduction): non-symmetric flux form, see set_coeffs */
#define RKL_ACROSS_POLE 4 /* set_coeffs (conduction): theta-ghosts beyond a pole at phi + pi, see set_coeffs */
#define RKL_FORCE_ODD 1 /* rkl2_superstep: round s up to an odd number (Sec. 3) */

/* Create a context for one grid on the current CUDA device.
 * prec = RKL_F64: every step in FP64.
 * prec = RKL_F32MIX (mixed precision; same FP64 inputs and outputs): set_coeffs also
 *   keeps FP32 copies of the operator; rkl2_superstep runs the stages in FP32 on the
 *   increments Y_j - Y_0 with FP64 stage coefficients, M0 = F(Y0) in FP64 and the
 *   result Y_0 + (Y_s - Y_0) formed in FP64; be_pcg_solve is FP64 iterative refinement
 *   (FP64 residual and stopping test, FP32 PCG correction solves whose dot products
 *   are accumulated in FP64 from FP32 partials of a few cells, FP64 update), so it
 *   meets the same rtol; iters_out then counts FP32 iterations.  apply_F stays FP64.
 * cuda_stream: a cudaStream_t (NULL = legacy default stream) on which all work of
 * this context is queued.  Allocates the geometry tables; coefficient, stage and
 * Krylov buffers are allocated on first use and kept until rkl_destroy. */
int rkl_create(rkl_ctx **ctx, const rkl_grid *g, int prec, void *cuda_stream);

/* Synchronise the context's stream and free everything it owns. NULL is a no-op. */
int rkl_destroy(rkl_ctx *ctx);

/* Re-bind the context to another stream (subsequent calls only). */
int rkl_set_stream(rkl_ctx *ctx, void *cuda_stream);

const char *rkl_strerror(int code);
const char *rkl_last_error(const rkl_ctx *ctx);

/* Kernel families timed by the optional profiler. */
enum {
  RKL_K_SETUP = 0,       /* set_coeffs kernels (one record per call) */
  RKL_K_APPLY_F = 1,
  RKL_K_RKL2_FIRST = 2,  /* stage 1: M0 = F(Y0), Y1 */
  RKL_K_RKL2_STAGE = 3,  /* fused stencil + stage j >= 2 */
  RKL_K_PCG_INIT = 4,    /* r0, first preconditioner application, p0 */
  RKL_K_SPMV = 5,        /* y = (W + dt S) p, p.y */
  RKL_K_PCG_UPDATE = 6,  /* x, r update (+ Jacobi z, r.z, r.r) */
  RKL_K_PCG_PUPDATE = 7, /* p = z + beta p */
  RKL_K_BILU_FACTOR = 8,
  RKL_K_BILU_APPLY = 9,  /* block-ILU0 solve + r.z, r.r */
  RKL_K_COUNT = 10
};

/* Per-kernel timing with CUDA events recorded on the context's stream around every
 * launch (instrumentation; no paper counterpart).  on != 0 clears the counters and starts
 * recording, 0 stops.  PCG launches queued after convergence, which return at once, are
 * not counted.  rkl_profile_read synchronises the stream and returns the total time (ms)
 * and the number of counted launches of one family. */
int rkl_profile_enable(rkl_ctx *ctx, int on);
int rkl_profile_read(rkl_ctx *ctx, int kernel, double *total_ms, long long *launches);

/* Measured FP64 fused-multiply-add throughput of the current device in TFLOP/s (2 flop
 * per FMA), the roof of the FP64 stencil kernels (instrumentation for the roofline; no
 * paper counterpart).  Runs a kernel of 8 independent FMA chains per thread on 8 CTAs of
 * 256 threads per SM, for about 50 ms, on cuda_stream (NULL = legacy default stream),
 * three times after a warm-up, and reports the fastest; synchronises the stream.  It
 * allocates and frees a small result buffer (2.5 MB on 152 SMs). */
int rkl_fp64_peak(void *cuda_stream, double *tflops_out);

/* Number of CUDA kernels this context has launched since rkl_create (instrumentation:
 * every launch of every entry point is counted, including PCG iterations queued after
 * convergence that return at once).  -1 for a NULL context.  No paper counterpart. */
long long rkl_kernel_launches(const rkl_ctx *ctx);

/* Eq. 5 (Sec. 3): number of RKL2 stages for dt/dt_exp, read as
 * s = ceil((sqrt(9 + 16 dt/dt_exp) - 1) / 2), at least 2, odd with RKL_FORCE_ODD.
 * Returns s, or RKL_EINVAL for a non-positive or non-finite ratio. */
int rkl2_stage_count(double dt_over_dt_exp, int flags);

/* Freeze the operator's coefficients for one large step (lagged diffusivity, Sec. 1;
 * Sec. 4.1 for the coefficients) and compute the explicit Euler limit
 * dt_exp = 2 / max_i sum_j |M_ij| (App. B, Eqs. 6-7, Gershgorin row sums).
 *   op = RKL_OP_CONDUCTION: a = T [N] (K), b = bhat [3N] (r, theta, phi unit-vector
 *        components), c = n [N] (cm^-3), kappa0 (cgs, 9e-7 in the paper);
 *        flags may hold RKL_BETA_TCUT and RKL_FLUX_FORM.  By default S is the
 *        symmetric Hessian of the discrete energy; with RKL_FLUX_FORM row c is minus
 *        the divergence of the face fluxes A_f (D^aa g_f + sum_b D^ab ghat_b) through
 *        the faces of c (the "standard" scheme of Sec. 4.2), a non-symmetric operator
 *        (about 7% antisymmetric on coronal fields) with the same symmetric part,
 *        stored as full 19-entry rows (152 B per cell instead of 80).  Every solver
 *        accepts it; PCG then runs as for "slightly non-symmetric" operators (Sec. 2.1)
 *        and still stops on the true residual.  rkl2_superstep_noalloc does not.
 *        With RKL_ACROSS_POLE (symmetric form only; needs nth >= 2 and an even
 *        nph >= 6, else RKL_EINVAL) the theta-difference of a cell next to a pole is
 *        taken across the pole (Sec. 4.2 boundaries): its ghost is the cell of the same
 *        row at phi + pi instead of the cell itself, which makes the difference a centred
 *        one along the meridian continued through the pole (consistent there, where the
 *        mirror ghost is not) and couples each pole cell to five cells of the antipodal
 *        column.  S stays symmetric with zero row sums; it is no longer positive
 *        semi-definite to rounding: one or two eigenvalues are slightly negative (about
 *        -1e-5 of the largest at 6 theta rows, -1e-7 at 24), so RKL2 lets those modes grow
 *        by about exp(|lambda| dt) per step and BE stays definite while dt |lambda| is
 *        below the smallest W.  The block-ILU0 preconditioner drops the across-pole
 *        couplings (they leave every block, like those across the phi seam).
 *   op = RKL_OP_VISCOSITY:  a = rho [N] (g cm^-3), b = NULL, c = nu [N] (cm^2/s);
 *        kappa0 is ignored; RKL_FLUX_FORM is RKL_EINVAL, other flags are ignored
 *        (the 7-point viscosity operator has no transverse differences).
 * dt_exp_out (host, may be NULL) receives dt_exp in seconds.  Invalidates any
 * cached preconditioner.  RKL_ENONFINITE if an input is NaN/Inf or T, n, rho, nu <= 0. */
int set_coeffs(rkl_ctx *ctx, int op, const double *a, const double *b, const double *c,
               double kappa0, int flags, double *dt_exp_out);

/* Fu = F(u) = -W^{-1} S u for each of ncomp components (Eq. 1).  u and Fu must not
 * overlap.  One stencil pass per component. */
int apply_F(rkl_ctx *ctx, const double *u, double *Fu, int ncomp);

/* In place u <- Y_s, one RKL2 super-step of size dt (Fig. 2, coefficients of Sec. 3,
 * with the M0 weight gamma~_j = -(1 - b_{j-1}) mu~_j).  s > 0 uses exactly s stages
 * (s >= 2); s == 0 takes s from Eq. 5 with dt/dt_exp (and RKL_FORCE_ODD in flags).
 * s_used (host, may be NULL) receives the number of stages run.  Stability needs
 * dt <= dt_exp (s^2 + s - 2)/4, which Eq. 5 guarantees when dt_exp is set_coeffs'. */
int rkl2_superstep(rkl_ctx *ctx, double *u, int ncomp, double dt, double dt_exp, int s,
                   int flags, int *s_used);

/* Damping variants of the super-step discussed in Sec. 6: an explicit-Euler prefix over
 * a fraction of dt (sub-steps no larger than dt_exp), then `cycles` equal sub-cycles of
 * RKL2 (or of first-order RKL1), each with the minimal stable number of stages plus
 * `extra_stages`.  euler_fraction = 0, cycles = 1, extra_stages = 0 and RKL2 is exactly
 * rkl2_superstep with s from Eq. 5. */
enum { RKL_SCHEME_RKL2 = 0, RKL_SCHEME_RKL1 = 1 };
typedef struct {
  int scheme;             /* RKL_SCHEME_RKL2 or RKL_SCHEME_RKL1 */
  int cycles;             /* sub-cycles of the super-time-stepping part, >= 1 */
  int extra_stages;       /* stages beyond the minimal stable count, >= 0 */
  double euler_fraction;  /* leading fraction of dt taken by explicit Euler, in [0, 1) */
  int flags;              /* RKL_FORCE_ODD (RKL2 stage counts) */
} rkl_sts_options;

/* In place u <- advance by dt with the variant in *opt (FP64 kernels, any context
 * precision).  stages_used (host, may be NULL) receives the total number of operator
 * applications (Euler sub-steps + stages of all cycles). */
int sts_advance(rkl_ctx *ctx, double *u, int ncomp, double dt, double dt_exp,
                const rkl_sts_options *opt, int *stages_used);

/* In place backward-Euler step (Eqs. 2-4): solve (W + dt S) x = W u for each
 * component by PCG (Fig. 1), from x0 (or from u when x0 is NULL), stopping when
 * ||r||_2 <= rtol ||W u||_2 (tested after r.z as in Fig. 1) or after maxit
 * products A p.  pc = RKL_PC_JACOBI (PC1) or RKL_PC_BILU0 (PC2: zero-fill ILU of
 * every block[0] x block[1] x block[2] sub-domain, couplings between blocks and
 * across the phi seam dropped, App. A); block is ignored for PC1.  For PC2 the grid
 * must be divisible by the block, which holds at most 4096 cells (else RKL_EINVAL).
 * rtol <= 0 runs exactly maxit iterations.
 * iters_out / relres_out (host, may be NULL) receive ncomp values each: the number
 * of A p products and the final ||r||/||W u||.  Returns RKL_ENOTCONV if some
 * component did not converge, RKL_EBREAKDOWN on p.Ap <= 0. */
int be_pcg_solve(rkl_ctx *ctx, double *u, int ncomp, double dt, int pc, const int block[3],
                 double rtol, int maxit, const double *x0, int *iters_out,
                 double *relres_out);

/* Allocation-free conduction super-step: set_coeffs(RKL_OP_CONDUCTION) followed by
 * rkl2_superstep, without a context, for callers that cannot call cudaMalloc -- a host
 * code whose own pool owns all device memory and fixes its footprint at start-up, or a
 * time loop that cannot afford the device-wide synchronisation that cudaMalloc and
 * cudaFree may cause.  The paper has no counterpart: this packages the same operator
 * set-up and super-step with no memory management.
 * Everything kept between kernels (geometry tables, frozen coefficients, W, 1/W, M0 and
 * two stage fields, the Gershgorin maximum) lives in one static device array of this
 * library, about 12.6 MiB, which a GPU holds from its first use until the process exits;
 * hence nr <= 1024, nth <= 1024 and nr*nth*nph <= 65536 cells (RKL_EINVAL beyond).
 * T [N], bhat [3N], n [N] and u [N] must be device pointers (RKL_EINVAL otherwise); u is
 * advanced in place.  kappa0 and coeff_flags are those of set_coeffs (RKL_BETA_TCUT
 * only: RKL_FLUX_FORM and RKL_ACROSS_POLE are RKL_EINVAL); dt and flags are those of rkl2_superstep; s > 0
 * runs exactly s stages, s == 0 the stage count that rkl2_stage_count gives for dt over
 * the dt_exp computed here.  dt_exp_out and s_used (host, may be NULL) receive dt_exp and
 * the number of stages.
 * The first call on a device looks up the device address of the static array with that
 * device current (cudaGetSymbolAddress); make that first call before any stream capture.
 * All calls on a device share the array, which keeps the last call's contents: calls
 * that overlap on the GPU (several streams, or host threads driving the same device)
 * race on it and must be serialised by the caller.  The host-side steps (the address
 * look-up, the staging of the geometry tables) are serialised by the library, so calls
 * from several host threads on different devices do not interfere.  The call returns once dt_exp is known (one small device-to-host read);
 * the stage kernels then run asynchronously on cuda_stream. */
int rkl2_superstep_noalloc(const rkl_grid *g, const double *T, const double *bhat,
                           const double *n, double kappa0, int coeff_flags, double *u,
                           double dt, int s, int flags, void *cuda_stream, double *dt_exp_out,
                           int *s_used);

#ifdef __cplusplus
}
#endif

#endif /* RKLPCG_H */
