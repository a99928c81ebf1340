// internal.cuh -- shared definitions of the rklpcg CUDA library (not part of the ABI).
//
// Operator storage.  The frozen operator is M = -W^{-1} S with S symmetric positive
// semi-definite.  S is kept once per cell as its "forward" off-diagonal entries (to
// the neighbours at lexicographically positive offsets) plus its diagonal, in
// structure-of-arrays form coef[slot * N + cell]:
//   conduction (19-point): 9 forward slots FWD[0..8] + diagonal in slot 9
//   viscosity  (7-point):  3 forward slots FWD[0..2] + diagonal in slot 3
// The entry of row c towards c - FWD[m] is the forward entry FWD[m] stored at the
// neighbour c - FWD[m], so S is exactly symmetric by construction.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <type_traits>
#include <vector>

#include "../../include/rklpcg.h"

#define RKL_RSUN_CM 6.96e10  // default length unit of the radial faces (rkl_grid.rsun_cm = 0)
#define RKL_KBOLTZ 1.380649e-16
#define RKL_TCUT 5.0e5
#define RKL_PI 3.14159265358979323846

namespace rkl {

// lexicographically positive neighbour offsets FWD[m] = (di, dj, dk) along (r, theta, phi):
//   m: 0 (1,0,0)  1 (0,1,0)  2 (0,0,1)  3 (-1,1,0)  4 (1,1,0)
//      5 (-1,0,1) 6 (1,0,1)  7 (0,-1,1) 8 (0,1,1)
__host__ __device__ constexpr int fwd_di(int m) {
  return (m == 0 || m == 4 || m == 6) ? 1 : ((m == 3 || m == 5) ? -1 : 0);
}
__host__ __device__ constexpr int fwd_dj(int m) {
  return (m == 1 || m == 3 || m == 4 || m == 8) ? 1 : (m == 7 ? -1 : 0);
}
__host__ __device__ constexpr int fwd_dk(int m) { return (m == 2 || m >= 5) ? 1 : 0; }

enum { NCOEF_COND = 10, NCOEF_VISC = 4, NCOEF_FULL = 19 };

// Operator kinds of a context (template argument OP of the kernels): the two public
// operators with symmetric storage, conduction in the non-symmetric flux form
// (RKL_FLUX_FORM) with full-row storage, and symmetric conduction with across-pole
// theta-ghosts (RKL_ACROSS_POLE).
enum { OPK_COND = RKL_OP_CONDUCTION, OPK_VISC = RKL_OP_VISCOSITY, OPK_FLUX = 2, OPK_POLE = 3 };

__host__ __device__ constexpr int op_ncoef(int op) {
  return op == OPK_VISC ? NCOEF_VISC : (op == OPK_FLUX ? NCOEF_FULL : NCOEF_COND);
}

// Across-pole couplings (OPK_POLE).  With the theta-ghost beyond a pole taken at phi + pi,
// a cell X = (i, j0, k) of a pole row (j0 = 0 or nth - 1) couples to the five cells
// (i + PDI[q], j0, k + nph/2 + PDK[q]) of the antipodal column.  Their entries are kept
// after the 10 symmetric slots, at coef + 10 N, as [q][side][k][i] with side 0 for j0 = 0
// and 1 for j0 = nth - 1 (full rows: the entry of X towards Y is stored at X and, equal,
// at Y).  Every coefficient array holds room for them.
__host__ __device__ constexpr int pole_di(int q) { return q == 1 ? 1 : (q == 2 ? -1 : 0); }
__host__ __device__ constexpr int pole_dk(int q) { return q == 3 ? 1 : (q == 4 ? -1 : 0); }
enum { NPOLE = 5 };

// f(std::integral_constant<int, OP>{}) for the operator kind op of a context
template <typename F>
inline void op_dispatch(int op, F &&f) {
  if (op == OPK_COND) f(std::integral_constant<int, OPK_COND>{});
  else if (op == OPK_FLUX) f(std::integral_constant<int, OPK_FLUX>{});
  else if (op == OPK_POLE) f(std::integral_constant<int, OPK_POLE>{});
  else f(std::integral_constant<int, OPK_VISC>{});
}

struct Dims {
  int nr, nth, nph;
  long long N;
  long long nrt;  // nr * nth (one phi layer)
};

// doubles (or floats) of the across-pole entries that follow the slots of an operator
__host__ __device__ inline long long pole_extra(const Dims &d) { return (long long)NPOLE * 2 * d.nr * d.nph; }

// Geometry tables in cm (device pointers); built on the host at rkl_create.
struct Geo {
  const double *rc;    // [nr]   cell-centre radius
  const double *hr;    // [nr]   rc[i+1] - rc[i] (last entry unused)
  const double *dr;    // [nr]   span of the centred r-difference (mirror ghosts at ends)
  const double *ar;    // [nr]   rf[i+1]^2 (r-face area over the solid angle)
  const double *a2;    // [nr]   (rf[i+1]^2 - rf[i]^2)/2
  const double *v3;    // [nr]   (rf[i+1]^3 - rf[i]^3)/3
  const double *dcos;  // [nth]  cos(theta_j) - cos(theta_{j+1}) (faces)
  const double *stf;   // [nth]  sin of the upper theta face
  const double *stc;   // [nth]  sin of the cell-centre theta
  double dth, dph;
};

// Scalars of one PCG solve, resident on the device.
struct PcgState {
  double rr;       // r.z
  double rnorm2;   // r.r
  double bnorm2;   // (W u).(W u)
  double pAp;
  double alpha, beta;
  double rtol2;    // rtol^2 (<= 0: never converge)
  int iters;
  int maxit;
  int status;      // 0 running, 1 converged, 2 breakdown, 3 maxit reached
  int loops;       // chunks run by the graph-driven loop (device-side bound)
};

enum { PCG_RUNNING = 0, PCG_CONVERGED = 1, PCG_BREAKDOWN = 2, PCG_MAXIT = 3 };

// block-ILU0 level schedule of one block shape and coupling pattern (device pointers).
// G blocks are solved together by one CTA; their factors are stored group by group as
// [slot][G * bs] with the cells of one wavefront of all G blocks contiguous.
struct IluPlan {
  int bi, bj, bk, bs;     // block dims and cells per block
  int pat;                // coupling pattern kept by the factorisation: 19 or 7 points
  int nlev;               // number of wavefront levels
  int nbi, nbj, nbk;      // blocks along r, theta, phi
  int nblocks, G, ngroups;
  const int *lev_start;   // [nlev+1] offsets into lev_cell
  const int *lev_cell;    // [bs] block-local index (li + bi*(lj + bj*lk)) in level order
  const int *pos_of;      // [bs] level-order position of a block-local index
};

// wavefront of a block-local cell: li + 2 lj + 3 lk for the 19-point pattern (each of its
// nine lower neighbours, (1,-1,0) and (0,1,-1) included, lies on an earlier wavefront),
// li + lj + lk for the 7-point one
__host__ __device__ constexpr int ilu_level(int pat, int li, int lj, int lk) {
  return pat == 7 ? li + lj + lk : li + 2 * lj + 3 * lk;
}
// factor slots per cell: 19-point 0 U_ii, 1..9 L (lower), 10..18 U (upper), 19 1/U_ii;
// 7-point 0 U_ii, 1..3 L, 4..6 U, 7 1/U_ii.  lu_slot maps the generic slot s (0 diagonal,
// 1 + m the lower coupling -FWD[m], 10 + m the upper +FWD[m], 19 the inverse) to the
// stored one, -1 where the pattern has none.
__host__ __device__ constexpr int ilu_nslots(int pat) { return pat == 7 ? 8 : 20; }
__host__ __device__ constexpr int lu_slot(int pat, int s) {
  return pat != 7 ? s : (s <= 3 ? s : (s >= 10 && s <= 12 ? s - 6 : (s == 19 ? 7 : -1)));
}

}  // namespace rkl

struct ProfRec {
  int kind, tag;
  cudaEvent_t a, b;
};

struct rkl_ctx {
  rkl::Dims d;
  int device;
  cudaStream_t stream;
  std::string err;
  std::vector<double> rf;
  double rsun_cm = RKL_RSUN_CM;  // length unit of rf (cm)
  int nsm;

  // geometry
  double *geo_buf = nullptr;
  rkl::Geo geo;

  // frozen operator
  int op = -1;  // operator kind (OPK_*) once set_coeffs succeeded
  double dt_exp = 0.0;
  double *coef = nullptr;   // coef_slots * N (NCOEF_COND at create, NCOEF_FULL for the flux form)
                            // + pole_extra (across-pole entries at coef + 10 N)
  int coef_slots = 0;
  double *W = nullptr;      // N
  double *invW = nullptr;   // N
  double *scratch = nullptr;  // 10 * N: kappa/mu + face scalars during set_coeffs
  unsigned long long *d_lammax = nullptr;
  int *d_flag = nullptr;

  // RKL2
  double *M0 = nullptr, *Ya = nullptr, *Yb = nullptr;

  // mixed precision (prec == RKL_F32MIX): FP32 copies of the frozen operator and FP32
  // work fields
  int prec = RKL_F64;
  float *coef32 = nullptr, *W32 = nullptr, *invW32 = nullptr;
  int coef32_slots = 0;
  float *M0f = nullptr, *da32 = nullptr, *db32 = nullptr;
  float *r32 = nullptr, *p32 = nullptr, *y32 = nullptr, *z32 = nullptr, *e32 = nullptr,
        *dinv32 = nullptr;
  float *LU32 = nullptr;
  size_t lu32_cap = 0;
  double inner_rtol = 1e-4;

  // PCG
  double *r = nullptr, *p = nullptr, *y = nullptr, *zbuf = nullptr, *dinv = nullptr;
  double *acoef = nullptr;  // A = W + dt S in the operator's storage (FP64 solves)
  int acoef_slots = 0, acoef_valid = 0;
  double acoef_dt = 0.0;
  double *partials = nullptr;
  int npart = 0;
  int *d_kerr = nullptr;      // kernel error word, just after the PCG state
  int march_nchunk[2] = {0, 0};  // phi chunks of the marching FP32 kernels per operator (0: not used)
  unsigned int *counter = nullptr;
  rkl::PcgState *d_state = nullptr;
  rkl::PcgState *h_state = nullptr;  // pinned

  // block ILU0
  double *LU = nullptr;
  size_t lu_cap = 0;  // doubles
  int *plan_buf = nullptr;
  rkl::IluPlan plan{};
  int lu_blk[3] = {0, 0, 0};
  double lu_dt = 0.0;
  int lu_valid = 0;

  // number of kernels this context has launched (all entry points)
  long long launches = 0;

  // optional per-kernel event timing (profile.cu)
  int prof_on = 0;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<ProfRec> prof_pending;
  double prof_ms[RKL_K_COUNT] = {};
  long long prof_n[RKL_K_COUNT] = {};

  // CUDA graph of the last super-step's stage launches (rkl2_superstep), replayed when the
  // same call repeats; epoch counts set_coeffs calls (a new operator forces a re-capture)
  cudaGraphExec_t sts_exec = nullptr;
  cudaStream_t cap_stream = nullptr;  // private stream the launches are captured on
  int sts_s = 0, sts_ncomp = 0, sts_prec = -1, sts_op = -1;
  const double *sts_u = nullptr;
  double sts_dt = 0.0;
  long long sts_epoch = -1, sts_nkern = 0, epoch = 0;
  int sts_direct_done = 0;  // the first super-step runs without a graph (loads the kernels)

  // CUDA graph of the PCG loop (a WHILE node over chunks of iterations), kept for the
  // last solve's kernels, fields, dt, preconditioner and operator
  cudaGraphExec_t pcg_exec = nullptr;
  cudaGraph_t pcg_graph = nullptr;     // kept while pcg_exec lives (it owns the conditional handle)
  cudaStream_t pcg_stream = nullptr;   // the PCG graph's own capture stream
  unsigned long long pcg_key = 0;
  int pcg_kpc = 0;  // kernels per chunk of the cached graph (including the condition kernel)

  // host-pointer staging
  double *stage = nullptr;
  size_t stage_cap = 0;  // doubles
  double *stage2 = nullptr;
  size_t stage2_cap = 0;
};

namespace rkl {

// Brackets one launch (or a fixed group of launches) with events when profiling is on;
// tag = iteration index inside a PCG chunk, or -1.
struct ProfScope {
  rkl_ctx *ctx;
  int kind, tag;
  cudaEvent_t a;
  ProfScope(rkl_ctx *c, int k, int t = -1);
  ~ProfScope();
};
void prof_settle(rkl_ctx *ctx, int n_real, bool still_running, bool chunk);
void prof_release(rkl_ctx *ctx);

int set_error(rkl_ctx *ctx, int code, const std::string &msg);
int cuda_check(rkl_ctx *ctx, cudaError_t e, const char *what);
int ensure_buffer(rkl_ctx *ctx, double **buf, size_t count, const char *what);
int ensure_fbuffer(rkl_ctx *ctx, float **buf, size_t count, const char *what);

inline unsigned int grid_for(long long n, int block) {
  return (unsigned int)((n + block - 1) / block);
}

// ---- launch wrappers (defined in the .cu files) ----
// coeffs.cu
int launch_setup_conduction(rkl_ctx *ctx, const double *T, const double *bhat, const double *n,
                            double kappa0, int flags);
int launch_setup_viscosity(rkl_ctx *ctx, const double *rho, const double *nu);

// rkl2.cu
int launch_apply_F(rkl_ctx *ctx, const double *u, double *Fu);
int launch_rkl2_stage1(rkl_ctx *ctx, const double *Y0, double *M0, double *Y1, double mut1dt);
int launch_rkl2_stage(rkl_ctx *ctx, const double *Ym1, const double *Ym2, const double *Y0,
                      const double *M0, double *Yout, double mu, double nu, double mutdt,
                      double gtdt);

// context-free launchers (explicit buffers, conduction), used by the allocation-free
// super-step of noalloc.cu
int launch_setup_conduction_raw(const Dims &d, const Geo &g, cudaStream_t stream, const double *T,
                                const double *bhat, const double *n, double kappa0, int flags,
                                double *kappa, double *FS, double *W, double *invW, double *coef,
                                unsigned long long *lammax, int *flag);
int launch_rkl2_first_raw(const Dims &d, cudaStream_t stream, const double *coef,
                          const double *invW, const double *Y0, double *M0, double *Y1,
                          double mut1dt);
int launch_rkl2_stage_raw(const Dims &d, cudaStream_t stream, const double *coef,
                          const double *invW, const double *Ym1, const double *Ym2,
                          const double *Y0, const double *M0, double *Yout, double mu, double nu,
                          double mutdt, double gtdt);

int launch_to_float(rkl_ctx *ctx, const double *a, float *b, long long n);
int march_setup_stage(rkl_ctx *ctx);
int march_setup_spmv(rkl_ctx *ctx);
// RKL_ECUDA when a kernel's bounded wait ran out since the last check (the word is
// cleared); `word` is the value already read back with the PCG state, or nullptr to read it
int check_kerr(rkl_ctx *ctx, const int *word);
int launch_rkl2_first_mix(rkl_ctx *ctx, const double *Y0, float *M0f, float *d1, double mut1dt);
int launch_rkl2_stage_mix(rkl_ctx *ctx, const float *dm1, const float *dm2, const float *M0f,
                          float *dout, double *u, double mu, double nu, double mutdt, double cm0);

// pcg.cu
int pcg_solve_component(rkl_ctx *ctx, double *x, const double *u, const double *x0, double dt,
                        int pc, double rtol, int maxit, int *iters, double *relres,
                        int *status);
int bilu0_prepare(rkl_ctx *ctx, const int *block, double dt);

}  // namespace rkl
