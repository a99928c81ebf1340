// api.cu -- the C ABI declared in include/rklpcg.h: context, argument checks, host
// staging of host-memory arrays, the RKL2 stage loop and the PCG driver.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "internal.cuh"
#include "march.cuh"

namespace rkl {

int set_error(rkl_ctx *ctx, int code, const std::string &msg) {
  if (ctx) ctx->err = msg;
  return code;
}

int cuda_check(rkl_ctx *ctx, cudaError_t e, const char *what) {
  if (e == cudaSuccess) return RKL_OK;
  std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  if (e == cudaErrorMemoryAllocation) return set_error(ctx, RKL_ENOMEM, m);
  return set_error(ctx, RKL_ECUDA, m);
}

int ensure_buffer(rkl_ctx *ctx, double **buf, size_t count, const char *what) {
  if (*buf) return RKL_OK;
  return cuda_check(ctx, cudaMalloc((void **)buf, count * sizeof(double)), what);
}

int ensure_fbuffer(rkl_ctx *ctx, float **buf, size_t count, const char *what) {
  if (*buf) return RKL_OK;
  return cuda_check(ctx, cudaMalloc((void **)buf, count * sizeof(float)), what);
}

int check_kerr(rkl_ctx *ctx, const int *word) {
  int v = 0;
  if (word) {
    v = *word;
  } else {
    int rc = cuda_check(ctx, cudaMemcpy(&v, ctx->d_kerr, sizeof(int), cudaMemcpyDeviceToHost), "error word read");
    if (rc) return rc;
  }
  if (!v) return RKL_OK;
  int rc = cuda_check(ctx, cudaMemsetAsync(ctx->d_kerr, 0, sizeof(int), ctx->stream), "error word clear");
  if (rc) return rc;
  return set_error(ctx, RKL_ECUDA, "a kernel's bounded wait for its asynchronous copies ran out; its outputs hold NaN");
}

}  // namespace rkl

using namespace rkl;

namespace {

bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

// Build the geometry tables (cm) of the grid on the host and upload them.
int build_geometry(rkl_ctx *ctx) {
  const int nr = ctx->d.nr, nth = ctx->d.nth, nph = ctx->d.nph;
  const double *rf = ctx->rf.data();
  const double RS = ctx->rsun_cm;
  const double dth = RKL_PI / nth, dph = 2.0 * RKL_PI / nph;
  std::vector<double> rc(nr), hr(nr), dr(nr), ar(nr), a2(nr), v3(nr), dcos(nth), stf(nth), stc(nth);
  for (int i = 0; i < nr; i++) rc[i] = 0.5 * (rf[i] + rf[i + 1]);
  auto rghost = [&](int i) {
    if (i < 0) return 2.0 * rf[0] - rc[0];
    if (i >= nr) return 2.0 * rf[nr] - rc[nr - 1];
    return rc[i];
  };
  for (int i = 0; i < nr; i++) {
    hr[i] = (i + 1 < nr ? rc[i + 1] - rc[i] : 0.0) * RS;
    dr[i] = (rghost(i + 1) - rghost(i - 1)) * RS;
    ar[i] = rf[i + 1] * rf[i + 1] * RS * RS;
    a2[i] = 0.5 * (rf[i + 1] * rf[i + 1] - rf[i] * rf[i]) * RS * RS;
    v3[i] = (rf[i + 1] * rf[i + 1] * rf[i + 1] - rf[i] * rf[i] * rf[i]) / 3.0 * RS * RS * RS;
  }
  for (int j = 0; j < nth; j++) {
    dcos[j] = std::cos(j * dth) - std::cos((j + 1) * dth);
    stf[j] = std::sin((j + 1) * dth);
    stc[j] = std::sin((j + 0.5) * dth);
  }
  for (int i = 0; i < nr; i++) rc[i] *= RS;
  std::vector<double> all;
  for (auto *v : {&rc, &hr, &dr, &ar, &a2, &v3}) all.insert(all.end(), v->begin(), v->end());
  for (auto *v : {&dcos, &stf, &stc}) all.insert(all.end(), v->begin(), v->end());
  int rc_ = cuda_check(ctx, cudaMalloc(&ctx->geo_buf, all.size() * sizeof(double)), "alloc geometry");
  if (rc_) return rc_;
  rc_ = cuda_check(ctx, cudaMemcpy(ctx->geo_buf, all.data(), all.size() * sizeof(double),
                                   cudaMemcpyHostToDevice), "upload geometry");
  if (rc_) return rc_;
  const double *p = ctx->geo_buf;
  Geo &g = ctx->geo;
  g.rc = p; p += nr;
  g.hr = p; p += nr;
  g.dr = p; p += nr;
  g.ar = p; p += nr;
  g.a2 = p; p += nr;
  g.v3 = p; p += nr;
  g.dcos = p; p += nth;
  g.stf = p; p += nth;
  g.stc = p;
  g.dth = dth;
  g.dph = dph;
  return RKL_OK;
}

bool is_device_ptr(const void *p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Staging arena for host arrays.  Every entry point sizes the arena for all of its
// arguments (ensure_stage) before staging the first one, so that a view handed out
// for one argument is never invalidated by a reallocation for the next.
int ensure_stage(rkl_ctx *ctx, size_t need) {
  if (need <= ctx->stage_cap) return RKL_OK;
  if (ctx->stage) {
    int rc = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "staging resize");
    if (rc) return rc;
    cudaFree(ctx->stage);
    ctx->stage = nullptr;
    ctx->stage_cap = 0;
  }
  int rc = cuda_check(ctx, cudaMalloc(&ctx->stage, need * sizeof(double)), "alloc staging");
  if (rc) return rc;
  ctx->stage_cap = need;
  return RKL_OK;
}

int stage_view(rkl_ctx *ctx, size_t offset, size_t n, double **out) {
  if (offset + n > ctx->stage_cap) return set_error(ctx, RKL_ECUDA, "internal: staging arena too small");
  *out = ctx->stage + offset;
  return RKL_OK;
}

// Make `p` (n doubles) usable on the device; host arrays are copied in (if `in`).
int to_device(rkl_ctx *ctx, const double *p, size_t n, size_t offset, bool in, double **dev,
              bool *staged) {
  *staged = false;
  if (is_device_ptr(p)) {
    *dev = const_cast<double *>(p);
    return RKL_OK;
  }
  int rc = stage_view(ctx, offset, n, dev);
  if (rc) return rc;
  *staged = true;
  if (in)
    return cuda_check(ctx, cudaMemcpyAsync(*dev, p, n * sizeof(double), cudaMemcpyHostToDevice,
                                           ctx->stream), "host->device copy");
  return RKL_OK;
}

int from_device(rkl_ctx *ctx, double *host, const double *dev, size_t n) {
  return cuda_check(ctx, cudaMemcpyAsync(host, dev, n * sizeof(double), cudaMemcpyDeviceToHost,
                                         ctx->stream), "device->host copy");
}

int sync(rkl_ctx *ctx, const char *what) {
  int rc = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), what);
  return rc ? rc : check_kerr(ctx, nullptr);
}

// RKL2 coefficients of Sec. 3 for stage j (b_0 = b_1 = b_2 = 1/3)
double rkl_b(int j) { return j <= 2 ? 1.0 / 3.0 : ((double)j * j + j - 2.0) / (2.0 * j * (j + 1.0)); }

}  // namespace

extern "C" {

const char *rkl_strerror(int code) {
  switch (code) {
    case RKL_OK: return "ok";
    case RKL_EINVAL: return "invalid argument";
    case RKL_ENOMEM: return "out of device memory";
    case RKL_ECUDA: return "CUDA runtime error";
    case RKL_ENONFINITE: return "non-finite or non-positive input";
    case RKL_ENOTCONV: return "PCG did not converge within maxit";
    case RKL_EBREAKDOWN: return "PCG breakdown (p.Ap <= 0 or not finite)";
    case RKL_ESTATE: return "call out of order (set_coeffs first)";
    default: return "unknown error code";
  }
}

const char *rkl_last_error(const rkl_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

long long rkl_kernel_launches(const rkl_ctx *ctx) { return ctx ? ctx->launches : -1; }

int rkl2_stage_count(double ratio, int flags) {
  if (!(std::isfinite(ratio) && ratio > 0.0)) return RKL_EINVAL;
  double s = std::ceil((std::sqrt(9.0 + 16.0 * ratio) - 1.0) / 2.0);
  if (!(s < 1e8)) return RKL_EINVAL;
  int si = std::max(2, (int)s);
  if ((flags & RKL_FORCE_ODD) && si % 2 == 0) si++;
  return si;
}

int rkl_create(rkl_ctx **out, const rkl_grid *g, int prec, void *stream) {
  if (!out) return RKL_EINVAL;
  *out = nullptr;
  if (!g || !g->r_faces || (prec != RKL_F64 && prec != RKL_F32MIX)) return RKL_EINVAL;
  if (g->nr < 1 || g->nth < 1 || g->nph < 3) return RKL_EINVAL;
  if (g->nth > 65535 || g->nph > 65535) return RKL_EINVAL;  // 3-D launches put (j, k) on the grid
  if ((long long)g->nr * g->nth * g->nph > (1LL << 40)) return RKL_EINVAL;
  if (!(g->rsun_cm == 0.0 || finite_pos(g->rsun_cm))) return RKL_EINVAL;
  for (int i = 0; i <= g->nr; i++) {
    if (!finite_pos(g->r_faces[i])) return RKL_EINVAL;
    if (i > 0 && !(g->r_faces[i] > g->r_faces[i - 1])) return RKL_EINVAL;
  }
  rkl_ctx *ctx = new (std::nothrow) rkl_ctx();
  if (!ctx) return RKL_ENOMEM;
  ctx->d.nr = g->nr;
  ctx->d.nth = g->nth;
  ctx->d.nph = g->nph;
  ctx->d.nrt = (long long)g->nr * g->nth;
  ctx->d.N = ctx->d.nrt * g->nph;
  ctx->rf.assign(g->r_faces, g->r_faces + g->nr + 1);
  if (g->rsun_cm > 0.0) ctx->rsun_cm = g->rsun_cm;
  ctx->stream = (cudaStream_t)stream;
  ctx->prec = prec;
  int rc = cuda_check(ctx, cudaGetDevice(&ctx->device), "cudaGetDevice");
  if (!rc) rc = cuda_check(ctx, cudaDeviceGetAttribute(&ctx->nsm, cudaDevAttrMultiProcessorCount, ctx->device), "SM count");
  if (!rc) rc = build_geometry(ctx);
  const size_t N = (size_t)ctx->d.N;
  if (!rc)
    rc = cuda_check(ctx, cudaMalloc(&ctx->coef, (NCOEF_COND * N + pole_extra(ctx->d)) * sizeof(double)),
                    "alloc coefficients");
  if (!rc) ctx->coef_slots = NCOEF_COND;
  if (!rc) rc = cuda_check(ctx, cudaMalloc(&ctx->W, N * sizeof(double)), "alloc W");
  if (!rc) rc = cuda_check(ctx, cudaMalloc(&ctx->invW, N * sizeof(double)), "alloc 1/W");
  if (!rc) rc = cuda_check(ctx, cudaMalloc(&ctx->d_lammax, sizeof(unsigned long long) + 2 * sizeof(int)), "alloc flags");
  if (!rc) {
    ctx->d_flag = (int *)(ctx->d_lammax + 1);
    ctx->npart = 2 * ctx->nsm * 8;
    rc = cuda_check(ctx, cudaMalloc(&ctx->partials, (size_t)ctx->npart * sizeof(double)), "alloc partials");
  }
  if (!rc) rc = cuda_check(ctx, cudaMalloc(&ctx->counter, sizeof(unsigned int)), "alloc counter");
  if (!rc) rc = cuda_check(ctx, cudaMemset(ctx->counter, 0, sizeof(unsigned int)), "clear counter");
  // the PCG state, followed by the kernel error word (set by a bounded wait that ran out)
  if (!rc) rc = cuda_check(ctx, cudaMalloc(&ctx->d_state, sizeof(PcgState) + 16), "alloc PCG state");
  if (!rc) {
    ctx->d_kerr = (int *)(ctx->d_state + 1);
    rc = cuda_check(ctx, cudaMemset(ctx->d_kerr, 0, sizeof(int)), "clear error word");
  }
  if (!rc) rc = cuda_check(ctx, cudaMallocHost(&ctx->h_state, sizeof(PcgState) + 64), "alloc pinned state");
  if (!rc && march_ok(ctx->d.nr)) {  // FP32 conduction kernels fed by bulk copies
    int smem_sm = 0;
    rc = cuda_check(ctx, cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, ctx->device),
                    "shared memory per SM");
    for (int op = OPK_COND; !rc && op <= OPK_VISC; op++)
      ctx->march_nchunk[op] = march_chunks(ctx->d.nth, ctx->d.nph, ctx->d.nr, op, ctx->nsm, smem_sm, ctx->npart);
  }
  if (!rc && march_ok(ctx->d.nr)) {
    rc = march_setup_stage(ctx);
    if (!rc) rc = march_setup_spmv(ctx);
  }
  if (rc) {
    rkl_destroy(ctx);
    return rc;
  }
  *out = ctx;
  return RKL_OK;
}

int rkl_destroy(rkl_ctx *ctx) {
  if (!ctx) return RKL_OK;
  cudaStreamSynchronize(ctx->stream);
  if (ctx->sts_exec) cudaGraphExecDestroy(ctx->sts_exec);
  if (ctx->pcg_exec) cudaGraphExecDestroy(ctx->pcg_exec);
  if (ctx->pcg_graph) cudaGraphDestroy(ctx->pcg_graph);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  if (ctx->pcg_stream) cudaStreamDestroy(ctx->pcg_stream);
  prof_release(ctx);
  double *bufs[] = {ctx->geo_buf, ctx->coef, ctx->W, ctx->invW, ctx->scratch, ctx->M0, ctx->Ya, ctx->Yb,
                    ctx->r, ctx->p, ctx->y, ctx->zbuf, ctx->dinv, ctx->partials, ctx->LU, ctx->stage, ctx->stage2,
                    ctx->acoef};
  for (double *b : bufs)
    if (b) cudaFree(b);
  if (ctx->d_lammax) cudaFree(ctx->d_lammax);
  if (ctx->counter) cudaFree(ctx->counter);
  if (ctx->d_state) cudaFree(ctx->d_state);
  if (ctx->h_state) cudaFreeHost(ctx->h_state);
  if (ctx->plan_buf) cudaFree(ctx->plan_buf);
  float *fbufs[] = {ctx->coef32, ctx->W32, ctx->invW32, ctx->M0f, ctx->da32, ctx->db32, ctx->r32, ctx->p32,
                    ctx->y32, ctx->z32, ctx->e32, ctx->dinv32, ctx->LU32};
  for (float *b : fbufs)
    if (b) cudaFree(b);
  cudaGetLastError();  // a failed teardown call must not surface in another context's checks
  delete ctx;
  return RKL_OK;
}

int rkl_set_stream(rkl_ctx *ctx, void *stream) {
  if (!ctx) return RKL_EINVAL;
  cudaStreamSynchronize(ctx->stream);
  ctx->stream = (cudaStream_t)stream;
  return RKL_OK;
}

int set_coeffs(rkl_ctx *ctx, int op, const double *a, const double *b, const double *c,
               double kappa0, int flags, double *dt_exp_out) {
  if (!ctx) return RKL_EINVAL;
  if (op != RKL_OP_CONDUCTION && op != RKL_OP_VISCOSITY)
    return set_error(ctx, RKL_EINVAL, "set_coeffs: unknown operator");
  if (!a || !c || (op == RKL_OP_CONDUCTION && !b))
    return set_error(ctx, RKL_EINVAL, "set_coeffs: null input array");
  if (op == RKL_OP_CONDUCTION && !finite_pos(kappa0))
    return set_error(ctx, RKL_EINVAL, "set_coeffs: kappa0 must be finite and > 0");
  if (op == RKL_OP_VISCOSITY && (flags & RKL_FLUX_FORM))
    return set_error(ctx, RKL_EINVAL, "set_coeffs: the flux form is a conduction option");
  const bool pole = op == RKL_OP_CONDUCTION && (flags & RKL_ACROSS_POLE);
  if (pole && (flags & RKL_FLUX_FORM))
    return set_error(ctx, RKL_EINVAL, "set_coeffs: across-pole ghosts are built for the symmetric form only");
  if (pole && (ctx->d.nth < 2 || ctx->d.nph < 6 || ctx->d.nph % 2))
    return set_error(ctx, RKL_EINVAL, "set_coeffs: across-pole ghosts need nth >= 2 and an even nph >= 6");
  const size_t N = (size_t)ctx->d.N;
  const int kind = (op == RKL_OP_CONDUCTION && (flags & RKL_FLUX_FORM)) ? OPK_FLUX : (pole ? OPK_POLE : op);
  ctx->op = -1;
  ctx->lu_valid = 0;
  ctx->acoef_valid = 0;
  ctx->epoch += 1;
  int rc = ensure_buffer(ctx, &ctx->scratch, 10 * N, "alloc set_coeffs scratch");
  if (rc) return rc;
  if (op_ncoef(kind) > ctx->coef_slots) {  // full rows need 19 slots
    cudaStreamSynchronize(ctx->stream);
    cudaFree(ctx->coef);
    ctx->coef = nullptr;
    ctx->coef_slots = 0;
    if ((rc = cuda_check(ctx, cudaMalloc(&ctx->coef, (op_ncoef(kind) * N + pole_extra(ctx->d)) * sizeof(double)),
                         "alloc coefficients")))
      return rc;
    ctx->coef_slots = op_ncoef(kind);
  }
  double *da, *db = nullptr, *dc;
  bool sa, sb = false, sc;
  if (!is_device_ptr(a) || (b && !is_device_ptr(b)) || !is_device_ptr(c))
    if ((rc = ensure_stage(ctx, 5 * N))) return rc;
  if ((rc = to_device(ctx, a, N, 0, true, &da, &sa))) return rc;
  if (op == RKL_OP_CONDUCTION && (rc = to_device(ctx, b, 3 * N, N, true, &db, &sb))) return rc;
  if ((rc = to_device(ctx, c, N, 4 * N, true, &dc, &sc))) return rc;
  if ((rc = cuda_check(ctx, cudaMemsetAsync(ctx->d_lammax, 0, sizeof(unsigned long long) + 2 * sizeof(int), ctx->stream), "clear flags")))
    return rc;
  ctx->op = kind;
  rc = op == RKL_OP_CONDUCTION ? launch_setup_conduction(ctx, da, db, dc, kappa0, flags)
                               : launch_setup_viscosity(ctx, da, dc);
  if (rc) {
    ctx->op = -1;
    return rc;
  }
  unsigned long long hbuf[2] = {0, 0};
  if ((rc = cuda_check(ctx, cudaMemcpyAsync(hbuf, ctx->d_lammax, sizeof(unsigned long long) + 2 * sizeof(int),
                                            cudaMemcpyDeviceToHost, ctx->stream), "read dt_exp")) ||
      (rc = sync(ctx, "set_coeffs"))) {
    ctx->op = -1;
    return rc;
  }
  int flag;
  std::memcpy(&flag, &hbuf[1], sizeof(int));
  double lam;
  std::memcpy(&lam, &hbuf[0], sizeof(double));
  if (flag & 1) {
    ctx->op = -1;
    return set_error(ctx, RKL_ENONFINITE, "set_coeffs: non-finite or non-positive input value");
  }
  if (flag & 2) {
    ctx->op = -1;
    return set_error(ctx, RKL_ECUDA, "set_coeffs: internal stencil assembly error");
  }
  if (ctx->prec == RKL_F32MIX) {  // FP32 copies of the frozen operator
    const long long nslot = op_ncoef(kind);
    if (nslot > ctx->coef32_slots && ctx->coef32) {
      cudaStreamSynchronize(ctx->stream);
      cudaFree(ctx->coef32);
      ctx->coef32 = nullptr;
    }
    if (!ctx->coef32) ctx->coef32_slots = (int)std::max<long long>(nslot, NCOEF_COND);
    const long long nconv = nslot * (long long)N + (kind == OPK_POLE ? pole_extra(ctx->d) : 0);
    if ((rc = ensure_fbuffer(ctx, &ctx->coef32, (size_t)ctx->coef32_slots * N + pole_extra(ctx->d),
                             "alloc FP32 coefficients")) ||
        (rc = ensure_fbuffer(ctx, &ctx->W32, N, "alloc FP32 W")) ||
        (rc = ensure_fbuffer(ctx, &ctx->invW32, N, "alloc FP32 1/W")) ||
        (rc = launch_to_float(ctx, ctx->coef, ctx->coef32, nconv)) ||
        (rc = launch_to_float(ctx, ctx->W, ctx->W32, (long long)N)) ||
        (rc = launch_to_float(ctx, ctx->invW, ctx->invW32, (long long)N))) {
      ctx->op = -1;
      return rc;
    }
  }
  ctx->dt_exp = lam > 0.0 ? 2.0 / lam : INFINITY;
  if (dt_exp_out) *dt_exp_out = ctx->dt_exp;
  return RKL_OK;
}

int apply_F(rkl_ctx *ctx, const double *u, double *Fu, int ncomp) {
  if (!ctx) return RKL_EINVAL;
  if (!u || !Fu || ncomp < 1 || ncomp > 3) return set_error(ctx, RKL_EINVAL, "apply_F: bad arguments");
  if (ctx->op < 0) return set_error(ctx, RKL_ESTATE, "apply_F before set_coeffs");
  const size_t N = (size_t)ctx->d.N, tot = N * ncomp;
  double *du, *dF;
  bool su, sF;
  int rc;
  if (!is_device_ptr(u) || !is_device_ptr(Fu))
    if ((rc = ensure_stage(ctx, 2 * tot))) return rc;
  if ((rc = to_device(ctx, u, tot, 0, true, &du, &su))) return rc;
  if ((rc = to_device(ctx, Fu, tot, tot, false, &dF, &sF))) return rc;
  for (int q = 0; q < ncomp; q++)
    if ((rc = launch_apply_F(ctx, du + q * N, dF + q * N))) return rc;
  if (sF && (rc = from_device(ctx, Fu, dF, tot))) return rc;
  if (su || sF) return sync(ctx, "apply_F");
  return RKL_OK;
}

namespace {

// the stage launches of one super-step (Fig. 2) for ncomp components at du
int rkl2_stages(rkl_ctx *ctx, double *du, int ncomp, int s, double dt, double w1) {
  const size_t N = (size_t)ctx->d.N;
  int rc;
  if (ctx->prec == RKL_F32MIX) {
    for (int q = 0; q < ncomp; q++) {
      double *Y0 = du + q * N;
      if ((rc = launch_rkl2_first_mix(ctx, Y0, ctx->M0f, ctx->da32, w1 / 3.0 * dt))) return rc;
      float *dm1 = ctx->da32, *dm2 = nullptr;
      for (int j = 2; j <= s; j++) {
        double mu = (2.0 * j - 1.0) / j * rkl_b(j) / rkl_b(j - 1);
        double nu = -(j - 1.0) / j * rkl_b(j) / rkl_b(j - 2);
        double mut = w1 * mu;
        double gt = -(1.0 - rkl_b(j - 1)) * mut;
        const bool last = j == s;
        float *out = last ? nullptr : (j == 2 ? ctx->db32 : dm2);
        if ((rc = launch_rkl2_stage_mix(ctx, dm1, dm2, ctx->M0f, out, last ? Y0 : nullptr, mu, nu, mut * dt,
                                        (mut + gt) * dt)))
          return rc;
        dm2 = dm1;
        dm1 = out;
      }
    }
    return RKL_OK;
  }
  for (int q = 0; q < ncomp; q++) {
    double *Y0 = du + q * N;
    if ((rc = launch_rkl2_stage1(ctx, Y0, ctx->M0, ctx->Ya, w1 / 3.0 * dt))) return rc;
    double *ym1 = ctx->Ya, *ym2 = Y0;
    for (int j = 2; j <= s; j++) {
      double mu = (2.0 * j - 1.0) / j * rkl_b(j) / rkl_b(j - 1);
      double nu = -(j - 1.0) / j * rkl_b(j) / rkl_b(j - 2);
      double mut = w1 * mu;
      double gt = -(1.0 - rkl_b(j - 1)) * mut;
      double *out = (j == s) ? Y0 : (j == 2 ? ctx->Yb : ym2);
      if ((rc = launch_rkl2_stage(ctx, ym1, ym2, Y0, ctx->M0, out, mu, nu, mut * dt, gt * dt))) return rc;
      ym2 = ym1;
      ym1 = out;
    }
  }
  return RKL_OK;
}

// The same launches through a CUDA graph: a call that repeats the last one (same stage
// count, components, field, precision, operator, dt and frozen coefficients) replays the
// instantiated graph; otherwise the launches are captured again and the executable graph
// is updated in place (or re-instantiated when its shape changed).
int rkl2_stages_graph(rkl_ctx *ctx, double *du, int ncomp, int s, double dt, double w1) {
  const bool same_shape = ctx->sts_exec && ctx->sts_s == s && ctx->sts_ncomp == ncomp && ctx->sts_u == du &&
                          ctx->sts_prec == ctx->prec && ctx->sts_op == ctx->op;
  if (same_shape && ctx->sts_dt == dt && ctx->sts_epoch == ctx->epoch) {
    ctx->launches += ctx->sts_nkern;
    return cuda_check(ctx, cudaGraphLaunch(ctx->sts_exec, ctx->stream), "super-step graph launch");
  }
  // capture on a private stream (the caller's may be the legacy default stream, which
  // cannot be captured); the graph is then launched on the caller's stream
  int rc = RKL_OK;
  if (!ctx->cap_stream &&
      (rc = cuda_check(ctx, cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking), "capture stream")))
    return rc;
  const long long l0 = ctx->launches;
  cudaStream_t user = ctx->stream;
  ctx->stream = ctx->cap_stream;
  rc = cuda_check(ctx, cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal), "super-step capture");
  if (rc) {
    ctx->stream = user;
    return rc;
  }
  const int rc_launch = rkl2_stages(ctx, du, ncomp, s, dt, w1);
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(ctx->stream, &graph);
  ctx->stream = user;
  if (rc_launch || e != cudaSuccess || !graph) {
    if (graph) cudaGraphDestroy(graph);
    ctx->launches = l0;
    return rc_launch ? rc_launch : cuda_check(ctx, e, "super-step capture");
  }
  bool updated = false;
  if (same_shape) {
    cudaGraphExecUpdateResultInfo info;
    updated = cudaGraphExecUpdate(ctx->sts_exec, graph, &info) == cudaSuccess;
    if (!updated) cudaGetLastError();
  }
  if (!updated) {
    if (ctx->sts_exec) cudaGraphExecDestroy(ctx->sts_exec);
    cudaGetLastError();  // teardown of the previous graph is not an error of this call
    ctx->sts_exec = nullptr;
    rc = cuda_check(ctx, cudaGraphInstantiate(&ctx->sts_exec, graph, 0), "super-step graph instantiate");
  }
  cudaGraphDestroy(graph);
  if (rc) {
    ctx->sts_exec = nullptr;
    return rc;
  }
  ctx->sts_s = s;
  ctx->sts_ncomp = ncomp;
  ctx->sts_u = du;
  ctx->sts_prec = ctx->prec;
  ctx->sts_op = ctx->op;
  ctx->sts_dt = dt;
  ctx->sts_epoch = ctx->epoch;
  ctx->sts_nkern = ctx->launches - l0;
  return cuda_check(ctx, cudaGraphLaunch(ctx->sts_exec, ctx->stream), "super-step graph launch");
}

}  // namespace

int rkl2_superstep(rkl_ctx *ctx, double *u, int ncomp, double dt, double dt_exp, int s, int flags,
                   int *s_used) {
  if (!ctx) return RKL_EINVAL;
  if (!u || ncomp < 1 || ncomp > 3 || !(std::isfinite(dt) && dt > 0.0) || s < 0 || s == 1)
    return set_error(ctx, RKL_EINVAL, "rkl2_superstep: bad arguments");
  if (ctx->op < 0) return set_error(ctx, RKL_ESTATE, "rkl2_superstep before set_coeffs");
  if (s == 0) {
    if (!(dt_exp > 0.0)) return set_error(ctx, RKL_EINVAL, "rkl2_superstep: dt_exp must be > 0 when s == 0");
    s = std::isinf(dt_exp) ? 2 : rkl2_stage_count(dt / dt_exp, flags);
    if (s < 0) return set_error(ctx, RKL_EINVAL, "rkl2_superstep: stage count out of range");
  }
  const size_t N = (size_t)ctx->d.N, tot = N * ncomp;
  int rc;
  if ((rc = ensure_buffer(ctx, &ctx->M0, N, "alloc M0")) || (rc = ensure_buffer(ctx, &ctx->Ya, N, "alloc Y")) ||
      (rc = ensure_buffer(ctx, &ctx->Yb, N, "alloc Y")))
    return rc;
  double *du;
  bool su;
  if (!is_device_ptr(u) && (rc = ensure_stage(ctx, tot))) return rc;
  if ((rc = to_device(ctx, u, tot, 0, true, &du, &su))) return rc;
  if (ctx->prec == RKL_F32MIX &&
      ((rc = ensure_fbuffer(ctx, &ctx->M0f, N, "alloc M0 (FP32)")) ||
       (rc = ensure_fbuffer(ctx, &ctx->da32, N, "alloc increments")) ||
       (rc = ensure_fbuffer(ctx, &ctx->db32, N, "alloc increments"))))
    return rc;
  const double w1 = 4.0 / ((double)s * s + s - 2.0);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if ((rc = cuda_check(ctx, cudaStreamIsCapturing(ctx->stream, &cap), "stream capture query"))) return rc;
  // kernels are loaded on their first launch (lazy module loading), which a stream capture
  // does not allow: a context's first super-step runs without a graph
  if (ctx->prof_on || cap != cudaStreamCaptureStatusNone || s < 4 || !ctx->sts_direct_done) {
    if ((rc = rkl2_stages(ctx, du, ncomp, s, dt, w1))) return rc;
    ctx->sts_direct_done = 1;
  } else if ((rc = rkl2_stages_graph(ctx, du, ncomp, s, dt, w1))) {
    return rc;
  }
  if (s_used) *s_used = s;
  if (su) {
    if ((rc = from_device(ctx, u, du, tot))) return rc;
    return sync(ctx, "rkl2_superstep");
  }
  return RKL_OK;
}

namespace {

// s FP64 stages of RKL2 (scheme 0) or RKL1 (scheme 1) over dt, in place on Y0
int run_sts(rkl_ctx *ctx, double *Y0, int scheme, int s, double dt) {
  const bool rkl1 = scheme == RKL_SCHEME_RKL1;
  const double w1 = rkl1 ? 2.0 / ((double)s * s + s) : 4.0 / ((double)s * s + s - 2.0);
  int rc;
  if (s == 1) {  // RKL1 with one stage: explicit Euler, Y1 = Y0 + w1 dt M Y0 (w1 = 1)
    if ((rc = launch_rkl2_stage1(ctx, Y0, ctx->M0, ctx->Ya, w1 * dt))) return rc;
    return cuda_check(ctx, cudaMemcpyAsync(Y0, ctx->Ya, sizeof(double) * ctx->d.N, cudaMemcpyDeviceToDevice,
                                           ctx->stream), "stage copy");
  }
  if ((rc = launch_rkl2_stage1(ctx, Y0, ctx->M0, ctx->Ya, (rkl1 ? w1 : w1 / 3.0) * dt))) return rc;
  double *ym1 = ctx->Ya, *ym2 = Y0;
  for (int j = 2; j <= s; j++) {
    double mu, nu, mut, gt;
    if (rkl1) {
      mu = (2.0 * j - 1.0) / j;
      nu = -(j - 1.0) / j;
      mut = w1 * mu;
      gt = 0.0;
    } else {
      mu = (2.0 * j - 1.0) / j * rkl_b(j) / rkl_b(j - 1);
      nu = -(j - 1.0) / j * rkl_b(j) / rkl_b(j - 2);
      mut = w1 * mu;
      gt = -(1.0 - rkl_b(j - 1)) * mut;
    }
    double *out = (j == s) ? Y0 : (j == 2 ? ctx->Yb : ym2);
    if ((rc = launch_rkl2_stage(ctx, ym1, ym2, Y0, ctx->M0, out, mu, nu, mut * dt, gt * dt))) return rc;
    ym2 = ym1;
    ym1 = out;
  }
  return RKL_OK;
}

}  // namespace

int sts_advance(rkl_ctx *ctx, double *u, int ncomp, double dt, double dt_exp, const rkl_sts_options *opt,
                int *stages_used) {
  if (!ctx) return RKL_EINVAL;
  if (!u || !opt || ncomp < 1 || ncomp > 3 || !(std::isfinite(dt) && dt > 0.0) || !(dt_exp > 0.0) ||
      (opt->scheme != RKL_SCHEME_RKL2 && opt->scheme != RKL_SCHEME_RKL1) || opt->cycles < 1 ||
      opt->cycles > 100000 || opt->extra_stages < 0 || opt->extra_stages > 100000 ||
      !(opt->euler_fraction >= 0.0 && opt->euler_fraction < 1.0))
    return set_error(ctx, RKL_EINVAL, "sts_advance: bad arguments");
  if (ctx->op < 0) return set_error(ctx, RKL_ESTATE, "sts_advance before set_coeffs");
  const size_t N = (size_t)ctx->d.N, tot = N * ncomp;
  int rc;
  if ((rc = ensure_buffer(ctx, &ctx->M0, N, "alloc M0")) || (rc = ensure_buffer(ctx, &ctx->Ya, N, "alloc Y")) ||
      (rc = ensure_buffer(ctx, &ctx->Yb, N, "alloc Y")))
    return rc;
  double *du;
  bool su;
  if (!is_device_ptr(u) && (rc = ensure_stage(ctx, tot))) return rc;
  if ((rc = to_device(ctx, u, tot, 0, true, &du, &su))) return rc;
  // explicit Euler prefix: n_E sub-steps of h <= dt_exp covering euler_fraction * dt
  const double te = opt->euler_fraction * dt;
  const long long ne = te > 0.0 ? (long long)std::ceil(te / dt_exp) : 0;
  if (ne > 10000000) return set_error(ctx, RKL_EINVAL, "sts_advance: too many Euler sub-steps");
  const double tau = (dt - te) / opt->cycles;
  int s;
  if (opt->scheme == RKL_SCHEME_RKL2) {
    s = std::isinf(dt_exp) ? 2 : rkl2_stage_count(tau / dt_exp, 0);
    if (s < 0) return set_error(ctx, RKL_EINVAL, "sts_advance: stage count out of range");
    s += opt->extra_stages;
    if ((opt->flags & RKL_FORCE_ODD) && s % 2 == 0) s++;
  } else {
    const double r1 = tau / dt_exp;
    s = std::max(1, (int)std::ceil((std::sqrt(1.0 + 8.0 * r1) - 1.0) / 2.0)) + opt->extra_stages;
  }
  for (int q = 0; q < ncomp; q++) {
    double *Y0 = du + q * N;
    for (long long e = 0; e < ne; e++)
      if ((rc = run_sts(ctx, Y0, RKL_SCHEME_RKL1, 1, te / ne))) return rc;
    for (int cyc = 0; cyc < opt->cycles; cyc++)
      if ((rc = run_sts(ctx, Y0, opt->scheme, s, tau))) return rc;
  }
  if (stages_used) *stages_used = (int)std::min<long long>(ne + (long long)opt->cycles * s, INT32_MAX);
  if (su) {
    if ((rc = from_device(ctx, u, du, tot))) return rc;
    return sync(ctx, "sts_advance");
  }
  return RKL_OK;
}

int be_pcg_solve(rkl_ctx *ctx, double *u, int ncomp, double dt, int pc, const int block[3],
                 double rtol, int maxit, const double *x0, int *iters_out, double *relres_out) {
  if (!ctx) return RKL_EINVAL;
  if (!u || ncomp < 1 || ncomp > 3 || !(std::isfinite(dt) && dt > 0.0) || maxit < 0 || !std::isfinite(rtol))
    return set_error(ctx, RKL_EINVAL, "be_pcg_solve: bad arguments");
  if (pc != RKL_PC_JACOBI && pc != RKL_PC_BILU0) return set_error(ctx, RKL_EINVAL, "be_pcg_solve: unknown preconditioner");
  if (ctx->op < 0) return set_error(ctx, RKL_ESTATE, "be_pcg_solve before set_coeffs");
  int rc;
  if (pc == RKL_PC_BILU0) {
    if (!block || block[0] < 1 || block[1] < 1 || block[2] < 1 || ctx->d.nr % block[0] ||
        ctx->d.nth % block[1] || ctx->d.nph % block[2] || (long long)block[0] * block[1] * block[2] > 4096)
      return set_error(ctx, RKL_EINVAL, "be_pcg_solve: grid must be divisible by the ILU block (<= 4096 cells)");
    long long nblk = ctx->d.N / ((long long)block[0] * block[1] * block[2]);
    if (nblk > (1LL << 30)) return set_error(ctx, RKL_EINVAL, "be_pcg_solve: too many ILU blocks");
    if (2 * nblk > ctx->npart) {
      // one partial pair per ILU block for the r.z / r.r reductions of the block solve
      if ((rc = sync(ctx, "be_pcg_solve"))) return rc;
      cudaFree(ctx->partials);
      ctx->partials = nullptr;
      if ((rc = cuda_check(ctx, cudaMalloc(&ctx->partials, (size_t)(2 * nblk) * sizeof(double)), "alloc partials"))) {
        ctx->npart = 0;
        return rc;
      }
      ctx->npart = (int)(2 * nblk);
    }
    if ((rc = bilu0_prepare(ctx, block, dt))) return rc;
  }
  const size_t N = (size_t)ctx->d.N, tot = N * ncomp;
  double *du, *dx0 = nullptr;
  bool su, sx = false;
  if (!is_device_ptr(u) || (x0 && !is_device_ptr(x0)))
    if ((rc = ensure_stage(ctx, 2 * tot))) return rc;
  if ((rc = to_device(ctx, u, tot, 0, true, &du, &su))) return rc;
  if (x0 && (rc = to_device(ctx, x0, tot, tot, true, &dx0, &sx))) return rc;
  int worst = RKL_OK;
  for (int q = 0; q < ncomp; q++) {
    int it = 0, status = 0;
    double rel = 0.0;
    rc = pcg_solve_component(ctx, du + q * N, du + q * N, dx0 ? dx0 + q * N : nullptr, dt, pc, rtol,
                             maxit, &it, &rel, &status);
    if (rc) return rc;
    if (iters_out) iters_out[q] = it;
    if (relres_out) relres_out[q] = rel;
    if (status == PCG_BREAKDOWN) worst = RKL_EBREAKDOWN;
    else if (status == PCG_MAXIT && worst == RKL_OK) worst = RKL_ENOTCONV;
  }
  if (su) {
    if ((rc = from_device(ctx, u, du, tot)) || (rc = sync(ctx, "be_pcg_solve"))) return rc;
  }
  if (worst == RKL_EBREAKDOWN) return set_error(ctx, worst, "be_pcg_solve: breakdown (p.Ap <= 0)");
  if (worst == RKL_ENOTCONV) return set_error(ctx, worst, "be_pcg_solve: maxit reached");
  return RKL_OK;
}

}  // extern "C"
