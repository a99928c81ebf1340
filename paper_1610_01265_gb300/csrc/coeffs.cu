// coeffs.cu -- set_coeffs: freeze the operator for one large step (lagged diffusivity,
// Sec. 1), build the symmetric stencil S and W, and bound |lambda|max of M = -W^{-1} S
// by Gershgorin row sums (App. B, Eq. 7).
//
// Conduction (Sec. 4.1): S is the Hessian of the discrete energy
//   Q(u) = 1/2 sum_a sum_{a-faces f=(L,R)} Vt_f [ D_f^aa g_f^2 + sum_{b!=a} D_f^ab g_f ghat_b ]
// with g_f = (u_R - u_L)/h_f, ghat_b = (G_b(L) + G_b(R))/2, G_b(x) the centred
// b-difference at x (mirror ghosts beyond r and theta edges, phi periodic),
// Vt_f = A_f h_f, D_f = (D_L + D_R)/2, D_x = kappa_x bhat_x bhat_x^T.  Each face adds
// a small symmetric block to S; the assembly here is a gather: one thread per cell
// walks every face that touches its row (its own 6 faces and the 24 faces for which
// it is a transverse neighbour) and keeps the row in registers/local memory.
//
// Viscosity: Q_v = 1/2 sum_f Vt_f mu_f g_f^2 (7-point), mu = nu rho, W = rho V.
#include <cuda_runtime.h>

#include "internal.cuh"
#include "stencil.cuh"

namespace rkl {

namespace {

constexpr int BLK = 256;

struct C3 {
  int i, j, k;
};

__device__ __forceinline__ bool same(C3 a, C3 b) { return a.i == b.i && a.j == b.j && a.k == b.k; }

__device__ __forceinline__ int wrapk(const Dims &d, int k) {
  return k < 0 ? k + d.nph : (k >= d.nph ? k - d.nph : k);
}

__device__ __forceinline__ long long lin(const Dims &d, C3 x) {
  return ((long long)x.k * d.nth + x.j) * d.nr + x.i;
}

// one step along direction a (sign sg) without mirroring; false if it leaves r/theta range
__device__ __forceinline__ bool step(const Dims &d, C3 x, int a, int sg, C3 &out) {
  out = x;
  if (a == 0) {
    out.i += sg;
    return out.i >= 0 && out.i < d.nr;
  }
  if (a == 1) {
    out.j += sg;
    return out.j >= 0 && out.j < d.nth;
  }
  out.k = wrapk(d, x.k + sg);
  return true;
}

// transverse neighbour used by a centred difference: mirror ghost = the cell itself
__device__ __forceinline__ C3 mirror_step(const Dims &d, C3 x, int b, int sg) {
  C3 o;
  return step(d, x, b, sg, o) ? o : x;
}

__device__ __forceinline__ bool has_upper_face(const Dims &d, C3 x, int a) {
  return a == 0 ? x.i < d.nr - 1 : (a == 1 ? x.j < d.nth - 1 : true);
}

// span of the centred b-difference at x
__device__ __forceinline__ double cspan(const Geo &g, int b, C3 x) {
  if (b == 0) return g.dr[x.i];
  if (b == 1) return 2.0 * g.rc[x.i] * g.dth;
  return 2.0 * g.rc[x.i] * g.stc[x.j] * g.dph;
}

__device__ __forceinline__ int transverse(int a, int t) {
  return a == 0 ? (t ? 2 : 1) : (a == 1 ? (t ? 2 : 0) : (t ? 1 : 0));
}

__device__ __forceinline__ void row_add(double *row, const Dims &d, C3 c, C3 X, double v,
                                        int *flag) {
  int di = X.i - c.i, dj = X.j - c.j, dk = X.k - c.k;
  if (dk == d.nph - 1) dk = -1;
  else if (dk == -(d.nph - 1)) dk = 1;
  if (di < -1 || di > 1 || dj < -1 || dj > 1 || dk < -1 || dk > 1) {
    atomicOr(flag, 2);  // cannot happen for a face that touches c; reported, not trapped
    return;
  }
  row[(di + 1) + 3 * (dj + 1) + 9 * (dk + 1)] += v;
}

// contribution of the upper a-face of L (L, R = L + e_a) to row c of S
__device__ void face_into_row(double *row, const Dims &d, const Geo &g, const double *FS, C3 c,
                              int a, C3 L, int *flag) {
  C3 R;
  step(d, L, a, +1, R);
  long long l = lin(d, L);
  double alpha = FS[(3 * a + 0) * d.N + l];
  double beta[2] = {FS[(3 * a + 1) * d.N + l], FS[(3 * a + 2) * d.N + l]};
  double sc = same(c, R) ? 1.0 : (same(c, L) ? -1.0 : 0.0);
  if (sc != 0.0) {
    row_add(row, d, c, L, -alpha * sc, flag);
    row_add(row, d, c, R, alpha * sc, flag);
  }
  for (int t = 0; t < 2; t++) {
    int b = transverse(a, t);
    double gl = 0.5 / cspan(g, b, L), gr = 0.5 / cspan(g, b, R);
    C3 X[4] = {mirror_step(d, L, b, +1), mirror_step(d, L, b, -1), mirror_step(d, R, b, +1),
               mirror_step(d, R, b, -1)};
    double w[4] = {gl, -gl, gr, -gr};
    for (int q = 0; q < 4; q++) {
      // d^2 Q / du_c du_X from the g * ghat_b term: beta (sigma_c w_X + w_c sigma_X)
      if (sc != 0.0) row_add(row, d, c, X[q], beta[t] * sc * w[q], flag);
      if (same(X[q], c)) {
        row_add(row, d, c, L, -beta[t] * w[q], flag);
        row_add(row, d, c, R, beta[t] * w[q], flag);
      }
    }
  }
}

__global__ void k_cell_cond(Dims d, Geo g, const double *__restrict__ T,
                            const double *__restrict__ bhat, const double *__restrict__ n,
                            double kappa0, int flags, double *__restrict__ kappa,
                            double *__restrict__ W, double *__restrict__ invW, int *flag) {
  long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= d.N) return;
  int i, j, k;
  cell_coords(d, c, i, j, k);
  double t = T[c], nn = n[c];
  double b0 = bhat[c], b1 = bhat[d.N + c], b2 = bhat[2 * d.N + c];
  bool ok = isfinite(t) && t > 0.0 && isfinite(nn) && nn > 0.0 && isfinite(b0) &&
            isfinite(b1) && isfinite(b2);
  if (!ok) {
    atomicOr(flag, 1);
    t = 1.0;
    nn = 1.0;
  }
  double te = ((flags & RKL_BETA_TCUT) && t < RKL_TCUT) ? RKL_TCUT : t;
  kappa[c] = kappa0 * te * te * sqrt(te);
  double V = g.v3[i] * g.dcos[j] * g.dph;
  double w = 3.0 * RKL_KBOLTZ * nn * V;
  W[c] = w;
  invW[c] = 1.0 / w;
}

// alpha_f = Vt D^aa / h^2 and beta_f^b = Vt D^ab / (2h) of the three upper faces of c
__global__ void k_faces_cond(Dims d, Geo g, const double *__restrict__ bhat,
                             const double *__restrict__ kappa, double *__restrict__ FS) {
  long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= d.N) return;
  int i, j, k;
  cell_coords(d, c, i, j, k);
  const long long N = d.N;
  double bL[3] = {bhat[c], bhat[N + c], bhat[2 * N + c]};
  double kL = kappa[c];
  for (int a = 0; a < 3; a++) {
    double al = 0.0, be0 = 0.0, be1 = 0.0;
    bool ex = a == 0 ? i < d.nr - 1 : (a == 1 ? j < d.nth - 1 : true);
    if (ex) {
      long long R = c + (a == 0 ? 1LL
                                : (a == 1 ? (long long)d.nr
                                          : (k < d.nph - 1 ? d.nrt
                                                           : -(long long)(d.nph - 1) * d.nrt)));
      double h, A;
      if (a == 0) {
        h = g.hr[i];
        A = g.ar[i] * g.dcos[j] * g.dph;
      } else if (a == 1) {
        h = g.rc[i] * g.dth;
        A = g.a2[i] * g.stf[j] * g.dph;
      } else {
        h = g.rc[i] * g.stc[j] * g.dph;
        A = g.a2[i] * g.dth;
      }
      double Vt = A * h;
      double kR = kappa[R];
      double bR[3] = {bhat[R], bhat[N + R], bhat[2 * N + R]};
      int t0 = transverse(a, 0), t1 = transverse(a, 1);
      double Daa = 0.5 * (kL * bL[a] * bL[a] + kR * bR[a] * bR[a]);
      double Da0 = 0.5 * (kL * bL[a] * bL[t0] + kR * bR[a] * bR[t0]);
      double Da1 = 0.5 * (kL * bL[a] * bL[t1] + kR * bR[a] * bR[t1]);
      al = Vt * Daa / (h * h);
      be0 = 0.5 * Vt * Da0 / h;
      be1 = 0.5 * Vt * Da1 / h;
    }
    FS[(3 * a + 0) * N + c] = al;
    FS[(3 * a + 1) * N + c] = be0;
    FS[(3 * a + 2) * N + c] = be1;
  }
}

__global__ void k_assemble_cond(Dims d, Geo g, const double *__restrict__ FS,
                                const double *__restrict__ invW, double *__restrict__ coef,
                                unsigned long long *lammax, int *flag) {
  long long cl = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (cl >= d.N) return;
  C3 c;
  cell_coords(d, cl, c.i, c.j, c.k);
  double row[27];
#pragma unroll
  for (int q = 0; q < 27; q++) row[q] = 0.0;
  for (int a = 0; a < 3; a++) {
    C3 x;
    // own faces: upper (c = L) and lower (c = R)
    if (has_upper_face(d, c, a)) face_into_row(row, d, g, FS, c, a, c, flag);
    if (step(d, c, a, -1, x)) face_into_row(row, d, g, FS, c, a, x, flag);
    // a-faces of the transverse neighbours c +- e_b: c enters them through ghat_b
    for (int t = 0; t < 2; t++) {
      int b = transverse(a, t);
      for (int sg = -1; sg <= 1; sg += 2) {
        C3 nb, nbm;
        if (!step(d, c, b, sg, nb)) continue;
        if (has_upper_face(d, nb, a)) face_into_row(row, d, g, FS, c, a, nb, flag);
        if (step(d, nb, a, -1, nbm)) face_into_row(row, d, g, FS, c, a, nbm, flag);
      }
    }
  }
  double sum = 0.0;
#pragma unroll
  for (int q = 0; q < 27; q++) sum += fabs(row[q]);
#pragma unroll
  for (int m = 0; m < 9; m++)
    coef[m * d.N + cl] = row[(fwd_di(m) + 1) + 3 * (fwd_dj(m) + 1) + 9 * (fwd_dk(m) + 1)];
  coef[9 * d.N + cl] = row[13];
  double rs = sum * invW[cl];
  if (!isfinite(rs)) atomicOr(flag, 1);
  else atomicMax(lammax, (unsigned long long)__double_as_longlong(rs));
}

__global__ void k_cell_visc(Dims d, Geo g, const double *__restrict__ rho,
                            const double *__restrict__ nu, double *__restrict__ mu,
                            double *__restrict__ W, double *__restrict__ invW, int *flag) {
  long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= d.N) return;
  int i, j, k;
  cell_coords(d, c, i, j, k);
  double r = rho[c], v = nu[c];
  if (!(isfinite(r) && r > 0.0 && isfinite(v) && v > 0.0)) {
    atomicOr(flag, 1);
    r = 1.0;
    v = 1.0;
  }
  mu[c] = v * r;
  double w = r * (g.v3[i] * g.dcos[j] * g.dph);
  W[c] = w;
  invW[c] = 1.0 / w;
}

// alpha_f = A_f mu_f / h_f for the six faces of c; S_cc = sum alpha, forward = -alpha
__global__ void k_assemble_visc(Dims d, Geo g, const double *__restrict__ mu,
                                const double *__restrict__ invW, double *__restrict__ coef,
                                unsigned long long *lammax, int *flag) {
  long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= d.N) return;
  int i, j, k;
  cell_coords(d, c, i, j, k);
  Nbr n = neighbours(d, i, j, k);
  double m0 = mu[c];
  double diag = 0.0, fw[3] = {0.0, 0.0, 0.0};
  // r faces
  if (n.vrp) {
    double al = g.ar[i] * g.dcos[j] * g.dph * (0.5 * (m0 + mu[c + 1])) / g.hr[i];
    fw[0] = -al;
    diag += al;
  }
  if (n.vrm) diag += g.ar[i - 1] * g.dcos[j] * g.dph * (0.5 * (mu[c - 1] + m0)) / g.hr[i - 1];
  // theta faces
  double ht = g.rc[i] * g.dth;
  if (n.vtp) {
    double al = g.a2[i] * g.stf[j] * g.dph * (0.5 * (m0 + mu[c + n.tp])) / ht;
    fw[1] = -al;
    diag += al;
  }
  if (n.vtm) diag += g.a2[i] * g.stf[j - 1] * g.dph * (0.5 * (mu[c + n.tm] + m0)) / ht;
  // phi faces (periodic)
  double hp = g.rc[i] * g.stc[j] * g.dph, Ap = g.a2[i] * g.dth;
  {
    double al = Ap * (0.5 * (m0 + mu[c + n.pp])) / hp;
    fw[2] = -al;
    diag += al;
    diag += Ap * (0.5 * (mu[c + n.pm] + m0)) / hp;
  }
  coef[0 * d.N + c] = fw[0];
  coef[1 * d.N + c] = fw[1];
  coef[2 * d.N + c] = fw[2];
  coef[3 * d.N + c] = diag;
  double rs = 2.0 * diag * invW[c];
  if (!isfinite(rs)) atomicOr(flag, 1);
  else atomicMax(lammax, (unsigned long long)__double_as_longlong(rs));
}

}  // namespace

int launch_setup_conduction(rkl_ctx *ctx, const double *T, const double *bhat, const double *n,
                            double kappa0, int flags) {
  const Dims &d = ctx->d;
  unsigned grid = grid_for(d.N, BLK);
  double *kappa = ctx->scratch;
  double *FS = ctx->scratch + d.N;
  k_cell_cond<<<grid, BLK, 0, ctx->stream>>>(d, ctx->geo, T, bhat, n, kappa0, flags, kappa, ctx->W,
                                            ctx->invW, ctx->d_flag);
  k_faces_cond<<<grid, BLK, 0, ctx->stream>>>(d, ctx->geo, bhat, kappa, FS);
  k_assemble_cond<<<grid, BLK, 0, ctx->stream>>>(d, ctx->geo, FS, ctx->invW, ctx->coef,
                                                ctx->d_lammax, ctx->d_flag);
  ctx->launches += 3;
  return cuda_check(ctx, cudaGetLastError(), "set_coeffs(conduction) launch");
}

int launch_setup_conduction_raw(const Dims &d, const Geo &g, cudaStream_t stream, const double *T,
                                const double *bhat, const double *n, double kappa0, int flags,
                                double *kappa, double *FS, double *W, double *invW, double *coef,
                                unsigned long long *lammax, int *flag) {
  unsigned grid = grid_for(d.N, BLK);
  k_cell_cond<<<grid, BLK, 0, stream>>>(d, g, T, bhat, n, kappa0, flags, kappa, W, invW, flag);
  k_faces_cond<<<grid, BLK, 0, stream>>>(d, g, bhat, kappa, FS);
  k_assemble_cond<<<grid, BLK, 0, stream>>>(d, g, FS, invW, coef, lammax, flag);
  return cudaGetLastError() == cudaSuccess ? RKL_OK : RKL_ECUDA;
}

int launch_setup_viscosity(rkl_ctx *ctx, const double *rho, const double *nu) {
  const Dims &d = ctx->d;
  unsigned grid = grid_for(d.N, BLK);
  double *mu = ctx->scratch;
  k_cell_visc<<<grid, BLK, 0, ctx->stream>>>(d, ctx->geo, rho, nu, mu, ctx->W, ctx->invW,
                                            ctx->d_flag);
  k_assemble_visc<<<grid, BLK, 0, ctx->stream>>>(d, ctx->geo, mu, ctx->invW, ctx->coef,
                                                ctx->d_lammax, ctx->d_flag);
  ctx->launches += 2;
  return cuda_check(ctx, cudaGetLastError(), "set_coeffs(viscosity) launch");
}

}  // namespace rkl
