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
// it is a transverse neighbour) and keeps the row in registers.
//
// Flux form (RKL_FLUX_FORM): row c is minus the divergence of the face fluxes
// A_f (D_f^aa g_f + sum_b D_f^ab ghat_b) through the six faces of c -- the "standard",
// slightly non-symmetric scheme whose symmetric part is the S above -- stored as full
// 19-entry rows.
//
// Viscosity: Q_v = 1/2 sum_f Vt_f mu_f g_f^2 (7-point), mu = nu rho, W = rho V.
#include <cuda_runtime.h>

#include "internal.cuh"
#include "stencil.cuh"

namespace rkl {

namespace {

constexpr int BLK = 256;

// slot of offset (di, dj, dk) in a 27-entry row; t-th transverse direction of a; unit vector
__host__ __device__ constexpr int r27(int di, int dj, int dk) { return (di + 1) + 3 * (dj + 1) + 9 * (dk + 1); }
__host__ __device__ constexpr int tdir(int a, int t) { return a == 0 ? (t ? 2 : 1) : (a == 1 ? (t ? 2 : 0) : (t ? 1 : 0)); }
__host__ __device__ constexpr int ex_(int a, int x) { return a == x ? 1 : 0; }

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
  double kap = kappa0 * t * t * sqrt(t);
  if ((flags & RKL_BETA_TCUT) && t < RKL_TCUT) {  // beta_Tcut = (T / T_cut)^{5/2} (Sec. 4.1)
    const double q = t / RKL_TCUT;
    kap *= q * q * sqrt(q);
  }
  kappa[c] = kap;
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
      int t0 = tdir(a, 0), t1 = tdir(a, 1);
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

// ---- row assembly: every slot index known at compile time ----
//
// A face touching the row of cell c is one of 30 cases fixed by its direction A, the
// position of its L cell relative to c and the role of c (L, R, or a transverse
// neighbour entering through ghat_b).  Enumerating the cases with templates makes every
// target slot a compile-time constant; the only runtime choices are whether a face
// exists and whether a transverse neighbour is a mirror ghost (then the entry goes to
// L or R instead), so the 27-entry row stays in registers.


struct RowCell {
  int i, j;
  long long c;
  bool up[3], dn[3];         // does c + e_a / c - e_a exist (always true along phi)
  long long dup[3], ddn[3];  // index deltas of c + e_a / c - e_a (phi wrapped)
};

template <int DI, int DJ, int DK>
__device__ __forceinline__ bool has(const RowCell &C) {
  return (DI > 0 ? C.up[0] : (DI < 0 ? C.dn[0] : true)) && (DJ > 0 ? C.up[1] : (DJ < 0 ? C.dn[1] : true));
}

template <int DI, int DJ, int DK>
__device__ __forceinline__ long long idx(const RowCell &C) {
  return C.c + (DI > 0 ? C.dup[0] : (DI < 0 ? C.ddn[0] : 0)) + (DJ > 0 ? C.dup[1] : (DJ < 0 ? C.ddn[1] : 0)) +
         (DK > 0 ? C.dup[2] : (DK < 0 ? C.ddn[2] : 0));
}

template <int B, int DI, int DJ>
__device__ __forceinline__ double gam(const Geo &g, const RowCell &C) {  // 0.5 / span of G_B at c + (DI,DJ,.)
  const int i = C.i + DI, j = C.j + DJ;
  if (B == 0) return 0.5 / g.dr[i];
  if (B == 1) return 0.5 / (2.0 * g.rc[i] * g.dth);
  return 0.5 / (2.0 * g.rc[i] * g.stc[j] * g.dph);
}

template <int I1, int I0>
__device__ __forceinline__ void add_sel(double (&row)[27], bool first, double v) {
  if (first) row[I1] += v;
  else row[I0] += v;
}

// own face of c (c = L when SC = -1, c = R when SC = +1); L at offset (LI, LJ, LK).
// FLUX: the flux form takes the whole cross term of the face flux into the row (twice
// the symmetric share; the transverse neighbours' rows get nothing).
template <int A, int LI, int LJ, int LK, int SC, int FLUX>
__device__ __forceinline__ void own_face(double (&row)[27], const RowCell &C, const Geo &g,
                                         const double *__restrict__ FS, long long N) {
  constexpr int RI = LI + ex_(A, 0), RJ = LJ + ex_(A, 1), RK = LK + ex_(A, 2);
  if (!has<LI, LJ, LK>(C) || !has<RI, RJ, RK>(C)) return;
  const long long l = idx<LI, LJ, LK>(C);
  const double al = FS[(3 * A + 0) * N + l];
  row[r27(LI, LJ, LK)] += -al * SC;
  row[r27(RI, RJ, RK)] += al * SC;
#pragma unroll
  for (int t = 0; t < 2; t++) {
    // (t is unrolled; tdir is constexpr-folded)
    const double be = (FLUX ? 2.0 : 1.0) * FS[(3 * A + 1 + t) * N + l];
    if (t == 0) {
      constexpr int B = tdir(A, 0), EI = ex_(B, 0), EJ = ex_(B, 1), EK = ex_(B, 2);
      const bool exp_ = has<EI, EJ, EK>(C), exm = has<-EI, -EJ, -EK>(C);
      const double gl = gam<B, LI, LJ>(g, C), gr = gam<B, RI, RJ>(g, C);
      const double v = be * SC;
      add_sel<r27(LI + EI, LJ + EJ, LK + EK), r27(LI, LJ, LK)>(row, exp_, v * gl);
      add_sel<r27(LI - EI, LJ - EJ, LK - EK), r27(LI, LJ, LK)>(row, exm, -v * gl);
      add_sel<r27(RI + EI, RJ + EJ, RK + EK), r27(RI, RJ, RK)>(row, exp_, v * gr);
      add_sel<r27(RI - EI, RJ - EJ, RK - EK), r27(RI, RJ, RK)>(row, exm, -v * gr);
      const double wp = SC < 0 ? gl : gr, wm = SC < 0 ? -gl : -gr;  // ghosts of c itself
      // (column-side entries: c enters ghat_B of this face as its own mirror ghost; the
      // flux form has no column-side entries)
      if (!FLUX && !exp_) { row[r27(LI, LJ, LK)] -= be * wp; row[r27(RI, RJ, RK)] += be * wp; }
      if (!FLUX && !exm) { row[r27(LI, LJ, LK)] -= be * wm; row[r27(RI, RJ, RK)] += be * wm; }
    } else {
      constexpr int B = tdir(A, 1), EI = ex_(B, 0), EJ = ex_(B, 1), EK = ex_(B, 2);
      const bool exp_ = has<EI, EJ, EK>(C), exm = has<-EI, -EJ, -EK>(C);
      const double gl = gam<B, LI, LJ>(g, C), gr = gam<B, RI, RJ>(g, C);
      const double v = be * SC;
      add_sel<r27(LI + EI, LJ + EJ, LK + EK), r27(LI, LJ, LK)>(row, exp_, v * gl);
      add_sel<r27(LI - EI, LJ - EJ, LK - EK), r27(LI, LJ, LK)>(row, exm, -v * gl);
      add_sel<r27(RI + EI, RJ + EJ, RK + EK), r27(RI, RJ, RK)>(row, exp_, v * gr);
      add_sel<r27(RI - EI, RJ - EJ, RK - EK), r27(RI, RJ, RK)>(row, exm, -v * gr);
      const double wp = SC < 0 ? gl : gr, wm = SC < 0 ? -gl : -gr;
      if (!FLUX && !exp_) { row[r27(LI, LJ, LK)] -= be * wp; row[r27(RI, RJ, RK)] += be * wp; }
      if (!FLUX && !exm) { row[r27(LI, LJ, LK)] -= be * wm; row[r27(RI, RJ, RK)] += be * wm; }
    }
  }
}

// A-face of the transverse neighbour x = c + SG e_T(A,TT): the face U_A(x) (LOW = 0) or
// U_A(x - e_A) (LOW = 1); c enters it as the ghat_B neighbour of x (B = tdir(A, TT)).
template <int A, int TT, int SG, int LOW>
__device__ __forceinline__ void trans_face(double (&row)[27], const RowCell &C, const Geo &g,
                                           const double *__restrict__ FS, long long N) {
  constexpr int B = tdir(A, TT);
  constexpr int XI = SG * ex_(B, 0), XJ = SG * ex_(B, 1), XK = SG * ex_(B, 2);
  constexpr int LI = XI - LOW * ex_(A, 0), LJ = XJ - LOW * ex_(A, 1), LK = XK - LOW * ex_(A, 2);
  constexpr int RI = LI + ex_(A, 0), RJ = LJ + ex_(A, 1), RK = LK + ex_(A, 2);
  if (!has<LI, LJ, LK>(C) || !has<RI, RJ, RK>(C)) return;
  const long long l = idx<LI, LJ, LK>(C);
  const double be = FS[(3 * A + 1 + TT) * N + l];
  // c = x - SG e_B, x = L (LOW = 0) or R (LOW = 1): weight of c in ghat_B is -SG gamma_B(x)
  const double w = LOW ? -SG * gam<B, RI, RJ>(g, C) : -SG * gam<B, LI, LJ>(g, C);
  row[r27(LI, LJ, LK)] -= be * w;
  row[r27(RI, RJ, RK)] += be * w;
}

template <int A, int FLUX>
__device__ __forceinline__ void faces_of_direction(double (&row)[27], const RowCell &C, const Geo &g,
                                                   const double *__restrict__ FS, long long N) {
  own_face<A, 0, 0, 0, -1, FLUX>(row, C, g, FS, N);
  own_face<A, -ex_(A, 0), -ex_(A, 1), -ex_(A, 2), +1, FLUX>(row, C, g, FS, N);
  if (FLUX) return;
  trans_face<A, 0, +1, 0>(row, C, g, FS, N);
  trans_face<A, 0, +1, 1>(row, C, g, FS, N);
  trans_face<A, 0, -1, 0>(row, C, g, FS, N);
  trans_face<A, 0, -1, 1>(row, C, g, FS, N);
  trans_face<A, 1, +1, 0>(row, C, g, FS, N);
  trans_face<A, 1, +1, 1>(row, C, g, FS, N);
  trans_face<A, 1, -1, 0>(row, C, g, FS, N);
  trans_face<A, 1, -1, 1>(row, C, g, FS, N);
}

// Across-pole theta-ghosts (POLE): in the pole rows j0 = 0 (sigma = +1) and nth - 1
// (sigma = -1) the centred theta-difference G(X) of a cell X gains sigma (u_X - u_Xb) / d,
// d = 2 r_i dtheta, Xb the cell at phi + pi, over the mirror ghost.  With
// beta_f = Vt D^{a theta} / (2h) of an r- or phi-face f = (L, R) of the pole row the energy
// changes by 1/2 sigma beta_f (u_R - u_L) [(u_L - u_Lb)/d_L + (u_R - u_Rb)/d_R], whose
// Hessian adds, with gam_i = 1/(2 d_i):
//   diagonal        -2 A(X),  A(Y) = sigma gam_i (br(i,kY) + bp(i,kY) - br(i-1,kY) - bp(i,kY-1))
//   towards X + e_r  sigma br(i,k) (gam_i - gam_{i+1})         (towards X + e_phi: nothing)
//   antipodal (0, 0)     A(X) + A(Xb)
//             (+1, 0)    sigma br(i,k) gam_{i+1} - sigma br(i,kb) gam_i
//             (-1, 0)  -sigma br(i-1,k) gam_{i-1} + sigma br(i-1,kb) gam_i
//             (0, +1)    sigma bp(i,k) gam_i - sigma bp(i,kb) gam_i
//             (0, -1)  -sigma bp(i,k-1) gam_i + sigma bp(i,kb-1) gam_i
// (br, bp: beta of the r-face i -> i+1 and of the phi-face k -> k+1 in the pole row,
// zero where there is no face).  Each antipodal entry is the sum of a term from X's faces
// and one from Xb's, computed by the same expressions in both rows, so S stays exactly
// symmetric.
struct PoleRow {
  double diag, fwd_r, bwd_r;  // changes of the diagonal and of the entries towards X +- e_r
  double ap[NPOLE];           // antipodal entries, (di, dk) = (pole_di(q), pole_dk(q))
};

__device__ __forceinline__ double pole_gam(const Geo &g, int i) { return 0.5 / (2.0 * g.rc[i] * g.dth); }

__device__ PoleRow pole_row(const Dims &d, const Geo &g, const double *__restrict__ FS, int i, int j, int k) {
  const long long N = d.N;
  const double sg = j == 0 ? 1.0 : -1.0;
  const int kb = (k + d.nph / 2) % d.nph;
  auto cell = [&](int ii, int kk) { return ((long long)kk * d.nth + j) * d.nr + ii; };
  auto km = [&](int kk) { return kk > 0 ? kk - 1 : d.nph - 1; };
  auto br = [&](int ii, int kk) { return ii < 0 ? 0.0 : FS[1 * N + cell(ii, kk)]; };  // r-face, theta cross
  auto bp = [&](int ii, int kk) { return FS[8 * N + cell(ii, kk)]; };                 // phi-face, theta cross
  const double gi = pole_gam(g, i);
  auto A = [&](int kk) { return sg * gi * (((br(i, kk) + bp(i, kk)) - br(i - 1, kk)) - bp(i, km(kk))); };
  PoleRow p;
  const double a = A(k), ab = A(kb);
  p.diag = -2.0 * a;
  p.ap[0] = a + ab;
  p.fwd_r = 0.0;
  p.bwd_r = 0.0;
  p.ap[1] = 0.0;
  p.ap[2] = 0.0;
  if (i < d.nr - 1) {
    const double gp = pole_gam(g, i + 1);
    p.fwd_r = sg * br(i, k) * (gi - gp);
    p.ap[1] = sg * br(i, k) * gp - sg * br(i, kb) * gi;
  }
  if (i > 0) {
    const double gm = pole_gam(g, i - 1);
    p.bwd_r = sg * br(i - 1, k) * (gm - gi);
    p.ap[2] = -(sg * br(i - 1, k) * gm) + sg * br(i - 1, kb) * gi;
  }
  p.ap[3] = sg * bp(i, k) * gi - sg * bp(i, kb) * gi;
  p.ap[4] = -(sg * bp(i, km(k)) * gi) + sg * bp(i, km(kb)) * gi;
  return p;
}

template <int FLUX, int POLE>
__global__ void __launch_bounds__(BLK) k_assemble_cond_fast(Dims d, Geo g, const double *__restrict__ FS,
                                                            const double *__restrict__ invW,
                                                            double *__restrict__ coef,
                                                            unsigned long long *lammax, int *flag) {
  long long cl = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (cl >= d.N) return;
  RowCell C;
  int k;
  cell_coords(d, cl, C.i, C.j, k);
  C.c = cl;
  C.up[0] = C.i < d.nr - 1;
  C.dn[0] = C.i > 0;
  C.up[1] = C.j < d.nth - 1;
  C.dn[1] = C.j > 0;
  C.up[2] = C.dn[2] = true;
  C.dup[0] = 1;
  C.ddn[0] = -1;
  C.dup[1] = d.nr;
  C.ddn[1] = -(long long)d.nr;
  C.dup[2] = (k < d.nph - 1) ? d.nrt : -(long long)(d.nph - 1) * d.nrt;
  C.ddn[2] = (k > 0) ? -d.nrt : (long long)(d.nph - 1) * d.nrt;
  double row[27];
#pragma unroll
  for (int q = 0; q < 27; q++) row[q] = 0.0;
  faces_of_direction<0, FLUX>(row, C, g, FS, d.N);
  faces_of_direction<1, FLUX>(row, C, g, FS, d.N);
  faces_of_direction<2, FLUX>(row, C, g, FS, d.N);
  double sum = 0.0;
  if (POLE && (C.j == 0 || C.j == d.nth - 1)) {
    const PoleRow p = pole_row(d, g, FS, C.i, C.j, k);
    row[13] += p.diag;
    row[r27(1, 0, 0)] += p.fwd_r;
    row[r27(-1, 0, 0)] += p.bwd_r;
    const long long stride = 2LL * d.nph * d.nr;
    const long long e = ((long long)(C.j == 0 ? 0 : 1) * d.nph + k) * d.nr + C.i;
#pragma unroll
    for (int q = 0; q < NPOLE; q++) {
      coef[10 * d.N + q * stride + e] = p.ap[q];
      sum += fabs(p.ap[q]);
    }
  }
#pragma unroll
  for (int q = 0; q < 27; q++) sum += fabs(row[q]);
#pragma unroll
  for (int m = 0; m < 9; m++) coef[m * d.N + cl] = row[r27(fwd_di(m), fwd_dj(m), fwd_dk(m))];
  coef[9 * d.N + cl] = row[13];
  if (FLUX) {  // full rows: the backward entries in slots 10..18
#pragma unroll
    for (int m = 0; m < 9; m++) coef[(10 + m) * d.N + cl] = row[r27(-fwd_di(m), -fwd_dj(m), -fwd_dk(m))];
  }
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
  ProfScope prof(ctx, RKL_K_SETUP);
  const Dims &d = ctx->d;
  unsigned grid = grid_for(d.N, BLK);
  double *kappa = ctx->scratch;
  double *FS = ctx->scratch + d.N;
  k_cell_cond<<<grid, BLK, 0, ctx->stream>>>(d, ctx->geo, T, bhat, n, kappa0, flags, kappa, ctx->W,
                                            ctx->invW, ctx->d_flag);
  k_faces_cond<<<grid, BLK, 0, ctx->stream>>>(d, ctx->geo, bhat, kappa, FS);
  if (flags & RKL_FLUX_FORM)
    k_assemble_cond_fast<1, 0><<<grid, BLK, 0, ctx->stream>>>(d, ctx->geo, FS, ctx->invW, ctx->coef,
                                                             ctx->d_lammax, ctx->d_flag);
  else if (flags & RKL_ACROSS_POLE)
    k_assemble_cond_fast<0, 1><<<grid, BLK, 0, ctx->stream>>>(d, ctx->geo, FS, ctx->invW, ctx->coef,
                                                             ctx->d_lammax, ctx->d_flag);
  else
    k_assemble_cond_fast<0, 0><<<grid, BLK, 0, ctx->stream>>>(d, ctx->geo, FS, ctx->invW, ctx->coef,
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
  k_assemble_cond_fast<0, 0><<<grid, BLK, 0, stream>>>(d, g, FS, invW, coef, lammax, flag);
  return cudaGetLastError() == cudaSuccess ? RKL_OK : RKL_ECUDA;
}

int launch_setup_viscosity(rkl_ctx *ctx, const double *rho, const double *nu) {
  ProfScope prof(ctx, RKL_K_SETUP);
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
