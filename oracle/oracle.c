/*
 * oracle.c -- plain, slow, FP64 CPU oracle for the frozen-coefficient parabolic
 * operators of Caplan, Mikic, Linker & Lionello, "Advancing parabolic operators in
 * thermodynamic MHD models: explicit super time-stepping versus implicit schemes
 * with Krylov solvers" (arXiv:1610.01265).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg may load this file's library.  It shares no code with the CUDA
 * library: it is written from the paper's equations, step by step, in the paper's
 * order, with no blocking, fusion or reordering.
 *
 * What each function follows:
 *   geometry / coefficients  Sec. 4.1 eq. for dT/dt (conduction term, prefactor
 *                            (gamma-1) m_p / (2 k rho) = 1/(3 k n)), Sec. 4.2
 *                            (non-uniform spherical grid, 19-point conduction and
 *                            self-adjoint viscosity stencils), App. B (p = 19, 15).
 *   operator F(u)            Eq. 1 and Eq. 3: F(u) = M u with M = W^-1 K frozen
 *                            (lagged diffusivity, Sec. 1).  K = -S where S is the
 *                            Hessian of the discrete energy Q(u) below, so that K is
 *                            symmetric (the paper's "self-adjoint" requirement for
 *                            CG, Sec. 2.1) and K 1 = 0 (no flux through the r faces).
 *   dt_Euler                 App. B, Eq. 6 and the Gershgorin bound Eq. 7 (row sums).
 *   stage count s            Eq. 5 read as s = ceil((sqrt(9 + 16 dt/dt_E) - 1)/2).
 *   RKL2                     Fig. 2 and the coefficient list of Sec. 3, with the
 *                            M0 weight read as -(1 - b_{k-1}) mu~_k.
 *   BE + PCG                 Eqs. 2-4 and Fig. 1, solving the W-scaled symmetric
 *                            form (W - dt K) x = W u^n (identical to Eq. 4 in exact
 *                            arithmetic), p_{k+1} = z_{k+1} + beta_k p_k.
 *   PC1 / PC2                App. A: Jacobi, and zero-fill ILU (IKJ) of each
 *                            non-overlapping sub-domain block; forward solve with
 *                            unit L (j < i), backward solve divided by U_ii.
 *
 * Discrete energy (the reading of the "standard" anisotropic scheme that makes K
 * symmetric; the paper does not spell the scheme out):
 *   Q(u) = 1/2 sum_{a in r,t,p} sum_{a-faces f=(L,R)} Vt_f [ D_f^aa g_f^2
 *                                      + sum_{b != a} D_f^ab g_f ghat_b(f) ]
 *   g_f       = (u_R - u_L) / h_f            (centre-to-centre distance)
 *   ghat_b(f) = (G_b(L) + G_b(R)) / 2,  G_b(c) = (u_{c+e_b} - u_{c-e_b}) / d_b(c)
 *   Vt_f      = A_f h_f                       (face dual volume)
 *   D_f       = (D_L + D_R)/2,  D_c = kappa_c bhat_c bhat_c^T (local r,t,p frame)
 * r faces at r = r_min and r = r_max are omitted (zero flux); pole faces have zero
 * area.  Transverse neighbours beyond r or theta boundaries are mirror ghosts equal
 * to the cell itself (ghost centre mirrored through the boundary face); phi is
 * periodic.  With the across-pole option (Sec. 4.2 boundaries: a theta-difference next
 * to a pole taken across it) the theta-neighbour beyond a pole is instead the cell of
 * the same pole row half a revolution away, at phi + pi (the meridian continued
 * through the pole), which couples a pole cell to five cells of the antipodal column.
 * Viscosity: Q_v = 1/2 sum_f Vt_f mu_f g_f^2, mu = nu rho, per Cartesian
 * component, W = rho V.
 *
 * Storage: an operator S is kept as full rows of 24 slots, S[c*24 + s]: slot s < 19
 * the neighbour at offset OFF[s] (phi wrapped); slots 19..23, used by pole rows with the
 * across-pole option only, the antipodal cells (i + PDI[q], j, k + nph/2 + PDK[q]).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_RSUN 6.96e10
#define OR_KB 1.380649e-16
#define OR_PI 3.14159265358979323846
#define OR_TCUT 5.0e5
#define NS19 19
#define NPOLE 5
#define NS (NS19 + NPOLE)

/* antipodal couplings of a pole cell (i, j, k) with the across-pole option: the cells
   (i + PDI[q], j, k + nph/2 + PDK[q]) of the same pole row */
static const int PDI[NPOLE] = {0, 1, -1, 0, 0};
static const int PDK[NPOLE] = {0, 0, 0, 1, -1};

static const int OFF[NS19][3] = {
    {0, 0, 0},
    {-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {0, 0, 1},
    {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}, {1, 1, 0},
    {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1}, {1, 0, 1},
    {0, -1, -1}, {0, 1, -1}, {0, -1, 1}, {0, 1, 1}};

typedef struct {
  int nr, nth, nph;
  const double *rf;
  int pole; /* across-pole theta-ghosts (needs nth >= 2 and nph even, >= 6) */
} grid;

void or_offsets(int *out) { memcpy(out, OFF, sizeof(OFF)); }
void or_pole_offsets(int *di, int *dk) {
  memcpy(di, PDI, sizeof(PDI));
  memcpy(dk, PDK, sizeof(PDK));
}
static int pole_row(const grid *g, int j) { return j == 0 || j == g->nth - 1; }

int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Number of host threads the parallel loops use (timing only; the arithmetic of every
 * loop is the same whatever the count). */
void or_set_num_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

static long cidx(const grid *g, int i, int j, int k) {
  return ((long)k * g->nth + j) * g->nr + i;
}
static long ncell(const grid *g) { return (long)g->nr * g->nth * g->nph; }
static int wrapk(const grid *g, int k) { return ((k % g->nph) + g->nph) % g->nph; }

/* ---------------- geometry (lengths in R_sun, scaled to cm at the end) ---------------- */
static double rcen(const grid *g, int i) { return 0.5 * (g->rf[i] + g->rf[i + 1]); }
static double dth(const grid *g) { return OR_PI / g->nth; }
static double dph(const grid *g) { return 2.0 * OR_PI / g->nph; }
static double tface(const grid *g, int j) { return j * dth(g); }
static double tcen(const grid *g, int j) { return (j + 0.5) * dth(g); }

double or_cell_volume(const grid *g, int i, int j) {
  double r0 = g->rf[i], r1 = g->rf[i + 1];
  return (r1 * r1 * r1 - r0 * r0 * r0) / 3.0 * (cos(tface(g, j)) - cos(tface(g, j + 1))) *
         dph(g) * OR_RSUN * OR_RSUN * OR_RSUN;
}

/* face area and centre distance of the upper a-face of cell (i,j) (k is irrelevant) */
static double face_area(const grid *g, int a, int i, int j) {
  double s2 = OR_RSUN * OR_RSUN;
  if (a == 0) {
    double r = g->rf[i + 1];
    return r * r * (cos(tface(g, j)) - cos(tface(g, j + 1))) * dph(g) * s2;
  }
  double r0 = g->rf[i], r1 = g->rf[i + 1];
  if (a == 1) return 0.5 * (r1 * r1 - r0 * r0) * sin(tface(g, j + 1)) * dph(g) * s2;
  return 0.5 * (r1 * r1 - r0 * r0) * dth(g) * s2;
}
static double face_dist(const grid *g, int a, int i, int j) {
  if (a == 0) return (rcen(g, i + 1) - rcen(g, i)) * OR_RSUN;
  if (a == 1) return rcen(g, i) * dth(g) * OR_RSUN;
  return rcen(g, i) * sin(tcen(g, j)) * dph(g) * OR_RSUN;
}
/* radius of the (possibly ghost) cell centre at radial index i in [-1, nr] */
static double rghost(const grid *g, int i) {
  if (i < 0) return 2.0 * g->rf[0] - rcen(g, 0);
  if (i >= g->nr) return 2.0 * g->rf[g->nr] - rcen(g, g->nr - 1);
  return rcen(g, i);
}
/* distance spanned by the centred b-difference at cell (i,j) */
static double cdiff_dist(const grid *g, int b, int i, int j) {
  if (b == 0) return (rghost(g, i + 1) - rghost(g, i - 1)) * OR_RSUN;
  if (b == 1) return 2.0 * rcen(g, i) * dth(g) * OR_RSUN;
  return 2.0 * rcen(g, i) * sin(tcen(g, j)) * dph(g) * OR_RSUN;
}

/* neighbour of (i,j,k) one step along direction b with sign sg, mirror ghosts in r and
   theta (the ghost is the cell itself), periodic in phi; with the across-pole option the
   theta-step beyond a pole lands on the cell at phi + pi of the same row */
static void remap(const grid *g, int i, int j, int k, int b, int sg, int *o) {
  o[0] = i; o[1] = j; o[2] = k;
  if (b == 0) { int n = i + sg; if (n >= 0 && n < g->nr) o[0] = n; }
  else if (b == 1) {
    int n = j + sg;
    if (n >= 0 && n < g->nth) o[1] = n;
    else if (g->pole) o[2] = wrapk(g, k + g->nph / 2);
  }
  else o[2] = wrapk(g, k + sg);
}

/* slot of cell q relative to cell p; -1 if not in the 19-point stencil (nor, for a
   pole row with the across-pole option, among the five antipodal couplings) */
static int slot_of(const grid *g, const int *p, const int *q) {
  int d[3];
  d[0] = q[0] - p[0];
  d[1] = q[1] - p[1];
  d[2] = q[2] - p[2];
  if (d[2] == g->nph - 1) d[2] = -1;
  if (d[2] == -(g->nph - 1)) d[2] = 1;
  for (int s = 0; s < NS19; s++)
    if (OFF[s][0] == d[0] && OFF[s][1] == d[1] && OFF[s][2] == d[2]) return s;
  if (g->pole && d[1] == 0 && pole_row(g, p[1]))
    for (int q5 = 0; q5 < NPOLE; q5++)
      if (d[0] == PDI[q5] && wrapk(g, q[2] - p[2] - g->nph / 2 - PDK[q5]) == 0) return NS19 + q5;
  return -1;
}

/* neighbour cell index of slot s, or -1 if outside r/theta range (the antipodal slots
   s >= 19 exist for pole rows only) */
static long nbr(const grid *g, int i, int j, int k, int s) {
  if (s >= NS19) {
    int ii = i + PDI[s - NS19];
    if (!pole_row(g, j) || ii < 0 || ii >= g->nr) return -1;
    return cidx(g, ii, j, wrapk(g, k + g->nph / 2 + PDK[s - NS19]));
  }
  int ii = i + OFF[s][0], jj = j + OFF[s][1];
  if (ii < 0 || ii >= g->nr || jj < 0 || jj >= g->nth) return -1;
  return cidx(g, ii, jj, wrapk(g, k + OFF[s][2]));
}

/* ---------------- coefficients (Sec. 4.1) ---------------- */
static double kappa_of(double T, double kappa0, int beta_tcut) {
  /* beta_Tcut (Sec. 4.1) as printed: kappa0 T^{5/2} times (T / T_cut)^{5/2} below T_cut */
  double k = kappa0 * pow(T, 2.5);
  if (beta_tcut && T < OR_TCUT) k *= pow(T / OR_TCUT, 2.5);
  return k;
}

static void cell_tensor(const double *T, const double *bhat, long N, long c, double kappa0,
                        int flags, double D[3][3]) {
  double kap = kappa_of(T[c], kappa0, flags & 1);
  double b[3] = {bhat[c], bhat[N + c], bhat[2 * N + c]};
  for (int a = 0; a < 3; a++)
    for (int e = 0; e < 3; e++)
      D[a][e] = (flags & 2) ? (a == e ? kap : 0.0) : kap * b[a] * b[e];
}

static void add_entry(const grid *g, double *S, const int *p, const int *q, double v) {
  int s = slot_of(g, p, q);
  if (s < 0) abort();
  S[cidx(g, p[0], p[1], p[2]) * NS + s] += v;
}

/* upper a-face of cell (i,j,k): R = cell + e_a (phi wrapped); returns 0 if no face */
static int face_cells(const grid *g, int a, int i, int j, int k, int *L, int *R) {
  L[0] = i; L[1] = j; L[2] = k;
  R[0] = i; R[1] = j; R[2] = k;
  if (a == 0) { if (i + 1 >= g->nr) return 0; R[0] = i + 1; }
  else if (a == 1) { if (j + 1 >= g->nth) return 0; R[1] = j + 1; }
  else R[2] = wrapk(g, k + 1);
  return 1;
}

/*
 * Conduction: assemble S = Hessian of Q (24 slots per row, zeroed here) and
 * W = 3 k_B n V.  flags: bit0 = beta_Tcut, bit1 = isotropic test hook (bhat bhat^T -> I),
 * bit2 = flux form: row c is minus the divergence of the face fluxes
 * A_f (D_f^aa g_f + sum_{b!=a} D_f^ab ghat_b(f)) through the faces of c, the "standard"
 * non-symmetric scheme whose symmetric part is the Hessian of Q (Sec. 4.2; PCG is used
 * for such slightly non-symmetric operators, Sec. 2.1); bit3 = across-pole theta-ghosts
 * (needs nth >= 2 and an even nph >= 6).
 */
int or_assemble_conduction(int nr, int nth, int nph, const double *rf, const double *T,
                           const double *bhat, const double *n, double kappa0, int flags,
                           double *S, double *W) {
  grid g = {nr, nth, nph, rf, (flags & 8) != 0};
  if (nr < 1 || nth < 1 || nph < 3) return -1;
  if (g.pole && (nth < 2 || nph < 6 || nph % 2)) return -1;
  long N = ncell(&g);
  memset(S, 0, sizeof(double) * NS * N);
  for (int k = 0; k < nph; k++)
    for (int j = 0; j < nth; j++)
      for (int i = 0; i < nr; i++) {
        long c = cidx(&g, i, j, k);
        W[c] = 3.0 * OR_KB * n[c] * or_cell_volume(&g, i, j);
      }
  for (int a = 0; a < 3; a++)
    for (int k = 0; k < nph; k++)
      for (int j = 0; j < nth; j++)
        for (int i = 0; i < nr; i++) {
          int L[3], R[3];
          if (!face_cells(&g, a, i, j, k, L, R)) continue;
          long cl = cidx(&g, L[0], L[1], L[2]), cr = cidx(&g, R[0], R[1], R[2]);
          double DL[3][3], DR[3][3], Df[3][3];
          cell_tensor(T, bhat, N, cl, kappa0, flags, DL);
          cell_tensor(T, bhat, N, cr, kappa0, flags, DR);
          for (int x = 0; x < 3; x++)
            for (int y = 0; y < 3; y++) Df[x][y] = 0.5 * (DL[x][y] + DR[x][y]);
          double h = face_dist(&g, a, i, j);
          double Vt = face_area(&g, a, i, j) * h;
          /* normal part: Vt D^aa g^2 / 2 */
          double alpha = Vt * Df[a][a] / (h * h);
          add_entry(&g, S, L, L, alpha);
          add_entry(&g, S, R, R, alpha);
          add_entry(&g, S, L, R, -alpha);
          add_entry(&g, S, R, L, -alpha);
          /* cross part: Vt D^ab g ghat_b / 2 */
          for (int b = 0; b < 3; b++) {
            if (b == a) continue;
            double coef = 0.5 * Vt * Df[a][b] / h;
            int X[4][3];
            double w[4];
            remap(&g, L[0], L[1], L[2], b, +1, X[0]);
            remap(&g, L[0], L[1], L[2], b, -1, X[1]);
            remap(&g, R[0], R[1], R[2], b, +1, X[2]);
            remap(&g, R[0], R[1], R[2], b, -1, X[3]);
            double gl = 0.5 / cdiff_dist(&g, b, L[0], L[1]);
            double gr = 0.5 / cdiff_dist(&g, b, R[0], R[1]);
            w[0] = gl; w[1] = -gl; w[2] = gr; w[3] = -gr;
            for (int x = 0; x < 4; x++) {
              double vL = coef * (-1.0) * w[x];
              double vR = coef * (+1.0) * w[x];
              if (flags & 4) {
                /* flux form: the face flux A_f (D^aa g + sum_b D^ab ghat_b) enters the rows
                   of L and R only (the divergence of the flux), so the cross terms are not
                   mirrored into the rows of the ghat_b neighbours */
                add_entry(&g, S, L, X[x], 2.0 * vL);
                add_entry(&g, S, R, X[x], 2.0 * vR);
              } else {
                add_entry(&g, S, L, X[x], vL);
                add_entry(&g, S, X[x], L, vL);
                add_entry(&g, S, R, X[x], vR);
                add_entry(&g, S, X[x], R, vR);
              }
            }
          }
        }
  return 0;
}

/* Q(u) evaluated directly from its face definition (used to pin the assembly). */
double or_energy_conduction(int nr, int nth, int nph, const double *rf, const double *T,
                            const double *bhat, const double *n, double kappa0, int flags,
                            const double *u) {
  grid g = {nr, nth, nph, rf, (flags & 8) != 0};
  long N = ncell(&g);
  (void)n;
  double Q = 0.0;
  for (int a = 0; a < 3; a++)
    for (int k = 0; k < nph; k++)
      for (int j = 0; j < nth; j++)
        for (int i = 0; i < nr; i++) {
          int L[3], R[3];
          if (!face_cells(&g, a, i, j, k, L, R)) continue;
          long cl = cidx(&g, L[0], L[1], L[2]), cr = cidx(&g, R[0], R[1], R[2]);
          double DL[3][3], DR[3][3];
          cell_tensor(T, bhat, N, cl, kappa0, flags, DL);
          cell_tensor(T, bhat, N, cr, kappa0, flags, DR);
          double h = face_dist(&g, a, i, j);
          double Vt = face_area(&g, a, i, j) * h;
          double gf = (u[cr] - u[cl]) / h;
          double e = 0.5 * (DL[a][a] + DR[a][a]) * gf * gf;
          for (int b = 0; b < 3; b++) {
            if (b == a) continue;
            int P[3], M[3];
            remap(&g, L[0], L[1], L[2], b, +1, P);
            remap(&g, L[0], L[1], L[2], b, -1, M);
            double GL = (u[cidx(&g, P[0], P[1], P[2])] - u[cidx(&g, M[0], M[1], M[2])]) /
                        cdiff_dist(&g, b, L[0], L[1]);
            remap(&g, R[0], R[1], R[2], b, +1, P);
            remap(&g, R[0], R[1], R[2], b, -1, M);
            double GR = (u[cidx(&g, P[0], P[1], P[2])] - u[cidx(&g, M[0], M[1], M[2])]) /
                        cdiff_dist(&g, b, R[0], R[1]);
            e += 0.5 * (DL[a][b] + DR[a][b]) * gf * 0.5 * (GL + GR);
          }
          Q += 0.5 * Vt * e;
        }
  return Q;
}

/* Viscosity (Sec. 4.1, (1/rho) div(nu rho grad v)): 7-point S per Cartesian component,
   mu = nu rho, mu_f = (mu_L + mu_R)/2, W = rho V. */
int or_assemble_viscosity(int nr, int nth, int nph, const double *rf, const double *rho,
                          const double *nu, double *S, double *W) {
  grid g = {nr, nth, nph, rf, 0};
  if (nr < 1 || nth < 1 || nph < 3) return -1;
  long N = ncell(&g);
  memset(S, 0, sizeof(double) * NS * N);
  for (int k = 0; k < nph; k++)
    for (int j = 0; j < nth; j++)
      for (int i = 0; i < nr; i++) {
        long c = cidx(&g, i, j, k);
        W[c] = rho[c] * or_cell_volume(&g, i, j);
      }
  for (int a = 0; a < 3; a++)
    for (int k = 0; k < nph; k++)
      for (int j = 0; j < nth; j++)
        for (int i = 0; i < nr; i++) {
          int L[3], R[3];
          if (!face_cells(&g, a, i, j, k, L, R)) continue;
          long cl = cidx(&g, L[0], L[1], L[2]), cr = cidx(&g, R[0], R[1], R[2]);
          double muf = 0.5 * (nu[cl] * rho[cl] + nu[cr] * rho[cr]);
          double h = face_dist(&g, a, i, j);
          double alpha = face_area(&g, a, i, j) * h * muf / (h * h);
          add_entry(&g, S, L, L, alpha);
          add_entry(&g, S, R, R, alpha);
          add_entry(&g, S, L, R, -alpha);
          add_entry(&g, S, R, L, -alpha);
        }
  return 0;
}

/* ---------------- operator apply: F(u) = M u = -W^-1 S u ---------------- */
static void s_apply(const grid *g, const double *S, const double *u, double *out) {
#pragma omp parallel for schedule(static)
  for (int k = 0; k < g->nph; k++)
    for (int j = 0; j < g->nth; j++)
      for (int i = 0; i < g->nr; i++) {
        long c = cidx(g, i, j, k);
        double acc = 0.0;
        for (int s = 0; s < NS; s++) {
          long q = nbr(g, i, j, k, s);
          if (q >= 0) acc += S[c * NS + s] * u[q];
        }
        out[c] = acc;
      }
}

int or_apply_F(int nr, int nth, int nph, const double *rf, const double *S, const double *W,
               const double *u, double *Fu) {
  grid g = {nr, nth, nph, rf, 0};
  long N = ncell(&g);
  s_apply(&g, S, u, Fu);
#pragma omp parallel for schedule(static)
  for (long c = 0; c < N; c++) Fu[c] = -Fu[c] / W[c];
  return 0;
}

/* ---------------- App. B: Gershgorin bound on |lambda|max of M ---------------- */
double or_gershgorin_dt(int nr, int nth, int nph, const double *rf, const double *S,
                        const double *W, double *lam_out) {
  grid g = {nr, nth, nph, rf, 0};
  long N = ncell(&g);
  double lam = 0.0;
  for (long c = 0; c < N; c++) {
    double row = 0.0;
    for (int s = 0; s < NS; s++) row += fabs(S[c * NS + s]);
    row /= W[c];
    if (row > lam) lam = row;
  }
  if (lam_out) *lam_out = lam;
  return 2.0 / lam;
}

/* ---------------- Sec. 3: RKL2 ---------------- */
int or_rkl2_stages(double ratio, int force_odd) {
  double s = ceil((sqrt(9.0 + 16.0 * ratio) - 1.0) / 2.0);
  int si = (int)s;
  if (si < 2) si = 2;
  if (force_odd && si % 2 == 0) si++;
  return si;
}

static double rkl_b(int j) {
  if (j <= 2) return 1.0 / 3.0;
  return ((double)j * j + j - 2.0) / (2.0 * j * (j + 1.0));
}

/* arrays of length s+1 indexed by stage j; entries j=0 unused, j=1 only mut[1] */
void or_rkl2_coeffs(int s, double *mu, double *nu, double *mut, double *gt) {
  double w1 = 4.0 / ((double)s * s + s - 2.0);
  for (int j = 0; j <= s; j++) mu[j] = nu[j] = mut[j] = gt[j] = 0.0;
  mut[1] = w1 / 3.0;
  for (int j = 2; j <= s; j++) {
    mu[j] = (2.0 * j - 1.0) / j * rkl_b(j) / rkl_b(j - 1);
    nu[j] = -(j - 1.0) / j * rkl_b(j) / rkl_b(j - 2);
    mut[j] = w1 * mu[j];
    gt[j] = -(1.0 - rkl_b(j - 1)) * mut[j];
  }
}

int or_rkl2_superstep(int nr, int nth, int nph, const double *rf, const double *S,
                      const double *W, double *u, double dt, int s) {
  grid g = {nr, nth, nph, rf, 0};
  long N = ncell(&g);
  if (s < 2) return -1;
  double *mu = malloc(sizeof(double) * (s + 1)), *nu = malloc(sizeof(double) * (s + 1));
  double *mut = malloc(sizeof(double) * (s + 1)), *gt = malloc(sizeof(double) * (s + 1));
  double *Y0 = malloc(sizeof(double) * N), *M0 = malloc(sizeof(double) * N);
  double *Ya = malloc(sizeof(double) * N), *Yb = malloc(sizeof(double) * N);
  double *Fy = malloc(sizeof(double) * N);
  or_rkl2_coeffs(s, mu, nu, mut, gt);
  memcpy(Y0, u, sizeof(double) * N);
  or_apply_F(nr, nth, nph, rf, S, W, Y0, M0);
  /* Ya = Y_{j-1}, Yb = Y_{j-2} */
#pragma omp parallel for schedule(static)
  for (long c = 0; c < N; c++) {
    Ya[c] = Y0[c] + mut[1] * dt * M0[c];
    Yb[c] = Y0[c];
  }
  for (int j = 2; j <= s; j++) {
    or_apply_F(nr, nth, nph, rf, S, W, Ya, Fy);
#pragma omp parallel for schedule(static)
    for (long c = 0; c < N; c++) {
      double y = mu[j] * Ya[c] + nu[j] * Yb[c] + (1.0 - mu[j] - nu[j]) * Y0[c] +
                 mut[j] * dt * Fy[c] + gt[j] * dt * M0[c];
      Yb[c] = Ya[c];
      Ya[c] = y;
    }
  }
  memcpy(u, Ya, sizeof(double) * N);
  free(mu); free(nu); free(mut); free(gt);
  free(Y0); free(M0); free(Ya); free(Yb); free(Fy);
  return 0;
}

/* ---------------- Sec. 6: first-order RKL1 (its remark on extra stages) ----------------
 * Y_1 = Y_0 + mu~_1 dt M Y_0,  Y_j = mu_j Y_{j-1} + nu_j Y_{j-2} + mu~_j dt M Y_{j-1},
 * mu_j = (2j-1)/j, nu_j = -(j-1)/j, mu~_j = w1 mu_j, w1 = 2/(s^2+s); stable for
 * dt <= dt_E (s^2+s)/2. */
int or_rkl1_stages(double ratio) {
  double s = ceil((sqrt(1.0 + 8.0 * ratio) - 1.0) / 2.0);
  int si = (int)s;
  return si < 1 ? 1 : si;
}

void or_rkl1_coeffs(int s, double *mu, double *nu, double *mut) {
  double w1 = 2.0 / ((double)s * s + s);
  for (int j = 0; j <= s; j++) mu[j] = nu[j] = mut[j] = 0.0;
  mut[1] = w1;
  for (int j = 2; j <= s; j++) {
    mu[j] = (2.0 * j - 1.0) / j;
    nu[j] = -(j - 1.0) / j;
    mut[j] = w1 * mu[j];
  }
}

int or_rkl1_superstep(int nr, int nth, int nph, const double *rf, const double *S,
                      const double *W, double *u, double dt, int s) {
  grid g = {nr, nth, nph, rf, 0};
  long N = ncell(&g);
  if (s < 1) return -1;
  double *mu = malloc(sizeof(double) * (s + 1)), *nu = malloc(sizeof(double) * (s + 1));
  double *mut = malloc(sizeof(double) * (s + 1));
  double *Ya = malloc(sizeof(double) * N), *Yb = malloc(sizeof(double) * N);
  double *Fy = malloc(sizeof(double) * N);
  or_rkl1_coeffs(s, mu, nu, mut);
  or_apply_F(nr, nth, nph, rf, S, W, u, Fy);
  for (long c = 0; c < N; c++) {
    Yb[c] = u[c];
    Ya[c] = u[c] + mut[1] * dt * Fy[c];
  }
  for (int j = 2; j <= s; j++) {
    or_apply_F(nr, nth, nph, rf, S, W, Ya, Fy);
    for (long c = 0; c < N; c++) {
      double y = mu[j] * Ya[c] + nu[j] * Yb[c] + mut[j] * dt * Fy[c];
      Yb[c] = Ya[c];
      Ya[c] = y;
    }
  }
  memcpy(u, Ya, sizeof(double) * N);
  free(mu); free(nu); free(mut); free(Ya); free(Yb); free(Fy);
  return 0;
}

/* ---------------- Sec. 2 / App. A: BE + PCG ---------------- */
/* A = W + dt S in 19-slot rows */
static void build_A(const grid *g, const double *S, const double *W, double dt, double *A) {
  long N = ncell(g);
#pragma omp parallel for schedule(static)
  for (long c = 0; c < N; c++) {
    for (int s = 0; s < NS; s++) A[c * NS + s] = dt * S[c * NS + s];
    A[c * NS] += W[c];
  }
}

/* Structural pattern of the operator: 19 points (conduction) or the 7 points of the
   centre and face neighbours (viscosity); App. A's "LU_ij != 0" means this pattern. */
static int g_npat = 19;

/* is the slot-s neighbour of (i,j,k) inside the same block (no phi wrap) and in the
   operator's pattern? */
static int in_block(const grid *g, const int *blk, int i, int j, int k, int s) {
  if (s >= NS19) return 0; /* antipodal couplings: dropped like those across the phi seam */
  int ii = i + OFF[s][0], jj = j + OFF[s][1], kk = k + OFF[s][2];
  (void)g;
  if (g_npat == 7 && s >= 7) return 0;
  if (ii < 0 || jj < 0 || kk < 0) return 0;
  if (ii / blk[0] != i / blk[0] || jj / blk[1] != j / blk[1] || kk / blk[2] != k / blk[2])
    return 0;
  if (ii >= g->nr || jj >= g->nth || kk >= g->nph) return 0;
  return 1;
}
static long local_index(const int *blk, int i, int j, int k) {
  return (i % blk[0]) + (long)blk[0] * ((j % blk[1]) + (long)blk[1] * (k % blk[2]));
}

/* pattern slots of cell (i,j,k) inside its block, sorted by neighbour local index */
static int block_row(const grid *g, const int *blk, int i, int j, int k, int *slots,
                     long *lidx) {
  int m = 0;
  for (int s = 0; s < NS; s++) {
    if (!in_block(g, blk, i, j, k, s)) continue;
    long li = local_index(blk, i + OFF[s][0], j + OFF[s][1], k + OFF[s][2]);
    int p = m++;
    while (p > 0 && lidx[p - 1] > li) { lidx[p] = lidx[p - 1]; slots[p] = slots[p - 1]; p--; }
    lidx[p] = li;
    slots[p] = s;
  }
  return m;
}
static int slot_by_offset(int di, int dj, int dk) {
  for (int s = 0; s < NS19; s++)
    if (OFF[s][0] == di && OFF[s][1] == dj && OFF[s][2] == dk) return s;
  return -1;
}

/* zero-fill IKJ ILU of every block of A (App. A, PC2); LU uses the 19-slot layout and
   only slots inside the block are meaningful (others are set to zero). */
int or_bilu0_factor(int nr, int nth, int nph, const double *rf, const int *blk, int npat,
                    const double *A, double *LU) {
  grid g = {nr, nth, nph, rf, 0};
  if (npat != 19 && npat != 7) return -1;
  g_npat = npat;
  long N = ncell(&g);
  if (nr % blk[0] || nth % blk[1] || nph % blk[2]) return -1;
  for (long c = 0; c < N * NS; c++) LU[c] = 0.0;
  for (int k = 0; k < nph; k++)
    for (int j = 0; j < nth; j++)
      for (int i = 0; i < nr; i++)
        for (int s = 0; s < NS; s++)
          if (in_block(&g, blk, i, j, k, s)) LU[cidx(&g, i, j, k) * NS + s] = A[cidx(&g, i, j, k) * NS + s];
  int nbk = nph / blk[2], nbj = nth / blk[1], nbi = nr / blk[0];
#pragma omp parallel for schedule(dynamic) collapse(3)
  for (int bk = 0; bk < nbk; bk++)
    for (int bj = 0; bj < nbj; bj++)
      for (int bi = 0; bi < nbi; bi++) {
        /* rows in block-local lexicographic order (r fastest) */
        for (int lk = 0; lk < blk[2]; lk++)
          for (int lj = 0; lj < blk[1]; lj++)
            for (int li = 0; li < blk[0]; li++) {
              int i = bi * blk[0] + li, j = bj * blk[1] + lj, k = bk * blk[2] + lk;
              long c = cidx(&g, i, j, k);
              long me = local_index(blk, i, j, k);
              int slots[NS];
              long lidx[NS];
              int m = block_row(&g, blk, i, j, k, slots, lidx);
              for (int p = 0; p < m && lidx[p] < me; p++) {
                int sk = slots[p];
                int ki = i + OFF[sk][0], kj = j + OFF[sk][1], kk = k + OFF[sk][2];
                long kc = cidx(&g, ki, kj, kk);
                LU[c * NS + sk] /= LU[kc * NS + 0];
                for (int q = p + 1; q < m; q++) {
                  int sj = slots[q];
                  int s3 = slot_by_offset(OFF[sj][0] - OFF[sk][0], OFF[sj][1] - OFF[sk][1],
                                          OFF[sj][2] - OFF[sk][2]);
                  if (s3 < 0) continue;
                  LU[c * NS + sj] -= LU[c * NS + sk] * LU[kc * NS + s3];
                }
              }
            }
      }
  return 0;
}

int or_bilu0_apply(int nr, int nth, int nph, const double *rf, const int *blk, int npat,
                   const double *LU, const double *r, double *z) {
  grid g = {nr, nth, nph, rf, 0};
  if (npat != 19 && npat != 7) return -1;
  g_npat = npat;
  int nbk = nph / blk[2], nbj = nth / blk[1], nbi = nr / blk[0];
#pragma omp parallel for schedule(dynamic) collapse(3)
  for (int bk = 0; bk < nbk; bk++)
    for (int bj = 0; bj < nbj; bj++)
      for (int bi = 0; bi < nbi; bi++) {
        /* forward: z* = r - L z* (unit lower) */
        for (int lk = 0; lk < blk[2]; lk++)
          for (int lj = 0; lj < blk[1]; lj++)
            for (int li = 0; li < blk[0]; li++) {
              int i = bi * blk[0] + li, j = bj * blk[1] + lj, k = bk * blk[2] + lk;
              long c = cidx(&g, i, j, k), me = local_index(blk, i, j, k);
              double v = r[c];
              for (int s = 0; s < NS; s++) {
                if (!in_block(&g, blk, i, j, k, s)) continue;
                if (local_index(blk, i + OFF[s][0], j + OFF[s][1], k + OFF[s][2]) >= me) continue;
                v -= LU[c * NS + s] * z[cidx(&g, i + OFF[s][0], j + OFF[s][1], k + OFF[s][2])];
              }
              z[c] = v;
            }
        /* backward: z = (z* - U z) / U_ii */
        for (int lk = blk[2] - 1; lk >= 0; lk--)
          for (int lj = blk[1] - 1; lj >= 0; lj--)
            for (int li = blk[0] - 1; li >= 0; li--) {
              int i = bi * blk[0] + li, j = bj * blk[1] + lj, k = bk * blk[2] + lk;
              long c = cidx(&g, i, j, k), me = local_index(blk, i, j, k);
              double v = z[c];
              for (int s = 0; s < NS; s++) {
                if (!in_block(&g, blk, i, j, k, s)) continue;
                if (local_index(blk, i + OFF[s][0], j + OFF[s][1], k + OFF[s][2]) <= me) continue;
                v -= LU[c * NS + s] * z[cidx(&g, i + OFF[s][0], j + OFF[s][1], k + OFF[s][2])];
              }
              z[c] = v / LU[c * NS + 0];
            }
      }
  return 0;
}

static double dot(long N, const double *a, const double *b) {
  double s = 0.0;
  for (long c = 0; c < N; c++) s += a[c] * b[c];
  return s;
}

/*
 * In-place BE step u <- x solving (W + dt S) x = W u (pc: 1 = PC1 Jacobi, 2 = PC2 block
 * ILU0 with block dims blk).  Stops when ||r||_2 <= rtol ||b||_2 (checked after r.z, the
 * order of Fig. 1) or after maxit products A p.  fixed_iters > 0 runs exactly that many
 * iterations with no convergence test.  Returns 0 converged, 1 maxit reached,
 * 2 breakdown (p.Ap <= 0 or not finite), -1 bad arguments.  npat = 19 (conduction) or
 * 7 (viscosity) is the operator's structural pattern used by PC2.
 */
int or_be_pcg(int nr, int nth, int nph, const double *rf, const double *S, const double *W,
              double *u, double dt, int pc, const int *blk, int npat, double rtol, int maxit,
              const double *x0, int fixed_iters, int *iters_out, double *relres_out) {
  grid g = {nr, nth, nph, rf, 0};
  long N = ncell(&g);
  if (pc != 1 && pc != 2) return -1;
  if (npat != 19 && npat != 7) return -1;
  if (pc == 2 && (nr % blk[0] || nth % blk[1] || nph % blk[2])) return -1;
  double *A = malloc(sizeof(double) * N * NS), *LU = NULL;
  double *b = malloc(sizeof(double) * N), *x = malloc(sizeof(double) * N);
  double *r = malloc(sizeof(double) * N), *z = malloc(sizeof(double) * N);
  double *p = malloc(sizeof(double) * N), *y = malloc(sizeof(double) * N);
  build_A(&g, S, W, dt, A);
  if (pc == 2) {
    LU = malloc(sizeof(double) * N * NS);
    or_bilu0_factor(nr, nth, nph, rf, blk, npat, A, LU);
  }
  for (long c = 0; c < N; c++) {
    b[c] = W[c] * u[c];
    x[c] = x0 ? x0[c] : u[c];
  }
  s_apply(&g, A, x, y);
  for (long c = 0; c < N; c++) r[c] = b[c] - y[c];
#define PRECOND()                                                    \
  do {                                                               \
    if (pc == 1)                                                     \
      for (long c = 0; c < N; c++) z[c] = r[c] / A[c * NS];          \
    else                                                             \
      or_bilu0_apply(nr, nth, nph, rf, blk, npat, LU, r, z);         \
  } while (0)
  PRECOND();
  for (long c = 0; c < N; c++) p[c] = z[c];
  double rr = dot(N, r, z);
  double bnorm = sqrt(dot(N, b, b));
  double rnorm = sqrt(dot(N, r, r));
  int it = 0, status = 1;
  if (fixed_iters <= 0 && rnorm <= rtol * bnorm) status = 0;
  int limit = fixed_iters > 0 ? fixed_iters : maxit;
  while (status == 1 && it < limit) {
    s_apply(&g, A, p, y);
    double py = dot(N, p, y);
    if (!(py > 0.0) || !isfinite(py)) { status = 2; break; }
    double alpha = rr / py;
    for (long c = 0; c < N; c++) {
      x[c] += alpha * p[c];
      r[c] -= alpha * y[c];
    }
    PRECOND();
    double rold = rr;
    rr = dot(N, r, z);
    rnorm = sqrt(dot(N, r, r));
    it++;
    if (fixed_iters <= 0 && rnorm <= rtol * bnorm) { status = 0; break; }
    double beta = rr / rold;
    for (long c = 0; c < N; c++) p[c] = z[c] + beta * p[c];
  }
#undef PRECOND
  if (fixed_iters > 0 && status == 1) status = 0;
  memcpy(u, x, sizeof(double) * N);
  if (iters_out) *iters_out = it;
  if (relres_out) *relres_out = rnorm / bnorm;
  free(A); free(LU); free(b); free(x); free(r); free(z); free(p); free(y);
  return status;
}
