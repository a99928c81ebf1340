// noalloc.cu -- rkl2_superstep_noalloc: one conduction RKL2 super-step straight from the
// fields, for callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc: a host code that owns all device memory through
// its own pool and sizes its footprint once at start-up, or a time loop that cannot
// afford the device-wide synchronisation cudaMalloc/cudaFree may impose.  This entry
// point needs no context: every intermediate it uses (geometry tables, frozen
// coefficients, W and 1/W, M0 and the two stage buffers, the Gershgorin maximum) lives in
// the file-scope device array below, of a fixed maximum size, which every GPU that loads
// the library holds until the process exits.  The kernels are the ones the context path
// runs, so the result equals rkl_create + set_coeffs + rkl2_superstep.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "internal.cuh"

#define RKL_NOALLOC_MAX_CELLS 65536
#define RKL_NOALLOC_MAX_NR 1024
#define RKL_NOALLOC_MAX_NTH 1024
#define RKL_NOALLOC_MAX_DEVICES 64

namespace {

using namespace rkl;

constexpr size_t kGeo = 6 * RKL_NOALLOC_MAX_NR + 3 * RKL_NOALLOC_MAX_NTH;
constexpr size_t kCells = RKL_NOALLOC_MAX_CELLS;
// layout (doubles): geometry | kappa + face scalars (10N) | coefficients (10N) | W | 1/W |
//                   M0 | Y_a | Y_b | Gershgorin maximum + flag word (2)
constexpr size_t kOffKappa = kGeo;
constexpr size_t kOffCoef = kOffKappa + 10 * kCells;
constexpr size_t kOffW = kOffCoef + 10 * kCells;
constexpr size_t kOffInvW = kOffW + kCells;
constexpr size_t kOffM0 = kOffInvW + kCells;
constexpr size_t kOffYa = kOffM0 + kCells;
constexpr size_t kOffYb = kOffYa + kCells;
constexpr size_t kOffLam = kOffYb + kCells;
constexpr size_t kScratchDoubles = kOffLam + 2;

// Shared by every call on a device; holds the previous call's contents.
static __device__ __align__(256) double rkl_noalloc_scratch[kScratchDoubles];

// Device address of rkl_noalloc_scratch per device, looked up once (host-side name of a
// __device__ array is not a device address).
static double *g_scratch_addr[RKL_NOALLOC_MAX_DEVICES] = {nullptr};
// Host copy of the geometry tables of the call being staged (no heap use).
static double g_geo_host[kGeo];
// Guards g_scratch_addr and g_geo_host: calls from several host threads (on one device or
// on several) serialise the address look-up and the fill + upload of the geometry tables.
// An upload from pageable memory returns once the source has been staged, so the buffer
// is free again when the lock is released.
static std::mutex g_host_mu;

bool device_resident(const void *p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

double stage_b(int j) { return j <= 2 ? 1.0 / 3.0 : ((double)j * j + j - 2.0) / (2.0 * j * (j + 1.0)); }

// Geometry tables in cm at fixed offsets (slot stride MAX_NR / MAX_NTH); same formulas
// and operation order as the context path.
void fill_geometry(const rkl_grid *g) {
  const int nr = g->nr, nth = g->nth, nph = g->nph;
  const double *rf = g->r_faces;
  const double RS = g->rsun_cm > 0.0 ? g->rsun_cm : RKL_RSUN_CM;
  const double dth = RKL_PI / nth;
  (void)nph;
  double *rc = g_geo_host, *hr = rc + RKL_NOALLOC_MAX_NR, *dr = hr + RKL_NOALLOC_MAX_NR;
  double *ar = dr + RKL_NOALLOC_MAX_NR, *a2 = ar + RKL_NOALLOC_MAX_NR, *v3 = a2 + RKL_NOALLOC_MAX_NR;
  double *dcos = v3 + RKL_NOALLOC_MAX_NR, *stf = dcos + RKL_NOALLOC_MAX_NTH, *stc = stf + RKL_NOALLOC_MAX_NTH;
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
}

}  // namespace

extern "C" int rkl2_superstep_noalloc(const rkl_grid *g, const double *T, const double *bhat,
                                      const double *n, double kappa0, int coeff_flags, double *u,
                                      double dt, int s, int flags, void *cuda_stream,
                                      double *dt_exp_out, int *s_used) {
  // ---- arguments (nothing is touched on the device before they pass) ----
  if (!g || !g->r_faces || g->nr < 1 || g->nth < 1 || g->nph < 3) return RKL_EINVAL;
  if (!(g->rsun_cm == 0.0 || (std::isfinite(g->rsun_cm) && g->rsun_cm > 0.0))) return RKL_EINVAL;
  if (g->nr > RKL_NOALLOC_MAX_NR || g->nth > RKL_NOALLOC_MAX_NTH ||
      (long long)g->nr * g->nth * g->nph > RKL_NOALLOC_MAX_CELLS)
    return RKL_EINVAL;  // larger than the static scratch
  for (int i = 0; i <= g->nr; i++) {
    if (!(std::isfinite(g->r_faces[i]) && g->r_faces[i] > 0.0)) return RKL_EINVAL;
    if (i > 0 && !(g->r_faces[i] > g->r_faces[i - 1])) return RKL_EINVAL;
  }
  if (!T || !bhat || !n || !u) return RKL_EINVAL;
  if (!(std::isfinite(kappa0) && kappa0 > 0.0) || !(std::isfinite(dt) && dt > 0.0)) return RKL_EINVAL;
  if (s < 0 || s == 1) return RKL_EINVAL;
  if (coeff_flags & (RKL_FLUX_FORM | RKL_ACROSS_POLE)) return RKL_EINVAL;  // not in the static layout
  if (!device_resident(T) || !device_resident(bhat) || !device_resident(n) || !device_resident(u))
    return RKL_EINVAL;  // no host staging here: that would need device buffers
  cudaStream_t stream = (cudaStream_t)cuda_stream;

  // ---- per-device set-up: the device address of the static scratch ----
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= RKL_NOALLOC_MAX_DEVICES) return RKL_ECUDA;
  std::unique_lock<std::mutex> host_lock(g_host_mu);
  if (!g_scratch_addr[dev]) {
    double *p = nullptr;
    if (cudaGetSymbolAddress((void **)&p, rkl_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return RKL_ECUDA;
    }
    g_scratch_addr[dev] = p;
  }
  double *sc = g_scratch_addr[dev];

  Dims d;
  d.nr = g->nr;
  d.nth = g->nth;
  d.nph = g->nph;
  d.nrt = (long long)g->nr * g->nth;
  d.N = d.nrt * g->nph;
  Geo geo;
  geo.rc = sc;
  geo.hr = sc + RKL_NOALLOC_MAX_NR;
  geo.dr = sc + 2 * RKL_NOALLOC_MAX_NR;
  geo.ar = sc + 3 * RKL_NOALLOC_MAX_NR;
  geo.a2 = sc + 4 * RKL_NOALLOC_MAX_NR;
  geo.v3 = sc + 5 * RKL_NOALLOC_MAX_NR;
  geo.dcos = sc + 6 * RKL_NOALLOC_MAX_NR;
  geo.stf = geo.dcos + RKL_NOALLOC_MAX_NTH;
  geo.stc = geo.stf + RKL_NOALLOC_MAX_NTH;
  geo.dth = RKL_PI / g->nth;
  geo.dph = 2.0 * RKL_PI / g->nph;
  double *kappa = sc + kOffKappa, *FS = kappa + kCells;  // FS spans 9 * MAX_CELLS
  double *coef = sc + kOffCoef, *W = sc + kOffW, *invW = sc + kOffInvW;
  double *M0 = sc + kOffM0, *Ya = sc + kOffYa, *Yb = sc + kOffYb;
  unsigned long long *lam = (unsigned long long *)(sc + kOffLam);
  int *flag = (int *)(sc + kOffLam + 1);

  // The kernels index coefficient slots as slot * N: with N < MAX_CELLS the 10 slots
  // of coef and the 9 face-scalar slots stay inside their regions.
  fill_geometry(g);
  if (cudaMemcpyAsync(sc, g_geo_host, kGeo * sizeof(double), cudaMemcpyHostToDevice, stream) != cudaSuccess)
    return RKL_ECUDA;
  host_lock.unlock();
  // the Gershgorin maximum and the error flag must start at zero on every call
  if (cudaMemsetAsync(lam, 0, 2 * sizeof(double), stream) != cudaSuccess) return RKL_ECUDA;
  if (launch_setup_conduction_raw(d, geo, stream, T, bhat, n, kappa0, coeff_flags, kappa, FS, W, invW,
                                  coef, lam, flag) != RKL_OK)
    return RKL_ECUDA;
  unsigned long long hb[2] = {0, 0};
  if (cudaMemcpyAsync(hb, lam, 2 * sizeof(double), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
      cudaStreamSynchronize(stream) != cudaSuccess)
    return RKL_ECUDA;
  int hflag;
  double lmax;
  std::memcpy(&hflag, &hb[1], sizeof(int));
  std::memcpy(&lmax, &hb[0], sizeof(double));
  if (hflag & 1) return RKL_ENONFINITE;
  if (hflag & 2) return RKL_ECUDA;
  const double dt_exp = lmax > 0.0 ? 2.0 / lmax : INFINITY;
  if (s == 0) s = std::isinf(dt_exp) ? 2 : rkl2_stage_count(dt / dt_exp, flags);
  if (s < 2) return RKL_EINVAL;

  // ---- the super-step (Fig. 2), same buffer rotation as rkl2_superstep ----
  const double w1 = 4.0 / ((double)s * s + s - 2.0);
  if (launch_rkl2_first_raw(d, stream, coef, invW, u, M0, Ya, w1 / 3.0 * dt) != RKL_OK) return RKL_ECUDA;
  double *ym1 = Ya, *ym2 = u;
  for (int j = 2; j <= s; j++) {
    const double mu = (2.0 * j - 1.0) / j * stage_b(j) / stage_b(j - 1);
    const double nu = -(j - 1.0) / j * stage_b(j) / stage_b(j - 2);
    const double mut = w1 * mu;
    const double gt = -(1.0 - stage_b(j - 1)) * mut;
    double *out = (j == s) ? u : (j == 2 ? Yb : ym2);
    if (launch_rkl2_stage_raw(d, stream, coef, invW, ym1, ym2, u, M0, out, mu, nu, mut * dt, gt * dt) != RKL_OK)
      return RKL_ECUDA;
    ym2 = ym1;
    ym1 = out;
  }
  if (dt_exp_out) *dt_exp_out = dt_exp;
  if (s_used) *s_used = s;
  return RKL_OK;
}
