// pcg.cu -- backward Euler by preconditioned CG (Sec. 2, Eqs. 2-4, Fig. 1) with point
// Jacobi (PC1) or non-overlapping block ILU0 (PC2, App. A).
//
// System: (W + dt S) x = W u^n, the W-scaled symmetric form of Eq. 4.  Every scalar
// of the iteration (alpha, beta, r.z, the residual norm, the status) stays on the
// device: each dot product is a deterministic two-level reduction (fixed-order block
// sums, then the last block to finish sums the block partials in a fixed order).
// Kernels of an iteration read the status word first and return at once when the
// solve has converged, broken down or hit maxit, so the host launches iterations in
// chunks and reads the status back once per chunk.
//
// Block ILU0: one CTA per sub-domain block; rows are processed in wavefronts
// l = li + 2 lj + 3 lk (every lower neighbour of the 19-point pattern has a smaller
// l), the factors are stored per block in wavefront order so that a wavefront's rows
// are contiguous, and the triangular solves run in shared memory.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "internal.cuh"
#include "stencil.cuh"
#include "march.cuh"

namespace rkl {

namespace {

constexpr int RB = 256;   // block size of grid-stride reduction kernels
constexpr int NSL = 19;   // slots of an ILU row: 0 diag, 1+m = -FWD[m], 10+m = +FWD[m]

__host__ __device__ constexpr int slot_di(int s) { return s == 0 ? 0 : (s < 10 ? -fwd_di(s - 1) : fwd_di(s - 10)); }
__host__ __device__ constexpr int slot_dj(int s) { return s == 0 ? 0 : (s < 10 ? -fwd_dj(s - 1) : fwd_dj(s - 10)); }
__host__ __device__ constexpr int slot_dk(int s) { return s == 0 ? 0 : (s < 10 ? -fwd_dk(s - 1) : fwd_dk(s - 10)); }

// Sum NV per-thread values over the whole grid.  Returns true (in every thread of the
// last block to finish) with the totals in tot[] of thread 0.  Blocks must be 1-D with a
// multiple of 32 threads, at most BS (threadIdx.x is the thread's rank; one counter
// increment per block); bid / nb are the block's linear index and the number of blocks.
// The order of the sums depends only on the launch shape, so the result is reproducible.
template <int NV, int BS>
__device__ bool grid_sum(double (&v)[NV], double *partials, unsigned int *counter,
                         double (&tot)[NV], unsigned int bid, unsigned int nb) {
  __shared__ double sh[NV][BS / 32];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NV; q++) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_down_sync(0xffffffffu, v[q], o);
    if (lane == 0) sh[q][warp] = v[q];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < NV; q++) {
      double s = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += sh[q][w];
      partials[(size_t)bid * NV + q] = s;
    }
    __threadfence();
    unsigned int t = atomicAdd(counter, 1u);
    last = (t == nb - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
#pragma unroll
  for (int q = 0; q < NV; q++) {
    double s = 0.0;
    for (unsigned int b = threadIdx.x; b < nb; b += blockDim.x) s += __ldcg(&partials[(size_t)b * NV + q]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) sh[q][warp] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < NV; q++) {
      double s = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += sh[q][w];
      tot[q] = s;
    }
    *counter = 0u;
  }
  return true;
}

template <int NV, int BS>
__device__ bool grid_sum(double (&v)[NV], double *partials, unsigned int *counter, double (&tot)[NV]) {
  return grid_sum<NV, BS>(v, partials, counter, tot, blockIdx.x, gridDim.x);
}

// r.z and r.r after a preconditioner application: the convergence test of Fig. 1
__device__ void finalize_dots(PcgState *st, double rz, double rn, bool init) {
  if (init) {
    st->rr = rz;
    st->rnorm2 = rn;
    st->iters = 0;
    if (!isfinite(rz) || !isfinite(rn)) st->status = PCG_BREAKDOWN;
    else st->status = (rn <= st->rtol2 * st->bnorm2) ? PCG_CONVERGED : PCG_RUNNING;
    return;
  }
  double rold = st->rr;
  st->rr = rz;
  st->rnorm2 = rn;
  st->iters += 1;
  if (!isfinite(rz) || !isfinite(rn)) st->status = PCG_BREAKDOWN;
  else if (rn <= st->rtol2 * st->bnorm2) st->status = PCG_CONVERGED;
  else if (st->iters >= st->maxit) st->status = PCG_MAXIT;
  else st->beta = rz / rold;
}

// r0 = W u - (W x0 + dt S x0); ||W u||^2 and ||r0||^2; Jacobi diagonal 1/(W + dt S_cc)
template <int OP>
__global__ void __launch_bounds__(RB) k_r0(Dims d, const double *__restrict__ coef,
                                           const double *__restrict__ W, double dt,
                                           const double *u, const double *x0,
                                           double *__restrict__ r, double *__restrict__ dinv,
                                           double *partials, unsigned int *counter,
                                           PcgState *st) {
  double v[2] = {0.0, 0.0};
  for (long long c = (long long)blockIdx.x * RB + threadIdx.x; c < d.N; c += (long long)gridDim.x * RB) {
    int i, j, k;
    cell_coords(d, c, i, j, k);
    Nbr n = neighbours(d, i, j, k);
    double w = W[c];
    double ax = fma(w, x0[c], dt * S_apply<OP>(d, coef, x0, c, n));
    double b = w * u[c];
    const double rv = b - ax;
    r[c] = rv;
    if (dinv) dinv[c] = 1.0 / fma(dt, S_diag<OP>(d, coef, c), w);
    v[0] = fma(b, b, v[0]);
    v[1] = fma(rv, rv, v[1]);
  }
  double tot[2];
  if (grid_sum<2, RB>(v, partials, counter, tot) && threadIdx.x == 0) {
    st->bnorm2 = tot[0];
    st->rnorm2 = tot[1];
  }
}

// Iteration kernels are templated on the field type T: double for the FP64 solve, float
// for the inner solve of the mixed-precision path.  Dot products always accumulate in
// FP64 and the iteration scalars (alpha, beta, norms) are FP64.
template <typename T>
__global__ void __launch_bounds__(RB) k_jacobi_init(long long N, const T *__restrict__ r,
                                                    const T *__restrict__ dinv,
                                                    T *__restrict__ p, double *partials,
                                                    unsigned int *counter, PcgState *st) {
  double v[2] = {0.0, 0.0};
  for (long long c = (long long)blockIdx.x * RB + threadIdx.x; c < N; c += (long long)gridDim.x * RB) {
    const T rv = r[c], z = rv * dinv[c];
    p[c] = z;
    v[0] = fma((double)rv, (double)z, v[0]);
    v[1] = fma((double)rv, (double)rv, v[1]);
  }
  double tot[2];
  if (grid_sum<2, RB>(v, partials, counter, tot) && threadIdx.x == 0) finalize_dots(st, tot[0], tot[1], true);
}

// y = A p = W p + dt S p ; alpha = r.z / p.y
template <int OP, typename T>
__global__ void __launch_bounds__(RB) k_spmv(Dims d, const T *__restrict__ coef,
                                             const T *__restrict__ W, T dt,
                                             const T *__restrict__ p,
                                             T *__restrict__ y, double *partials,
                                             unsigned int *counter, PcgState *st) {
  if (st->status != PCG_RUNNING) return;
  double v[1] = {0.0};
  for (long long c = (long long)blockIdx.x * RB + threadIdx.x; c < d.N; c += (long long)gridDim.x * RB) {
    int i, j, k;
    cell_coords(d, c, i, j, k);
    Nbr n = neighbours(d, i, j, k);
    const T pc = p[c];
    const T yv = fma(W[c], pc, dt * S_apply<OP, T>(d, coef, p, c, n));
    y[c] = yv;
    v[0] = fma((double)pc, (double)yv, v[0]);
  }
  double tot[1];
  if (grid_sum<1, RB>(v, partials, counter, tot) && threadIdx.x == 0) {
    double pAp = tot[0];
    st->pAp = pAp;
    if (!(pAp > 0.0) || !isfinite(pAp)) st->status = PCG_BREAKDOWN;
    else st->alpha = st->rr / pAp;
  }
}

// A = W + dt S in the storage of S (off-diagonal slots dt S, diagonal slot W + dt S_cc),
// built once per FP64 solve so that an iteration's y = A p is the stencil alone (19 FP64
// instructions per conduction row instead of 21)
template <int OP>
__global__ void __launch_bounds__(RB) k_assemble_A(Dims d, const double *__restrict__ coef,
                                                   const double *__restrict__ W, double dt,
                                                   double *__restrict__ acoef) {
  constexpr int NS = op_ncoef(OP), DIAG = OP == OPK_VISC ? 3 : 9;
  for (long long c = (long long)blockIdx.x * RB + threadIdx.x; c < d.N; c += (long long)gridDim.x * RB) {
#pragma unroll
    for (int s = 0; s < NS; s++)
      acoef[s * d.N + c] = s == DIAG ? fma(dt, coef[s * d.N + c], W[c]) : dt * coef[s * d.N + c];
  }
  if (OP == OPK_POLE) {  // the across-pole entries after the slots
    const long long np = pole_extra(d), o = (long long)NS * d.N;
    for (long long e = (long long)blockIdx.x * RB + threadIdx.x; e < np; e += (long long)gridDim.x * RB)
      acoef[o + e] = dt * coef[o + e];
  }
}

// y = A p with A from k_assemble_A ; alpha = r.z / p.y
template <int OP>
__global__ void __launch_bounds__(RB, 4) k_spmv_a(Dims d, const double *__restrict__ acoef,
                                               const double *__restrict__ p, double *__restrict__ y,
                                               double *partials, unsigned int *counter, PcgState *st) {
  if (st->status != PCG_RUNNING) return;
  double v[1] = {0.0};
  for (long long c = (long long)blockIdx.x * RB + threadIdx.x; c < d.N; c += (long long)gridDim.x * RB) {
    int i, j, k;
    cell_coords(d, c, i, j, k);
    Nbr n = neighbours(d, i, j, k);
    const double yv = S_apply<OP, double>(d, acoef, p, c, n);
    y[c] = yv;
    v[0] = fma(p[c], yv, v[0]);
  }
  double tot[1];
  if (grid_sum<1, RB>(v, partials, counter, tot) && threadIdx.x == 0) {
    double pAp = tot[0];
    st->pAp = pAp;
    if (!(pAp > 0.0) || !isfinite(pAp)) st->status = PCG_BREAKDOWN;
    else st->alpha = st->rr / pAp;
  }
}

// FP32 y = A p for the symmetric 19-point conduction operator, marching along phi like
// k_rkl2_stage_mix_march (rkl2.cu): a CTA owns a 32 x 8 (r, theta) tile and a chunk of
// phi planes, one thread per cell of the tile and its halo stages p and the
// coefficients once per plane in shared memory.  Same sums, same order as k_spmv per
// cell; p.y is accumulated per thread over its planes, then reduced over the grid.
constexpr int MR = 32, MT = 8, MHR = MR + 2, MHT = MT + 2, MPL = MHR * MHT;
constexpr int MTHREADS = 352;

__global__ void __launch_bounds__(MTHREADS) k_spmv_march(Dims d, const float *__restrict__ coef,
                                                         const float *__restrict__ W, float dt,
                                                         const float *__restrict__ p, float *__restrict__ y,
                                                         double *partials, unsigned int *counter, PcgState *st,
                                                         int kchunk) {
  if (st->status != PCG_RUNNING) return;
  __shared__ float sd[3][MPL];
  __shared__ float sc[4][MPL];
  __shared__ float sp[2][5][MPL];
  const int t = threadIdx.x;
  const bool active = t < MPL;
  const int tx = t % MHR, ty = t / MHR;
  const int i = blockIdx.x * MR + tx - 1, j = blockIdx.y * MT + ty - 1;
  const bool inside = active && i >= 0 && i < d.nr && j >= 0 && j < d.nth;
  const bool interior = inside && tx >= 1 && tx <= MR && ty >= 1 && ty <= MT;
  const long long col = inside ? (long long)j * d.nr + i : 0;
  const long long N = d.N;
  const int k0 = blockIdx.z * kchunk, k1 = min(k0 + kchunk, d.nph);
  auto wrap = [&](int k) { return k < 0 ? k + d.nph : (k >= d.nph ? k - d.nph : k); };
  auto cell = [&](int k) { return (long long)wrap(k) * d.nrt + col; };
  auto rs = [&](int k) { return (k - k0 + 1) % 3; };
  const int fw[4] = {0, 1, 3, 4}, bw[5] = {2, 5, 6, 7, 8};
  double v[1] = {0.0};
  float nf[10], nd = 0.0f, nw = 0.0f;  // next plane's loads, issued one plane ahead
  auto fetch = [&](int k) {
    const long long c = cell(k);
#pragma unroll
    for (int m = 0; m < 10; m++) nf[m] = inside ? coef[m * N + c] : 0.0f;
    nd = inside ? p[cell(k + 1)] : 0.0f;
    if (interior) nw = W[c];
  };
  if (active) {
    const long long cm = cell(k0 - 1);
    sd[rs(k0 - 1)][t] = inside ? p[cm] : 0.0f;
    sd[rs(k0)][t] = inside ? p[cell(k0)] : 0.0f;
#pragma unroll
    for (int q = 0; q < 5; q++) sp[(k0 + 1) & 1][q][t] = inside ? coef[bw[q] * N + cm] : 0.0f;
    fetch(k0);
  }
  for (int k = k0; k < k1; k++) {
    float cf[10];
    const float wc = nw;
    if (active) {
#pragma unroll
      for (int m = 0; m < 10; m++) cf[m] = nf[m];
      sd[rs(k + 1)][t] = nd;
#pragma unroll
      for (int q = 0; q < 4; q++) sc[q][t] = cf[fw[q]];
#pragma unroll
      for (int q = 0; q < 5; q++) sp[k & 1][q][t] = cf[bw[q]];
    }
    __syncthreads();
    if (active && k + 1 < k1) fetch(k + 1);
    if (interior) {
      const float *D0 = sd[rs(k)], *Dp = sd[rs(k + 1)], *Dm = sd[rs(k - 1)];
      const float(*P)[MPL] = sp[(k + 1) & 1];
      float acc = cf[9] * D0[t];
      acc = fmaf(cf[0], D0[t + 1], acc);
      acc = fmaf(cf[1], D0[t + MHR], acc);
      acc = fmaf(cf[2], Dp[t], acc);
      acc = fmaf(cf[3], D0[t - 1 + MHR], acc);
      acc = fmaf(cf[4], D0[t + 1 + MHR], acc);
      acc = fmaf(cf[5], Dp[t - 1], acc);
      acc = fmaf(cf[6], Dp[t + 1], acc);
      acc = fmaf(cf[7], Dp[t - MHR], acc);
      acc = fmaf(cf[8], Dp[t + MHR], acc);
      acc = fmaf(sc[0][t - 1], D0[t - 1], acc);
      acc = fmaf(sc[1][t - MHR], D0[t - MHR], acc);
      acc = fmaf(P[0][t], Dm[t], acc);
      acc = fmaf(sc[2][t + 1 - MHR], D0[t + 1 - MHR], acc);
      acc = fmaf(sc[3][t - 1 - MHR], D0[t - 1 - MHR], acc);
      acc = fmaf(P[1][t + 1], Dm[t + 1], acc);
      acc = fmaf(P[2][t - 1], Dm[t - 1], acc);
      acc = fmaf(P[3][t + MHR], Dm[t + MHR], acc);
      acc = fmaf(P[4][t - MHR], Dm[t - MHR], acc);
      const float pc = D0[t];
      const float yv = fmaf(wc, pc, dt * acc);
      y[cell(k)] = yv;
      v[0] = fma((double)pc, (double)yv, v[0]);
    }
    __syncthreads();
  }
  double tot[1];
  const unsigned int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
  const unsigned int nb = gridDim.x * gridDim.y * gridDim.z;
  if (grid_sum<1, MTHREADS>(v, partials, counter, tot, bid, nb) && threadIdx.x == 0) {
    double pAp = tot[0];
    st->pAp = pAp;
    if (!(pAp > 0.0) || !isfinite(pAp)) st->status = PCG_BREAKDOWN;
    else st->alpha = st->rr / pAp;
  }
}

// FP32 y = A p = W p + dt S p for symmetric conduction and viscosity, marching along phi
// with the planes of p and of the coefficients brought in by bulk copies (march.cuh); per
// cell the arithmetic of k_spmv<OP, float>.  alpha = r.z / p.y as in k_spmv.
struct SpmvEpi {
  const float *__restrict__ W;
  float *__restrict__ y;
  float dt;
  double dot;
  float4 w, wn;
  __device__ __forceinline__ void load(long long c) { wn = *reinterpret_cast<const float4 *>(W + c); }
  __device__ __forceinline__ void advance() { w = wn; }
  // p.y: the four products of a thread's cells in a plane are summed in FP32 and that
  // partial is accumulated in FP64 (one conversion and one FP64 add per four cells instead
  // of three FP64 operations per cell, which bound this kernel on the FP64 pipe)
  __device__ __forceinline__ void store(long long c, const float (&s)[4], const float (&pc)[4]) {
    const float wv[4] = {w.x, w.y, w.z, w.w};
    float yv[4], part = 0.f;
#pragma unroll
    for (int e = 0; e < 4; e++) {
      yv[e] = fmaf(wv[e], pc[e], dt * s[e]);
      part = fmaf(pc[e], yv[e], part);
    }
    dot += (double)part;
    *reinterpret_cast<float4 *>(y + c) = make_float4(yv[0], yv[1], yv[2], yv[3]);
  }
  __device__ __forceinline__ void poison(long long c) {
    const float q = __int_as_float(0x7fc00000);
    *reinterpret_cast<float4 *>(y + c) = make_float4(q, q, q, q);
    dot = __longlong_as_double(0x7ff8000000000000LL);
  }
};

template <int OP>
__global__ void __launch_bounds__(MARCH_MAX_THREADS, 1) k_spmv_tma(Dims d, int nchunk, const float *__restrict__ coef,
                                                              const float *__restrict__ W, float dt,
                                                              const float *__restrict__ p, float *__restrict__ y,
                                                              double *partials, unsigned int *counter,
                                                              PcgState *st, int *kerr) {
  if (st->status != PCG_RUNNING) return;
  SpmvEpi e{W, y, dt, 0.0};
  march32<OP>(d, nchunk, coef, p, e, kerr);
  double v[1] = {e.dot}, tot[1];
  if (grid_sum<1, MARCH_MAX_THREADS>(v, partials, counter, tot) && threadIdx.x == 0) {
    double pAp = tot[0];
    st->pAp = pAp;
    if (!(pAp > 0.0) || !isfinite(pAp) || atomicAdd(kerr, 0) != 0) st->status = PCG_BREAKDOWN;
    else st->alpha = st->rr / pAp;
  }
}

// x += alpha p ; r -= alpha y ; z = r / diag(A) ; r.z, r.r
template <typename T>
__global__ void __launch_bounds__(RB) k_update_jacobi(long long N, T *__restrict__ x,
                                                      const T *__restrict__ p,
                                                      T *__restrict__ r,
                                                      const T *__restrict__ y,
                                                      const T *__restrict__ dinv,
                                                      double *partials, unsigned int *counter,
                                                      PcgState *st) {
  if (st->status != PCG_RUNNING) return;
  const T a = (T)st->alpha;
  double v[2] = {0.0, 0.0};
  if constexpr (std::is_same<T, float>::value) {
    // FP32 with N a multiple of 4: four cells per step with 16-byte accesses; the products
    // of the four are summed in FP32 and accumulated in FP64 (one conversion and one add
    // per dot and four cells instead of four FP64 operations per cell, which bound the
    // kernel on the FP64 pipe)
    if ((N & 3) == 0) {
      const long long N4 = N >> 2;
      for (long long g = (long long)blockIdx.x * RB + threadIdx.x; g < N4; g += (long long)gridDim.x * RB) {
        float4 X = reinterpret_cast<float4 *>(x)[g], R = reinterpret_cast<float4 *>(r)[g];
        const float4 P = reinterpret_cast<const float4 *>(p)[g], Y = reinterpret_cast<const float4 *>(y)[g];
        const float4 D = reinterpret_cast<const float4 *>(dinv)[g];
        X = make_float4(fmaf(a, P.x, X.x), fmaf(a, P.y, X.y), fmaf(a, P.z, X.z), fmaf(a, P.w, X.w));
        R = make_float4(fmaf(-a, Y.x, R.x), fmaf(-a, Y.y, R.y), fmaf(-a, Y.z, R.z), fmaf(-a, Y.w, R.w));
        reinterpret_cast<float4 *>(x)[g] = X;
        reinterpret_cast<float4 *>(r)[g] = R;
        const float rz = fmaf(R.w, R.w * D.w, fmaf(R.z, R.z * D.z, fmaf(R.y, R.y * D.y, R.x * (R.x * D.x))));
        const float rr = fmaf(R.w, R.w, fmaf(R.z, R.z, fmaf(R.y, R.y, R.x * R.x)));
        v[0] += (double)rz;
        v[1] += (double)rr;
      }
      double tot[2];
      if (grid_sum<2, RB>(v, partials, counter, tot) && threadIdx.x == 0) finalize_dots(st, tot[0], tot[1], false);
      return;
    }
  }
  if constexpr (std::is_same<T, double>::value) {
    // FP64 with N even and 16-byte aligned arrays (x may be the caller's): two cells per
    // step with 16-byte accesses and two independent partial sums per dot (added in a
    // fixed order, so the result is reproducible)
    const uintptr_t al = (uintptr_t)x | (uintptr_t)p | (uintptr_t)r | (uintptr_t)y | (uintptr_t)dinv;
    if ((N & 1) == 0 && (al & 15) == 0) {
      const long long N2 = N >> 1;
      double w[2] = {0.0, 0.0};
      for (long long g = (long long)blockIdx.x * RB + threadIdx.x; g < N2; g += (long long)gridDim.x * RB) {
        double2 X = reinterpret_cast<double2 *>(x)[g], R = reinterpret_cast<double2 *>(r)[g];
        const double2 P = reinterpret_cast<const double2 *>(p)[g], Y = reinterpret_cast<const double2 *>(y)[g];
        const double2 D = reinterpret_cast<const double2 *>(dinv)[g];
        X.x = fma(a, P.x, X.x);
        X.y = fma(a, P.y, X.y);
        R.x = fma(-a, Y.x, R.x);
        R.y = fma(-a, Y.y, R.y);
        reinterpret_cast<double2 *>(x)[g] = X;
        reinterpret_cast<double2 *>(r)[g] = R;
        v[0] = fma(R.x, R.x * D.x, v[0]);
        w[0] = fma(R.y, R.y * D.y, w[0]);
        v[1] = fma(R.x, R.x, v[1]);
        w[1] = fma(R.y, R.y, w[1]);
      }
      v[0] += w[0];
      v[1] += w[1];
      double tot[2];
      if (grid_sum<2, RB>(v, partials, counter, tot) && threadIdx.x == 0) finalize_dots(st, tot[0], tot[1], false);
      return;
    }
  }
  for (long long c = (long long)blockIdx.x * RB + threadIdx.x; c < N; c += (long long)gridDim.x * RB) {
    x[c] = fma(a, p[c], x[c]);
    const T rv = fma(-a, y[c], r[c]);
    r[c] = rv;
    const T z = rv * dinv[c];
    v[0] = fma((double)rv, (double)z, v[0]);
    v[1] = fma((double)rv, (double)rv, v[1]);
  }
  double tot[2];
  if (grid_sum<2, RB>(v, partials, counter, tot) && threadIdx.x == 0) finalize_dots(st, tot[0], tot[1], false);
}

template <typename T>
__global__ void __launch_bounds__(RB) k_pupdate_jacobi(long long N, const T *__restrict__ r,
                                                       const T *__restrict__ dinv,
                                                       T *__restrict__ p,
                                                       const PcgState *st) {
  if (st->status != PCG_RUNNING) return;
  const T b = (T)st->beta;
  for (long long c = (long long)blockIdx.x * RB + threadIdx.x; c < N; c += (long long)gridDim.x * RB)
    p[c] = fma(b, p[c], r[c] * dinv[c]);
}

// x += alpha p ; r -= alpha y ; r.r for the convergence test of the block-ILU0 solve that
// follows (this kernel is bound by memory, so its FP64 product is free; FP32 fields sum the
// products of four cells in FP32 before the FP64 accumulation)
template <typename T>
__global__ void __launch_bounds__(RB) k_xr_update(long long N, T *__restrict__ x,
                                                  const T *__restrict__ p,
                                                  T *__restrict__ r,
                                                  const T *__restrict__ y,
                                                  double *partials, unsigned int *counter,
                                                  PcgState *st) {
  if (st->status != PCG_RUNNING) return;
  const T a = (T)st->alpha;
  double v[1] = {0.0};
  T part = T(0);
  int cnt = 0;
  for (long long c = (long long)blockIdx.x * RB + threadIdx.x; c < N; c += (long long)gridDim.x * RB) {
    x[c] = fma(a, p[c], x[c]);
    const T rv = fma(-a, y[c], r[c]);
    r[c] = rv;
    if constexpr (std::is_same<T, float>::value) {
      part = fmaf(rv, rv, part);
      if (++cnt == 4) {
        v[0] += (double)part;
        part = 0.f;
        cnt = 0;
      }
    } else {
      v[0] = fma(rv, rv, v[0]);
    }
  }
  v[0] += (double)part;
  double tot[1];
  if (grid_sum<1, RB>(v, partials, counter, tot) && threadIdx.x == 0) st->rnorm2 = tot[0];
}

template <typename T>
__global__ void __launch_bounds__(RB) k_pupdate_z(long long N, const T *__restrict__ z,
                                                  T *__restrict__ p, const PcgState *st,
                                                  int first) {
  if (st->status != PCG_RUNNING) return;
  const T b = first ? T(0) : (T)st->beta;
  for (long long c = (long long)blockIdx.x * RB + threadIdx.x; c < N; c += (long long)gridDim.x * RB)
    p[c] = first ? z[c] : fma(b, p[c], z[c]);
}

// mixed precision: the FP64 residual r scaled by 1/sigma into the FP32 right-hand side of
// the correction solve, whose starting guess is e = 0; ||r/sigma||^2 is the inner ||b||^2
__global__ void __launch_bounds__(RB) k_scale_to_f32(long long N, const double *__restrict__ r,
                                                     double inv_sigma, float *__restrict__ r32,
                                                     float *__restrict__ e32, double *partials,
                                                     unsigned int *counter, PcgState *st) {
  double v[1] = {0.0};
  for (long long c = (long long)blockIdx.x * RB + threadIdx.x; c < N; c += (long long)gridDim.x * RB) {
    const float rv = (float)(r[c] * inv_sigma);
    r32[c] = rv;
    e32[c] = 0.0f;
    v[0] = fma((double)rv, (double)rv, v[0]);
  }
  double tot[1];
  if (grid_sum<1, RB>(v, partials, counter, tot) && threadIdx.x == 0) {
    st->bnorm2 = tot[0];
    st->rnorm2 = tot[0];  // e = 0: the inner residual is the right-hand side
  }
}

// x += sigma e (FP64)
__global__ void __launch_bounds__(RB) k_correct(long long N, double *__restrict__ x, double sigma,
                                                const float *__restrict__ e32) {
  for (long long c = (long long)blockIdx.x * RB + threadIdx.x; c < N; c += (long long)gridDim.x * RB)
    x[c] = fma(sigma, (double)e32[c], x[c]);
}

// ---------------- block ILU0 ----------------

constexpr int GB = 256;  // threads of a block-ILU0 CTA (G blocks per CTA)

struct BlockCell {
  int li, lj, lk;
  long long c;
};

__device__ __forceinline__ BlockCell block_cell(const Dims &d, const IluPlan &pl, int blk, int l) {
  BlockCell b;
  int bI = blk % pl.nbi, bJ = (blk / pl.nbi) % pl.nbj, bK = blk / (pl.nbi * pl.nbj);
  b.li = l % pl.bi;
  b.lj = (l / pl.bi) % pl.bj;
  b.lk = l / (pl.bi * pl.bj);
  int i = bI * pl.bi + b.li, j = bJ * pl.bj + b.lj, k = bK * pl.bk + b.lk;
  b.c = ((long long)k * d.nth + j) * d.nr + i;
  return b;
}

// is the slot-s neighbour inside the block (no phi wrap), and part of the pattern
template <int OP>
__device__ __forceinline__ bool in_pattern(const IluPlan &pl, const BlockCell &b, int s) {
  if (OP == RKL_OP_VISCOSITY && s != 0 && (((s - 1) % 9) >= 3)) return false;  // 7-point
  int li = b.li + slot_di(s), lj = b.lj + slot_dj(s), lk = b.lk + slot_dk(s);
  return li >= 0 && li < pl.bi && lj >= 0 && lj < pl.bj && lk >= 0 && lk < pl.bk;
}

__device__ __forceinline__ int slot_ldelta(const IluPlan &pl, int s) {
  return slot_di(s) + pl.bi * (slot_dj(s) + pl.bj * slot_dk(s));
}

__host__ __device__ constexpr int lex_rank(int s) {
  return (slot_dk(s) + 1) * 9 + (slot_dj(s) + 1) * 3 + (slot_di(s) + 1);
}

__host__ __device__ constexpr int slot_of_offset(int di, int dj, int dk) {
  if (di == 0 && dj == 0 && dk == 0) return 0;
  for (int m = 0; m < 9; m++) {
    if (fwd_di(m) == di && fwd_dj(m) == dj && fwd_dk(m) == dk) return 10 + m;
    if (fwd_di(m) == -di && fwd_dj(m) == -dj && fwd_dk(m) == -dk) return 1 + m;
  }
  return -1;
}

template <int OP> constexpr int ilu_pat() { return OP == OPK_VISC ? 7 : 19; }

// position inside a group's [G * bs] slot array of block bb's local cell l
__device__ __forceinline__ int group_pos(const IluPlan &pl, int bb, int l) {
  int li = l % pl.bi, lj = (l / pl.bi) % pl.bj, lk = l / (pl.bi * pl.bj);
  int lev = ilu_level(pl.pat, li, lj, lk);
  int ls = pl.lev_start[lev], nl = pl.lev_start[lev + 1] - ls;
  return pl.G * ls + bb * nl + (pl.pos_of[l] - ls);
}

// zero-fill IKJ ILU of the rows of A = W + dt S of G blocks (App. A), wavefront by
// wavefront; rows of earlier wavefronts are read back from the group's factor array.
template <int OP>
__global__ void __launch_bounds__(GB) k_bilu_factor(Dims d, IluPlan pl,
                                                    const double *__restrict__ coef,
                                                    const double *__restrict__ W, double dt,
                                                    double *__restrict__ LU) {
  constexpr int PAT = ilu_pat<OP>();
  const int grp = blockIdx.x, b0 = grp * pl.G;
  const int gcount = min(pl.G, pl.nblocks - b0);
  const size_t gs = (size_t)pl.G * pl.bs;
  double *LUg = LU + (size_t)grp * ilu_nslots(PAT) * gs;
  const int nf = OP == RKL_OP_VISCOSITY ? 3 : 9;
  for (int lev = 0; lev < pl.nlev; lev++) {
    const int ls = pl.lev_start[lev], nl = pl.lev_start[lev + 1] - ls;
    for (int q = threadIdx.x; q < gcount * nl; q += GB) {
      const int bb = q / nl, l = pl.lev_cell[ls + (q - bb * nl)];
      const size_t p = (size_t)pl.G * ls + q;
      BlockCell b = block_cell(d, pl, b0 + bb, l);
      int mask = 0;  // bit s: slot s inside the block and the pattern
#pragma unroll
      for (int q2 = 0; q2 < NSL; q2++)
        if (in_pattern<OP>(pl, b, q2)) mask |= 1 << q2;
      double a[NSL];
      a[0] = fma(dt, S_diag<OP>(d, coef, b.c), W[b.c]);
#pragma unroll
      for (int m = 0; m < 9; m++) {
        a[1 + m] = 0.0;
        a[10 + m] = 0.0;
        if (m >= nf) continue;
        const long long off = fwd_di(m) + (long long)fwd_dj(m) * d.nr + (long long)fwd_dk(m) * d.nrt;
        if (mask & (1 << (10 + m))) a[10 + m] = dt * coef[m * d.N + b.c];
        if (mask & (1 << (1 + m)))  // full rows keep the backward entries themselves
          a[1 + m] = dt * (OP == OPK_FLUX ? coef[(10 + m) * d.N + b.c] : coef[m * d.N + b.c - off]);
      }
      // lower slots in increasing order of the neighbour's position (lexicographic); the
      // slot arithmetic is resolved at compile time, only the pattern mask is tested here
#pragma unroll
      for (int rk = 0; rk < 13; rk++) {
#pragma unroll
        for (int s = 1; s < 10; s++) {
          if (lex_rank(s) != rk) continue;
          // the loads do not depend on a[], so they are issued unconditionally (a slot outside
          // the pattern reads the row's own, valid position and the values are not used) and
          // the compiler can start them ahead of the eliminations before them
          const bool has = mask & (1 << s);
          const size_t kp = has ? (size_t)group_pos(pl, bb, l + slot_ldelta(pl, s)) : p;
          const double ukk = LUg[kp];  // U_kk, slot 0
          double u[NSL];
#pragma unroll
          for (int q2 = 0; q2 < NSL; q2++) {
            u[q2] = 0.0;
            if (lex_rank(q2) <= rk) continue;
            const int s3 = slot_of_offset(slot_di(q2) - slot_di(s), slot_dj(q2) - slot_dj(s),
                                          slot_dk(q2) - slot_dk(s));
            if (s3 < 0 || lu_slot(PAT, s3) < 0) continue;
            u[q2] = LUg[(size_t)lu_slot(PAT, s3) * gs + kp];
          }
          if (!has) continue;
          const double L = a[s] / ukk;
          a[s] = L;
#pragma unroll
          for (int q2 = 0; q2 < NSL; q2++) {
            if (lex_rank(q2) <= rk) continue;
            const int s3 = slot_of_offset(slot_di(q2) - slot_di(s), slot_dj(q2) - slot_dj(s),
                                          slot_dk(q2) - slot_dk(s));
            if (s3 < 0 || lu_slot(PAT, s3) < 0 || !(mask & (1 << q2))) continue;
            a[q2] -= L * u[q2];
          }
        }
      }
#pragma unroll
      for (int q2 = 0; q2 < NSL; q2++)
        if (lu_slot(PAT, q2) >= 0) LUg[(size_t)lu_slot(PAT, q2) * gs + p] = (mask & (1 << q2)) ? a[q2] : 0.0;
      LUg[(size_t)lu_slot(PAT, 19) * gs + p] = 1.0 / a[0];
    }
    __syncthreads();
  }
}

// z = (LU)^{-1} r on G blocks: residual staged in shared memory, forward (unit L) and
// backward (U, times 1/U_ii) sweeps wavefront by wavefront, then r.z and r.r.
// G is chosen so that a wavefront of the group has at most AB rows: each thread owns at
// most one row per wavefront and loads the factors of its next row before the barrier,
// so their latency overlaps the current wavefront.  Per-position data (local index,
// pattern mask, offset in the grid) is tabulated once per CTA in shared memory.
constexpr int AB = 384;
// the solve depends only on the pattern kept by the factorisation: the flux form keeps
// the 19-point pattern of symmetric conduction, and so does the across-pole form (its
// couplings to the antipodal column leave every block)
constexpr int ilu_op(int op) { return op == OPK_FLUX || op == OPK_POLE ? OPK_COND : op; }
constexpr int ILU_TAB_BYTES = (8192 + 64) * 8 + 4096 * 4 * 2 + 64 * 8;  // zs + tab + goff + base
// per-block stride of the staged residual: odd, so that the same local cell of the G
// blocks of a group falls into different shared-memory banks
__host__ __device__ constexpr int ilu_zstride(int bs) { return bs | 1; }

template <int OP, typename T>
__global__ void __launch_bounds__(AB) k_bilu_apply(Dims d, IluPlan pl,
                                                   const T *__restrict__ LU,
                                                   const T *__restrict__ r,
                                                   T *__restrict__ z, double *partials,
                                                   unsigned int *counter, PcgState *st,
                                                   int init) {
  if (!init && st->status != PCG_RUNNING) return;
  constexpr int PAT = ilu_pat<OP>();
  constexpr int NF = PAT == 7 ? 3 : 9;  // lower (and upper) couplings of a row
  constexpr int SU = lu_slot(PAT, 10), SINV = lu_slot(PAT, 19);
  extern __shared__ double smem[];
  const int bs = pl.bs;
  const int zst = ilu_zstride(bs);
  T *zs = reinterpret_cast<T *>(smem);                      // [G][zst] by local index
  long long *base = (long long *)(smem + ((size_t)pl.G * zst * sizeof(T) + 7) / 8);  // [G]
  int *tab = (int *)(base + pl.G);                          // [bs] level order: l | mask << 12
  int *goff = tab + bs;                                     // [bs] by local index
  const int grp = blockIdx.x, b0 = grp * pl.G;
  const int gcount = min(pl.G, pl.nblocks - b0);
  const size_t gs = (size_t)pl.G * bs;
  const T *LUg = LU + (size_t)grp * ilu_nslots(PAT) * gs;
  const int tid = threadIdx.x;

  for (int pp = tid; pp < bs; pp += AB) {
    const int l = pl.lev_cell[pp];
    BlockCell b;
    b.li = l % pl.bi;
    b.lj = (l / pl.bi) % pl.bj;
    b.lk = l / (pl.bi * pl.bj);
    int mask = 0;  // bit m: lower coupling m, bit 9 + m: upper coupling m
#pragma unroll
    for (int m = 0; m < NF; m++) {
      if (in_pattern<OP>(pl, b, 1 + m)) mask |= 1 << m;
      if (in_pattern<OP>(pl, b, 10 + m)) mask |= 1 << (9 + m);
    }
    tab[pp] = l | (mask << 12);
    goff[l] = (int)(b.li + (long long)d.nr * b.lj + d.nrt * b.lk);
  }
  for (int bb = tid; bb < gcount; bb += AB) {
    const int blk = b0 + bb;
    const int bI = blk % pl.nbi, bJ = (blk / pl.nbi) % pl.nbj, bK = blk / (pl.nbi * pl.nbj);
    base[bb] = ((long long)(bK * pl.bk) * d.nth + bJ * pl.bj) * d.nr + bI * pl.bi;
  }
  __syncthreads();
  for (int q = tid; q < gcount * bs; q += AB) {
    const int bb = q / bs;
    zs[bb * zst + (q - bb * bs)] = r[base[bb] + goff[q - bb * bs]];
  }
  int dl[NF];  // local-index offset of lower coupling m (of upper coupling m: -dl[m])
#pragma unroll
  for (int m = 0; m < NF; m++) dl[m] = slot_ldelta(pl, 1 + m);

  // ---- forward sweep: z* = r - L z* ----
  T pre[NF];
  {
    const int nl = pl.lev_start[1] - pl.lev_start[0];
    if (tid < gcount * nl) {
#pragma unroll
      for (int m = 0; m < NF; m++) pre[m] = LUg[(size_t)(1 + m) * gs + tid];
    }
  }
  __syncthreads();
  for (int lev = 0; lev < pl.nlev; lev++) {
    const int ls = pl.lev_start[lev], nl = pl.lev_start[lev + 1] - ls;
    T cur[NF];
#pragma unroll
    for (int m = 0; m < NF; m++) cur[m] = pre[m];
    if (lev + 1 < pl.nlev) {
      const int ls2 = pl.lev_start[lev + 1], nl2 = pl.lev_start[lev + 2] - ls2;
      if (tid < gcount * nl2) {
        const size_t p2 = (size_t)pl.G * ls2 + tid;
#pragma unroll
        for (int m = 0; m < NF; m++) pre[m] = LUg[(size_t)(1 + m) * gs + p2];
      }
    }
    for (int q = tid; q < gcount * nl; q += AB) {
      const int bb = q / nl;
      const int t = tab[ls + (q - bb * nl)], l = t & 0xfff, mask = t >> 12;
      T *zb = zs + bb * zst;
      T v = zb[l];
      if (q == tid) {
#pragma unroll
        for (int m = 0; m < NF; m++)
          if (mask & (1 << m)) v = fma(-cur[m], zb[l + dl[m]], v);
      } else {
        const size_t p = (size_t)pl.G * ls + q;
#pragma unroll
        for (int m = 0; m < NF; m++)
          if (mask & (1 << m)) v = fma(-LUg[(size_t)(1 + m) * gs + p], zb[l + dl[m]], v);
      }
      zb[l] = v;
    }
    __syncthreads();
  }

  // ---- backward sweep: z = (z* - U z) / U_ii ----
  T preb[NF + 1];
  {
    const int lsl = pl.lev_start[pl.nlev - 1], nl = pl.lev_start[pl.nlev] - lsl;
    if (tid < gcount * nl) {
      const size_t p = (size_t)pl.G * lsl + tid;
#pragma unroll
      for (int m = 0; m < NF; m++) preb[m] = LUg[(size_t)(SU + m) * gs + p];
      preb[NF] = LUg[(size_t)SINV * gs + p];
    }
  }
  for (int lev = pl.nlev - 1; lev >= 0; lev--) {
    const int ls = pl.lev_start[lev], nl = pl.lev_start[lev + 1] - ls;
    T cur[NF + 1];
#pragma unroll
    for (int m = 0; m <= NF; m++) cur[m] = preb[m];
    if (lev > 0) {
      const int ls2 = pl.lev_start[lev - 1], nl2 = ls - ls2;
      if (tid < gcount * nl2) {
        const size_t p2 = (size_t)pl.G * ls2 + tid;
#pragma unroll
        for (int m = 0; m < NF; m++) preb[m] = LUg[(size_t)(SU + m) * gs + p2];
        preb[NF] = LUg[(size_t)SINV * gs + p2];
      }
    }
    for (int q = tid; q < gcount * nl; q += AB) {
      const int bb = q / nl;
      const int t = tab[ls + (q - bb * nl)], l = t & 0xfff, mask = t >> 12;
      T *zb = zs + bb * zst;
      T v = zb[l];
      if (q == tid) {
#pragma unroll
        for (int m = 0; m < NF; m++)
          if (mask & (1 << (9 + m))) v = fma(-cur[m], zb[l - dl[m]], v);
        zb[l] = v * cur[NF];
      } else {
        const size_t p = (size_t)pl.G * ls + q;
#pragma unroll
        for (int m = 0; m < NF; m++)
          if (mask & (1 << (9 + m))) v = fma(-LUg[(size_t)(SU + m) * gs + p], zb[l - dl[m]], v);
        zb[l] = v * LUg[(size_t)SINV * gs + p];
      }
    }
    __syncthreads();
  }
  double v1[1] = {0.0};
  // r.z (r.r comes from the x, r update before this kernel): FP64 products per cell for
  // the FP64 solve; for the FP32 solve the products of four successive cells of a thread
  // are summed in FP32 before the FP64 accumulation, as in the FP32 SpMV and Jacobi update
  T prz = T(0);
  int cnt = 0;
  for (int q = tid; q < gcount * bs; q += AB) {
    const int bb = q / bs;
    const long long c = base[bb] + goff[q - bb * bs];
    const T zv = zs[bb * zst + (q - bb * bs)], rv = r[c];
    z[c] = zv;
    if constexpr (std::is_same<T, float>::value) {
      prz = fmaf(rv, zv, prz);
      if (++cnt == 4) {
        v1[0] += (double)prz;
        prz = 0.f;
        cnt = 0;
      }
    } else {
      v1[0] = fma(rv, zv, v1[0]);
    }
  }
  v1[0] += (double)prz;
  double tot[1];
  if (grid_sum<1, AB>(v1, partials, counter, tot) && threadIdx.x == 0)
    finalize_dots(st, tot[0], st->rnorm2, init != 0);
}

unsigned int march_grid(const rkl_ctx *ctx, int op) {
  const int TH = march_th(ctx->d.nr);
  return (unsigned)(((ctx->d.nth + TH - 1) / TH) * ctx->march_nchunk[op]);
}

unsigned int stride_grid(const rkl_ctx *ctx) {
  long long g = (ctx->d.N + RB - 1) / RB;
  long long cap = (long long)ctx->nsm * 8;
  return (unsigned int)std::max(1LL, std::min(g, cap));
}

}  // namespace

// the marching kernels may use up to the opt-in shared memory of a CTA, whatever the
// grid of the context (the attribute belongs to the kernel, not to a context)
int march_setup_spmv(rkl_ctx *ctx) {
  int optin = 0;
  int rc = cuda_check(ctx, cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device),
                      "shared memory opt-in");
  if (rc) return rc;
  for (int op = OPK_COND; op <= OPK_VISC; op++)
    if ((size_t)optin < march_smem(ctx->d.nr, op) + 1024) ctx->march_nchunk[op] = 0;
  rc = cuda_check(ctx, cudaFuncSetAttribute(k_spmv_tma<OPK_COND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            optin - 1024),
                  "bulk-copy SpMV shared memory");
  if (rc) return rc;
  return cuda_check(ctx, cudaFuncSetAttribute(k_spmv_tma<OPK_VISC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              optin - 1024),
                    "bulk-copy SpMV shared memory");
}

// Build the wavefront plan of a block shape and (re)factor A = W + dt S when the block
// shape, dt or the operator changed since the last factorisation.
int bilu0_prepare(rkl_ctx *ctx, const int *block, double dt) {
  const Dims &d = ctx->d;
  const int pat = ctx->op == OPK_VISC ? 7 : 19;  // pattern kept by the zero-fill ILU
  if (ctx->lu_valid && ctx->lu_blk[0] == block[0] && ctx->lu_blk[1] == block[1] &&
      ctx->lu_blk[2] == block[2] && ctx->lu_dt == dt && ctx->plan.pat == pat)
    return RKL_OK;
  int bi = block[0], bj = block[1], bk = block[2], bs = bi * bj * bk;
  if (ctx->plan.bs != bs || ctx->plan.bi != bi || ctx->plan.bj != bj || ctx->plan.bk != bk ||
      ctx->plan.pat != pat) {
    // wavefronts l = li + 2 lj + 3 lk (19-point: every lower neighbour, (1,-1,0) included,
    // has a smaller l) or l = li + lj + lk (7-point); lexicographic order within a wavefront
    const int nlev = ilu_level(pat, bi - 1, bj - 1, bk - 1) + 1;
    std::vector<int> start(nlev + 1, 0), cell(bs), pos(bs);
    for (int lk = 0; lk < bk; lk++)
      for (int lj = 0; lj < bj; lj++)
        for (int li = 0; li < bi; li++) start[ilu_level(pat, li, lj, lk) + 1]++;
    for (int l = 0; l < nlev; l++) start[l + 1] += start[l];
    std::vector<int> fill(start.begin(), start.end() - 1);
    for (int lk = 0; lk < bk; lk++)
      for (int lj = 0; lj < bj; lj++)
        for (int li = 0; li < bi; li++) {
          int l = li + bi * (lj + bj * lk);
          int p = fill[ilu_level(pat, li, lj, lk)]++;
          cell[p] = l;
          pos[l] = p;
        }
    if (ctx->plan_buf) {
      int rc0 = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "ILU plan resize");
      if (rc0) return rc0;
      cudaFree(ctx->plan_buf);
    }
    ctx->plan_buf = nullptr;
    size_t nint = (size_t)(nlev + 1) + 2 * (size_t)bs;
    if (cuda_check(ctx, cudaMalloc(&ctx->plan_buf, nint * sizeof(int)), "alloc ILU plan")) return RKL_ENOMEM;
    std::vector<int> host(nint);
    std::copy(start.begin(), start.end(), host.begin());
    std::copy(cell.begin(), cell.end(), host.begin() + nlev + 1);
    std::copy(pos.begin(), pos.end(), host.begin() + nlev + 1 + bs);
    int rc = cuda_check(ctx, cudaMemcpyAsync(ctx->plan_buf, host.data(), nint * sizeof(int),
                                             cudaMemcpyHostToDevice, ctx->stream),
                        "upload ILU plan");
    if (rc) return rc;
    rc = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "upload ILU plan");
    if (rc) return rc;
    IluPlan &pl = ctx->plan;
    pl.bi = bi; pl.bj = bj; pl.bk = bk; pl.bs = bs; pl.nlev = nlev; pl.pat = pat;
    pl.nbi = d.nr / bi; pl.nbj = d.nth / bj; pl.nbk = d.nph / bk;
    pl.nblocks = pl.nbi * pl.nbj * pl.nbk;
    // G blocks per CTA: enough rows per wavefront to fill the warps but at most AB rows
    // per wavefront of the group, and G * bs <= 8192 cells of shared memory
    int maxlev = 0;
    for (int l = 0; l < nlev; l++) maxlev = std::max(maxlev, start[l + 1] - start[l]);
    pl.G = std::max(1, std::min({64, 8192 / bs, AB / maxlev}));
    pl.ngroups = (pl.nblocks + pl.G - 1) / pl.G;
    pl.lev_start = ctx->plan_buf;
    pl.lev_cell = ctx->plan_buf + nlev + 1;
    pl.pos_of = ctx->plan_buf + nlev + 1 + bs;
    // the attribute is per function (shared by all contexts): always allow the largest group
    const int smem = ILU_TAB_BYTES;
    rc = cuda_check(ctx, cudaFuncSetAttribute(k_bilu_apply<RKL_OP_CONDUCTION, double>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize, smem),
                    "ILU shared memory");
    if (!rc)
      rc = cuda_check(ctx, cudaFuncSetAttribute(k_bilu_apply<RKL_OP_VISCOSITY, double>,
                                                cudaFuncAttributeMaxDynamicSharedMemorySize, smem),
                      "ILU shared memory");
    if (!rc)
      rc = cuda_check(ctx, cudaFuncSetAttribute(k_bilu_apply<RKL_OP_CONDUCTION, float>,
                                                cudaFuncAttributeMaxDynamicSharedMemorySize, smem),
                      "ILU shared memory");
    if (!rc)
      rc = cuda_check(ctx, cudaFuncSetAttribute(k_bilu_apply<RKL_OP_VISCOSITY, float>,
                                                cudaFuncAttributeMaxDynamicSharedMemorySize, smem),
                      "ILU shared memory");
    if (rc) return rc;
  }
  const size_t need = (size_t)ilu_nslots(pat) * ctx->plan.ngroups * ctx->plan.G * ctx->plan.bs;
  int rc;
  if (need > ctx->lu_cap) {
    if (ctx->LU) {
      if ((rc = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "ILU resize"))) return rc;
      cudaFree(ctx->LU);
      ctx->LU = nullptr;
      ctx->lu_cap = 0;
    }
    if ((rc = cuda_check(ctx, cudaMalloc(&ctx->LU, need * sizeof(double)), "block-ILU0 factors"))) return rc;
    ctx->lu_cap = need;
  }
  const unsigned int ngrp = (unsigned int)ctx->plan.ngroups;
  ProfScope prof(ctx, RKL_K_BILU_FACTOR);
  op_dispatch(ctx->op, [&](auto kind) {
    constexpr int OP = decltype(kind)::value;
      k_bilu_factor<OP><<<ngrp, GB, 0, ctx->stream>>>(d, ctx->plan, ctx->coef, ctx->W, dt, ctx->LU);
  });
  ctx->launches += 1;
  rc = cuda_check(ctx, cudaGetLastError(), "block-ILU0 factor launch");
  if (rc) return rc;
  if (ctx->prec == RKL_F32MIX) {  // FP32 copy of the factors for the correction solves
    if (need > ctx->lu32_cap) {
      if (ctx->LU32) {
        if ((rc = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "ILU resize"))) return rc;
        cudaFree(ctx->LU32);
        ctx->LU32 = nullptr;
        ctx->lu32_cap = 0;
      }
      if ((rc = cuda_check(ctx, cudaMalloc(&ctx->LU32, need * sizeof(float)), "FP32 block-ILU0 factors"))) return rc;
      ctx->lu32_cap = need;
    }
    if ((rc = launch_to_float(ctx, ctx->LU, ctx->LU32, (long long)need))) return rc;
  }
  ctx->lu_valid = 1;
  ctx->lu_blk[0] = bi; ctx->lu_blk[1] = bj; ctx->lu_blk[2] = bk;
  ctx->lu_dt = dt;
  return RKL_OK;
}

template <typename T>
struct PcgFields {
  T *x, *r, *p, *y, *z, *dinv;
  const T *coef, *W, *LU;
  const double *acoef;  // A = W + dt S for the FP64 iteration (NULL: y = W p + dt S p)
};

static int state_upload(rkl_ctx *ctx, double rtol, int maxit) {
  PcgState init{};
  init.rtol2 = rtol > 0.0 ? rtol * rtol : -1.0;
  init.maxit = maxit;
  init.status = PCG_RUNNING;
  *ctx->h_state = init;
  return cuda_check(ctx, cudaMemcpyAsync(ctx->d_state, ctx->h_state, sizeof(PcgState),
                                         cudaMemcpyHostToDevice, ctx->stream), "PCG state upload");
}

static int state_read(rkl_ctx *ctx) {
  int rc = cuda_check(ctx, cudaMemcpyAsync(ctx->h_state, ctx->d_state, sizeof(PcgState) + sizeof(int),
                                           cudaMemcpyDeviceToHost, ctx->stream), "PCG state read");
  if (rc) return rc;
  if ((rc = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "PCG iteration"))) return rc;
  return check_kerr(ctx, reinterpret_cast<const int *>(ctx->h_state + 1));
}

static size_t ilu_smem(const rkl_ctx *ctx, size_t elem) {
  const IluPlan &pl = ctx->plan;
  return ((elem * pl.G * ilu_zstride(pl.bs) + 7) / 8) * 8 + sizeof(long long) * pl.G + 2 * sizeof(int) * pl.bs;
}

// first preconditioner application once r (and for PC1 the diagonal) is in place and
// the state holds ||b||^2: z0 = P^-1 r0, p0 = z0, r.z, convergence test
template <int OP, typename T>
static void pcg_first(rkl_ctx *ctx, const PcgFields<T> &f, int pc) {
  const Dims &d = ctx->d;
  const unsigned g = stride_grid(ctx);
  if (pc == RKL_PC_JACOBI) {
    k_jacobi_init<T><<<g, RB, 0, ctx->stream>>>(d.N, f.r, f.dinv, f.p, ctx->partials, ctx->counter, ctx->d_state);
    ctx->launches += 1;
  } else {
    k_bilu_apply<ilu_op(OP), T><<<(unsigned)ctx->plan.ngroups, AB, ilu_smem(ctx, sizeof(T)), ctx->stream>>>(
        d, ctx->plan, f.LU, f.r, f.z, ctx->partials, ctx->counter, ctx->d_state, 1);
    k_pupdate_z<T><<<g, RB, 0, ctx->stream>>>(d.N, f.z, f.p, ctx->d_state, 1);
    ctx->launches += 2;
  }
}

// Launch configuration of the iteration kernels of one solve.
struct LoopCfg {
  unsigned g, nblk;
  size_t smem;
  bool march, tma;
  dim3 mgrid;
  int kchunk;
};

template <int OP, typename T>
static LoopCfg loop_cfg(const rkl_ctx *ctx, int pc) {
  const Dims &d = ctx->d;
  LoopCfg L;
  L.g = stride_grid(ctx);
  L.nblk = (unsigned)ctx->plan.ngroups;
  L.smem = pc == RKL_PC_BILU0 ? ilu_smem(ctx, sizeof(T)) : 0;
  // FP32 symmetric conduction: the phi-marching y = A p when its CTAs fit the partials
  const int nbx = (d.nr + MR - 1) / MR, nby = (d.nth + MT - 1) / MT;
  const int nz = std::max(1, std::min(d.nph, (8 * ctx->nsm + nbx * nby - 1) / (nbx * nby)));
  L.kchunk = (d.nph + nz - 1) / nz;
  L.mgrid = dim3(nbx, nby, (d.nph + L.kchunk - 1) / L.kchunk);
  // FP32 symmetric conduction or viscosity with nr a multiple of 4 up to 256: planes by
  // bulk copies
  L.tma = std::is_same<T, float>::value && (OP == OPK_COND || OP == OPK_VISC) && ctx->march_nchunk[OP] > 0;
  L.march = !L.tma && std::is_same<T, float>::value && OP == OPK_COND &&
            (long long)L.mgrid.x * L.mgrid.y * L.mgrid.z <= (long long)ctx->npart;
  return L;
}

// FP32 y = A p through the bulk-copy marching kernel (loop_cfg decides when it applies)
template <int OP, typename T>
static void launch_spmv_tma(rkl_ctx *ctx, const PcgFields<T> &f, double dt) {
  if constexpr ((OP == OPK_COND || OP == OPK_VISC) && std::is_same<T, float>::value) {
    const Dims &d = ctx->d;
    k_spmv_tma<OP><<<march_grid(ctx, OP), march_threads(d.nr), march_smem(d.nr, OP), ctx->stream>>>(
        d, ctx->march_nchunk[OP], f.coef, f.W, (float)dt, f.p, f.y, ctx->partials, ctx->counter, ctx->d_state,
        ctx->d_kerr);
  }
}

// `chunk` iterations of Fig. 1 on ctx->stream; every kernel returns at once when the
// device status has left "running"
template <int OP, typename T>
static void queue_chunk(rkl_ctx *ctx, const PcgFields<T> &f, double dt, int pc, const LoopCfg &L, int chunk) {
  const Dims &d = ctx->d;
  const long long N = d.N;
  const T tdt = (T)dt;
  for (int q = 0; q < chunk; q++) {
    {
      ProfScope prof(ctx, RKL_K_SPMV, q);
      if (L.tma)
        launch_spmv_tma<OP, T>(ctx, f, dt);
      else if (L.march)
        k_spmv_march<<<L.mgrid, MTHREADS, 0, ctx->stream>>>(d, (const float *)f.coef, (const float *)f.W, (float)dt,
                                                             (const float *)f.p, (float *)f.y, ctx->partials,
                                                             ctx->counter, ctx->d_state, L.kchunk);
      else if (f.acoef)
        k_spmv_a<OP><<<L.g, RB, 0, ctx->stream>>>(d, f.acoef, (const double *)f.p, (double *)f.y, ctx->partials,
                                                  ctx->counter, ctx->d_state);
      else
        k_spmv<OP, T><<<L.g, RB, 0, ctx->stream>>>(d, f.coef, f.W, tdt, f.p, f.y, ctx->partials, ctx->counter,
                                                   ctx->d_state);
    }
    if (pc == RKL_PC_JACOBI) {
      {
        ProfScope prof(ctx, RKL_K_PCG_UPDATE, q);
        k_update_jacobi<T><<<L.g, RB, 0, ctx->stream>>>(N, f.x, f.p, f.r, f.y, f.dinv, ctx->partials,
                                                        ctx->counter, ctx->d_state);
      }
      ProfScope prof(ctx, RKL_K_PCG_PUPDATE, q);
      k_pupdate_jacobi<T><<<L.g, RB, 0, ctx->stream>>>(N, f.r, f.dinv, f.p, ctx->d_state);
    } else {
      {
        ProfScope prof(ctx, RKL_K_PCG_UPDATE, q);
        k_xr_update<T><<<L.g, RB, 0, ctx->stream>>>(N, f.x, f.p, f.r, f.y, ctx->partials, ctx->counter,
                                                    ctx->d_state);
      }
      {
        ProfScope prof(ctx, RKL_K_BILU_APPLY, q);
        k_bilu_apply<ilu_op(OP), T><<<L.nblk, AB, L.smem, ctx->stream>>>(d, ctx->plan, f.LU, f.r, f.z,
                                                                         ctx->partials, ctx->counter,
                                                                         ctx->d_state, 0);
      }
      ProfScope prof(ctx, RKL_K_PCG_PUPDATE, q);
      k_pupdate_z<T><<<L.g, RB, 0, ctx->stream>>>(N, f.z, f.p, ctx->d_state, 0);
    }
  }
}

// Condition of the graph-driven loop: run another chunk while the solve is running and
// below maxit, and never more than maxit / chunk + 2 chunks (a bound that does not rely
// on the iteration state)
__global__ void k_pcg_continue(PcgState *st, int chunk, cudaGraphConditionalHandle h) {
  if (threadIdx.x != 0) return;
  const int l = ++st->loops;
  const bool go = st->status == PCG_RUNNING && st->iters < st->maxit && l <= st->maxit / chunk + 2;
  cudaGraphSetConditional(h, go ? 1u : 0u);
}

constexpr int PCG_CHUNK = 8;

// Fig. 1's loop as one CUDA graph: a WHILE node whose body is a chunk of iterations
// followed by k_pcg_continue; launched once, so the host waits once per solve.  The
// executable graph is kept for the next solve with the same kernels and arguments.
template <int OP, typename T>
static int pcg_loop_graph(rkl_ctx *ctx, const PcgFields<T> &f, double dt, int pc, const LoopCfg &L) {
  unsigned long long key = 1469598103934665603ULL;  // FNV-1a over the arguments
  auto mix = [&](const void *p, size_t n) {
    const unsigned char *b = (const unsigned char *)p;
    for (size_t q = 0; q < n; q++) key = (key ^ b[q]) * 1099511628211ULL;
  };
  const int op = OP, tsize = (int)sizeof(T);
  const void *ptrs[] = {f.x, f.r, f.p, f.y, f.z, f.dinv, f.coef, f.W, f.LU, f.acoef, ctx->partials, ctx->counter,
                        ctx->d_state, ctx->plan_buf};
  mix(&op, sizeof op);
  mix(&tsize, sizeof tsize);
  mix(&pc, sizeof pc);
  mix(&dt, sizeof dt);
  mix(ptrs, sizeof ptrs);
  mix(&L.g, sizeof L.g);
  mix(&L.nblk, sizeof L.nblk);
  mix(&L.smem, sizeof L.smem);
  mix(&L.march, sizeof L.march);
  mix(&L.tma, sizeof L.tma);
  mix(&L.kchunk, sizeof L.kchunk);
  int rc = RKL_OK;
  if (!ctx->pcg_exec || ctx->pcg_key != key) {
    if (ctx->pcg_exec) cudaGraphExecDestroy(ctx->pcg_exec);
    if (ctx->pcg_graph) cudaGraphDestroy(ctx->pcg_graph);
    cudaGetLastError();  // teardown of the previous graph is not an error of this solve
    ctx->pcg_exec = nullptr;
    ctx->pcg_graph = nullptr;
    if (!ctx->pcg_stream &&
        (rc = cuda_check(ctx, cudaStreamCreateWithFlags(&ctx->pcg_stream, cudaStreamNonBlocking), "capture stream")))
      return rc;
    cudaGraph_t graph = nullptr;
    if ((rc = cuda_check(ctx, cudaGraphCreate(&graph, 0), "PCG graph"))) return rc;
    cudaGraphConditionalHandle h;
    cudaGraphNodeParams np = {};
    cudaGraphNode_t node;
    rc = cuda_check(ctx, cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault), "PCG graph");
    if (!rc) {
      np.type = cudaGraphNodeTypeConditional;
      np.conditional.handle = h;
      np.conditional.type = cudaGraphCondTypeWhile;
      np.conditional.size = 1;
      rc = cuda_check(ctx, cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &np), "PCG graph");
    }
    if (!rc) {
      cudaGraph_t body = np.conditional.phGraph_out[0];
      cudaStream_t user = ctx->stream;
      ctx->stream = ctx->pcg_stream;
      rc = cuda_check(ctx, cudaStreamBeginCaptureToGraph(ctx->stream, body, nullptr, nullptr, 0,
                                                         cudaStreamCaptureModeThreadLocal), "PCG graph capture");
      if (!rc) {
        queue_chunk<OP, T>(ctx, f, dt, pc, L, PCG_CHUNK);
        k_pcg_continue<<<1, 32, 0, ctx->stream>>>(ctx->d_state, PCG_CHUNK, h);
        cudaGraph_t captured = nullptr;
        rc = cuda_check(ctx, cudaStreamEndCapture(ctx->stream, &captured), "PCG graph capture");
      }
      ctx->stream = user;
    }
    if (!rc) rc = cuda_check(ctx, cudaGraphInstantiate(&ctx->pcg_exec, graph, 0), "PCG graph instantiate");
    if (rc) {
      cudaGraphDestroy(graph);
      cudaGetLastError();
      ctx->pcg_exec = nullptr;
      return rc;
    }
    ctx->pcg_graph = graph;
    ctx->pcg_key = key;
    ctx->pcg_kpc = PCG_CHUNK * (pc == RKL_PC_JACOBI ? 3 : 4) + 1;
  }
  if ((rc = cuda_check(ctx, cudaGraphLaunch(ctx->pcg_exec, ctx->stream), "PCG graph launch"))) return rc;
  if ((rc = state_read(ctx))) return rc;
  ctx->launches += (long long)ctx->h_state->loops * ctx->pcg_kpc;
  return RKL_OK;
}

// Fig. 1's loop until the device status leaves "running" (converged, breakdown, maxit):
// through the graph above, or -- while the per-kernel profiler is on or the caller's stream
// is being captured -- queued by the host in chunks with a status read after each chunk
template <int OP, typename T>
static int pcg_loop(rkl_ctx *ctx, const PcgFields<T> &f, double dt, int pc, int maxit) {
  const LoopCfg L = loop_cfg<OP, T>(ctx, pc);
  int it_prev = 0, rc;
  if ((rc = state_read(ctx))) return rc;
  if (ctx->h_state->status != PCG_RUNNING || ctx->h_state->iters >= maxit) return RKL_OK;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if ((rc = cuda_check(ctx, cudaStreamIsCapturing(ctx->stream, &cap), "stream capture query"))) return rc;
  if (!ctx->prof_on && cap == cudaStreamCaptureStatusNone) return pcg_loop_graph<OP, T>(ctx, f, dt, pc, L);
  // host-side bound: the device counts iterations and stops at maxit; should its status
  // ever stop advancing, the host stops queueing after maxit + 2 chunks
  long long queued = 0;
  for (bool first = true;; first = false) {
    if (!first && (rc = state_read(ctx))) return rc;
    const PcgState &h = *ctx->h_state;
    if (ctx->prof_on) prof_settle(ctx, h.iters - it_prev, h.status == PCG_RUNNING, true);
    it_prev = h.iters;
    if (h.status != PCG_RUNNING || h.iters >= maxit) break;
    if (queued > (long long)maxit + 2 * PCG_CHUNK)
      return set_error(ctx, RKL_ECUDA, "PCG: device iteration count is not advancing");
    queued += PCG_CHUNK;
    queue_chunk<OP, T>(ctx, f, dt, pc, L, PCG_CHUNK);
    ctx->launches += (long long)PCG_CHUNK * (pc == RKL_PC_JACOBI ? 3 : 4);
    if ((rc = cuda_check(ctx, cudaGetLastError(), "PCG iteration launch"))) return rc;
  }
  return RKL_OK;
}

template <int OP>
static int pcg_run(rkl_ctx *ctx, double *x, const double *u, const double *x0, double dt, int pc,
                   double rtol, int maxit, int *iters, double *relres, int *status) {
  const Dims &d = ctx->d;
  const long long N = d.N;
  int rc;
  if ((rc = ensure_buffer(ctx, &ctx->r, N, "PCG r")) || (rc = ensure_buffer(ctx, &ctx->p, N, "PCG p")) ||
      (rc = ensure_buffer(ctx, &ctx->y, N, "PCG y")) || (rc = ensure_buffer(ctx, &ctx->zbuf, N, "PCG z")) ||
      (rc = ensure_buffer(ctx, &ctx->dinv, N, "PCG diag")))
    return rc;
  if ((rc = state_upload(ctx, rtol, maxit))) return rc;
  const unsigned g = stride_grid(ctx);
  if (op_ncoef(OP) > ctx->acoef_slots) {
    cudaStreamSynchronize(ctx->stream);
    cudaFree(ctx->acoef);
    ctx->acoef = nullptr;
    ctx->acoef_slots = 0;
    if ((rc = cuda_check(ctx, cudaMalloc(&ctx->acoef, (op_ncoef(OP) * N + pole_extra(d)) * sizeof(double)),
                         "alloc A")))
      return rc;
    ctx->acoef_slots = op_ncoef(OP);
  }
  if (!ctx->acoef_valid || ctx->acoef_dt != dt) {
    ProfScope prof(ctx, RKL_K_PCG_INIT);
    k_assemble_A<OP><<<g, RB, 0, ctx->stream>>>(d, ctx->coef, ctx->W, dt, ctx->acoef);
    ctx->launches += 1;
    if ((rc = cuda_check(ctx, cudaGetLastError(), "A assembly launch"))) return rc;
    ctx->acoef_valid = 1;
    ctx->acoef_dt = dt;
  }
  PcgFields<double> f{x, ctx->r, ctx->p, ctx->y, ctx->zbuf, ctx->dinv, ctx->coef, ctx->W, ctx->LU, ctx->acoef};
  {
    ProfScope prof(ctx, RKL_K_PCG_INIT);
    k_r0<OP><<<g, RB, 0, ctx->stream>>>(d, ctx->coef, ctx->W, dt, u, x0 ? x0 : u, ctx->r,
                                        pc == RKL_PC_JACOBI ? ctx->dinv : nullptr, ctx->partials,
                                        ctx->counter, ctx->d_state);
    ctx->launches += 1;
    if (x0 && x0 != x &&
        (rc = cuda_check(ctx, cudaMemcpyAsync(x, x0, sizeof(double) * N, cudaMemcpyDeviceToDevice, ctx->stream),
                         "x0 copy")))
      return rc;
    pcg_first<OP, double>(ctx, f, pc);
  }
  if ((rc = cuda_check(ctx, cudaGetLastError(), "PCG init launch"))) return rc;
  if ((rc = pcg_loop<OP, double>(ctx, f, dt, pc, maxit))) return rc;
  const PcgState &h = *ctx->h_state;
  *iters = h.iters;
  *relres = h.bnorm2 > 0.0 ? std::sqrt(h.rnorm2 / h.bnorm2) : 0.0;
  int st = h.status;
  if (st == PCG_RUNNING) st = PCG_MAXIT;  // maxit == 0 without convergence
  *status = st;
  return RKL_OK;
}

// Mixed precision: FP64 iterative refinement around FP32 PCG.  Each outer step computes
// the FP64 residual r = W u - (W + dt S) x and its norm, stops when ||r|| <= rtol ||W u||,
// otherwise solves (W + dt S) e = r / sigma in FP32 (sigma = RMS of r) to the relative
// tolerance max(inner_rtol, 0.3 rtol ||b|| / ||r||) and updates x += sigma e in FP64.
// iters counts FP32 iterations.
template <int OP>
static int pcg_run_mixed(rkl_ctx *ctx, double *x, const double *u, const double *x0, double dt,
                         int pc, double rtol, int maxit, int *iters, double *relres, int *status) {
  const Dims &d = ctx->d;
  const long long N = d.N;
  int rc;
  if ((rc = ensure_buffer(ctx, &ctx->r, N, "PCG r")) || (rc = ensure_buffer(ctx, &ctx->dinv, N, "PCG diag")) ||
      (rc = ensure_buffer(ctx, &ctx->p, N, "copy of u^n")) ||
      (rc = ensure_fbuffer(ctx, &ctx->r32, N, "PCG r32")) || (rc = ensure_fbuffer(ctx, &ctx->p32, N, "PCG p32")) ||
      (rc = ensure_fbuffer(ctx, &ctx->y32, N, "PCG y32")) || (rc = ensure_fbuffer(ctx, &ctx->z32, N, "PCG z32")) ||
      (rc = ensure_fbuffer(ctx, &ctx->e32, N, "PCG e32")) || (rc = ensure_fbuffer(ctx, &ctx->dinv32, N, "PCG d32")))
    return rc;
  const unsigned g = stride_grid(ctx);
  PcgFields<float> f{ctx->e32, ctx->r32, ctx->p32, ctx->y32, ctx->z32, ctx->dinv32, ctx->coef32, ctx->W32, ctx->LU32,
                     nullptr};
  // x may share its buffer with u: keep u^n for the right-hand side W u^n of every
  // outer residual (the FP64 buffer p is not used by the mixed solve)
  double *un = ctx->p;
  if ((rc = cuda_check(ctx, cudaMemcpyAsync(un, u, sizeof(double) * N, cudaMemcpyDeviceToDevice, ctx->stream),
                       "copy of u^n")))
    return rc;
  int total = 0, st = PCG_MAXIT;
  double bn2 = 0.0, rn2 = 0.0;
  for (int outer = 0; outer < 64; outer++) {
    {
      ProfScope prof(ctx, RKL_K_PCG_INIT);
      const double *xs = outer == 0 ? (x0 ? x0 : un) : x;
      k_r0<OP><<<g, RB, 0, ctx->stream>>>(d, ctx->coef, ctx->W, dt, un, xs, ctx->r,
                                          outer == 0 && pc == RKL_PC_JACOBI ? ctx->dinv : nullptr,
                                          ctx->partials, ctx->counter, ctx->d_state);
      ctx->launches += 1;
      if (outer == 0 && pc == RKL_PC_JACOBI && (rc = launch_to_float(ctx, ctx->dinv, ctx->dinv32, N))) return rc;
      if (outer == 0 && x0 && x0 != x &&
          (rc = cuda_check(ctx, cudaMemcpyAsync(x, x0, sizeof(double) * N, cudaMemcpyDeviceToDevice, ctx->stream),
                           "x0 copy")))
        return rc;
    }
    if ((rc = state_read(ctx))) return rc;
    bn2 = ctx->h_state->bnorm2;
    rn2 = ctx->h_state->rnorm2;
    if (!std::isfinite(rn2) || !std::isfinite(bn2)) {
      st = PCG_BREAKDOWN;
      break;
    }
    if (rtol > 0.0 && rn2 <= rtol * rtol * bn2) {
      st = PCG_CONVERGED;
      break;
    }
    if (rn2 == 0.0) {
      st = PCG_CONVERGED;
      break;
    }
    if (total >= maxit) break;
    const double sigma = std::sqrt(rn2 / (double)N);
    // the correction only has to bring ||r|| down to the target: relative tolerance
    // max(inner_rtol, 0.3 rtol ||b|| / ||r||), at most 0.5
    double eta = ctx->inner_rtol;
    if (rtol > 0.0) eta = std::min(0.5, std::max(eta, 0.3 * rtol * std::sqrt(bn2 / rn2)));
    if ((rc = state_upload(ctx, eta, maxit - total))) return rc;
    {
      ProfScope prof(ctx, RKL_K_PCG_INIT);
      k_scale_to_f32<<<g, RB, 0, ctx->stream>>>(N, ctx->r, 1.0 / sigma, ctx->r32, ctx->e32, ctx->partials,
                                                ctx->counter, ctx->d_state);
      ctx->launches += 1;
      pcg_first<OP, float>(ctx, f, pc);
    }
    if ((rc = cuda_check(ctx, cudaGetLastError(), "mixed PCG init launch"))) return rc;
    if ((rc = pcg_loop<OP, float>(ctx, f, dt, pc, maxit - total))) return rc;
    const PcgState &h = *ctx->h_state;
    total += h.iters;
    if (h.status == PCG_BREAKDOWN) {
      st = PCG_BREAKDOWN;
      break;
    }
    k_correct<<<g, RB, 0, ctx->stream>>>(N, x, sigma, ctx->e32);
    ctx->launches += 1;
    if ((rc = cuda_check(ctx, cudaGetLastError(), "mixed PCG correction launch"))) return rc;
  }
  *iters = total;
  *relres = bn2 > 0.0 ? std::sqrt(rn2 / bn2) : 0.0;
  *status = st;
  return RKL_OK;
}

int pcg_solve_component(rkl_ctx *ctx, double *x, const double *u, const double *x0, double dt,
                        int pc, double rtol, int maxit, int *iters, double *relres, int *status) {
  if (ctx->prec == RKL_F32MIX) {
    int rc = RKL_OK;
    op_dispatch(ctx->op, [&](auto kind) {
      rc = pcg_run_mixed<decltype(kind)::value>(ctx, x, u, x0, dt, pc, rtol, maxit, iters, relres, status);
    });
    return rc;
  }
  int rc = RKL_OK;
  op_dispatch(ctx->op, [&](auto kind) {
    rc = pcg_run<decltype(kind)::value>(ctx, x, u, x0, dt, pc, rtol, maxit, iters, relres, status);
  });
  return rc;
}

}  // namespace rkl
