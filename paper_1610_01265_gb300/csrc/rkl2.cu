// rkl2.cu -- operator apply and the fused stencil + RKL2 stage kernels (Fig. 2).
//
// Each stage j >= 2 is one pass over the grid: the stencil of Y_{j-1} and the
// pointwise recurrence
//   Y_j = mu_j Y_{j-1} + nu_j Y_{j-2} + (1 - mu_j - nu_j) Y_0
//         + mu~_j dt M Y_{j-1} + gamma~_j dt M Y_0,      M Y = -W^{-1} S Y,
// so the stage streams Y_{j-1} (stencil, reused through L1/L2), Y_{j-2}, Y_0, M_0,
// the 10 stored coefficients and 1/W, and writes Y_j in place of Y_{j-2}.
// FP64 work per cell: 19 (stencil) + 6 (recurrence) DP instructions.
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.cuh"
#include "stencil.cuh"
#include "march.cuh"

namespace rkl {

namespace {

constexpr int BLK = 256;

template <int OP>
__global__ void __launch_bounds__(BLK) k_apply_F(Dims d, const double *__restrict__ coef,
                                                 const double *__restrict__ invW,
                                                 const double *__restrict__ u,
                                                 double *__restrict__ Fu) {
  long long c = (long long)blockIdx.x * BLK + threadIdx.x;
  if (c >= d.N) return;
  int i, j, k;
  cell_coords(d, c, i, j, k);
  Nbr n = neighbours(d, i, j, k);
  Fu[c] = -invW[c] * S_apply<OP>(d, coef, u, c, n);
}

template <int OP>
__global__ void __launch_bounds__(BLK) k_rkl2_first(Dims d, const double *__restrict__ coef,
                                                const double *__restrict__ invW,
                                                const double *__restrict__ Y0,
                                                double *__restrict__ M0, double *__restrict__ Y1,
                                                double mut1dt) {
  long long c = (long long)blockIdx.x * BLK + threadIdx.x;
  if (c >= d.N) return;
  int i, j, k;
  cell_coords(d, c, i, j, k);
  Nbr n = neighbours(d, i, j, k);
  double m0 = -invW[c] * S_apply<OP>(d, coef, Y0, c, n);
  M0[c] = m0;
  Y1[c] = fma(mut1dt, m0, Y0[c]);
}

// Yout may alias Ym2 or Y0 (read and written at the same cell only); never Ym1.
template <int OP>
__global__ void __launch_bounds__(BLK) k_rkl2_stage(Dims d, const double *__restrict__ coef,
                                               const double *__restrict__ invW,
                                               const double *__restrict__ Ym1,
                                               const double *Ym2, const double *Y0,
                                               const double *__restrict__ M0, double *Yout,
                                               double mu, double nu, double om, double mutdt,
                                               double gtdt) {
  long long c = (long long)blockIdx.x * BLK + threadIdx.x;
  if (c >= d.N) return;
  int i, j, k;
  cell_coords(d, c, i, j, k);
  Nbr n = neighbours(d, i, j, k);
  double f = -invW[c] * S_apply<OP>(d, coef, Ym1, c, n);
  double y = mu * Ym1[c];
  y = fma(nu, Ym2[c], y);
  y = fma(om, Y0[c], y);
  y = fma(mutdt, f, y);
  y = fma(gtdt, M0[c], y);
  Yout[c] = y;
}

// ---- mixed precision (FP32 stages on increments, FP64 kept where it matters) ----
//
// With Y_j = Y_0 + delta_j the recurrence of Fig. 2 becomes
//   delta_j = mu_j delta_{j-1} + nu_j delta_{j-2} + mu~_j dt M delta_{j-1}
//             + (mu~_j + gamma~_j) dt M_0,       delta_0 = 0, delta_1 = mu~_1 dt M_0,
// because M Y_{j-1} = M_0 + M delta_{j-1}.  M_0 = M Y_0 is computed in FP64 (the large
// values of Y_0 cancel in the stencil); the increments, the stencil on them and the
// recurrence run in FP32; the last stage writes u = Y_0 + delta_s in FP64.

template <int OP>
__global__ void __launch_bounds__(BLK) k_rkl2_first_mix(Dims d, const double *__restrict__ coef,
                                                        const double *__restrict__ invW,
                                                        const double *__restrict__ Y0,
                                                        float *__restrict__ M0f,
                                                        float *__restrict__ d1, double mut1dt) {
  long long c = (long long)blockIdx.x * BLK + threadIdx.x;
  if (c >= d.N) return;
  int i, j, k;
  cell_coords(d, c, i, j, k);
  Nbr n = neighbours(d, i, j, k);
  const double m0 = -invW[c] * S_apply<OP>(d, coef, Y0, c, n);
  M0f[c] = (float)m0;
  d1[c] = (float)(mut1dt * m0);
}

// dm2 == nullptr stands for delta_0 = 0; u != nullptr marks the last stage (u += delta_s)
template <int OP>
__global__ void __launch_bounds__(BLK) k_rkl2_stage_mix(Dims d, const float *__restrict__ coef,
                                                        const float *__restrict__ invW,
                                                        const float *__restrict__ dm1,
                                                        const float *dm2,
                                                        const float *__restrict__ M0f,
                                                        float *dout, double *u, float mu, float nu,
                                                        float mutdt, float cm0) {
  // 3-D launch: i and j from a 2-D block, k from the grid (no index division)
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y, k = blockIdx.z;
  if (i >= d.nr || j >= d.nth) return;
  const long long c = ((long long)k * d.nth + j) * d.nr + i;
  Nbr n = neighbours(d, i, j, k);
  const float f = -invW[c] * S_apply<OP, float>(d, coef, dm1, c, n);
  float y = mu * dm1[c];
  if (dm2) y = fmaf(nu, dm2[c], y);
  y = fmaf(mutdt, f, y);
  y = fmaf(cm0, M0f[c], y);
  if (u) u[c] += (double)y;
  else dout[c] = y;
}

// The same stage for symmetric conduction and viscosity, marching along phi with the
// planes of delta_{j-1} and of the coefficients brought in by bulk copies (march.cuh);
// per cell the arithmetic of k_rkl2_stage_mix<OP>.  Yout may alias dm2 (each cell is read
// by its own thread, a plane ahead of its write).  LAST (u += delta_s in FP64) is a
// separate instantiation, so that the other stages issue no FP64 instruction at all.
template <bool LAST>
struct StageEpi {
  const float *__restrict__ invW;
  const float *dm2;
  const float *__restrict__ M0f;
  float *dout;
  double *u;
  float mu, nu, mutdt, cm0;
  float4 w, m, z, wn, mn, zn;
  __device__ __forceinline__ void load(long long c) {
    wn = *reinterpret_cast<const float4 *>(invW + c);
    mn = *reinterpret_cast<const float4 *>(M0f + c);
    zn = dm2 ? *reinterpret_cast<const float4 *>(dm2 + c) : make_float4(0.f, 0.f, 0.f, 0.f);
  }
  __device__ __forceinline__ void advance() {
    w = wn;
    m = mn;
    z = zn;
  }
  __device__ __forceinline__ void store(long long c, const float (&s)[4], const float (&uc)[4]) {
    const float wv[4] = {w.x, w.y, w.z, w.w}, mv[4] = {m.x, m.y, m.z, m.w}, zv[4] = {z.x, z.y, z.z, z.w};
    float y[4];
#pragma unroll
    for (int e = 0; e < 4; e++) {
      const float f = -wv[e] * s[e];
      float t = mu * uc[e];
      if (dm2) t = fmaf(nu, zv[e], t);
      t = fmaf(mutdt, f, t);
      y[e] = fmaf(cm0, mv[e], t);
    }
    if constexpr (LAST) {
#pragma unroll
      for (int e = 0; e < 4; e++) u[c + e] += (double)y[e];
    } else {
      *reinterpret_cast<float4 *>(dout + c) = make_float4(y[0], y[1], y[2], y[3]);
    }
  }
  __device__ __forceinline__ void poison(long long c) {
    const float q = __int_as_float(0x7fc00000);
    if constexpr (LAST) {
#pragma unroll
      for (int e = 0; e < 4; e++) u[c + e] = (double)q;
    } else {
      *reinterpret_cast<float4 *>(dout + c) = make_float4(q, q, q, q);
    }
  }
};

template <int OP, bool LAST>
__global__ void __launch_bounds__(MARCH_MAX_THREADS, 1) k_rkl2_stage_mix_tma(Dims d, int nchunk,
                                                                        const float *__restrict__ coef,
                                                                        const float *__restrict__ invW,
                                                                        const float *__restrict__ dm1,
                                                                        const float *dm2,
                                                                        const float *__restrict__ M0f,
                                                                        float *dout, double *u, float mu,
                                                                        float nu, float mutdt, float cm0,
                                                                        int *kerr) {
  StageEpi<LAST> e{invW, dm2, M0f, dout, u, mu, nu, mutdt, cm0};
  march32<OP>(d, nchunk, coef, dm1, e, kerr);
}

__global__ void __launch_bounds__(BLK) k_to_float(long long n, const double *__restrict__ a,
                                                  float *__restrict__ b) {
  for (long long c = (long long)blockIdx.x * BLK + threadIdx.x; c < n; c += (long long)gridDim.x * BLK)
    b[c] = (float)a[c];
}

}  // namespace

int march_setup_stage(rkl_ctx *ctx) {
  int optin = 0;
  int rc = cuda_check(ctx, cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device),
                      "shared memory opt-in");
  if (rc) return rc;
  for (int op = OPK_COND; op <= OPK_VISC; op++)
    if ((size_t)optin < march_smem(ctx->d.nr, op) + 1024) ctx->march_nchunk[op] = 0;
  const void *kerns[] = {(const void *)k_rkl2_stage_mix_tma<OPK_COND, false>,
                         (const void *)k_rkl2_stage_mix_tma<OPK_COND, true>,
                         (const void *)k_rkl2_stage_mix_tma<OPK_VISC, false>,
                         (const void *)k_rkl2_stage_mix_tma<OPK_VISC, true>};
  for (const void *k : kerns)
    if ((rc = cuda_check(ctx, cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - 1024),
                         "bulk-copy stage shared memory")))
      return rc;
  return RKL_OK;
}

int launch_to_float(rkl_ctx *ctx, const double *a, float *b, long long n) {
  long long g = std::min<long long>((n + BLK - 1) / BLK, (long long)ctx->nsm * 16);
  k_to_float<<<(unsigned)std::max(1LL, g), BLK, 0, ctx->stream>>>(n, a, b);
  ctx->launches += 1;
  return cuda_check(ctx, cudaGetLastError(), "FP32 conversion launch");
}

int launch_rkl2_first_mix(rkl_ctx *ctx, const double *Y0, float *M0f, float *d1, double mut1dt) {
  ProfScope prof(ctx, RKL_K_RKL2_FIRST);
  unsigned grid = grid_for(ctx->d.N, BLK);
  op_dispatch(ctx->op, [&](auto kind) {
    constexpr int OP = decltype(kind)::value;
      k_rkl2_first_mix<OP><<<grid, BLK, 0, ctx->stream>>>(ctx->d, ctx->coef, ctx->invW, Y0, M0f, d1, mut1dt);
  });
  ctx->launches += 1;
  return cuda_check(ctx, cudaGetLastError(), "mixed rkl2 stage-1 launch");
}

int launch_rkl2_stage_mix(rkl_ctx *ctx, const float *dm1, const float *dm2, const float *M0f,
                          float *dout, double *u, double mu, double nu, double mutdt, double cm0) {
  ProfScope prof(ctx, RKL_K_RKL2_STAGE);
  if ((ctx->op == OPK_COND || ctx->op == OPK_VISC) && ctx->march_nchunk[ctx->op] > 0) {
    const int TH = march_th(ctx->d.nr), nchunk = ctx->march_nchunk[ctx->op];
    const unsigned grid = (unsigned)(((ctx->d.nth + TH - 1) / TH) * nchunk);
    const dim3 block(march_threads(ctx->d.nr));
    const size_t smem = march_smem(ctx->d.nr, ctx->op);
    auto go = [&](auto kern) {
      kern<<<grid, block, smem, ctx->stream>>>(ctx->d, nchunk, ctx->coef32, ctx->invW32, dm1, dm2, M0f, dout, u,
                                                (float)mu, (float)nu, (float)mutdt, (float)cm0, ctx->d_kerr);
    };
    if (ctx->op == OPK_COND)
      u ? go(k_rkl2_stage_mix_tma<OPK_COND, true>) : go(k_rkl2_stage_mix_tma<OPK_COND, false>);
    else
      u ? go(k_rkl2_stage_mix_tma<OPK_VISC, true>) : go(k_rkl2_stage_mix_tma<OPK_VISC, false>);
    ctx->launches += 1;
    return cuda_check(ctx, cudaGetLastError(), "mixed rkl2 stage launch");
  }
  // a block of 256 threads: the whole (padded) r line when it is short, several theta rows
  const unsigned bx = (unsigned)std::min(256, ((ctx->d.nr + 31) / 32) * 32), by = 256 / bx;
  const dim3 block(bx, by), grid(grid_for(ctx->d.nr, bx), grid_for(ctx->d.nth, by), (unsigned)ctx->d.nph);
  op_dispatch(ctx->op, [&](auto kind) {
    constexpr int OP = decltype(kind)::value;
      k_rkl2_stage_mix<OP><<<grid, block, 0, ctx->stream>>>(
          ctx->d, ctx->coef32, ctx->invW32, dm1, dm2, M0f, dout, u, (float)mu, (float)nu, (float)mutdt, (float)cm0);
  });
  ctx->launches += 1;
  return cuda_check(ctx, cudaGetLastError(), "mixed rkl2 stage launch");
}

int launch_apply_F(rkl_ctx *ctx, const double *u, double *Fu) {
  ProfScope prof(ctx, RKL_K_APPLY_F);
  unsigned grid = grid_for(ctx->d.N, BLK);
  op_dispatch(ctx->op, [&](auto kind) {
    constexpr int OP = decltype(kind)::value;
      k_apply_F<OP><<<grid, BLK, 0, ctx->stream>>>(ctx->d, ctx->coef, ctx->invW, u, Fu);
  });
  ctx->launches += 1;
  return cuda_check(ctx, cudaGetLastError(), "apply_F launch");
}

int launch_rkl2_stage1(rkl_ctx *ctx, const double *Y0, double *M0, double *Y1, double mut1dt) {
  ProfScope prof(ctx, RKL_K_RKL2_FIRST);
  unsigned grid = grid_for(ctx->d.N, BLK);
  op_dispatch(ctx->op, [&](auto kind) {
    constexpr int OP = decltype(kind)::value;
      k_rkl2_first<OP><<<grid, BLK, 0, ctx->stream>>>(ctx->d, ctx->coef, ctx->invW, Y0, M0,
                                                                Y1, mut1dt);
  });
  ctx->launches += 1;
  return cuda_check(ctx, cudaGetLastError(), "rkl2 stage-1 launch");
}

int launch_rkl2_stage(rkl_ctx *ctx, const double *Ym1, const double *Ym2, const double *Y0,
                      const double *M0, double *Yout, double mu, double nu, double mutdt,
                      double gtdt) {
  ProfScope prof(ctx, RKL_K_RKL2_STAGE);
  unsigned grid = grid_for(ctx->d.N, BLK);
  double om = 1.0 - mu - nu;
  op_dispatch(ctx->op, [&](auto kind) {
    constexpr int OP = decltype(kind)::value;
      k_rkl2_stage<OP><<<grid, BLK, 0, ctx->stream>>>(ctx->d, ctx->coef, ctx->invW, Ym1,
                                                               Ym2, Y0, M0, Yout, mu, nu, om, mutdt,
                                                               gtdt);
  });
  ctx->launches += 1;
  return cuda_check(ctx, cudaGetLastError(), "rkl2 stage launch");
}

int launch_rkl2_first_raw(const Dims &d, cudaStream_t stream, const double *coef,
                          const double *invW, const double *Y0, double *M0, double *Y1,
                          double mut1dt) {
  k_rkl2_first<RKL_OP_CONDUCTION><<<grid_for(d.N, BLK), BLK, 0, stream>>>(d, coef, invW, Y0, M0, Y1, mut1dt);
  return cudaGetLastError() == cudaSuccess ? RKL_OK : RKL_ECUDA;
}

int launch_rkl2_stage_raw(const Dims &d, cudaStream_t stream, const double *coef,
                          const double *invW, const double *Ym1, const double *Ym2,
                          const double *Y0, const double *M0, double *Yout, double mu, double nu,
                          double mutdt, double gtdt) {
  k_rkl2_stage<RKL_OP_CONDUCTION><<<grid_for(d.N, BLK), BLK, 0, stream>>>(
      d, coef, invW, Ym1, Ym2, Y0, M0, Yout, mu, nu, 1.0 - mu - nu, mutdt, gtdt);
  return cudaGetLastError() == cudaSuccess ? RKL_OK : RKL_ECUDA;
}

}  // namespace rkl
