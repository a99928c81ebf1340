// stencil.cuh -- (S u)_c for the stored symmetric operators (see internal.cuh).
//
// Row c of S is  S_cc u_c + sum_m F_m(c) u_{c+FWD[m]} + sum_m F_m(c-FWD[m]) u_{c-FWD[m]}
// where F_m is the forward entry stored at slot m.  A neighbour outside the r or
// theta range does not exist: its forward entry is stored as zero and its index is
// clamped onto the cell itself (a valid address); the backward entry of a missing
// neighbour is masked to zero (the clamped address holds an unrelated entry).
// phi wraps.  The FP64 cost is one DMUL + 18 DFMA (19-point) or 6 DFMA (7-point).
#pragma once
#include "internal.cuh"

namespace rkl {

struct Nbr {
  long long rp, rm, tp, tm, pp, pm;  // index deltas (clamped to 0 at r/theta edges)
  bool vrp, vrm, vtp, vtm;            // does the neighbour exist
};

__device__ __forceinline__ void cell_coords(const Dims &d, long long c, int &i, int &j, int &k) {
  long long q = c / d.nr;
  i = (int)(c - q * d.nr);
  long long kk = q / d.nth;
  k = (int)kk;
  j = (int)(q - kk * d.nth);
}

__device__ __forceinline__ Nbr neighbours(const Dims &d, int i, int j, int k) {
  Nbr n;
  n.vrp = i < d.nr - 1;
  n.vrm = i > 0;
  n.vtp = j < d.nth - 1;
  n.vtm = j > 0;
  n.rp = n.vrp ? 1 : 0;
  n.rm = n.vrm ? -1 : 0;
  n.tp = n.vtp ? (long long)d.nr : 0;
  n.tm = n.vtm ? -(long long)d.nr : 0;
  n.pp = (k < d.nph - 1) ? d.nrt : -(long long)(d.nph - 1) * d.nrt;
  n.pm = (k > 0) ? -d.nrt : (long long)(d.nph - 1) * d.nrt;
  return n;
}

// 19-point conduction operator, coef = [10][N] (9 forward + diagonal); T = double, or
// float for the mixed-precision path (FP32 coefficients and fields, FP32 accumulation)
template <typename T>
__device__ __forceinline__ T S_apply_cond(const Dims &d, const T *__restrict__ coef,
                                          const T *__restrict__ u, long long c, const Nbr &n) {
  const long long N = d.N;
  const long long f[9] = {c + n.rp,        c + n.tp,        c + n.pp,
                          c + n.rm + n.tp, c + n.rp + n.tp, c + n.rm + n.pp,
                          c + n.rp + n.pp, c + n.tm + n.pp, c + n.tp + n.pp};
  const long long b[9] = {c + n.rm,        c + n.tm,        c + n.pm,
                          c + n.rp + n.tm, c + n.rm + n.tm, c + n.rp + n.pm,
                          c + n.rm + n.pm, c + n.tp + n.pm, c + n.tm + n.pm};
  const bool bv[9] = {n.vrm, n.vtm, true, n.vrp && n.vtm, n.vrm && n.vtm,
                      n.vrp, n.vrm, n.vtp, n.vtm};
  T acc = coef[9 * N + c] * u[c];
#pragma unroll
  for (int m = 0; m < 9; m++) acc = fma(coef[m * N + c], u[f[m]], acc);
#pragma unroll
  for (int m = 0; m < 9; m++) {
    T cb = bv[m] ? coef[m * N + b[m]] : T(0);
    acc = fma(cb, u[b[m]], acc);
  }
  return acc;
}

// 7-point viscosity operator, coef = [4][N] (3 forward + diagonal)
template <typename T>
__device__ __forceinline__ T S_apply_visc(const Dims &d, const T *__restrict__ coef,
                                          const T *__restrict__ u, long long c, const Nbr &n) {
  const long long N = d.N;
  T acc = coef[3 * N + c] * u[c];
  acc = fma(coef[0 * N + c], u[c + n.rp], acc);
  acc = fma(coef[1 * N + c], u[c + n.tp], acc);
  acc = fma(coef[2 * N + c], u[c + n.pp], acc);
  acc = fma(n.vrm ? coef[0 * N + c + n.rm] : T(0), u[c + n.rm], acc);
  acc = fma(n.vtm ? coef[1 * N + c + n.tm] : T(0), u[c + n.tm], acc);
  acc = fma(coef[2 * N + c + n.pm], u[c + n.pm], acc);
  return acc;
}

// 19-point operator stored as full rows, coef = [19][N]: slot m < 9 the entry towards
// c + FWD[m], slot 9 the diagonal, slot 10 + m the entry towards c - FWD[m] (zero for a
// missing neighbour, whose index is clamped onto a valid cell).  Used for the
// non-symmetric flux form of conduction.
template <typename T>
__device__ __forceinline__ T S_apply_full(const Dims &d, const T *__restrict__ coef,
                                          const T *__restrict__ u, long long c, const Nbr &n) {
  const long long N = d.N;
  const long long f[9] = {c + n.rp,        c + n.tp,        c + n.pp,
                          c + n.rm + n.tp, c + n.rp + n.tp, c + n.rm + n.pp,
                          c + n.rp + n.pp, c + n.tm + n.pp, c + n.tp + n.pp};
  const long long b[9] = {c + n.rm,        c + n.tm,        c + n.pm,
                          c + n.rp + n.tm, c + n.rm + n.tm, c + n.rp + n.pm,
                          c + n.rm + n.pm, c + n.tp + n.pm, c + n.tm + n.pm};
  T acc = coef[9 * N + c] * u[c];
#pragma unroll
  for (int m = 0; m < 9; m++) acc = fma(coef[m * N + c], u[f[m]], acc);
#pragma unroll
  for (int m = 0; m < 9; m++) acc = fma(coef[(10 + m) * N + c], u[b[m]], acc);
  return acc;
}

// Symmetric 19-point conduction with across-pole theta-ghosts: the stored symmetric part
// plus, in the two pole rows (nth >= 2), the five couplings to the antipodal column kept
// at coef + 10 N (internal.cuh).  Other rows are exactly S_apply_cond.
template <typename T>
__device__ __forceinline__ T S_apply_pole(const Dims &d, const T *__restrict__ coef,
                                          const T *__restrict__ u, long long c, const Nbr &n) {
  T acc = S_apply_cond<T>(d, coef, u, c, n);
  if (n.vtm && n.vtp) return acc;
  const long long q = c / d.nr;
  const int i = (int)(c - q * d.nr), k = (int)(q / d.nth);
  const int side = n.vtm ? 1 : 0;  // j = 0 has no theta-minus neighbour
  const T *P = coef + 10 * d.N;
  const long long stride = 2LL * d.nph * d.nr, e = ((long long)side * d.nph + k) * d.nr + i;
  const int h = d.nph / 2;
  const int kb = k + h < d.nph ? k + h : k + h - d.nph;
  const long long cb = c + (long long)(kb - k) * d.nrt;  // the antipodal cell (same i, j)
  acc = fma(P[e], u[cb], acc);
  if (i < d.nr - 1) acc = fma(P[stride + e], u[cb + 1], acc);
  if (i > 0) acc = fma(P[2 * stride + e], u[cb - 1], acc);
  acc = fma(P[3 * stride + e], u[cb + (kb < d.nph - 1 ? d.nrt : -(long long)(d.nph - 1) * d.nrt)], acc);
  acc = fma(P[4 * stride + e], u[cb + (kb > 0 ? -d.nrt : (long long)(d.nph - 1) * d.nrt)], acc);
  return acc;
}

template <int OP, typename T>
__device__ __forceinline__ T S_apply(const Dims &d, const T *__restrict__ coef,
                                     const T *__restrict__ u, long long c, const Nbr &n) {
  if (OP == RKL_OP_CONDUCTION) return S_apply_cond<T>(d, coef, u, c, n);
  if (OP == OPK_FLUX) return S_apply_full<T>(d, coef, u, c, n);
  if (OP == OPK_POLE) return S_apply_pole<T>(d, coef, u, c, n);
  return S_apply_visc<T>(d, coef, u, c, n);
}

template <int OP, typename T>
__device__ __forceinline__ T S_diag(const Dims &d, const T *__restrict__ coef, long long c) {
  return coef[(OP == RKL_OP_VISCOSITY ? 3 : 9) * d.N + c];
}

}  // namespace rkl
