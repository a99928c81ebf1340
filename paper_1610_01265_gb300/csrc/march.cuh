// march.cuh -- FP32 stencils (19-point conduction, 7-point viscosity) marching along phi,
// with every plane brought into shared memory by bulk asynchronous copies (the TMA
// engine, cp.async.bulk) that signal mbarriers.
//
// A CTA owns a tile of TH theta rows (all nr cells of each row, four consecutive r cells
// per thread; march_th below) and a chunk [k0, k1) of phi planes.  For each plane it
// holds in shared memory
//   u     rows j0-1 .. j0+TH: the tile and its theta halo          ring of MU = 5 planes
//   coef  the slots of the tile's own rows (10 conduction, 4 viscosity), plus halo rows:
//         conduction slots 1, 3, 4, 8 of row j0-1 and slot 7 of row j0+th,
//         viscosity slot 1 of row j0-1                               ring of MC = 4 planes
// which is all that the stencil of plane k reads: u of planes k-1, k, k+1, the
// coefficients of plane k, and the backward entries held by plane k-1 (conduction slots
// 2, 5, 6, 7, 8; viscosity slot 2).  Each plane of every stream is copied once per tile,
// so the only traffic above the algorithmic bytes is the theta halo, which the
// neighbouring tile reads from L2.
// While plane k is computed, the copies of u up to plane k+3 and of the coefficients
// up to plane k+2 are in flight.  One elected thread issues them, in batches that each
// complete one of three mbarriers:
//   prologue    u(k0-1), u(k0), u(k0+1), coef(k0-1), coef(k0)   barrier 0, waited at k0
//               u(k0+2), coef(k0+1)                             barrier 1, waited at k0+1
//               u(k0+3), coef(k0+2)                             barrier 2, waited at k0+2
//   after k     u(k+4), coef(k+3)                  barrier (k-k0)%3, waited at k+3
// A batch refills the ring slots that plane k-1 vacated, after the barrier that ends
// plane k.  Pointwise streams (1/W, M_0, delta_{j-2}; W) are read by each thread with
// 16-byte loads one plane ahead.  Waits are bounded: a wait that runs out sets the
// kernel error word, the CTA stops, writes NaN over the rest of its outputs and waits
// (bounded) for the copies it has in flight before it returns.
//
// Per cell, the products and the order of the sums are those of S_apply_cond and
// S_apply_visc.
#pragma once
#include <algorithm>
#include <cstdint>

#include "internal.cuh"

namespace rkl {

constexpr int MARCH_MAX_THREADS = 256, MARCH_MU = 5, MARCH_MC = 4, MARCH_NB = 3;
constexpr long long MARCH_WAIT_CYCLES = 4000000000LL;  // ~2 s at the maximum SM clock

// the marching kernels take grids with nr a multiple of 4 and at most 256
__host__ __device__ inline bool march_ok(int nr) { return nr % 4 == 0 && nr >= 4 && nr <= 256; }
// theta rows per tile: at least 4 (halo rows cost 2 per tile) and at least 512 cells per
// plane; a CTA has one thread per four cells of a tile plane, rounded up to whole warps,
// so tiles of nr <= 128 take 128 threads and (conduction) about 108 KB of shared memory,
// two CTAs per SM; tiles of nr = 256 take 256 threads and about 215 KB (viscosity needs
// less than half of these)
__host__ __device__ inline int march_th(int nr) { return 128 / (nr / 4) > 4 ? 128 / (nr / 4) : 4; }
__host__ __device__ inline int march_threads(int nr) { return ((nr / 4) * march_th(nr) + 31) / 32 * 32; }
// coefficient slots of a tile row and halo rows per plane
__host__ __device__ constexpr int march_ns(int op) { return op == OPK_VISC ? 4 : 10; }
__host__ __device__ constexpr int march_nh(int op) { return op == OPK_VISC ? 1 : 5; }
__host__ __device__ inline size_t march_smem(int nr, int op) {
  const int TH = march_th(nr);
  return sizeof(float) *
         ((size_t)MARCH_MU * (TH + 2) * nr + (size_t)MARCH_MC * (march_ns(op) * TH + march_nh(op)) * nr);
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
// global -> shared copy of `bytes` (a multiple of 16, both addresses 16-byte aligned)
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// wait for the phase of `parity` to complete; false once MARCH_WAIT_CYCLES have passed
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > MARCH_WAIT_CYCLES) return false;
  return true;
}

__device__ __forceinline__ float4 lds4(const float *p) { return *reinterpret_cast<const float4 *>(p); }

// a row of u around the four cells: x[0] = u(i0-1), x[1..4] = u(i0..i0+3), x[5] = u(i0+4);
// a missing r neighbour is clamped onto the cell itself, as in neighbours().  (Taking
// the neighbours from the adjacent lanes by shuffles instead was slower.)
__device__ __forceinline__ void row6(const float *row, int i0, int nr, float (&x)[6]) {
  const float4 v = lds4(row + i0);
  x[1] = v.x;
  x[2] = v.y;
  x[3] = v.z;
  x[4] = v.w;
  x[0] = i0 > 0 ? row[i0 - 1] : v.x;
  x[5] = i0 + 4 < nr ? row[i0 + 4] : v.w;
}
__device__ __forceinline__ void row4(const float *row, int i0, float (&x)[4]) {
  const float4 v = lds4(row + i0);
  x[0] = v.x;
  x[1] = v.y;
  x[2] = v.z;
  x[3] = v.w;
}
// entries of the cells one step down (L: i0-1 .. i0+2) or up (R: i0+1 .. i0+4) in r;
// outside the row 0 (masked by the caller)
__device__ __forceinline__ void row4L(const float *row, int i0, float (&x)[4]) {
  const float4 v = lds4(row + i0);
  x[0] = i0 > 0 ? row[i0 - 1] : 0.f;
  x[1] = v.x;
  x[2] = v.y;
  x[3] = v.z;
}
__device__ __forceinline__ void row4R(const float *row, int i0, int nr, float (&x)[4]) {
  const float4 v = lds4(row + i0);
  x[0] = v.y;
  x[1] = v.z;
  x[2] = v.w;
  x[3] = i0 + 4 < nr ? row[i0 + 4] : 0.f;
}

// The marching loop.  Epi supplies the pointwise part of a kernel:
//   void load(long long c)          16-byte loads of the pointwise inputs of cells c..c+3
//   void advance()                  make the loaded plane current
//   void store(long long c, const float (&s)[4], const float (&uc)[4])
//                                   outputs of cells c..c+3 from (S u) and u there
//   void poison(long long c)        NaN over the outputs of cells c..c+3
// Returns false when a wait ran out (the kernel error word is then set).
template <int OP, class Epi>
__device__ __forceinline__ bool march32(const Dims &d, int nchunk, const float *__restrict__ coef,
                                        const float *__restrict__ u, Epi &epi, int *kerr) {
  constexpr int NS = march_ns(OP), NH = march_nh(OP);
  extern __shared__ __align__(16) float msm[];
  __shared__ __align__(8) uint64_t bars[MARCH_NB];
  const int nr = d.nr, nth = d.nth, nph = d.nph, nq = nr >> 2, TH = march_th(nr);
  const int ntile = (nth + TH - 1) / TH;
  const int tile = (int)(blockIdx.x % (unsigned)ntile), chunk = (int)(blockIdx.x / (unsigned)ntile);
  const int j0 = tile * TH, th = min(TH, nth - j0);
  const int k0 = (int)((long long)chunk * nph / nchunk), k1 = (int)((long long)(chunk + 1) * nph / nchunk);
  const long long N = d.N;
  const int utile = (TH + 2) * nr, ctile = (NS * TH + NH) * nr, slot = TH * nr;
  float *ubuf = msm, *cbuf = msm + (size_t)MARCH_MU * utile;
  const int tid = threadIdx.x, tx = tid % nq, ty = tid / nq;
  const bool active = ty < th;
  const int i0 = 4 * tx, j = j0 + ty;
  const bool vtp = j < nth - 1, vtm = j > 0;
  const int jm = vtm ? j - 1 : j, jp = vtp ? j + 1 : j;

  // bytes of one plane of u (rows j0-1 .. j0+th inside the grid) and of coefficients
  const int rlo = max(j0 - 1, 0), rhi = min(j0 + th, nth - 1);
  const unsigned UB = (unsigned)((rhi - rlo + 1) * nr * 4);
  const unsigned CB =
      OP == OPK_VISC ? (unsigned)((4 * th + (j0 > 0 ? 1 : 0)) * nr * 4)
                     : (unsigned)((10 * th + (j0 > 0 ? 4 : 0) + (j0 + th < nth ? 1 : 0)) * nr * 4);
  auto wrapk = [nph](int p) { return p < 0 ? p + nph : (p >= nph ? p - nph : p); };
  auto issue_u = [&](int p, uint64_t *bar) {
    float *dst = ubuf + (size_t)((p - k0 + 1) % MARCH_MU) * utile + (rlo - j0 + 1) * nr;
    bulk_g2s(dst, u + ((long long)wrapk(p) * nth + rlo) * nr, UB, bar);
  };
  auto issue_c = [&](int p, uint64_t *bar) {
    float *dst = cbuf + (size_t)((p - k0 + 1) % MARCH_MC) * ctile;
    const long long row0 = ((long long)wrapk(p) * nth + j0) * nr;
    for (int m = 0; m < NS; m++) bulk_g2s(dst + m * slot, coef + m * N + row0, (unsigned)(th * nr * 4), bar);
    float *h = dst + NS * slot;
    if (OP == OPK_VISC) {
      if (j0 > 0) bulk_g2s(h, coef + 1 * N + row0 - nr, (unsigned)(nr * 4), bar);
      return;
    }
    if (j0 > 0) {
      bulk_g2s(h + 0 * nr, coef + 1 * N + row0 - nr, (unsigned)(nr * 4), bar);
      bulk_g2s(h + 1 * nr, coef + 3 * N + row0 - nr, (unsigned)(nr * 4), bar);
      bulk_g2s(h + 2 * nr, coef + 4 * N + row0 - nr, (unsigned)(nr * 4), bar);
      bulk_g2s(h + 3 * nr, coef + 8 * N + row0 - nr, (unsigned)(nr * 4), bar);
    }
    if (j0 + th < nth) bulk_g2s(h + 4 * nr, coef + 7 * N + row0 + (long long)th * nr, (unsigned)(nr * 4), bar);
  };

  if (tid == 0) {
    for (int b = 0; b < MARCH_NB; b++) mbar_init(&bars[b], 1);
    mbar_fence_init();
  }
  __syncthreads();
  if (tid == 0) {
    mbar_expect_tx(&bars[0], 3 * UB + 2 * CB);
    issue_u(k0 - 1, &bars[0]);
    issue_u(k0, &bars[0]);
    issue_u(k0 + 1, &bars[0]);
    issue_c(k0 - 1, &bars[0]);
    issue_c(k0, &bars[0]);
    for (int q = 1; q <= 2; q++)
      if (k0 + q < k1) {
        mbar_expect_tx(&bars[q], UB + CB);
        issue_u(k0 + q + 1, &bars[q]);
        issue_c(k0 + q, &bars[q]);
      }
  }
  const long long cbase = (long long)j * nr + i0;  // cell i0 of row j in plane 0
  if (active) epi.load(cbase + (long long)k0 * d.nrt);
  int kfail = -1;
  for (int k = k0; k < k1; k++) {
    const int it = k - k0;
    epi.advance();
    if (active && k + 1 < k1) epi.load(cbase + (long long)(k + 1) * d.nrt);
    const bool ok = mbar_wait(&bars[it % MARCH_NB], (unsigned)(it / MARCH_NB) & 1u);
    if (ok && active) {
      const float *uk = ubuf + (size_t)((it + 1) % MARCH_MU) * utile;
      const float *ukm = ubuf + (size_t)(it % MARCH_MU) * utile;
      const float *ukp = ubuf + (size_t)((it + 2) % MARCH_MU) * utile;
      const float *ck = cbuf + (size_t)((it + 1) % MARCH_MC) * ctile;
      const float *ckm = cbuf + (size_t)(it % MARCH_MC) * ctile;
      const int ro = (j - j0 + 1) * nr, rom = (jm - j0 + 1) * nr, rop = (jp - j0 + 1) * nr;
      const int co = (j - j0) * nr;
      const bool first = j == j0, last = j + 1 == j0 + th;
      float s[4], uc[4];
      if constexpr (OP == OPK_VISC) {
        float S0[6], TP[4], TM[4], PP[4], PM[4], C[4][4], B0[4], B1[4], B2[4];
        row6(uk + ro, i0, nr, S0);
        row4(uk + rop, i0, TP);
        row4(uk + rom, i0, TM);
        row4(ukp + ro, i0, PP);
        row4(ukm + ro, i0, PM);
#pragma unroll
        for (int m = 0; m < 4; m++) row4(ck + m * slot + co, i0, C[m]);
        row4L(ck + co, i0, B0);
        row4(first ? ck + 4 * slot : ck + 1 * slot + co - nr, i0, B1);
        row4(ckm + 2 * slot + co, i0, B2);
#pragma unroll
        for (int e = 0; e < 4; e++) {
          const bool vrm = e > 0 || i0 > 0;
          float acc = C[3][e] * S0[e + 1];
          acc = fmaf(C[0][e], S0[e + 2], acc);
          acc = fmaf(C[1][e], TP[e], acc);
          acc = fmaf(C[2][e], PP[e], acc);
          acc = fmaf(vrm ? B0[e] : 0.f, S0[e], acc);
          acc = fmaf(vtm ? B1[e] : 0.f, TM[e], acc);
          acc = fmaf(B2[e], PM[e], acc);
          s[e] = acc;
          uc[e] = S0[e + 1];
        }
      } else {
        float S0[6], TP[6], TM[6], PP[6], PM[6], G0[4], G1[4], G2[4], G3[4];
        row6(uk + ro, i0, nr, S0);
        row6(uk + rop, i0, nr, TP);
        row6(uk + rom, i0, nr, TM);
        row6(ukp + ro, i0, nr, PP);
        row6(ukm + ro, i0, nr, PM);
        row4(ukp + rom, i0, G0);  // tm + pp
        row4(ukp + rop, i0, G1);  // tp + pp
        row4(ukm + rop, i0, G2);  // tp + pm
        row4(ukm + rom, i0, G3);  // tm + pm
        float C[10][4];
#pragma unroll
        for (int m = 0; m < 10; m++) row4(ck + m * slot + co, i0, C[m]);
        float B0[4], B1[4], B2[4], B3[4], B4[4], B5[4], B6[4], B7[4], B8[4];
        row4L(ck + co, i0, B0);
        const float *h = ck + 10 * slot, *hm = ckm + 10 * slot;
        row4(first ? h + 0 * nr : ck + 1 * slot + co - nr, i0, B1);
        row4R(first ? h + 1 * nr : ck + 3 * slot + co - nr, i0, nr, B3);
        row4L(first ? h + 2 * nr : ck + 4 * slot + co - nr, i0, B4);
        row4(ckm + 2 * slot + co, i0, B2);
        row4R(ckm + 5 * slot + co, i0, nr, B5);
        row4L(ckm + 6 * slot + co, i0, B6);
        row4(last ? hm + 4 * nr : ckm + 7 * slot + co + nr, i0, B7);
        row4(first ? hm + 3 * nr : ckm + 8 * slot + co - nr, i0, B8);
#pragma unroll
        for (int e = 0; e < 4; e++) {
          const bool vrm = e > 0 || i0 > 0, vrp = e < 3 || i0 + 4 < nr;
          float acc = C[9][e] * S0[e + 1];
          acc = fmaf(C[0][e], S0[e + 2], acc);
          acc = fmaf(C[1][e], TP[e + 1], acc);
          acc = fmaf(C[2][e], PP[e + 1], acc);
          acc = fmaf(C[3][e], TP[e], acc);
          acc = fmaf(C[4][e], TP[e + 2], acc);
          acc = fmaf(C[5][e], PP[e], acc);
          acc = fmaf(C[6][e], PP[e + 2], acc);
          acc = fmaf(C[7][e], G0[e], acc);
          acc = fmaf(C[8][e], G1[e], acc);
          acc = fmaf(vrm ? B0[e] : 0.f, S0[e], acc);
          acc = fmaf(vtm ? B1[e] : 0.f, TM[e + 1], acc);
          acc = fmaf(B2[e], PM[e + 1], acc);
          acc = fmaf(vrp && vtm ? B3[e] : 0.f, TM[e + 2], acc);
          acc = fmaf(vrm && vtm ? B4[e] : 0.f, TM[e], acc);
          acc = fmaf(vrp ? B5[e] : 0.f, PM[e + 2], acc);
          acc = fmaf(vrm ? B6[e] : 0.f, PM[e], acc);
          acc = fmaf(vtp ? B7[e] : 0.f, G2[e], acc);
          acc = fmaf(vtm ? B8[e] : 0.f, G3[e], acc);
          s[e] = acc;
          uc[e] = S0[e + 1];
        }
      }
      epi.store(cbase + (long long)k * d.nrt, s, uc);
    }
    // the slots of plane k-1 are free once every thread is past plane k
    if (__syncthreads_or(!ok)) {
      kfail = k;
      break;
    }
    if (tid == 0 && k + 3 < k1) {
      uint64_t *bar = &bars[it % MARCH_NB];
      mbar_expect_tx(bar, UB + CB);
      issue_u(k + 4, bar);
      issue_c(k + 3, bar);
    }
  }
  if (kfail < 0) return true;
  // a wait ran out: flag it, poison the outputs not written, and let the copies in
  // flight (the batches of planes kfail .. kfail+2) land before the CTA's memory goes
  if (tid == 0) atomicExch(kerr, 1);
  if (active)
    for (int k = kfail; k < k1; k++) epi.poison(cbase + (long long)k * d.nrt);
  if (tid == 0)
    for (int k = kfail; k < min(kfail + 3, k1); k++)
      (void)mbar_wait(&bars[(k - k0) % MARCH_NB], (unsigned)((k - k0) / MARCH_NB) & 1u);
  __syncthreads();
  return false;
}

// phi chunks per theta tile: the fewest waves of resident CTAs (as many per SM as its
// shared memory holds), each item paying about two planes of prologue
inline int march_chunks(int nth, int nph, int nr, int op, int nsm, int smem_per_sm, int max_items) {
  const int TH = march_th(nr), ntile = (nth + TH - 1) / TH;
  const long long slots =
      (long long)nsm * std::max<long long>(1, smem_per_sm / (long long)(march_smem(nr, op) + 1024));
  int best = 1;
  double best_cost = 1e300;
  for (int n = 1; n <= nph && (long long)n * ntile <= max_items; n++) {
    const long long items = (long long)n * ntile;
    const double cost = (double)((items + slots - 1) / slots) * ((double)nph / n + 2.0);
    if (cost < best_cost - 1e-9) {
      best_cost = cost;
      best = n;
    }
  }
  return best;
}

}  // namespace rkl
