// warmstart.cu -- learned initial guess for the backward-Euler + PCG solve (the PCG of
// Fig. 1 starts from any x0).  A 4-layer 3-D convolutional net maps (T, bhat, log dt) to
// Delta T; it is trained on the solver's own solutions, and PCG still runs to the same
// tolerance, so the net only moves the starting point.
//
// Net: conv3x3x3 5->32 ReLU, 32->32 ReLU, 32->32 ReLU, 32->1.  Parameters are FP32 (Adam
// state too); every pass uses BF16 copies of the weights, BF16 activations and FP32
// accumulation on the tensor cores.  Rounding points: features, weights, stored
// activations a1..a3, the output gradient dy and the back-propagated gradients dz1..dz3
// are BF16 (round to nearest even); biases, y and the parameter gradients (FP32 per CTA,
// FP64 across CTAs in a fixed order) are not.
//
// Two convolution paths, with the same rounding points:
//
// * Grids whose r extent is a multiple of 128 (tcgen05): activations are planar 8-channel
//   slabs [C/8][box][phi][theta][r][8]; the 32-channel layers (forward layers 1-3, the
//   adjoint of layers 2-4) run k_conv_tc (TMA-staged planes, MMAs issued by single threads
//   into TMEM accumulators, the three phi taps of a (theta, r) tap in one N = 96 MMA) and
//   the output layer runs k_conv_out_tc (D = a W on the tensor cores, the 27-tap
//   shift-sum on the CUDA cores).  See the comments above each kernel.
//
// * Other grids (mma.sync m16n8k16): channels-last BF16 activations [box][phi][theta][r][C]
//   with C = 32, or C = 16 for the 5 input features (channels 5..15 zero) and for dy
//   (channel 0).  Convolutions are implicit GEMMs over bricks of 32 (r) x 4 (theta) x
//   2 (phi) cells: the brick plus a one-cell halo (34 x 6 x 4 rows of C channels) is
//   staged in shared memory with cp.async, rows XOR-swizzled by 16-byte chunk so that
//   ldmatrix of eight consecutive rows is conflict-free, and each tap's A operand is read
//   with ldmatrix from per-lane row addresses (the neighbour of the lane's cell).  Weights
//   sit in shared memory in mma fragment order.  Forward: M = 256 cells, N = 32 channels,
//   K = 27 taps x C.  Data gradient: the same kernel with the adjoint weights
//   W'[ci][co][26 - tap] = W[co][ci][tap].
//
// A box is a whole grid (phi periodic) or a detached block (zero outside on every face); r
// and theta are always zero outside.  The weight gradient runs on mma.sync on every grid
// (its layout-aware staging reads either activation layout): per tap, M = Cout, N = Cin,
// K = cells, both operands through ldmatrix.trans; a persistent CTA accumulates its
// bricks in registers and a second kernel sums the per-CTA partials in FP64.  (On tcgen05
// a tap is a shift along K, so each instruction would carry one tap with M = 32 output
// channels padded to 64; at the per-instruction cost measured for these kernels that is
// slower than mma.sync.)
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/warmstart.h"
#include "internal.cuh"

namespace {

constexpr int NL = 4;
constexpr int L_CIN[NL] = {5, 32, 32, 32};
constexpr int L_COUT[NL] = {32, 32, 32, 1};
constexpr int NTAP = 27;

// brick and halo geometry
constexpr int BR = 32, BT = 4, BP = 2, BRICK = BR * BT * BP;
constexpr int HR = BR + 2, HT = BT + 2, HP = BP + 2, NH = HR * HT * HP;
constexpr int CONV_THREADS = 256;  // 8 warps, one brick row of 32 cells each
constexpr int WG_THREADS = 288;    // 9 warps, three taps each
constexpr int EW = 256;            // element-wise kernels

enum { EPI_RELU = 0, EPI_MASK = 1, EPI_F32 = 2 };

struct Boxes {
  int nr, nth, nph, nbox, periodic;
  int nbr, nbt, nbp;  // bricks per box along r, theta, phi
  long long nc;       // cells per box
  long long nbricks;
};

Boxes make_boxes(int nr, int nth, int nph, int nbox, int periodic) {
  Boxes b;
  b.nr = nr;
  b.nth = nth;
  b.nph = nph;
  b.nbox = nbox;
  b.periodic = periodic;
  b.nbr = (nr + BR - 1) / BR;
  b.nbt = (nth + BT - 1) / BT;
  b.nbp = (nph + BP - 1) / BP;
  b.nc = (long long)nr * nth * nph;
  b.nbricks = (long long)b.nbr * b.nbt * b.nbp * nbox;
  return b;
}

__device__ __forceinline__ unsigned smem_u32(const void *p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void cp_async16(void *dst, const void *src, int bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(dst)), "l"(src), "r"(bytes));
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n" ::);
  asm volatile("cp.async.wait_group 0;\n" ::);
}

__device__ __forceinline__ void ldsm_x4(unsigned addr, unsigned &r0, unsigned &r1, unsigned &r2, unsigned &r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr));
}
__device__ __forceinline__ void ldsm_x4_t(unsigned addr, unsigned &r0, unsigned &r1, unsigned &r2, unsigned &r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr));
}

// D += A B, m16n8k16, BF16 inputs, FP32 accumulators
__device__ __forceinline__ void mma_bf16(float *d, unsigned a0, unsigned a1, unsigned a2, unsigned a3, unsigned b0,
                                         unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// 16-byte chunk swizzle of a staged row of C channels (C * 2 bytes)
template <int C>
__device__ __forceinline__ int swz(int row) {
  return C == 32 ? ((row >> 1) & 3) : ((row >> 2) & 1);
}
template <int C>
__device__ __forceinline__ unsigned row_chunk(unsigned base, int row, int chunk) {
  return base + row * (C * 2) + ((chunk ^ swz<C>(row)) << 4);
}

struct BrickPos {
  int b, i0, j0, k0;
};

__device__ __forceinline__ BrickPos brick_pos(const Boxes &g, long long id) {
  BrickPos p;
  const long long per_box = (long long)g.nbr * g.nbt * g.nbp;
  p.b = (int)(id / per_box);
  long long r = id - (long long)p.b * per_box;
  const int br = (int)(r % g.nbr);
  r /= g.nbr;
  const int bt = (int)(r % g.nbt);
  const int bp = (int)(r / g.nbt);
  p.i0 = br * BR;
  p.j0 = bt * BT;
  p.k0 = bp * BP;
  return p;
}

// global cell index of (i, j, k) in box b, or -1 outside (phi wraps when periodic)
__device__ __forceinline__ long long cell_index(const Boxes &g, int b, int i, int j, int k) {
  if (i < 0 || i >= g.nr || j < 0 || j >= g.nth) return -1;
  if (k < 0 || k >= g.nph) {
    if (!g.periodic) return -1;
    k = ((k % g.nph) + g.nph) % g.nph;
  }
  return (long long)b * g.nc + ((long long)k * g.nth + j) * g.nr + i;
}

// 8 channels (16 bytes) c of a cell of a C-channel BF16 activation: channels-last
// [cells][C] when ss = 0, else planar 8-channel slabs [C / 8][cells][8] with slab stride ss
// elements (the layout of the grids on the tcgen05 path)
__device__ __forceinline__ const __nv_bfloat16 *chunk_ptr(const __nv_bfloat16 *src, long long cell, int c, int C,
                                                          long long ss) {
  return ss ? src + c * ss + cell * 8 : src + cell * C + c * 8;
}

// stage the brick's halo rows of a C-channel activation (zero outside the box)
template <int C>
__device__ __forceinline__ void stage_halo(const Boxes &g, const BrickPos &p, const __nv_bfloat16 *src,
                                           unsigned char *halo, long long ss = 0) {
  constexpr int NCH = C / 8;
  for (int q = threadIdx.x; q < NH * NCH; q += blockDim.x) {
    const int h = q / NCH, c = q - h * NCH;
    const int hr = h % HR, ht = (h / HR) % HT, hp = h / (HR * HT);
    const long long cell = cell_index(g, p.b, p.i0 + hr - 1, p.j0 + ht - 1, p.k0 + hp - 1);
    const __nv_bfloat16 *gp = cell >= 0 ? chunk_ptr(src, cell, c, C, ss) : src;
    cp_async16(halo + h * (C * 2) + ((c ^ swz<C>(h)) << 4), gp, cell >= 0 ? 16 : 0);
  }
}

// stage the brick's own rows of a C-channel tensor (zero outside the box)
template <int C>
__device__ __forceinline__ void stage_brick(const Boxes &g, const BrickPos &p, const __nv_bfloat16 *src,
                                            unsigned char *dst, long long ss = 0) {
  constexpr int NCH = C / 8;
  for (int q = threadIdx.x; q < BRICK * NCH; q += blockDim.x) {
    const int r = q / NCH, c = q - r * NCH;
    const int ir = r % BR, it = (r / BR) % BT, ip = r / (BR * BT);
    const int i = p.i0 + ir, j = p.j0 + it, k = p.k0 + ip;
    const long long cell = (k < g.nph) ? cell_index(g, p.b, i, j, k) : -1;
    const __nv_bfloat16 *gp = cell >= 0 ? chunk_ptr(src, cell, c, C, ss) : src;
    cp_async16(dst + r * (C * 2) + ((c ^ swz<C>(r)) << 4), gp, cell >= 0 ? 16 : 0);
  }
}

__device__ __forceinline__ int halo_row(int ir, int it, int ip, int tap) {
  const int dr = tap % 3 - 1, dt = (tap / 3) % 3 - 1, dp = tap / 9 - 1;
  return (ir + 1 + dr) + HR * ((it + 1 + dt) + HT * (ip + 1 + dp));
}

struct ConvArgs {
  Boxes g;
  const __nv_bfloat16 *in;  // [cells][CIN]
  const uint2 *wfrag;       // [27][CIN/16][NT][32] B fragments
  const float *bias;        // [nbias] (EPI_RELU, EPI_F32) or NULL
  int nbias;
  const __nv_bfloat16 *mask;  // [cells][32] (EPI_MASK): zero where mask <= 0
  void *out;                // [cells][32] BF16, or [cells] FP32 (EPI_F32)
};

template <int CIN, int NT>
constexpr int conv_smem_bytes() {
  return NTAP * (CIN / 16) * NT * 32 * 8 + 128 + NH * CIN * 2;
}

// out = epilogue(sum_tap sum_ci W[.][ci][tap] in[ci][x + d(tap)]) over one box set
template <int CIN, int NT, int EPI>
__global__ void __launch_bounds__(CONV_THREADS, 2) k_conv(ConvArgs a) {
  constexpr int KS = CIN / 16;
  constexpr int WF_BYTES = NTAP * KS * NT * 32 * 8;
  extern __shared__ __align__(128) unsigned char smem[];
  uint2 *wf = reinterpret_cast<uint2 *>(smem);
  float *bias_s = reinterpret_cast<float *>(smem + WF_BYTES);
  unsigned char *halo = smem + WF_BYTES + 128;
  const unsigned halo_u = smem_u32(halo);

  for (int q = threadIdx.x; q < WF_BYTES / 16; q += CONV_THREADS)
    cp_async16(smem + q * 16, reinterpret_cast<const unsigned char *>(a.wfrag) + q * 16, 16);
  if (threadIdx.x < 32) bias_s[threadIdx.x] = (a.bias && (int)threadIdx.x < a.nbias) ? a.bias[threadIdx.x] : 0.0f;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int it = warp & 3, ip = warp >> 2;
  const int g = lane >> 2, q = lane & 3;
  const int mi = lane >> 3;
  const int row_in = (lane & 7) + ((mi & 1) << 3);  // ldmatrix row of this lane in an m-tile
  const int chunk_sel = mi >> 1;

  for (long long id = blockIdx.x; id < a.g.nbricks; id += gridDim.x) {
    const BrickPos p = brick_pos(a.g, id);
    stage_halo<CIN>(a.g, p, a.in, halo);
    cp_async_wait_all();
    __syncthreads();

    float acc[2][NT][4];
#pragma unroll
    for (int mt = 0; mt < 2; mt++)
#pragma unroll
      for (int nt = 0; nt < NT; nt++)
#pragma unroll
        for (int e = 0; e < 4; e++) acc[mt][nt][e] = 0.0f;

#pragma unroll 1
    for (int tap = 0; tap < NTAP; tap++) {
      const int h0 = halo_row(row_in, it, ip, tap);
#pragma unroll
      for (int ks = 0; ks < KS; ks++) {
        uint2 bf[NT];
#pragma unroll
        for (int nt = 0; nt < NT; nt++) bf[nt] = wf[((tap * KS + ks) * NT + nt) * 32 + lane];
#pragma unroll
        for (int mt = 0; mt < 2; mt++) {
          unsigned a0, a1, a2, a3;
          ldsm_x4(row_chunk<CIN>(halo_u, h0 + mt * 16, 2 * ks + chunk_sel), a0, a1, a2, a3);
#pragma unroll
          for (int nt = 0; nt < NT; nt++) mma_bf16(acc[mt][nt], a0, a1, a2, a3, bf[nt].x, bf[nt].y);
        }
      }
    }

    // epilogue: rows g and g + 8 of each m-tile, columns nt*8 + 2q, +1
#pragma unroll
    for (int mt = 0; mt < 2; mt++)
#pragma unroll
      for (int half = 0; half < 2; half++) {
        const int ir = mt * 16 + g + 8 * half;
        const int i = p.i0 + ir, j = p.j0 + it, k = p.k0 + ip;
        if (i >= a.g.nr || j >= a.g.nth || k >= a.g.nph) continue;
        const long long cell = (long long)p.b * a.g.nc + ((long long)k * a.g.nth + j) * a.g.nr + i;
        if (EPI == EPI_F32) {
          if (q == 0) reinterpret_cast<float *>(a.out)[cell] = acc[mt][0][2 * half] + bias_s[0];
        } else {
#pragma unroll
          for (int nt = 0; nt < NT; nt++) {
            const int col = nt * 8 + 2 * q;
            float v0 = acc[mt][nt][2 * half], v1 = acc[mt][nt][2 * half + 1];
            if (EPI == EPI_RELU) {
              v0 = fmaxf(v0 + bias_s[col], 0.0f);
              v1 = fmaxf(v1 + bias_s[col + 1], 0.0f);
            } else {
              const __nv_bfloat162 m = *reinterpret_cast<const __nv_bfloat162 *>(a.mask + cell * 32 + col);
              if (!(__low2float(m) > 0.0f)) v0 = 0.0f;
              if (!(__high2float(m) > 0.0f)) v1 = 0.0f;
            }
            *reinterpret_cast<__nv_bfloat162 *>(reinterpret_cast<__nv_bfloat16 *>(a.out) + cell * 32 + col) =
                __floats2bfloat162_rn(v0, v1);
          }
        }
      }
    __syncthreads();  // the halo is restaged next
  }
}

// ---- tcgen05 implicit-GEMM convolution: CIN in {16, 32} -> 32 channels, grids with nr a
// multiple of 128 ----
//
// A work unit is one column of TC_T = 2 theta rows x 128 r cells of one box over TC_C = 8
// consecutive output phi planes.  Its input planes k0 - 1 .. k0 + 8 are staged one by one:
// the 4 theta lines (the two rows and their halo) x 130 r cells (with the r halo) of the
// input, channels-last BF16, in the no-swizzle K-major layout of the tensor-core descriptors
// (for every 8-channel slab one 16-byte row per cell, rows contiguous:
// [slab][line][130 cells][8 channels]), brought in by one 5-D TMA copy (zero fill outside the
// box in r and theta).
//
// The cost of a tcgen05.mma here is set by the instruction count, not its size, so each MMA
// carries the three phi taps of one (theta, r) tap: for staged line l, output row t (theta
// offset dt = l - 1 - t) and r offset dr, A is the window of 128 rows of line l starting at
// 1 + dr (M = 128 cells, K = 16 channels per instruction) and B stacks the weights of
// (dt, dr, dp = +1, 0, -1) for the 32 output channels (N = 96), so that one instruction adds
// input plane k into the accumulators of output planes k - 1, k, k + 1.  TMEM holds the
// unit's 8 output planes x 2 rows x 32 FP32 channels ([row][plane][channel], all 512
// columns), so the three planes are adjacent columns (at the ends of a unit the window is cut
// to 64 or 32 columns).  36 MMAs per input plane, 45 per output plane instead of 108.
//
// The CTA is warp-specialised and its roles meet only at mbarriers:
//   warp 0     loads input planes into a ring of TC_RING slots (full[s] / empty[s]);
//   warps 1, 3 one thread each issues the MMAs of one output row for each input plane (two
//              issuers, as the issue of a tcgen05.mma, not its execution, sets the rate here),
//              frees the plane's ring slot by a commit, and commits output plane q as
//              complete (tfull[q]) after input plane q + 1;
//   warp 2     allocates and frees the TMEM columns;
//   warps 4-7  epilogue: TMEM -> registers (warp w reads TMEM lanes 32 (w mod 4) ..), then
//              zeros the plane's columns for the next unit (all MMAs accumulate) and frees
//              them (tempty[q]); bias + ReLU or the ReLU mask of the adjoint, BF16 stores.
// Every wait is bounded; one that runs out raises a shared abort flag that ends all roles,
// the kernel error word is set, and the CTA waits (bounded) for its copies and MMAs in
// flight before it frees TMEM and returns.
constexpr int TC_R = 128, TC_T = 2, TC_LINES = TC_T + 2, TC_ROWS = TC_R + 2, TC_PROWS = TC_LINES * TC_ROWS;
constexpr int TC_RING = 5, TC_THREADS = 256, TC_C = 8, TC_TMEM_COLS = 512;
constexpr int TC_CHUNK = 32;  // phi planes per unit of the output layer (k_conv_out_tc)
constexpr long long TC_WAIT = 4000000000LL;  // ~2 s at the maximum SM clock

template <int CIN> constexpr int tc_wbytes() { return NTAP * (CIN / 8) * 32 * 16; }
template <int CIN> constexpr int tc_plane_bytes() { return (CIN / 8) * TC_PROWS * 16; }
// weights, ring, 128 bytes of alignment slack, bias + barriers + TMEM slot + abort flag
// (at least 120000 bytes, so that one CTA, which holds all 512 TMEM columns, runs per SM)
template <int CIN> constexpr int tc_smem_bytes() {
  return tc_wbytes<CIN>() + TC_RING * tc_plane_bytes<CIN>() + 512 > 120000
             ? tc_wbytes<CIN>() + TC_RING * tc_plane_bytes<CIN>() + 512
             : 120000;
}

__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}
// kind::f16 instruction descriptor: FP32 accumulate, BF16 A and B, both K-major, M = 128, N
__host__ __device__ constexpr uint32_t tc_idesc(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | (8u << 24);
}

// D[tmem] (+)= A B^T, M = 128, K = 16, N from the instruction descriptor, BF16 in, FP32 accumulate
__device__ __forceinline__ void umma_bf16(uint32_t d, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}
// arrive on `bar` once every tcgen05 operation this thread has issued so far has completed
__device__ __forceinline__ void umma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tc_bar_init(uint64_t *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void tc_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void tc_expect_tx(uint64_t *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool tc_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// wait for the phase of `parity`; false when another role has aborted, or after TC_WAIT
// cycles (which raises the abort flag)
__device__ __forceinline__ bool tc_wait(uint64_t *bar, uint32_t parity, volatile int *abort_s) {
  const long long t0 = clock64();
  while (!tc_try_wait(bar, parity)) {
    if (*abort_s) return false;
    if (clock64() - t0 > TC_WAIT) {
      *abort_s = 1;
      return false;
    }
  }
  return true;
}
// teardown wait: ignores the abort flag, still bounded
__device__ __forceinline__ void tc_drain(uint64_t *bar, uint32_t parity) {
  const long long t0 = clock64();
  while (!tc_try_wait(bar, parity) && clock64() - t0 <= TC_WAIT) {
  }
}
// 5-D tiled TMA load of one box into shared memory, completing on `bar`
__device__ __forceinline__ void tma_load_5d(void *dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                            int c4, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, "
      "%6}], [%7];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(smem_u32(bar))
      : "memory");
}

// 32 consecutive TMEM columns of this thread's lane (32x32b shape, one lane per thread)
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}
// store 32 consecutive TMEM columns of this thread's lane
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
      "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
      "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]), "r"(r[17]), "r"(r[18]),
      "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]),
      "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
      : "memory");
}

struct TcArgs {
  Boxes g;
  const __nv_bfloat16 *wum;   // [27][CIN / 8][32][8] weight blocks (rows = output channel)
  const float *bias;          // [32] (EPI_RELU) or NULL
  const __nv_bfloat16 *mask;  // [cells][32] (EPI_MASK)
  __nv_bfloat16 *out;         // [cells][32]
  long long ss;               // slab stride of mask and out (planar [4][cells][8])
  long long nunits;
  int nchunk;                 // phi chunks per column
  int *kerr;                  // set when a bounded wait runs out
};

struct TcUnit {
  int b, i0, j0, k0, k1;
};
// unit -> (box, theta pair, r segment, phi chunk), the chunk fastest
__device__ __forceinline__ TcUnit tc_unit(const Boxes &g, int nchunk, int chunk, long long u) {
  TcUnit p;
  const int ch = (int)(u % nchunk);
  u /= nchunk;
  const int nseg = g.nr / TC_R, npair = (g.nth + TC_T - 1) / TC_T;
  const int seg = (int)(u % nseg);
  u /= nseg;
  const int pair = (int)(u % npair);
  p.b = (int)(u / npair);
  p.i0 = seg * TC_R;
  p.j0 = pair * TC_T;
  p.k0 = ch * chunk;
  p.k1 = min(g.nph, p.k0 + chunk);
  return p;
}

// in: the tensor map of the [cells][CIN] input, dims {8 channels, r, theta, CIN / 8 slabs,
// box * phi}, box {8, 130, 4, CIN / 8, 1}
template <int CIN, int EPI>
__global__ void __launch_bounds__(TC_THREADS, 1) k_conv_tc(const __grid_constant__ CUtensorMap in, TcArgs a) {
  constexpr int NS = CIN / 8, PB = tc_plane_bytes<CIN>(), SLAB = TC_PROWS * 16;
  constexpr int BSLAB = 96 * 16, BBLK = NS * BSLAB;  // B block of one (dt, dr): [slab][96 rows][8 channels]
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char *smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  unsigned char *wsm = smem;                      // weights, 9 B blocks
  unsigned char *ring = smem + tc_wbytes<CIN>();  // TC_RING staged planes
  float *bias_s = reinterpret_cast<float *>(ring + TC_RING * PB);
  uint64_t *full = reinterpret_cast<uint64_t *>(bias_s + 32);
  uint64_t *empty = full + TC_RING;
  uint64_t *tfull = empty + TC_RING;  // [TC_C]
  uint64_t *tempty = tfull + TC_C;    // [TC_C]
  uint64_t *done = tempty + TC_C;  // [2], one per MMA issuer
  uint32_t *tslot = reinterpret_cast<uint32_t *>(done + 2);
  volatile int *abort_s = reinterpret_cast<volatile int *>(tslot + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t wsm_u = smem_u32(wsm), ring_u = smem_u32(ring);
  const int nph = a.g.nph;

  for (int q = tid; q < tc_wbytes<CIN>() / 16; q += TC_THREADS)
    cp_async16(wsm + q * 16, reinterpret_cast<const unsigned char *>(a.wum) + q * 16, 16);
  if (tid < 32) bias_s[tid] = (EPI == EPI_RELU && a.bias) ? a.bias[tid] : 0.0f;
  if (tid == 0) {
    for (int s = 0; s < TC_RING; s++) {
      tc_bar_init(&full[s], 1);
      tc_bar_init(&empty[s], TC_T);  // one commit per MMA issuer
    }
    for (int q = 0; q < TC_C; q++) {
      tc_bar_init(&tfull[q], TC_T);
      tc_bar_init(&tempty[q], 4);
    }
    tc_bar_init(&done[0], 1);
    tc_bar_init(&done[1], 1);
    *abort_s = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(TC_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  cp_async_wait_all();
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // weights, for the tensor cores
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  if (warp >= 4) {  // the accumulators start at zero (every MMA accumulates)
    uint32_t z[32];
#pragma unroll
    for (int c = 0; c < 32; c++) z[c] = 0u;
    for (int c0 = 0; c0 < TC_TMEM_COLS; c0 += 32) tmem_st32(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + c0, z);
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

  if (warp == 0) {
    // ---- producer: planes k0 - 1 .. k1 of each unit, fill f into slot f mod TC_RING ----
    long long f = 0;
    bool ok = true;
    for (long long u = blockIdx.x; u < a.nunits && ok; u += gridDim.x) {
      const TcUnit p = tc_unit(a.g, a.nchunk, TC_C, u);
      for (int k = p.k0 - 1; k <= p.k1; k++, f++) {
        const int s = (int)(f % TC_RING);
        bool w = true;
        if (lane == 0) w = tc_wait(&empty[s], (uint32_t)((f / TC_RING) & 1) ^ 1u, abort_s);
        if (!__shfl_sync(0xffffffffu, w, 0)) {
          ok = false;
          break;
        }
        int kk = k;
        bool zero = false;
        if (kk < 0 || kk >= nph) {
          if (a.g.periodic) kk = ((kk % nph) + nph) % nph;
          else zero = true;
        }
        unsigned char *dst = ring + s * PB;
        if (!zero) {
          if (lane == 0) {
            tc_expect_tx(&full[s], PB);
            tma_load_5d(dst, &in, 0, p.i0 - 1, p.j0 - 1, 0, p.b * nph + kk, &full[s]);
          }
        } else {  // outside a non-periodic box: zeros, written by the warp
          for (int q = lane; q < PB / 16; q += 32) reinterpret_cast<uint4 *>(dst)[q] = make_uint4(0, 0, 0, 0);
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          __syncwarp();
          if (lane == 0) tc_arrive(&full[s]);
        }
      }
    }
    // teardown: the copies still in flight (the last fill of each slot) land before exit
    if (lane == 0)
      for (long long fi = f - 1; fi >= 0 && fi >= f - TC_RING; fi--)
        tc_drain(&full[fi % TC_RING], (uint32_t)((fi / TC_RING) & 1));
  } else if (warp == 1 || warp == 3) {
    // ---- MMA issuers: warp 1 the MMAs of output row 0, warp 3 those of row 1 ----
    const int tt = warp == 1 ? 0 : 1;
    if (lane == 0) {
      long long f = 0;    // fill of the unit's input plane k0 - 1
      uint32_t par = 0;   // bit q: uses of output slot q so far, mod 2
      bool ok = true;
      for (long long u = blockIdx.x; u < a.nunits && ok; u += gridDim.x) {
        const TcUnit p = tc_unit(a.g, a.nchunk, TC_C, u);
        const int nc = p.k1 - p.k0;  // output planes of the unit
        uint32_t ready = 0;          // output slots known free in this unit
        for (int qi = -1; qi <= nc && ok; qi++) {  // input plane k0 + qi
          const long long fi = f + qi + 1;
          const int s = (int)(fi % TC_RING);
          ok = tc_wait(&full[s], (uint32_t)((fi / TC_RING) & 1), abort_s);
          // output planes lo .. hi take this input plane (dp = input - output = +1, 0, -1)
          const int lo = qi - 1 > 0 ? qi - 1 : 0, hi = qi + 1 < nc - 1 ? qi + 1 : nc - 1;
          for (int q = lo; q <= hi && ok; q++)
            if (!((ready >> q) & 1u)) {
              ok = tc_wait(&tempty[q], ((par >> q) & 1u) ^ 1u, abort_s);
              ready |= 1u << q;
            }
          if (!ok) break;
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t idesc = tc_idesc(32 * (hi - lo + 1));
          const uint32_t brow = (uint32_t)(lo - (qi - 1)) * 32;  // first B row: dp = +1, 0, -1 blocks of 32
          const uint64_t ad0 = umma_desc(ring_u + (uint32_t)s * PB, SLAB, 128);
          const uint64_t bd0 = umma_desc(wsm_u + brow * 16, BSLAB, 128);
#pragma unroll
          for (int l = 0; l < TC_LINES; l++)
#pragma unroll
            for (int t = 0; t < TC_T; t++) {
              const int dt = l - 1 - t;
              if (t != tt || dt < -1 || dt > 1) continue;
#pragma unroll
              for (int dr = -1; dr <= 1; dr++)
#pragma unroll
                for (int ks = 0; ks < CIN / 16; ks++) {
                  const uint64_t ad = ad0 + ((uint32_t)((l * TC_ROWS + 1 + dr) * 16 + 2 * ks * SLAB) >> 4);
                  const uint64_t bd = bd0 + ((uint32_t)(((dt + 1) * 3 + (dr + 1)) * BBLK + 2 * ks * BSLAB) >> 4);
                  umma_bf16(tmem + t * (TC_C * 32) + lo * 32, ad, bd, idesc, 1u);
                }
            }
          umma_commit(&empty[s]);                    // this input plane is read
          if (qi >= 1) umma_commit(&tfull[qi - 1]);  // output plane qi - 1 has all its inputs
        }
        if (!ok) break;
        par ^= (1u << nc) - 1u;
        f += nc + 2;
      }
      umma_commit(&done[tt]);  // teardown: every MMA issued has completed
      tc_drain(&done[tt], 0);
    }
    __syncwarp();
  } else if (warp >= 4) {
    // ---- epilogue: output plane k0 + q from TMEM slot q ----
    const int q4 = warp & 3, m = 32 * q4 + lane;
    uint32_t par = 0;
    bool ok = true;
    uint32_t z[32];
#pragma unroll
    for (int c = 0; c < 32; c++) z[c] = 0u;
    for (long long u = blockIdx.x; u < a.nunits && ok; u += gridDim.x) {
      const TcUnit p = tc_unit(a.g, a.nchunk, TC_C, u);
      const int nc = p.k1 - p.k0;
      const bool row1 = p.j0 + 1 < a.g.nth;  // an odd theta count leaves the last pair one row
      for (int q = 0; q < nc; q++) {
        const int k = p.k0 + q;
        long long cell[TC_T];
#pragma unroll
        for (int t = 0; t < TC_T; t++)
          cell[t] = (long long)p.b * a.g.nc + ((long long)k * a.g.nth + (p.j0 + t)) * a.g.nr + p.i0 + m;
        uint4 mk[TC_T][4];
        if (EPI == EPI_MASK) {  // issued before the wait, so that their latency hides behind it
#pragma unroll
          for (int t = 0; t < TC_T; t++)
#pragma unroll
            for (int v = 0; v < 4; v++)
              mk[t][v] = (t == 0 || row1) ? *reinterpret_cast<const uint4 *>(a.mask + v * a.ss + cell[t] * 8)
                                          : make_uint4(0, 0, 0, 0);
        }
        const bool w = tc_wait(&tfull[q], (par >> q) & 1u, abort_s);
        if (!__all_sync(0xffffffffu, w)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        uint32_t r[TC_T][32];
#pragma unroll
        for (int t = 0; t < TC_T; t++) tmem_ld32(tmem + ((uint32_t)(32 * q4) << 16) + t * (TC_C * 32) + q * 32, r[t]);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int t = 0; t < TC_T; t++) tmem_st32(tmem + ((uint32_t)(32 * q4) << 16) + t * (TC_C * 32) + q * 32, z);
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) tc_arrive(&tempty[q]);  // slot q is zero again: the next unit may accumulate
#pragma unroll
        for (int t = 0; t < TC_T; t++) {
          if (t > 0 && !row1) break;
          __align__(16) __nv_bfloat16 o[32];
          if (EPI == EPI_RELU) {
#pragma unroll
            for (int c = 0; c < 32; c++) o[c] = __float2bfloat16_rn(fmaxf(__uint_as_float(r[t][c]) + bias_s[c], 0.0f));
          } else {
            const __nv_bfloat16 *mb = reinterpret_cast<const __nv_bfloat16 *>(mk[t]);
#pragma unroll
            for (int c = 0; c < 32; c++)
              o[c] = __float2bfloat16_rn(__bfloat162float(mb[c]) > 0.0f ? __uint_as_float(r[t][c]) : 0.0f);
          }
#pragma unroll
          for (int v = 0; v < 4; v++)
            *reinterpret_cast<uint4 *>(a.out + v * a.ss + cell[t] * 8) = reinterpret_cast<const uint4 *>(o)[v];
        }
      }
      par ^= (1u << nc) - 1u;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (tid == 0 && *abort_s) atomicOr(a.kerr, 1);
  if (warp == 2) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS));
  }
}

// ---- output layer (32 channels -> 1) on tcgen05, grids with nr a multiple of 128 ----
//
// y(x) = bias + sum over taps of sum_ci a(x + d(tap))[ci] W[ci][tap].  Per staged input plane
// the tensor cores form D[x][tap] = sum_ci a(x)[ci] W[ci][tap] for the plane's 4 lines (M = 128
// cells, N = 32 >= 27 taps, K = 32), and y is the sum over taps of D at the tap's neighbour,
// y(x) = bias + sum_tap D[x + d(tap)][tap]: every input is multiplied once, not once per tap.
// Units and staging are those of k_conv_tc (one 5-D TMA copy per plane, ring of TO_RING);
// D of the two r-halo cells of each line (outside the 128-cell tile) is formed on the CUDA
// cores.  Input plane k adds its contributions to the outputs of planes k - 1, k, k + 1, held
// in registers, one output cell per thread.
//
// Roles, synchronised by bounded mbarrier waits as in k_conv_tc:
//   warp 0     TMA producer (ring slot s is free once the MMAs of its plane and the r-halo
//              sums that read it are done: empty[s] takes two arrivals);
//   warp 1     allocates TMEM and issues the 8 MMAs of each plane into one of TO_NBUF TMEM
//              buffers (tfull / tempty), running up to TO_NBUF - 1 planes ahead;
//   warps 2-9  math: TMEM -> D tile in shared memory (double-buffered), r-halo D, one named
//              barrier per plane (which also ANDs the waits' outcomes, so that all math warps
//              leave together if one wait gives up), the 27-tap sums and the y stores.
constexpr int TO_RING = 3, TO_NBUF = 4, TO_TMEM_COLS = 512, TO_THREADS = 320;
constexpr int TO_DS_FLOATS = TC_LINES * NTAP * TC_ROWS;  // D of one plane, [line][tap][130 cells]
constexpr int to_smem_bytes() { return TO_RING * tc_plane_bytes<32>() + 2 * TO_DS_FLOATS * 4 + 2048 + NTAP * 32 * 4 + 512; }

struct ToArgs {
  Boxes g;
  const __nv_bfloat16 *w;  // [32 ci][27 taps], BF16
  const float *bias;       // [1]
  float *y;                // [cells]
  long long nunits;
  int nchunk;
  int *kerr;
};

// barrier 1 over the 256 math threads; returns the AND of v over them
__device__ __forceinline__ bool math_bar_and(bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.and.pred q, 1, 256, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)v)
      : "memory");
  return r != 0;
}

__global__ void __launch_bounds__(TO_THREADS, 1) k_conv_out_tc(const __grid_constant__ CUtensorMap in, ToArgs a) {
  constexpr int PB = tc_plane_bytes<32>(), SLAB = TC_PROWS * 16;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char *smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  unsigned char *ring = smem;                                      // TO_RING staged planes
  float *ds0 = reinterpret_cast<float *>(ring + TO_RING * PB);     // 2 x [4][27][130]
  __nv_bfloat16 *wb = reinterpret_cast<__nv_bfloat16 *>(ds0 + 2 * TO_DS_FLOATS);  // B: [4 slabs][32 taps][8 ci]
  float *wf = reinterpret_cast<float *>(wb + 1024);                // [27 taps][32 ci], FP32, for the r halo
  uint64_t *full = reinterpret_cast<uint64_t *>(wf + NTAP * 32);   // [TO_RING]
  uint64_t *empty = full + TO_RING;                                // [TO_RING]
  uint64_t *tfull = empty + TO_RING;                               // [TO_NBUF]
  uint64_t *tempty = tfull + TO_NBUF;                              // [TO_NBUF]
  uint64_t *done = tempty + TO_NBUF;
  uint32_t *tslot = reinterpret_cast<uint32_t *>(done + 1);
  volatile int *abort_s = reinterpret_cast<volatile int *>(tslot + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t ring_u = smem_u32(ring), wb_u = smem_u32(wb);
  const int nph = a.g.nph;

  for (int q = tid; q < 1024; q += TO_THREADS) {
    const int slab = q >> 8, n = (q >> 3) & 31, ci = slab * 8 + (q & 7);
    wb[q] = n < NTAP ? a.w[ci * NTAP + n] : __float2bfloat16(0.0f);
  }
  for (int q = tid; q < NTAP * 32; q += TO_THREADS) wf[q] = __bfloat162float(a.w[(q & 31) * NTAP + (q >> 5)]);
  if (tid == 0) {
    for (int s = 0; s < TO_RING; s++) {
      tc_bar_init(&full[s], 1);
      tc_bar_init(&empty[s], 2);
    }
    for (int b = 0; b < TO_NBUF; b++) {
      tc_bar_init(&tfull[b], 1);
      tc_bar_init(&tempty[b], 8);
    }
    tc_bar_init(done, 1);
    *abort_s = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(TO_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // B, for the tensor cores
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;

  if (warp == 0) {
    // ---- producer: planes k0 - 1 .. k1 of each unit, fill f into slot f mod TO_RING ----
    long long f = 0;
    bool ok = true;
    for (long long u = blockIdx.x; u < a.nunits && ok; u += gridDim.x) {
      const TcUnit p = tc_unit(a.g, a.nchunk, TC_CHUNK, u);
      for (int k = p.k0 - 1; k <= p.k1; k++, f++) {
        const int s = (int)(f % TO_RING);
        bool w = true;
        if (lane == 0) w = tc_wait(&empty[s], (uint32_t)((f / TO_RING) & 1) ^ 1u, abort_s);
        if (!__shfl_sync(0xffffffffu, w, 0)) {
          ok = false;
          break;
        }
        int kk = k;
        bool zero = false;
        if (kk < 0 || kk >= nph) {
          if (a.g.periodic) kk = ((kk % nph) + nph) % nph;
          else zero = true;
        }
        unsigned char *dst = ring + s * PB;
        if (!zero) {
          if (lane == 0) {
            tc_expect_tx(&full[s], PB);
            tma_load_5d(dst, &in, 0, p.i0 - 1, p.j0 - 1, 0, p.b * nph + kk, &full[s]);
          }
        } else {  // outside a non-periodic box: zeros, written by the warp
          for (int q = lane; q < PB / 16; q += 32) reinterpret_cast<uint4 *>(dst)[q] = make_uint4(0, 0, 0, 0);
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          __syncwarp();
          if (lane == 0) tc_arrive(&full[s]);
        }
      }
    }
    if (lane == 0)
      for (long long fi = f - 1; fi >= 0 && fi >= f - TO_RING; fi--)
        tc_drain(&full[fi % TO_RING], (uint32_t)((fi / TO_RING) & 1));
  } else if (warp == 1) {
    // ---- MMA issuer: D of plane g (all units in order) into TMEM buffer g mod TO_NBUF ----
    if (lane == 0) {
      long long g = 0;
      bool ok = true;
      for (long long u = blockIdx.x; u < a.nunits && ok; u += gridDim.x) {
        const TcUnit p = tc_unit(a.g, a.nchunk, TC_CHUNK, u);
        for (int k = p.k0 - 1; k <= p.k1; k++, g++) {
          const int s = (int)(g % TO_RING), buf = (int)(g % TO_NBUF);
          ok = tc_wait(&full[s], (uint32_t)((g / TO_RING) & 1), abort_s);
          if (ok) ok = tc_wait(&tempty[buf], (uint32_t)((g / TO_NBUF) & 1) ^ 1u, abort_s);
          if (!ok) break;
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
          for (int L = 0; L < TC_LINES; L++)
#pragma unroll
            for (int ks = 0; ks < 2; ks++)
              umma_bf16(tmem + buf * 128 + L * 32,
                        umma_desc(ring_u + s * PB + (L * TC_ROWS + 1) * 16 + 2 * ks * SLAB, SLAB, 128),
                        umma_desc(wb_u + 2 * ks * 512, 512, 128), tc_idesc(32), ks > 0 ? 1u : 0u);
          umma_commit(&tfull[buf]);
          umma_commit(&empty[s]);  // one of the slot's two arrivals
        }
      }
      umma_commit(done);
      tc_drain(done, 0);
    }
    __syncwarp();
  } else {
    // ---- math warps ----
    const int mt = tid - 64;                         // 0 .. 255
    const int t_out = mt >> 7, i_out = mt & 127;     // this thread's output cell in the tile
    const int q4 = warp & 3, m = 32 * q4 + lane;     // TMEM lane = tile cell
    const int L0 = warp < 6 ? 0 : 2;                 // this warp's two lines of D
    const float bias = a.bias[0];
    long long g = 0;
    bool ok = true;
    for (long long u = blockIdx.x; u < a.nunits && ok; u += gridDim.x) {
      const TcUnit p = tc_unit(a.g, a.nchunk, TC_CHUNK, u);
      float acc_prev = 0.0f, acc_cur = 0.0f, acc_next = 0.0f;  // outputs k - 1, k, k + 1
      for (int k = p.k0 - 1; k <= p.k1; k++, g++) {
        const int s = (int)(g % TO_RING), buf = (int)(g % TO_NBUF);
        float *ds = ds0 + (g & 1) * TO_DS_FLOATS;
        bool w = tc_wait(&tfull[buf], (uint32_t)((g / TO_NBUF) & 1), abort_s);
        w = __all_sync(0xffffffffu, w);
        if (w) {
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          uint32_t r[2][32];
#pragma unroll
          for (int h = 0; h < 2; h++) tmem_ld32(tmem + ((uint32_t)(32 * q4) << 16) + buf * 128 + (L0 + h) * 32, r[h]);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
          asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
          __syncwarp();
          if (lane == 0) tc_arrive(&tempty[buf]);
#pragma unroll
          for (int h = 0; h < 2; h++)
#pragma unroll
            for (int tap = 0; tap < NTAP; tap++)
              ds[((L0 + h) * NTAP + tap) * TC_ROWS + 1 + m] = __uint_as_float(r[h][tap]);
        }
        // D of the r-halo cells (rows 0 and 129 of each line); outside the box (the ends of
        // the r range) the staged rows are zero and so is D, written without the products
        if (w && mt < 8 * NTAP) {
          const int hc = mt / NTAP, tap = mt - hc * NTAP, L = hc >> 1, row = (hc & 1) ? TC_ROWS - 1 : 0;
          const bool inside = row == 0 ? p.i0 > 0 : p.i0 + TC_R < a.g.nr;
          float dsum = 0.0f;
          if (inside) w = tc_wait(&full[s], (uint32_t)((g / TO_RING) & 1), abort_s);
          if (inside && w) {
            const unsigned char *src = ring + s * PB + (L * TC_ROWS + row) * 16;
            const float *wt = wf + tap * 32;
#pragma unroll
            for (int slab = 0; slab < 4; slab++) {
              const uint4 v = *reinterpret_cast<const uint4 *>(src + slab * SLAB);
              const __nv_bfloat16 *x = reinterpret_cast<const __nv_bfloat16 *>(&v);
#pragma unroll
              for (int c = 0; c < 8; c++) dsum = fmaf(__bfloat162float(x[c]), wt[slab * 8 + c], dsum);
            }
          }
          ds[(L * NTAP + tap) * TC_ROWS + row] = dsum;
        }
        if (!math_bar_and(w)) {  // ds complete, slot s no longer read by the math warps
          ok = false;
          break;
        }
        if (mt == 0) tc_arrive(&empty[s]);
        // contributions of input plane k: tap (dr, dt, dp) takes D at (i + dr, j + dt) of the
        // plane k = output plane + dp
        float c[3];
#pragma unroll
        for (int dp = 0; dp < 3; dp++) {
          float sum = 0.0f;
#pragma unroll
          for (int dt = 0; dt < 3; dt++)
#pragma unroll
            for (int dr = 0; dr < 3; dr++)
              sum += ds[((t_out + dt) * NTAP + dp * 9 + dt * 3 + dr) * TC_ROWS + i_out + dr];
          c[dp] = sum;
        }
        acc_prev += c[2];  // output k - 1 (dp = +1): complete now
        acc_cur += c[1];
        acc_next += c[0];
        const int ko = k - 1;
        if (ko >= p.k0 && ko < p.k1 && p.j0 + t_out < a.g.nth)
          a.y[(long long)p.b * a.g.nc + ((long long)ko * a.g.nth + p.j0 + t_out) * a.g.nr + p.i0 + i_out] =
              bias + acc_prev;
        acc_prev = acc_cur;
        acc_cur = acc_next;
        acc_next = 0.0f;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (tid == 0 && *abort_s) atomicOr(a.kerr, 1);
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TO_TMEM_COLS));
  }
}

struct WgArgs {
  Boxes g;
  const __nv_bfloat16 *in;    // [cells][CIN] layer input activation
  const __nv_bfloat16 *dout;  // [cells][COUT] gradient at the layer's output
  float *part;                // [gridDim.x][27][COUT][CIN]
  float *partb;               // [gridDim.x][COUT]
  long long ss;               // slab stride of in and dout (0: channels-last)
};

template <int CIN, int COUT>
constexpr int wgrad_smem_bytes() {
  return NH * CIN * 2 + BRICK * COUT * 2;
}

// per-CTA partial dW[tap][co][ci] = sum_x dout[x][co] in[x + d(tap)][ci] and db[co]
template <int CIN, int COUT>
__global__ void __launch_bounds__(WG_THREADS, 1) k_wgrad(WgArgs a) {
  constexpr int MT = COUT / 16, NT = CIN / 8;
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned char *halo = smem;
  unsigned char *dsm = smem + NH * CIN * 2;
  const unsigned halo_u = smem_u32(halo), dsm_u = smem_u32(dsm);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, q = lane & 3, mi = lane >> 3;

  float acc[3][MT][NT][4];
  float accb[MT][4];
#pragma unroll
  for (int t = 0; t < 3; t++)
#pragma unroll
    for (int mt = 0; mt < MT; mt++)
#pragma unroll
      for (int nt = 0; nt < NT; nt++)
#pragma unroll
        for (int e = 0; e < 4; e++) acc[t][mt][nt][e] = 0.0f;
#pragma unroll
  for (int mt = 0; mt < MT; mt++)
#pragma unroll
    for (int e = 0; e < 4; e++) accb[mt][e] = 0.0f;
  const unsigned ones = 0x3F803F80u;  // two BF16 1.0

  for (long long id = blockIdx.x; id < a.g.nbricks; id += gridDim.x) {
    const BrickPos p = brick_pos(a.g, id);
    stage_halo<CIN>(a.g, p, a.in, halo, a.ss);
    stage_brick<COUT>(a.g, p, a.dout, dsm, a.ss);
    cp_async_wait_all();
    __syncthreads();
#pragma unroll 1
    for (int kk = 0; kk < BRICK / 16; kk++) {
      // A = dout^T (m = output channel, k = cell): matrices (cells 0-7 | 8-15) x (co lo | hi)
      unsigned af[MT][4];
      const int arow = kk * 16 + (lane & 7) + ((mi >> 1) << 3);
#pragma unroll
      for (int mt = 0; mt < MT; mt++)
        ldsm_x4_t(row_chunk<COUT>(dsm_u, arow, mt * 2 + (mi & 1)), af[mt][0], af[mt][1], af[mt][2], af[mt][3]);
      if (warp == 0) {
#pragma unroll
        for (int mt = 0; mt < MT; mt++) mma_bf16(accb[mt], af[mt][0], af[mt][1], af[mt][2], af[mt][3], ones, ones);
      }
      // B = shifted input (k = cell, n = input channel): matrices (cells 0-7 | 8-15) x (chunk nt | nt+1)
      const int bcell = kk * 16 + (lane & 7) + ((mi & 1) << 3);
      const int ir = bcell % BR, it = (bcell / BR) % BT, ip = bcell / (BR * BT);
#pragma unroll
      for (int t = 0; t < 3; t++) {
        const int h = halo_row(ir, it, ip, warp * 3 + t);
#pragma unroll
        for (int np = 0; np < NT / 2; np++) {
          unsigned b0, b1, b2, b3;
          ldsm_x4_t(row_chunk<CIN>(halo_u, h, np * 2 + (mi >> 1)), b0, b1, b2, b3);
#pragma unroll
          for (int mt = 0; mt < MT; mt++) {
            mma_bf16(acc[t][mt][2 * np], af[mt][0], af[mt][1], af[mt][2], af[mt][3], b0, b1);
            mma_bf16(acc[t][mt][2 * np + 1], af[mt][0], af[mt][1], af[mt][2], af[mt][3], b2, b3);
          }
        }
      }
    }
    __syncthreads();
  }

  float *part = a.part + (size_t)blockIdx.x * NTAP * COUT * CIN;
#pragma unroll
  for (int t = 0; t < 3; t++) {
    const int tap = warp * 3 + t;
#pragma unroll
    for (int mt = 0; mt < MT; mt++)
#pragma unroll
      for (int nt = 0; nt < NT; nt++)
#pragma unroll
        for (int half = 0; half < 2; half++) {
          const int co = mt * 16 + g + 8 * half, ci = nt * 8 + 2 * q;
          float *dst = part + ((size_t)tap * COUT + co) * CIN + ci;
          dst[0] = acc[t][mt][nt][2 * half];
          dst[1] = acc[t][mt][nt][2 * half + 1];
        }
  }
  if (warp == 0 && q == 0) {
#pragma unroll
    for (int mt = 0; mt < MT; mt++) {
      a.partb[(size_t)blockIdx.x * COUT + mt * 16 + g] = accb[mt][0];
      a.partb[(size_t)blockIdx.x * COUT + mt * 16 + g + 8] = accb[mt][2];
    }
  }
}

// dW in parameter order [co][ci][tap] (real channel counts) and db: fixed-order FP64 sums
__global__ void k_wgrad_reduce(int nblk, int CIN, int COUT, int cin, int cout, const float *__restrict__ part,
                               const float *__restrict__ partb, float *__restrict__ gw, float *__restrict__ gb) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  const int nw = cout * cin * NTAP;
  if (idx < nw) {
    const int co = idx / (cin * NTAP), ci = (idx / NTAP) % cin, tap = idx % NTAP;
    double s = 0.0;
    for (int b = 0; b < nblk; b++) s += part[(((size_t)b * NTAP + tap) * COUT + co) * CIN + ci];
    gw[idx] = (float)s;
  } else if (idx < nw + cout) {
    const int co = idx - nw;
    double s = 0.0;
    for (int b = 0; b < nblk; b++) s += partb[(size_t)b * COUT + co];
    gb[co] = (float)s;
  }
}

// B fragments of one layer in [tap][ks][nt][lane] order.  Forward: B[k][n] = W[n][k][tap]
// with n = output channel, k = input channel; adjoint: B[k][n] = W[k][n][26 - tap].
// Channels beyond the layer's real counts are zero.
__global__ void k_wfrag(const __nv_bfloat16 *__restrict__ w, int cin, int cout, int KS, int NT, int adjoint,
                        uint2 *__restrict__ out) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= NTAP * KS * NT * 32) return;
  const int lane = idx % 32, nt = (idx / 32) % NT, ks = (idx / (32 * NT)) % KS, tap = idx / (32 * NT * KS);
  const int g = lane >> 2, q = lane & 3;
  const int n = nt * 8 + g;
  auto elem = [&](int k) -> __nv_bfloat16 {
    const int kc = ks * 16 + k;
    int co, ci, t;
    if (!adjoint) {
      co = n;
      ci = kc;
      t = tap;
    } else {
      co = kc;
      ci = n;
      t = NTAP - 1 - tap;
    }
    if (co >= cout || ci >= cin) return __float2bfloat16(0.0f);
    return w[((size_t)co * cin + ci) * NTAP + t];
  };
  auto pack = [&](int k) -> unsigned {
    const __nv_bfloat16 lo = elem(k), hi = elem(k + 1);
    return (unsigned)__bfloat16_as_ushort(lo) | ((unsigned)__bfloat16_as_ushort(hi) << 16);
  };
  out[idx] = make_uint2(pack(2 * q), pack(2 * q + 8));
}

// B blocks of the tcgen05 convolution, [dt + 1][dr + 1][cin / 8][96][8]: row n = 32 dpi + c with
// dp = 1 - dpi (the phi offsets +1, 0, -1 in that order) and c the output channel of the
// convolution, 8 consecutive input channels per 16-byte row; forward B[n][k] = W[c][k][tap],
// adjoint B[n][k] = W[k][c][26 - tap], tap = (dr + 1) + 3 (dt + 1) + 9 (dp + 1).  Channels
// beyond the layer's real counts are zero.
__global__ void k_wumma(const __nv_bfloat16 *__restrict__ w, int cin, int cout, int CIN, int adjoint,
                        __nv_bfloat16 *__restrict__ out) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= NTAP * CIN * 32) return;
  const int e = idx % 8, n = (idx / 8) % 96, slab = (idx / 768) % (CIN / 8), blk = idx / (768 * (CIN / 8));
  const int dti = blk / 3, dri = blk % 3, dpi = n / 32, c = n % 32, k = slab * 8 + e;
  const int tap = dri + 3 * dti + 9 * (2 - dpi);
  int co, ci, t;
  if (!adjoint) {
    co = c;
    ci = k;
    t = tap;
  } else {
    co = k;
    ci = c;
    t = NTAP - 1 - tap;
  }
  out[idx] = (co < cout && ci < cin) ? w[((size_t)co * cin + ci) * NTAP + t] : __float2bfloat16(0.0f);
}

__global__ void __launch_bounds__(EW) k_to_bf16(int n, const float *__restrict__ a, __nv_bfloat16 *__restrict__ b) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < n) b[q] = __float2bfloat16_rn(a[q]);
}

// 16 BF16 channels of one cell into a 16-channel activation (layout as chunk_ptr)
__device__ __forceinline__ void store16(__nv_bfloat16 *out, long long c, long long ss, const __nv_bfloat16 (&v)[16]) {
  uint4 *d0 = reinterpret_cast<uint4 *>(ss ? out + c * 8 : out + c * 16);
  uint4 *d1 = reinterpret_cast<uint4 *>(ss ? out + ss + c * 8 : out + c * 16 + 8);
  *d0 = reinterpret_cast<const uint4 *>(v)[0];
  *d1 = reinterpret_cast<const uint4 *>(v)[1];
}

// FP32 channel-major [5][cells] -> 16-channel BF16 activation (slab stride ss, 0: channels-last)
__global__ void __launch_bounds__(EW) k_pack_input(long long cells, const float *__restrict__ in,
                                                   __nv_bfloat16 *__restrict__ out, long long ss) {
  const long long c = (long long)blockIdx.x * EW + threadIdx.x;
  if (c >= cells) return;
  __align__(16) __nv_bfloat16 v[16];
#pragma unroll
  for (int ch = 0; ch < 16; ch++) v[ch] = __float2bfloat16_rn(ch < 5 ? in[ch * cells + c] : 0.0f);
  store16(out, c, ss, v);
}

// features of one grid straight into the packed layout: (T - 1e6)/1e6, bhat, log10 dt
__global__ void __launch_bounds__(EW) k_features(long long N, const double *__restrict__ T,
                                                 const double *__restrict__ bhat, float logdt,
                                                 __nv_bfloat16 *__restrict__ out, float *__restrict__ f32,
                                                 long long ss) {
  const long long c = (long long)blockIdx.x * EW + threadIdx.x;
  if (c >= N) return;
  float f[5] = {(float)((T[c] - 1e6) * 1e-6), (float)bhat[c], (float)bhat[N + c], (float)bhat[2 * N + c], logdt};
  __align__(16) __nv_bfloat16 v[16];
#pragma unroll
  for (int ch = 0; ch < 16; ch++) v[ch] = __float2bfloat16_rn(ch < 5 ? f[ch] : 0.0f);
  store16(out, c, ss, v);
  if (f32) {
#pragma unroll
    for (int ch = 0; ch < 5; ch++) f32[ch * N + c] = f[ch];
  }
}

// sum of the loss weights (fixed-order block partials)
__global__ void __launch_bounds__(EW) k_sum(long long n, const float *__restrict__ w, double *__restrict__ part) {
  __shared__ double red[EW];
  double s = 0.0;
  for (long long q = (long long)blockIdx.x * EW + threadIdx.x; q < n; q += (long long)gridDim.x * EW)
    s += w ? (double)w[q] : 1.0;
  red[threadIdx.x] = s;
  __syncthreads();
  for (int h = EW / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// dy = 2 w (y - t) / sum w into channel 0 of a 16-channel BF16 tensor; partial sums of w e^2
__global__ void __launch_bounds__(EW) k_loss(long long n, const float *__restrict__ y, const float *__restrict__ t,
                                             const float *__restrict__ w, const double *__restrict__ wpart,
                                             int nwpart, __nv_bfloat16 *__restrict__ dy, double *__restrict__ part,
                                             long long ss) {
  __shared__ double red[EW];
  __shared__ float scale_s;
  if (threadIdx.x == 0) {
    double ws = 0.0;
    for (int b = 0; b < nwpart; b++) ws += wpart[b];
    scale_s = (float)(2.0 / ws);
  }
  __syncthreads();
  const float scale = scale_s;
  double s = 0.0;
  for (long long q = (long long)blockIdx.x * EW + threadIdx.x; q < n; q += (long long)gridDim.x * EW) {
    const float wq = w ? w[q] : 1.0f;
    const float e = y[q] - t[q];
    __align__(16) __nv_bfloat16 v[16];
    v[0] = __float2bfloat16_rn(scale * wq * e);
#pragma unroll
    for (int ch = 1; ch < 16; ch++) v[ch] = __float2bfloat16_rn(0.0f);
    store16(dy, q, ss, v);
    s += (double)wq * (double)e * (double)e;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int h = EW / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// Adam with bias correction (c1 = 1 - b1^t, c2 = 1 - b2^t); the complements om = 1 - b
// come from the host in FP64 (1 - 0.999f in FP32 is off by 1.3e-5 relative)
__global__ void __launch_bounds__(EW) k_adam(int n, float *__restrict__ p, const float *__restrict__ g,
                                             float *__restrict__ m, float *__restrict__ v, float lr, float b1,
                                             float om1, float b2, float om2, float eps, float c1, float c2) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const float gq = g[q];
  const float mq = b1 * m[q] + om1 * gq;
  const float vq = b2 * v[q] + om2 * gq * gq;
  m[q] = mq;
  v[q] = vq;
  p[q] = p[q] - lr * (mq / c1) / (sqrtf(vq / c2) + eps);
}

// x0 = T + scale y
__global__ void __launch_bounds__(EW) k_guess(long long N, const double *__restrict__ T, const float *__restrict__ y,
                                              double scale, double *__restrict__ x0) {
  const long long c = (long long)blockIdx.x * EW + threadIdx.x;
  if (c < N) x0[c] = fma(scale, (double)y[c], T[c]);
}

// training target out = (x - base) / unit in FP32
__global__ void __launch_bounds__(EW) k_target(long long N, const double *__restrict__ x, const double *__restrict__ base,
                                               double inv_unit, float *__restrict__ out) {
  const long long c = (long long)blockIdx.x * EW + threadIdx.x;
  if (c < N) out[c] = (float)((x[c] - base[c]) * inv_unit);
}

// SplitMix64 (Steele, Lea & Flood 2014), one step per counter from state seed
double splitmix_uniform(unsigned long long seed, unsigned long long ctr) {
  unsigned long long z = seed + 0x9E3779B97F4A7C15ULL * (ctr + 1);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  z ^= z >> 31;
  return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

}  // namespace

struct rkl_ws {
  cudaStream_t stream = nullptr;
  int nsm = 0;
  size_t woff[NL], boff[NL], bw_off[NL];  // FP32 weight/bias offsets, BF16 weight offsets
  int nparam = 0, nweight = 0;
  float *param = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
  __nv_bfloat16 *wbf = nullptr;
  uint2 *wfrag[NL] = {nullptr, nullptr, nullptr, nullptr};  // forward fragments
  uint2 *wadj[NL] = {nullptr, nullptr, nullptr, nullptr};   // adjoint fragments (layers 1..3)
  __nv_bfloat16 *wum[NL] = {nullptr, nullptr, nullptr, nullptr};   // tcgen05 weight blocks (layers 0..2)
  __nv_bfloat16 *wuma[NL] = {nullptr, nullptr, nullptr, nullptr};  // tcgen05 adjoint blocks (layers 1..3)
  int *kerr = nullptr;  // set by a tcgen05 convolution whose bounded wait ran out
  long long step = 0;
  unsigned char *arena = nullptr;
  size_t arena_cap = 0;
  float *part = nullptr;  // weight-gradient partials
  size_t part_cap = 0;
  double *red = nullptr;  // loss partials (2 x 1024)
  long long launches = 0;
  char err[256] = {0};
};

using namespace rkl;

namespace {

constexpr int RED_BLOCKS = 1024;

int ws_cuda(rkl_ws *ws, cudaError_t e) {
  if (e == cudaSuccess) return RKL_OK;
  if (ws) snprintf(ws->err, sizeof(ws->err), "%s", cudaGetErrorString(e));
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? RKL_ENOMEM : RKL_ECUDA;
}

int frag_ks(int l) { return L_CIN[l] <= 16 ? 1 : 2; }
// channels of a tcgen05 convolution input (K padded to a multiple of 16)
int tc_cin(int c) { return c <= 16 ? 16 : 32; }
int frag_nt(int l) { return L_COUT[l] == 1 ? 1 : 4; }
size_t frag_count(int l) { return (size_t)NTAP * frag_ks(l) * frag_nt(l) * 32; }
// adjoint of layer l (l >= 1): input = gradient at its output (16 channels for l = 3)
size_t adj_count(int l) { return (size_t)NTAP * (L_COUT[l] == 1 ? 1 : 2) * 4 * 32; }

template <typename K>
int set_smem(rkl_ws *ws, K kernel, int bytes) {
  return ws_cuda(ws, cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
}

int configure_kernels(rkl_ws *ws) {
  int rc = set_smem(ws, k_conv<16, 4, EPI_RELU>, conv_smem_bytes<16, 4>());
  if (!rc) rc = set_smem(ws, k_conv<32, 4, EPI_RELU>, conv_smem_bytes<32, 4>());
  if (!rc) rc = set_smem(ws, k_conv<32, 1, EPI_F32>, conv_smem_bytes<32, 1>());
  if (!rc) rc = set_smem(ws, k_conv<16, 4, EPI_MASK>, conv_smem_bytes<16, 4>());
  if (!rc) rc = set_smem(ws, k_conv<32, 4, EPI_MASK>, conv_smem_bytes<32, 4>());
  if (!rc) rc = set_smem(ws, k_wgrad<16, 32>, wgrad_smem_bytes<16, 32>());
  if (!rc) rc = set_smem(ws, k_wgrad<32, 32>, wgrad_smem_bytes<32, 32>());
  if (!rc) rc = set_smem(ws, k_wgrad<32, 16>, wgrad_smem_bytes<32, 16>());
  if (!rc) rc = set_smem(ws, k_conv_tc<16, EPI_RELU>, tc_smem_bytes<16>());
  if (!rc) rc = set_smem(ws, k_conv_tc<32, EPI_RELU>, tc_smem_bytes<32>());
  if (!rc) rc = set_smem(ws, k_conv_tc<16, EPI_MASK>, tc_smem_bytes<16>());
  if (!rc) rc = set_smem(ws, k_conv_tc<32, EPI_MASK>, tc_smem_bytes<32>());
  if (!rc) rc = set_smem(ws, k_conv_out_tc, to_smem_bytes());
  return rc;
}

// BF16 weights and mma fragments from the FP32 parameters
int refresh_weights(rkl_ws *ws) {
  for (int l = 0; l < NL; l++) {
    const int nw = L_COUT[l] * L_CIN[l] * NTAP;
    k_to_bf16<<<(nw + EW - 1) / EW, EW, 0, ws->stream>>>(nw, ws->param + ws->woff[l], ws->wbf + ws->bw_off[l]);
    const int nf = (int)frag_count(l);
    k_wfrag<<<(nf + EW - 1) / EW, EW, 0, ws->stream>>>(ws->wbf + ws->bw_off[l], L_CIN[l], L_COUT[l], frag_ks(l),
                                                      frag_nt(l), 0, ws->wfrag[l]);
    ws->launches += 2;
    if (l > 0) {
      const int na = (int)adj_count(l);
      k_wfrag<<<(na + EW - 1) / EW, EW, 0, ws->stream>>>(ws->wbf + ws->bw_off[l], L_CIN[l], L_COUT[l],
                                                        L_COUT[l] == 1 ? 1 : 2, 4, 1, ws->wadj[l]);
      ws->launches += 1;
    }
    if (l < NL - 1) {  // tcgen05 forward blocks: input channels padded to 16 or 32
      const int CIN = tc_cin(L_CIN[l]), n = NTAP * CIN * 32;
      k_wumma<<<(n + EW - 1) / EW, EW, 0, ws->stream>>>(ws->wbf + ws->bw_off[l], L_CIN[l], L_COUT[l], CIN, 0,
                                                       ws->wum[l]);
      ws->launches += 1;
    }
    if (l > 0) {  // tcgen05 adjoint blocks: the adjoint's input is the gradient at the output
      const int CIN = tc_cin(L_COUT[l]), n = NTAP * CIN * 32;
      k_wumma<<<(n + EW - 1) / EW, EW, 0, ws->stream>>>(ws->wbf + ws->bw_off[l], L_CIN[l], L_COUT[l], CIN, 1,
                                                       ws->wuma[l]);
      ws->launches += 1;
    }
  }
  return ws_cuda(ws, cudaGetLastError());
}

int ensure_arena(rkl_ws *ws, size_t bytes) {
  if (bytes <= ws->arena_cap) return RKL_OK;
  if (ws->arena) {
    cudaStreamSynchronize(ws->stream);
    cudaFree(ws->arena);
    ws->arena = nullptr;
    ws->arena_cap = 0;
  }
  int rc = ws_cuda(ws, cudaMalloc(&ws->arena, bytes));
  if (!rc) ws->arena_cap = bytes;
  return rc;
}

int ensure_part(rkl_ws *ws, size_t floats) {
  if (floats <= ws->part_cap) return RKL_OK;
  if (ws->part) {
    cudaStreamSynchronize(ws->stream);
    cudaFree(ws->part);
    ws->part = nullptr;
    ws->part_cap = 0;
  }
  int rc = ws_cuda(ws, cudaMalloc(&ws->part, floats * sizeof(float)));
  if (!rc) ws->part_cap = floats;
  return rc;
}

// the tcgen05 convolution takes 16- or 32-channel inputs, 32 outputs, and grids whose r
// extent is a multiple of 128 (one UMMA tile per r line)
bool tc_applies(const Boxes &g) { return g.nr % TC_R == 0; }

// cuTensorMapEncodeTiled, fetched once through the runtime (no link against the driver library)
typedef CUresult (*TmapEncodeFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
TmapEncodeFn tmap_encoder() {
  static TmapEncodeFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<TmapEncodeFn>(p);
  });
  return fn;
}

// tensor map of a planar [cin / 8][cells][8] BF16 activation viewed as {8 channels, r, theta,
// cin / 8 slabs, box * phi}, box {8, 130, 4, cin / 8, 1}: a box lands in shared memory as
// [slab][line][r][8 channels], and each line of a slab is one contiguous run of 130 x 16 bytes
int tc_tmap(rkl_ws *ws, const Boxes &g, const __nv_bfloat16 *in, int cin, CUtensorMap *map) {
  const TmapEncodeFn enc = tmap_encoder();
  if (!enc) {
    snprintf(ws->err, sizeof(ws->err), "%s", "cuTensorMapEncodeTiled is not available");
    return RKL_ECUDA;
  }
  const cuuint64_t dims[5] = {8, (cuuint64_t)g.nr, (cuuint64_t)g.nth, (cuuint64_t)(cin / 8),
                              (cuuint64_t)g.nbox * (cuuint64_t)g.nph};
  const cuuint64_t strides[4] = {16, (cuuint64_t)g.nr * 16, (cuuint64_t)(g.nc * g.nbox) * 16,
                                 (cuuint64_t)g.nth * g.nr * 16};
  const cuuint32_t box[5] = {8, (cuuint32_t)TC_ROWS, (cuuint32_t)TC_LINES, (cuuint32_t)(cin / 8), 1};
  const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  const CUresult cr = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<__nv_bfloat16 *>(in), dims, strides,
                          box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (cr != CUDA_SUCCESS) {
    snprintf(ws->err, sizeof(ws->err), "cuTensorMapEncodeTiled failed (%d)", (int)cr);
    return RKL_ECUDA;
  }
  return RKL_OK;
}

template <int CIN, int EPI>
int launch_conv_tc(rkl_ws *ws, const Boxes &g, const __nv_bfloat16 *in, const __nv_bfloat16 *wum, const float *bias,
                   const __nv_bfloat16 *mask, __nv_bfloat16 *out) {
  CUtensorMap map;
  if (int rc = tc_tmap(ws, g, in, CIN, &map)) return rc;
  TcArgs a;
  a.g = g;
  a.wum = wum;
  a.bias = bias;
  a.mask = mask;
  a.out = out;
  a.ss = 8 * g.nc * g.nbox;
  a.nchunk = (g.nph + TC_C - 1) / TC_C;
  a.nunits = (long long)g.nbox * (g.nr / TC_R) * ((g.nth + TC_T - 1) / TC_T) * a.nchunk;
  a.kerr = ws->kerr;
  const long long grid = a.nunits < ws->nsm ? a.nunits : ws->nsm;
  k_conv_tc<CIN, EPI><<<(unsigned)grid, TC_THREADS, tc_smem_bytes<CIN>(), ws->stream>>>(map, a);
  ws->launches += 1;
  return RKL_OK;
}

int launch_conv_out_tc(rkl_ws *ws, const Boxes &g, const __nv_bfloat16 *in, const __nv_bfloat16 *w,
                       const float *bias, float *y) {
  CUtensorMap map;
  if (int rc = tc_tmap(ws, g, in, 32, &map)) return rc;
  ToArgs a;
  a.g = g;
  a.w = w;
  a.bias = bias;
  a.y = y;
  a.nchunk = (g.nph + TC_CHUNK - 1) / TC_CHUNK;
  a.nunits = (long long)g.nbox * (g.nr / TC_R) * ((g.nth + TC_T - 1) / TC_T) * a.nchunk;
  a.kerr = ws->kerr;
  const long long grid = a.nunits < ws->nsm ? a.nunits : ws->nsm;
  k_conv_out_tc<<<(unsigned)grid, TO_THREADS, to_smem_bytes(), ws->stream>>>(map, a);
  ws->launches += 1;
  return RKL_OK;
}

int conv_grid(const rkl_ws *ws, const Boxes &g) {
  const long long cap = 2LL * ws->nsm;
  return (int)(g.nbricks < cap ? g.nbricks : cap);
}

template <int CIN, int NT, int EPI>
void launch_conv(rkl_ws *ws, const Boxes &g, const __nv_bfloat16 *in, const uint2 *wf, const float *bias,
                 const __nv_bfloat16 *mask, void *out) {
  ConvArgs a{g, in, wf, bias, bias ? (NT == 1 ? 1 : 32) : 0, mask, out};
  k_conv<CIN, NT, EPI><<<conv_grid(ws, g), CONV_THREADS, conv_smem_bytes<CIN, NT>(), ws->stream>>>(a);
  ws->launches += 1;
}

template <int CIN, int COUT>
int launch_wgrad(rkl_ws *ws, const Boxes &g, const __nv_bfloat16 *in, const __nv_bfloat16 *dout, int l,
                 long long ss) {
  const int nblk = (int)(g.nbricks < ws->nsm ? g.nbricks : ws->nsm);
  const size_t need = (size_t)nblk * (NTAP * COUT * CIN + COUT);
  int rc = ensure_part(ws, need);
  if (rc) return rc;
  WgArgs a{g, in, dout, ws->part, ws->part + (size_t)nblk * NTAP * COUT * CIN, ss};
  k_wgrad<CIN, COUT><<<nblk, WG_THREADS, wgrad_smem_bytes<CIN, COUT>(), ws->stream>>>(a);
  const int nout = L_COUT[l] * L_CIN[l] * NTAP + L_COUT[l];
  k_wgrad_reduce<<<(nout + EW - 1) / EW, EW, 0, ws->stream>>>(nblk, CIN, COUT, L_CIN[l], L_COUT[l], a.part, a.partb,
                                                             ws->grad + ws->woff[l], ws->grad + ws->boff[l]);
  ws->launches += 2;
  return RKL_OK;
}

// buffers of one pass over `cells` cells, carved from the arena (256-byte aligned)
struct Bufs {
  __nv_bfloat16 *a0, *a1, *a2, *a3, *dy, *dzA, *dzB;
  float *y;
};

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

int carve(rkl_ws *ws, long long cells, bool training, Bufs &b) {
  const size_t s16 = align256((size_t)cells * 16 * 2), s32 = align256((size_t)cells * 32 * 2),
               sf = align256((size_t)cells * 4);
  const size_t total = training ? (2 * s16 + 5 * s32 + sf) : (s16 + 2 * s32 + sf);
  int rc = ensure_arena(ws, total);
  if (rc) return rc;
  unsigned char *p = ws->arena;
  auto take = [&](size_t s) {
    unsigned char *q = p;
    p += s;
    return q;
  };
  b.a0 = (__nv_bfloat16 *)take(s16);
  b.a1 = (__nv_bfloat16 *)take(s32);
  b.a2 = (__nv_bfloat16 *)take(s32);
  if (training) {
    b.a3 = (__nv_bfloat16 *)take(s32);
    b.dy = (__nv_bfloat16 *)take(s16);
    b.dzA = (__nv_bfloat16 *)take(s32);
    b.dzB = (__nv_bfloat16 *)take(s32);
  } else {
    b.a3 = b.a1;  // a1 is dead once a2 exists
    b.dy = b.dzA = b.dzB = nullptr;
  }
  b.y = (float *)take(sf);
  return RKL_OK;
}

int run_forward(rkl_ws *ws, const Boxes &g, const Bufs &b) {
  int rc = RKL_OK;
  if (tc_applies(g)) {
    rc = launch_conv_tc<16, EPI_RELU>(ws, g, b.a0, ws->wum[0], ws->param + ws->boff[0], nullptr, b.a1);
    if (!rc) rc = launch_conv_tc<32, EPI_RELU>(ws, g, b.a1, ws->wum[1], ws->param + ws->boff[1], nullptr, b.a2);
    if (!rc) rc = launch_conv_tc<32, EPI_RELU>(ws, g, b.a2, ws->wum[2], ws->param + ws->boff[2], nullptr, b.a3);
  } else {
    launch_conv<16, 4, EPI_RELU>(ws, g, b.a0, ws->wfrag[0], ws->param + ws->boff[0], nullptr, b.a1);
    launch_conv<32, 4, EPI_RELU>(ws, g, b.a1, ws->wfrag[1], ws->param + ws->boff[1], nullptr, b.a2);
    launch_conv<32, 4, EPI_RELU>(ws, g, b.a2, ws->wfrag[2], ws->param + ws->boff[2], nullptr, b.a3);
  }
  if (rc) return rc;
  if (tc_applies(g)) return launch_conv_out_tc(ws, g, b.a3, ws->wbf + ws->bw_off[3], ws->param + ws->boff[3], b.y);
  launch_conv<32, 1, EPI_F32>(ws, g, b.a3, ws->wfrag[3], ws->param + ws->boff[3], nullptr, b.y);
  return RKL_OK;
}

bool valid_box(const int box[3], int nbox) {
  return box && nbox >= 1 && box[0] >= 1 && box[1] >= 1 && box[2] >= 1;
}

}  // namespace

extern "C" {

int ws_num_params(void) {
  int n = 0;
  for (int l = 0; l < NL; l++) n += L_COUT[l] * L_CIN[l] * NTAP + L_COUT[l];
  return n;
}

int ws_create(rkl_ws **out, unsigned long long seed, void *cuda_stream) {
  if (!out) return RKL_EINVAL;
  *out = nullptr;
  rkl_ws *ws = new (std::nothrow) rkl_ws();
  if (!ws) return RKL_ENOMEM;
  ws->stream = (cudaStream_t)cuda_stream;
  size_t off = 0, boff = 0;
  for (int l = 0; l < NL; l++) {
    ws->woff[l] = off;
    ws->boff[l] = off + (size_t)L_COUT[l] * L_CIN[l] * NTAP;
    ws->bw_off[l] = boff;
    off = ws->boff[l] + L_COUT[l];
    boff += (size_t)L_COUT[l] * L_CIN[l] * NTAP;
  }
  ws->nparam = (int)off;
  ws->nweight = (int)boff;
  int dev = 0;
  int rc = ws_cuda(ws, cudaGetDevice(&dev));
  if (!rc) rc = ws_cuda(ws, cudaDeviceGetAttribute(&ws->nsm, cudaDevAttrMultiProcessorCount, dev));
  const size_t pb = sizeof(float) * ws->nparam;
  if (!rc) rc = ws_cuda(ws, cudaMalloc(&ws->param, pb));
  if (!rc) rc = ws_cuda(ws, cudaMalloc(&ws->grad, pb));
  if (!rc) rc = ws_cuda(ws, cudaMalloc(&ws->m, pb));
  if (!rc) rc = ws_cuda(ws, cudaMalloc(&ws->v, pb));
  if (!rc) rc = ws_cuda(ws, cudaMalloc(&ws->wbf, sizeof(__nv_bfloat16) * ws->nweight));
  if (!rc) rc = ws_cuda(ws, cudaMalloc(&ws->red, sizeof(double) * 2 * RED_BLOCKS));
  for (int l = 0; l < NL && !rc; l++) {
    rc = ws_cuda(ws, cudaMalloc(&ws->wfrag[l], sizeof(uint2) * frag_count(l)));
    if (!rc && l > 0) rc = ws_cuda(ws, cudaMalloc(&ws->wadj[l], sizeof(uint2) * adj_count(l)));
    if (!rc && l < NL - 1)
      rc = ws_cuda(ws, cudaMalloc(&ws->wum[l], sizeof(__nv_bfloat16) * NTAP * tc_cin(L_CIN[l]) * 32));
    if (!rc && l > 0)
      rc = ws_cuda(ws, cudaMalloc(&ws->wuma[l], sizeof(__nv_bfloat16) * NTAP * tc_cin(L_COUT[l]) * 32));
  }
  if (!rc) rc = ws_cuda(ws, cudaMalloc(&ws->kerr, sizeof(int)));
  if (!rc) rc = ws_cuda(ws, cudaMemset(ws->kerr, 0, sizeof(int)));
  if (!rc) rc = configure_kernels(ws);
  if (!rc) {
    std::vector<float> p(ws->nparam, 0.0f);
    for (int l = 0; l < NL; l++) {
      const size_t nw = (size_t)L_COUT[l] * L_CIN[l] * NTAP;
      const double a = std::sqrt(6.0 / (L_CIN[l] * (double)NTAP));
      for (size_t q = 0; q < nw; q++)
        p[ws->woff[l] + q] = (float)((2.0 * splitmix_uniform(seed, ws->woff[l] + q) - 1.0) * a);
    }
    rc = ws_set_params(ws, p.data(), ws->nparam);
  }
  if (!rc) rc = ws_cuda(ws, cudaMemsetAsync(ws->grad, 0, pb, ws->stream));
  if (rc) {
    ws_destroy(ws);
    return rc;
  }
  *out = ws;
  return RKL_OK;
}

int ws_destroy(rkl_ws *ws) {
  if (!ws) return RKL_OK;
  cudaStreamSynchronize(ws->stream);
  void *bufs[] = {ws->param, ws->grad, ws->m, ws->v, ws->wbf, ws->arena, ws->part, ws->red};
  for (void *b : bufs)
    if (b) cudaFree(b);
  for (int l = 0; l < NL; l++) {
    if (ws->wfrag[l]) cudaFree(ws->wfrag[l]);
    if (ws->wadj[l]) cudaFree(ws->wadj[l]);
    if (ws->wum[l]) cudaFree(ws->wum[l]);
    if (ws->wuma[l]) cudaFree(ws->wuma[l]);
  }
  if (ws->kerr) cudaFree(ws->kerr);
  cudaGetLastError();
  delete ws;
  return RKL_OK;
}

const char *ws_last_error(const rkl_ws *ws) { return ws ? ws->err : ""; }

long long ws_kernel_launches(const rkl_ws *ws) { return ws ? ws->launches : 0; }

int ws_set_stream(rkl_ws *ws, void *cuda_stream) {
  if (!ws) return RKL_EINVAL;
  ws->stream = (cudaStream_t)cuda_stream;
  return RKL_OK;
}

int ws_set_params(rkl_ws *ws, const float *params, int n) {
  if (!ws || !params || n != ws->nparam) return RKL_EINVAL;
  const size_t pb = sizeof(float) * n;
  int rc = ws_cuda(ws, cudaMemcpyAsync(ws->param, params, pb, cudaMemcpyDefault, ws->stream));
  if (!rc) rc = ws_cuda(ws, cudaMemsetAsync(ws->m, 0, pb, ws->stream));
  if (!rc) rc = ws_cuda(ws, cudaMemsetAsync(ws->v, 0, pb, ws->stream));
  if (!rc) rc = refresh_weights(ws);
  if (!rc) rc = ws_cuda(ws, cudaStreamSynchronize(ws->stream));
  ws->step = 0;
  return rc;
}

int ws_get_params(rkl_ws *ws, float *params, int n) {
  if (!ws || !params || n != ws->nparam) return RKL_EINVAL;
  int rc = ws_cuda(ws, cudaMemcpyAsync(params, ws->param, sizeof(float) * n, cudaMemcpyDefault, ws->stream));
  if (!rc) rc = ws_cuda(ws, cudaStreamSynchronize(ws->stream));
  return rc;
}

int ws_get_grads(rkl_ws *ws, float *grads, int n) {
  if (!ws || !grads || n != ws->nparam) return RKL_EINVAL;
  int rc = ws_cuda(ws, cudaMemcpyAsync(grads, ws->grad, sizeof(float) * n, cudaMemcpyDefault, ws->stream));
  if (!rc) rc = ws_cuda(ws, cudaStreamSynchronize(ws->stream));
  return rc;
}

int ws_set_grads(rkl_ws *ws, const float *grads, int n) {
  if (!ws || !grads || n != ws->nparam) return RKL_EINVAL;
  return ws_cuda(ws, cudaMemcpyAsync(ws->grad, grads, sizeof(float) * n, cudaMemcpyDefault, ws->stream));
}

int ws_forward(rkl_ws *ws, const int box[3], int nbox, int periodic_phi, const float *in, float *out) {
  if (!ws || !valid_box(box, nbox) || !in || !out) return RKL_EINVAL;
  const Boxes g = make_boxes(box[0], box[1], box[2], nbox, periodic_phi ? 1 : 0);
  const long long cells = g.nc * nbox;
  Bufs b;
  int rc = carve(ws, cells, false, b);
  if (rc) return rc;
  k_pack_input<<<(unsigned)((cells + EW - 1) / EW), EW, 0, ws->stream>>>(cells, in, b.a0,
                                                                       tc_applies(g) ? 8 * cells : 0);
  ws->launches += 1;
  Bufs o = b;
  o.y = out;
  if ((rc = run_forward(ws, g, o))) return rc;
  return ws_cuda(ws, cudaGetLastError());
}

int ws_loss_grad(rkl_ws *ws, const int box[3], int nbox, int periodic_phi, const float *in, const float *target,
                 const float *weight, double *loss_out) {
  if (!ws || !valid_box(box, nbox) || !in || !target) return RKL_EINVAL;
  const Boxes g = make_boxes(box[0], box[1], box[2], nbox, periodic_phi ? 1 : 0);
  const long long cells = g.nc * nbox;
  Bufs b;
  int rc = carve(ws, cells, true, b);
  if (rc) return rc;
  const unsigned eg = (unsigned)((cells + EW - 1) / EW);
  const long long ss = tc_applies(g) ? 8 * cells : 0;  // planar activations on the tcgen05 path
  k_pack_input<<<eg, EW, 0, ws->stream>>>(cells, in, b.a0, ss);
  if ((rc = run_forward(ws, g, b))) return rc;
  k_sum<<<RED_BLOCKS, EW, 0, ws->stream>>>(cells, weight, ws->red);
  k_loss<<<RED_BLOCKS, EW, 0, ws->stream>>>(cells, b.y, target, weight, ws->red, RED_BLOCKS, b.dy,
                                            ws->red + RED_BLOCKS, ss);
  ws->launches += 3;
  // layer 4: dW4 from (dy, a3); dz3 = W4^T dy masked by a3 > 0
  if ((rc = launch_wgrad<32, 16>(ws, g, b.a3, b.dy, 3, ss))) return rc;
  if (tc_applies(g)) {
    if ((rc = launch_conv_tc<16, EPI_MASK>(ws, g, b.dy, ws->wuma[3], nullptr, b.a3, b.dzA))) return rc;
  } else {
    launch_conv<16, 4, EPI_MASK>(ws, g, b.dy, ws->wadj[3], nullptr, b.a3, b.dzA);
  }
  // layer 3: dW3 from (dz3, a2); dz2 = W3^T dz3 masked by a2 > 0
  if ((rc = launch_wgrad<32, 32>(ws, g, b.a2, b.dzA, 2, ss))) return rc;
  if (tc_applies(g)) {
    if ((rc = launch_conv_tc<32, EPI_MASK>(ws, g, b.dzA, ws->wuma[2], nullptr, b.a2, b.dzB))) return rc;
  } else {
    launch_conv<32, 4, EPI_MASK>(ws, g, b.dzA, ws->wadj[2], nullptr, b.a2, b.dzB);
  }
  // layer 2: dW2 from (dz2, a1); dz1 = W2^T dz2 masked by a1 > 0
  if ((rc = launch_wgrad<32, 32>(ws, g, b.a1, b.dzB, 1, ss))) return rc;
  if (tc_applies(g)) {
    if ((rc = launch_conv_tc<32, EPI_MASK>(ws, g, b.dzB, ws->wuma[1], nullptr, b.a1, b.dzA))) return rc;
  } else {
    launch_conv<32, 4, EPI_MASK>(ws, g, b.dzB, ws->wadj[1], nullptr, b.a1, b.dzA);
  }
  // layer 1: dW1 from (dz1, a0)
  if ((rc = launch_wgrad<16, 32>(ws, g, b.a0, b.dzA, 0, ss))) return rc;
  if ((rc = ws_cuda(ws, cudaGetLastError()))) return rc;
  if (loss_out) {
    std::vector<double> h(2 * RED_BLOCKS);
    rc = ws_cuda(ws, cudaMemcpyAsync(h.data(), ws->red, sizeof(double) * 2 * RED_BLOCKS, cudaMemcpyDeviceToHost,
                                     ws->stream));
    if (!rc) rc = ws_check(ws);
    if (rc) return rc;
    double wsum = 0.0, l = 0.0;
    for (int q = 0; q < RED_BLOCKS; q++) wsum += h[q];
    for (int q = 0; q < RED_BLOCKS; q++) l += h[RED_BLOCKS + q];
    *loss_out = l / wsum;
  }
  return RKL_OK;
}

int ws_adam(rkl_ws *ws, double lr) {
  if (!ws || !(lr > 0.0) || !std::isfinite(lr)) return RKL_EINVAL;
  ws->step += 1;
  const double b1 = 0.9, b2 = 0.999;
  const float c1 = (float)(1.0 - std::pow(b1, (double)ws->step));
  const float c2 = (float)(1.0 - std::pow(b2, (double)ws->step));
  k_adam<<<(ws->nparam + EW - 1) / EW, EW, 0, ws->stream>>>(ws->nparam, ws->param, ws->grad, ws->m, ws->v, (float)lr,
                                                           (float)b1, (float)(1.0 - b1), (float)b2,
                                                           (float)(1.0 - b2), 1e-8f, c1, c2);
  ws->launches += 1;
  int rc = ws_cuda(ws, cudaGetLastError());
  if (!rc) rc = refresh_weights(ws);
  return rc;
}

int ws_features(rkl_ws *ws, const rkl_grid *grid, const double *T, const double *bhat, double dt, float *feat) {
  if (!ws || !grid || grid->nr < 1 || grid->nth < 1 || grid->nph < 1 || !T || !bhat || !feat || !(dt > 0.0) ||
      !std::isfinite(dt))
    return RKL_EINVAL;
  const long long N = (long long)grid->nr * grid->nth * grid->nph;
  Bufs b;
  int rc = carve(ws, N, false, b);
  if (rc) return rc;
  k_features<<<(unsigned)((N + EW - 1) / EW), EW, 0, ws->stream>>>(N, T, bhat, (float)std::log10(dt), b.a0, feat,
                                                                   0);
  ws->launches += 1;
  return ws_cuda(ws, cudaGetLastError());
}

int ws_guess(rkl_ws *ws, const rkl_grid *grid, const double *T, const double *bhat, double dt, double scale,
             double *x0) {
  if (!ws || !grid || grid->nr < 1 || grid->nth < 1 || grid->nph < 1 || !T || !bhat || !x0 || !(dt > 0.0) ||
      !std::isfinite(dt) || !std::isfinite(scale))
    return RKL_EINVAL;
  const long long N = (long long)grid->nr * grid->nth * grid->nph;
  const Boxes g = make_boxes(grid->nr, grid->nth, grid->nph, 1, 1);
  Bufs b;
  int rc = carve(ws, N, false, b);
  if (rc) return rc;
  const unsigned eg = (unsigned)((N + EW - 1) / EW);
  k_features<<<eg, EW, 0, ws->stream>>>(N, T, bhat, (float)std::log10(dt), b.a0, nullptr, tc_applies(g) ? 8 * N : 0);
  if ((rc = run_forward(ws, g, b))) return rc;
  k_guess<<<eg, EW, 0, ws->stream>>>(N, T, b.y, scale, x0);
  ws->launches += 2;
  return ws_cuda(ws, cudaGetLastError());
}

int ws_check(rkl_ws *ws) {
  if (!ws) return RKL_EINVAL;
  int flag = 0;
  int rc = ws_cuda(ws, cudaMemcpyAsync(&flag, ws->kerr, sizeof(int), cudaMemcpyDeviceToHost, ws->stream));
  if (!rc) rc = ws_cuda(ws, cudaStreamSynchronize(ws->stream));
  if (rc) return rc;
  if (flag) {
    snprintf(ws->err, sizeof(ws->err), "%s",
             "a tensor-core convolution gave up waiting for its MMAs; its outputs are not valid");
    rc = ws_cuda(ws, cudaMemsetAsync(ws->kerr, 0, sizeof(int), ws->stream));
    return rc ? rc : RKL_ECUDA;
  }
  return RKL_OK;
}

int ws_target(rkl_ws *ws, long long n, const double *x, const double *base, double unit, float *target) {
  if (!ws || n < 1 || !x || !base || !target || !(unit > 0.0) || !std::isfinite(unit)) return RKL_EINVAL;
  k_target<<<(unsigned)((n + EW - 1) / EW), EW, 0, ws->stream>>>(n, x, base, 1.0 / unit, target);
  ws->launches += 1;
  return ws_cuda(ws, cudaGetLastError());
}

}  // extern "C"
