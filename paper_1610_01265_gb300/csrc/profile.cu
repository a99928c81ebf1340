// profile.cu -- optional per-kernel timing with CUDA events on the context's stream.
//
// When enabled, every launch (or the three set-up kernels together) is bracketed by a
// pair of events recorded on the context's stream.  Records are settled at the host
// synchronisation points the library already has (PCG status reads, set_coeffs) or when
// the caller reads the counters.  PCG iterations are queued in chunks and the kernels
// of iterations past convergence return at once; those launches are recognised from the
// iteration count read back after the chunk and are not counted, so the per-launch
// average of a kernel is the duration of launches that did the work.
//
// rkl_fp64_peak measures the device's FP64 FMA throughput, the roof of the FP64 stencil
// kernels on this part.
#include <cuda_runtime.h>

#include "internal.cuh"

namespace rkl {

static cudaEvent_t take_event(rkl_ctx *ctx) {
  if (!ctx->ev_pool.empty()) {
    cudaEvent_t e = ctx->ev_pool.back();
    ctx->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

ProfScope::ProfScope(rkl_ctx *c, int k, int t) : ctx(c), kind(k), tag(t), a(nullptr) {
  if (!ctx->prof_on) return;
  a = take_event(ctx);
  if (a) cudaEventRecord(a, ctx->stream);
}

ProfScope::~ProfScope() {
  if (!ctx->prof_on || !a) return;
  cudaEvent_t b = take_event(ctx);
  if (!b) {
    ctx->ev_pool.push_back(a);
    return;
  }
  cudaEventRecord(b, ctx->stream);
  ctx->prof_pending.push_back({kind, tag, a, b});
  if (ctx->prof_pending.size() > 16384) prof_settle(ctx, 0, false, false);
}

// Accumulate pending records (the stream is synchronised first).  Records tagged with an
// iteration index q >= 0 belong to the PCG chunk just read back (chunk = true): n_real
// iterations of it did work, and the p-update of the last of them did not run when the
// solve ended there.  Outside a chunk settlement, tagged records are left pending.
void prof_settle(rkl_ctx *ctx, int n_real, bool still_running, bool chunk) {
  if (ctx->prof_pending.empty()) return;
  cudaStreamSynchronize(ctx->stream);
  std::vector<ProfRec> left;
  for (const ProfRec &r : ctx->prof_pending) {
    bool keep = true;
    if (r.tag >= 0) {
      if (!chunk) {
        left.push_back(r);
        continue;
      }
      keep = r.tag < n_real;
      if (r.kind == RKL_K_PCG_PUPDATE && r.tag == n_real - 1 && !still_running) keep = false;
    }
    float ms = 0.0f;
    if (keep && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      ctx->prof_ms[r.kind] += ms;
      ctx->prof_n[r.kind] += 1;
    }
    cudaGetLastError();
    ctx->ev_pool.push_back(r.a);
    ctx->ev_pool.push_back(r.b);
  }
  ctx->prof_pending.swap(left);
}

void prof_release(rkl_ctx *ctx) {
  for (const ProfRec &r : ctx->prof_pending) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  ctx->prof_pending.clear();
  for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
  ctx->ev_pool.clear();
}

namespace {

constexpr int PEAK_CHAINS = 8;    // independent FMA chains per thread
constexpr int PEAK_THREADS = 256;

// PEAK_CHAINS independent a <- a * b + c chains per thread (b < 1: every chain converges to
// c / (1 - b), so the values stay finite); the sums are stored so that no chain is dead code.
// b and c are moved into registers first (an FMA whose operands come from the constant
// bank does not issue at the full FP64 rate).
__global__ void __launch_bounds__(PEAK_THREADS) k_dfma_peak(int iters, double b_in, double c_in, double *out) {
  const double b = __shfl_sync(0xffffffffu, b_in, 0), c = __shfl_sync(0xffffffffu, c_in, 0);
  double a[PEAK_CHAINS];
#pragma unroll
  for (int q = 0; q < PEAK_CHAINS; q++) a[q] = 1e-3 * threadIdx.x + q;
#pragma unroll 4
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int q = 0; q < PEAK_CHAINS; q++) a[q] = fma(a[q], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < PEAK_CHAINS; q++) s += a[q];
  out[(size_t)blockIdx.x * PEAK_THREADS + threadIdx.x] = s;
}

}  // namespace

}  // namespace rkl

using namespace rkl;

extern "C" int rkl_fp64_peak(void *cuda_stream, double *tflops_out) {
  if (!tflops_out) return RKL_EINVAL;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1) {
    cudaGetLastError();
    return RKL_ECUDA;
  }
  const unsigned grid = (unsigned)nsm * 8;  // 8 CTAs of 256 threads per SM
  const int iters = 16384;
  double *out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = RKL_OK;
  if (cudaMalloc(&out, (size_t)grid * PEAK_THREADS * sizeof(double)) != cudaSuccess || !out) rc = RKL_ENOMEM;
  if (!rc && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) rc = RKL_ECUDA;
  float best = 0.0f;
  if (!rc) {
    k_dfma_peak<<<grid, PEAK_THREADS, 0, st>>>(iters / 8, 0.999999, 1e-6, out);  // warm-up
    for (int rep = 0; rep < 3 && !rc; rep++) {
      cudaEventRecord(e0, st);
      k_dfma_peak<<<grid, PEAK_THREADS, 0, st>>>(iters, 0.999999, 1e-6, out);
      cudaEventRecord(e1, st);
      float ms = 0.0f;
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
        rc = RKL_ECUDA;
      else if (ms > 0.0f && (best == 0.0f || ms < best))
        best = ms;
    }
  }
  if (!rc && cudaGetLastError() != cudaSuccess) rc = RKL_ECUDA;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (out) cudaFree(out);
  cudaGetLastError();
  if (rc) return rc;
  if (!(best > 0.0f)) return RKL_ECUDA;
  const double flop = 2.0 * PEAK_CHAINS * (double)iters * grid * PEAK_THREADS;
  *tflops_out = flop / (best * 1e-3) / 1e12;
  return RKL_OK;
}

extern "C" int rkl_profile_enable(rkl_ctx *ctx, int on) {
  if (!ctx) return RKL_EINVAL;
  prof_settle(ctx, 0, false, false);
  for (int k = 0; k < RKL_K_COUNT; k++) {
    ctx->prof_ms[k] = 0.0;
    ctx->prof_n[k] = 0;
  }
  ctx->prof_on = on ? 1 : 0;
  return RKL_OK;
}

extern "C" int rkl_profile_read(rkl_ctx *ctx, int kernel, double *total_ms, long long *launches) {
  if (!ctx || kernel < 0 || kernel >= RKL_K_COUNT) return RKL_EINVAL;
  prof_settle(ctx, 0, false, false);
  if (total_ms) *total_ms = ctx->prof_ms[kernel];
  if (launches) *launches = ctx->prof_n[kernel];
  return RKL_OK;
}
