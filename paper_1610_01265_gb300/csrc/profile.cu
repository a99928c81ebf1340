// profile.cu -- optional per-kernel timing with CUDA events on the context's stream.
//
// When enabled, every launch (or the three set-up kernels together) is bracketed by a
// pair of events recorded on the context's stream.  Records are settled at the host
// synchronisation points the library already has (PCG status reads, set_coeffs) or when
// the caller reads the counters.  PCG iterations are queued in chunks and the kernels
// of iterations past convergence return at once; those launches are recognised from the
// iteration count read back after the chunk and are not counted, so the per-launch
// average of a kernel is the duration of launches that did the work.
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

}  // namespace rkl

using namespace rkl;

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
