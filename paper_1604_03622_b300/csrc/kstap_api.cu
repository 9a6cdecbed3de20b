// libkstap: C ABI (include/kstap.h) over the Kron-STAP kernels.
#include <cuda_runtime.h>

#include <cmath>
#include <complex>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/kstap.h"
#include "kstap_kernels.cuh"

using kstap::Geom;

struct kstap_ctx {
  kstap_params prm;
  int V = 0;
  cudaStream_t stream = nullptr;
  size_t budget = 0;
  int device = 0;
  // bank, transposed for the detect kernel: aT [p][V], bT [q][V], norms [2V]
  float2* bank_aT = nullptr;
  float2* bank_bT = nullptr;
  float* bank_n2 = nullptr;
  // workspace
  void* ws = nullptr;
  size_t ws_bytes = 0;
  std::string err;
  // optional per-kernel timing: events around every launch on ctx->stream
  bool profile = false;
  cudaEvent_t ev[kstap_nkernels + 1][2] = {};
  float kernel_ms[kstap_nkernels] = {};
  int kernel_launches[kstap_nkernels] = {};
  bool ev_pending[kstap_nkernels] = {};
};

namespace {

thread_local std::string g_create_err;

// Records the start event of kernel `k` (profiling mode only).
void prof_begin(kstap_ctx* ctx, int k) {
  if (!ctx->profile) return;
  if (!ctx->ev[k][0]) {
    cudaEventCreate(&ctx->ev[k][0]);
    cudaEventCreate(&ctx->ev[k][1]);
  }
  cudaEventRecord(ctx->ev[k][0], ctx->stream);
}

// Records the end event of kernel `k`; the elapsed time is collected lazily.
void prof_end(kstap_ctx* ctx, int k) {
  if (!ctx->profile) return;
  cudaEventRecord(ctx->ev[k][1], ctx->stream);
  ctx->ev_pending[k] = true;
}

// Folds finished launches into the per-kernel totals (synchronises on each
// pending end event; called before the next launch of the same kernel and by
// kstap_kernel_times).
void prof_collect(kstap_ctx* ctx, int k) {
  if (!ctx->ev_pending[k]) return;
  cudaEventSynchronize(ctx->ev[k][1]);
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, ctx->ev[k][0], ctx->ev[k][1]) == cudaSuccess) {
    ctx->kernel_ms[k] += ms;
    ctx->kernel_launches[k] += 1;
  }
  ctx->ev_pending[k] = false;
}

kstap_status fail(kstap_ctx* ctx, kstap_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (ctx)
    ctx->err = buf;
  else
    g_create_err = buf;
  return st;
}

#define KSTAP_CUDA(ctx, call)                                                            \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return fail((ctx), KSTAP_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));   \
  } while (0)

int ceil_log2(long v) {
  int k = 0;
  while ((1L << k) < v) ++k;
  return k;
}

bool valid_params(const kstap_params* p, std::string& why) {
  if (!p) {
    why = "params is NULL";
    return false;
  }
  if (p->p != 3) {
    why = "this build supports p == 3";
    return false;
  }
  if (p->q != 8 && p->q != 16 && p->q != 32) {
    why = "q must be 8, 16 or 32";
    return false;
  }
  if (p->r_a != 1) {
    why = "r_a must be 1 (rank-one spatial clutter model)";
    return false;
  }
  if (p->r_b < 1 || p->r_b > kstap::kRbMax || p->r_b >= p->q) {
    why = "r_b must satisfy 1 <= r_b <= 4 and r_b < q";
    return false;
  }
  if (p->ring_r < 0 || p->ring_a < 0 || p->guard_r < 0 || p->guard_a < 0 ||
      p->guard_r > p->ring_r || p->guard_a > p->ring_a) {
    why = "need ring >= guard >= 0";
    return false;
  }
  if (p->ring_r > 12 || p->ring_a > 24) {
    why = "ring_r <= 12 and ring_a <= 24 in this build";
    return false;
  }
  const long nbox = (2L * p->ring_r + 1) * (2L * p->ring_a + 1);
  const long n = nbox - (2L * p->guard_r + 1) * (2L * p->guard_a + 1);
  if (n < 1) {
    why = "training ring is empty (n < 1)";
    return false;
  }
  if (nbox > 1024) {
    why = "(2 ring_r + 1)(2 ring_a + 1) must be <= 1024";
    return false;
  }
  return true;
}

Geom make_geom(const kstap_ctx* ctx, int H_in, int W_in) {
  const kstap_params& p = ctx->prm;
  Geom g;
  g.p = p.p;
  g.q = p.q;
  g.r_a = p.r_a;
  g.r_b = p.r_b;
  g.Rr = p.ring_r;
  g.Ra = p.ring_a;
  g.Gr = p.guard_r;
  g.Ga = p.guard_a;
  g.H_in = H_in;
  g.W_in = W_in;
  g.H = H_in - 2 * p.ring_r;
  g.W = W_in - 2 * p.ring_a - p.q + 1;
  const long nbox = (2L * p.ring_r + 1) * (2L * p.ring_a + 1);
  g.n = (int)(nbox - (2L * p.guard_r + 1) * (2L * p.guard_a + 1));
  g.V = ctx->V;
  // |Y| < 2^B per component keeps every box sum of products below 2^62:
  // 2B + 1 + ceil(log2(nbox)) <= 62.
  g.B = (61 - ceil_log2(nbox)) / 2;
  if (g.B > 26) g.B = 26;
  g.max_iter = p.max_iter > 0 ? p.max_iter : 64;
  g.eps = p.eps > 0 ? (float)p.eps : 2e-6f;
  g.tau = p.tau;
  g.tc = (p.q >= 32) ? 16 : kstap::kTileCells;
  return g;
}

// workspace layout (struct of arrays per cell, plus the optional lag store)
struct WsLayout {
  size_t flags, Mw, Sw, aw, Lw, total;
};

WsLayout ws_layout(int p, int q, size_t H, size_t W, bool lag_store) {
  const size_t PP = (size_t)p * p, NE = PP * (PP + 1) / 2, ncell = H * W;
  auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
  WsLayout L;
  L.flags = 0;
  L.Mw = 256;
  L.Sw = up(L.Mw + ncell * NE * sizeof(float2));
  L.aw = up(L.Sw + ncell * PP * sizeof(float2));
  L.Lw = up(L.aw + ncell * PP * sizeof(float2));
  L.total = L.Lw + (lag_store ? up(H * q * PP * (W + q - 1) * sizeof(float4)) : 0);
  return L;
}

size_t smem_moments(const Geom& g) {
  const int P = g.p, PP = P * P, TC = kstap::kTileCells, TR = kstap::kMomRows;
  const int NRT = 2 * g.Rr + TR, WT = TC + 2 * g.Ra + g.q - 1, NUmax = TC + g.q - 1;
  size_t b = (size_t)P * NRT * WT * 8;
  b += (b & 15);
  b += 2 * (size_t)PP * WT * 16;
  b += (size_t)TR * PP * NUmax * 8;
  return b;
}

size_t smem_bfit(const Geom& g, bool from_store) {
  const int P = g.p, PP = P * P, Q = g.q, TC = g.tc, R = g.r_b;
  const int NR = 2 * g.Rr + 1, WT = TC + 2 * g.Ra + Q - 1, NUmax = TC + Q - 1;
  size_t b = (size_t)TC * (Q * (Q + 1) / 2) * 16;
  b += (size_t)TC * PP * 8;
  // the eigen phase's basis scratch reuses the (then dead) lag and box-sum buffers
  const size_t vs = (size_t)(kstap::kThreads / 32) * (32 / Q) * Q * R * 8;
  const size_t lagb = (size_t)PP * NUmax * 16 + (from_store ? 0 : 2 * (size_t)PP * WT * 16);
  b += std::max(vs, lagb);
  if (!from_store) b += (size_t)P * NR * WT * 8;
  return b;
}

size_t smem_detect(const Geom& g) {
  const int P = g.p, Q = g.q, V = g.V, R = g.r_b;
  const size_t CS = 2 * (size_t)P * Q + 2 * (size_t)Q * R + 2 * P + 2 * (size_t)P * R;
  const size_t cells = (kstap::kThreads / 32) * (32 / Q);
  return (size_t)(P + Q) * V * 8 + 2 * (size_t)V * 4 + cells * CS * 8;
}

// Enqueues the fit (scale, moments, flip-flop, B / U_B) on stream s with the
// given scratch; ctx (may be NULL) receives errors and profiling events.
template <int P, int Q, int R>
kstap_status enqueue_fit(kstap_ctx* ctx, const Geom& g, const float2* Y, char* scratch,
                         const WsLayout& L, bool lag_store, const kstap_factors* f,
                         cudaStream_t s) {
  unsigned* maxbits = (unsigned*)(scratch + L.flags);
  float4* Lw = lag_store ? (float4*)(scratch + L.Lw) : nullptr;
  float2* Mw = (float2*)(scratch + L.Mw);
  float2* Sw = (float2*)(scratch + L.Sw);
  float2* aw = (float2*)(scratch + L.aw);
  const size_t ncell = (size_t)g.H * g.W;
  KSTAP_CUDA(ctx, cudaMemsetAsync(maxbits, 0, 8, s));   // the scale words must start at zero
  const size_t nfloat = 2 * (size_t)g.p * g.H_in * g.W_in;
  int blocks = (int)std::min<size_t>((nfloat + 1023) / 1024, 148 * 16);
  if (blocks < 1) blocks = 1;
  if (ctx) prof_collect(ctx, KSTAP_K_SCALE), prof_begin(ctx, KSTAP_K_SCALE);
  kstap::k_frame_maxabs<<<blocks, 256, 0, s>>>((const float*)Y, nfloat, maxbits, maxbits + 1);
  if (ctx) prof_end(ctx, KSTAP_K_SCALE);
  KSTAP_CUDA(ctx, cudaGetLastError());

  const size_t sm1 = smem_moments(g);
  KSTAP_CUDA(ctx, cudaFuncSetAttribute(kstap::k_moments<P, Q>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1));
  dim3 grid1((g.W + kstap::kTileCells - 1) / kstap::kTileCells,
             (g.H + kstap::kMomRows - 1) / kstap::kMomRows);
  if (ctx) prof_collect(ctx, KSTAP_K_MOMENTS), prof_begin(ctx, KSTAP_K_MOMENTS);
  kstap::k_moments<P, Q><<<grid1, kstap::kMomThreads, sm1, s>>>(Y, g, maxbits, Mw, Sw, Lw);
  if (ctx) prof_end(ctx, KSTAP_K_MOMENTS);
  KSTAP_CUDA(ctx, cudaGetLastError());

  if (ctx) prof_collect(ctx, KSTAP_K_FLIPFLOP), prof_begin(ctx, KSTAP_K_FLIPFLOP);
  kstap::k_flipflop<P><<<(unsigned)((ncell + 127) / 128), 128, 0, s>>>(
      Mw, Sw, g, ncell, aw, (float2*)f->UA, f->lamA, f->iters, f->eta);
  if (ctx) prof_end(ctx, KSTAP_K_FLIPFLOP);
  KSTAP_CUDA(ctx, cudaGetLastError());

  const size_t sm3 = smem_bfit(g, lag_store);
  auto kb = lag_store ? kstap::k_bfit<P, Q, R, true> : kstap::k_bfit<P, Q, R, false>;
  KSTAP_CUDA(ctx, cudaFuncSetAttribute(kb, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm3));
  dim3 grid3((g.W + g.tc - 1) / g.tc, g.H);
  if (ctx) prof_collect(ctx, KSTAP_K_BFIT), prof_begin(ctx, KSTAP_K_BFIT);
  kb<<<grid3, kstap::kThreads, sm3, s>>>(Y, g, maxbits, aw, Lw, (float2*)f->UB_hi,
                                          (float2*)f->UB_lo, f->lamB);
  if (ctx) prof_end(ctx, KSTAP_K_BFIT);
  KSTAP_CUDA(ctx, cudaGetLastError());
  return KSTAP_OK;
}

kstap_status dispatch_fit(kstap_ctx* ctx, const Geom& g, const float2* Y, char* scratch,
                          const WsLayout& L, bool lag_store, const kstap_factors* f,
                          cudaStream_t s) {
#define KSTAP_FIT(QQ, RR)        \
  if (g.q == QQ && g.r_b == RR) \
    return enqueue_fit<3, QQ, RR>(ctx, g, Y, scratch, L, lag_store, f, s);
  KSTAP_FIT(8, 1) KSTAP_FIT(8, 2) KSTAP_FIT(8, 3) KSTAP_FIT(8, 4)
  KSTAP_FIT(16, 1) KSTAP_FIT(16, 2) KSTAP_FIT(16, 3) KSTAP_FIT(16, 4)
  KSTAP_FIT(32, 1) KSTAP_FIT(32, 2) KSTAP_FIT(32, 3) KSTAP_FIT(32, 4)
#undef KSTAP_FIT
  return fail(ctx, KSTAP_EINVAL, "unsupported (q, r_b)");
}

template <int P, int Q, int R>
kstap_status launch_detect(kstap_ctx* ctx, const Geom& g, const float2* Y, const kstap_factors* f,
                           float* Tmax, int32_t* vidx, uint8_t* map, float* T_all) {
  const size_t ncell = (size_t)g.H * g.W;
  const size_t sm = smem_detect(g);
  KSTAP_CUDA(ctx, cudaFuncSetAttribute(kstap::k_detect<P, Q, R>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  const size_t per_block = (kstap::kThreads / 32) * (32 / Q);
  const unsigned grid = (unsigned)((ncell + per_block - 1) / per_block);
  prof_collect(ctx, KSTAP_K_DETECT);
  prof_begin(ctx, KSTAP_K_DETECT);
  kstap::k_detect<P, Q, R><<<grid, kstap::kThreads, sm, ctx->stream>>>(
      Y, g, ctx->bank_aT, ctx->bank_bT, ctx->bank_n2, (const float2*)f->UA,
      (const float2*)f->UB_hi, (const float2*)f->UB_lo, Tmax, vidx, map, T_all);
  prof_end(ctx, KSTAP_K_DETECT);
  KSTAP_CUDA(ctx, cudaGetLastError());
  return KSTAP_OK;
}

kstap_status check_frame(kstap_ctx* ctx, const kstap_c64* Y, int H_in, int W_in) {
  if (!ctx) return KSTAP_EINVAL;
  if (!Y) return fail(ctx, KSTAP_EINVAL, "Y is NULL");
  const kstap_params& p = ctx->prm;
  if (H_in < 2 * p.ring_r + 1 || W_in < 2 * p.ring_a + p.q)
    return fail(ctx, KSTAP_EINVAL, "frame %dx%d smaller than the training box plus window", H_in,
                W_in);
  if ((size_t)p.p * H_in * W_in > ((size_t)1 << 40))
    return fail(ctx, KSTAP_EINVAL, "frame too large");
  return KSTAP_OK;
}

}  // namespace

extern "C" {

size_t kstap_workspace_bytes(const kstap_params* params, int H_in, int W_in) {
  std::string why;
  if (!valid_params(params, why)) return 0;
  const long H = H_in - 2L * params->ring_r;
  const long W = W_in - 2L * params->ring_a - params->q + 1;
  if (H < 1 || W < 1) return 0;
  return ws_layout(params->p, params->q, (size_t)H, (size_t)W, true).total;
}

kstap_status kstap_create(const kstap_params* params, const kstap_c64* bank_a,
                          const kstap_c64* bank_b, int V, size_t hbm_budget_bytes,
                          void* cuda_stream, kstap_ctx** out) {
  if (!out) return fail(nullptr, KSTAP_EINVAL, "out is NULL");
  *out = nullptr;
  std::string why;
  if (!valid_params(params, why)) return fail(nullptr, KSTAP_EINVAL, "%s", why.c_str());
  if (V < 1 || V > 256) return fail(nullptr, KSTAP_EINVAL, "V must be in [1, 256]");
  if (!bank_a || !bank_b) return fail(nullptr, KSTAP_EINVAL, "bank is NULL");
  kstap_ctx* ctx = new kstap_ctx();
  ctx->prm = *params;
  ctx->V = V;
  ctx->stream = (cudaStream_t)cuda_stream;
  ctx->budget = hbm_budget_bytes;
  cudaGetDevice(&ctx->device);
  const int p = params->p, q = params->q;
  std::vector<kstap_c64> ha((size_t)V * p), hb((size_t)V * q);
  cudaError_t e = cudaMemcpy(ha.data(), bank_a, ha.size() * sizeof(kstap_c64), cudaMemcpyDefault);
  if (e == cudaSuccess)
    e = cudaMemcpy(hb.data(), bank_b, hb.size() * sizeof(kstap_c64), cudaMemcpyDefault);
  if (e != cudaSuccess) {
    delete ctx;
    return fail(nullptr, KSTAP_ECUDA, "copying the bank failed: %s", cudaGetErrorString(e));
  }
  std::vector<float2> aT((size_t)p * V), bT((size_t)q * V);
  std::vector<float> n2(2 * (size_t)V);
  for (int v = 0; v < V; ++v) {
    double sa = 0, sb = 0;
    for (int i = 0; i < p; ++i) {
      const kstap_c64 z = ha[(size_t)v * p + i];
      aT[(size_t)i * V + v] = make_float2(z.re, z.im);
      sa += (double)z.re * z.re + (double)z.im * z.im;
    }
    for (int j = 0; j < q; ++j) {
      const kstap_c64 z = hb[(size_t)v * q + j];
      bT[(size_t)j * V + v] = make_float2(z.re, z.im);
      sb += (double)z.re * z.re + (double)z.im * z.im;
    }
    n2[v] = (float)sa;
    n2[V + v] = (float)sb;
  }
  e = cudaMalloc(&ctx->bank_aT, aT.size() * sizeof(float2));
  if (e == cudaSuccess) e = cudaMalloc(&ctx->bank_bT, bT.size() * sizeof(float2));
  if (e == cudaSuccess) e = cudaMalloc(&ctx->bank_n2, n2.size() * sizeof(float));
  if (e == cudaSuccess)
    e = cudaMemcpy(ctx->bank_aT, aT.data(), aT.size() * sizeof(float2), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(ctx->bank_bT, bT.data(), bT.size() * sizeof(float2), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(ctx->bank_n2, n2.data(), n2.size() * sizeof(float), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    kstap_destroy(ctx);
    return fail(nullptr, KSTAP_ECUDA, "bank upload failed: %s", cudaGetErrorString(e));
  }
  *out = ctx;
  return KSTAP_OK;
}

kstap_status kstap_fit_project(kstap_ctx* ctx, const kstap_c64* Y, int H_in, int W_in,
                               const kstap_factors* factors) {
  kstap_status st = check_frame(ctx, Y, H_in, W_in);
  if (st != KSTAP_OK) return st;
  if (!factors || !factors->UA || !factors->UB_hi || !factors->UB_lo)
    return fail(ctx, KSTAP_EINVAL, "factors (UA, UB_hi, UB_lo) must be non-NULL");
  const Geom g = make_geom(ctx, H_in, W_in);
  const size_t ncell = (size_t)g.H * g.W;
  const WsLayout L = ws_layout(g.p, g.q, g.H, g.W, true);
  if (L.total > ctx->ws_bytes) {
    if (ctx->budget && L.total > ctx->budget)
      return fail(ctx, KSTAP_ENOMEM, "workspace %zu B exceeds the HBM budget %zu B", L.total,
                  ctx->budget);
    if (ctx->ws) {
      KSTAP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
      cudaFree(ctx->ws);
      ctx->ws = nullptr;
      ctx->ws_bytes = 0;
    }
    cudaError_t e = cudaMalloc(&ctx->ws, L.total);
    if (e != cudaSuccess)
      return fail(ctx, KSTAP_ENOMEM, "workspace cudaMalloc(%zu) failed: %s", L.total,
                  cudaGetErrorString(e));
    ctx->ws_bytes = L.total;
  }
  return dispatch_fit(ctx, g, (const float2*)Y, (char*)ctx->ws, L, true, factors, ctx->stream);
}

kstap_status kstap_detect(kstap_ctx* ctx, const kstap_c64* Y, int H_in, int W_in,
                          const kstap_factors* factors, float* Tmax, int32_t* vidx, uint8_t* map,
                          float* T_all) {
  kstap_status st = check_frame(ctx, Y, H_in, W_in);
  if (st != KSTAP_OK) return st;
  if (!factors || !factors->UA || !factors->UB_hi || !factors->UB_lo)
    return fail(ctx, KSTAP_EINVAL, "factors (UA, UB_hi, UB_lo) must be non-NULL");
  if (!Tmax || !vidx || !map) return fail(ctx, KSTAP_EINVAL, "Tmax, vidx and map are required");
  const Geom g = make_geom(ctx, H_in, W_in);
  const float2* Yf = (const float2*)Y;
#define KSTAP_DET(QQ, RR)                                                                 \
  if (g.q == QQ && g.r_b == RR) return launch_detect<3, QQ, RR>(ctx, g, Yf, factors, Tmax, vidx, \
                                                                map, T_all);
  KSTAP_DET(8, 1) KSTAP_DET(8, 2) KSTAP_DET(8, 3) KSTAP_DET(8, 4)
  KSTAP_DET(16, 1) KSTAP_DET(16, 2) KSTAP_DET(16, 3) KSTAP_DET(16, 4)
  KSTAP_DET(32, 1) KSTAP_DET(32, 2) KSTAP_DET(32, 3) KSTAP_DET(32, 4)
#undef KSTAP_DET
  return fail(ctx, KSTAP_EINVAL, "unsupported q");
}

kstap_status kstap_set_profiling(kstap_ctx* ctx, int enable) {
  if (!ctx) return KSTAP_EINVAL;
  for (int k = 0; k < kstap_nkernels; ++k) {
    prof_collect(ctx, k);
    ctx->kernel_ms[k] = 0.f;
    ctx->kernel_launches[k] = 0;
  }
  ctx->profile = enable != 0;
  return KSTAP_OK;
}

kstap_status kstap_kernel_times(kstap_ctx* ctx, float* total_ms, int32_t* launches, int n) {
  if (!ctx || n < 0) return KSTAP_EINVAL;
  for (int k = 0; k < kstap_nkernels; ++k) prof_collect(ctx, k);
  for (int k = 0; k < n && k < kstap_nkernels; ++k) {
    if (total_ms) total_ms[k] = ctx->kernel_ms[k];
    if (launches) launches[k] = ctx->kernel_launches[k];
  }
  return KSTAP_OK;
}

kstap_status kstap_destroy(kstap_ctx* ctx) {
  if (!ctx) return KSTAP_EINVAL;
  if (ctx->ws || ctx->bank_aT) cudaStreamSynchronize(ctx->stream);
  for (int k = 0; k <= kstap_nkernels; ++k)
    if (ctx->ev[k][0]) {
      cudaEventDestroy(ctx->ev[k][0]);
      cudaEventDestroy(ctx->ev[k][1]);
    }
  cudaFree(ctx->ws);
  cudaFree(ctx->bank_aT);
  cudaFree(ctx->bank_bT);
  cudaFree(ctx->bank_n2);
  delete ctx;
  return KSTAP_OK;
}

const char* kstap_last_error(const kstap_ctx* ctx) {
  return ctx ? ctx->err.c_str() : g_create_err.c_str();
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free fit (kstap_fit_project_noalloc).  Its scratch -- the frame
// scale word and the per-cell moments M, block sums and flip-flop factor a --
// lives in this file-scope device array instead of a cudaMalloc'd workspace.
// Host code must not pass the array's name to a kernel: on the host it is only
// a stand-in symbol.  The device address is looked up once per device with
// cudaGetSymbolAddress and cached.
// ---------------------------------------------------------------------------
#define KSTAP_NOALLOC_MAX_CELLS 32768
#define KSTAP_NOALLOC_SCRATCH_BYTES (256 + (size_t)KSTAP_NOALLOC_MAX_CELLS * (45 + 9 + 9) * 8 + 1024)

static __device__ __align__(256) unsigned char g_noalloc_scratch[KSTAP_NOALLOC_SCRATCH_BYTES];

#include <mutex>

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device (looked up on
// the first call per device).
kstap_status noalloc_scratch(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess)
    return fail(nullptr, KSTAP_ECUDA, "cudaGetDevice failed: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices)
    return fail(nullptr, KSTAP_EINVAL, "device index %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return fail(nullptr, KSTAP_ECUDA, "cudaGetSymbolAddress(scratch) failed: %s",
                  cudaGetErrorString(e));
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return KSTAP_OK;
}

Geom noalloc_geom(const kstap_params& p, int H_in, int W_in) {
  Geom g;
  g.p = p.p;
  g.q = p.q;
  g.r_a = p.r_a;
  g.r_b = p.r_b;
  g.Rr = p.ring_r;
  g.Ra = p.ring_a;
  g.Gr = p.guard_r;
  g.Ga = p.guard_a;
  g.H_in = H_in;
  g.W_in = W_in;
  g.H = H_in - 2 * p.ring_r;
  g.W = W_in - 2 * p.ring_a - p.q + 1;
  const long nbox = (2L * p.ring_r + 1) * (2L * p.ring_a + 1);
  g.n = (int)(nbox - (2L * p.guard_r + 1) * (2L * p.guard_a + 1));
  g.V = 0;
  g.B = (61 - ceil_log2(nbox)) / 2;
  if (g.B > 26) g.B = 26;
  g.max_iter = p.max_iter > 0 ? p.max_iter : 64;
  g.eps = p.eps > 0 ? (float)p.eps : 2e-6f;
  g.tau = p.tau;
  g.tc = (p.q >= 32) ? 16 : kstap::kTileCells;
  return g;
}

}  // namespace

extern "C" kstap_status kstap_fit_project_noalloc(const kstap_params* params, const kstap_c64* Y,
                                                  int H_in, int W_in,
                                                  const kstap_factors* factors,
                                                  void* cuda_stream) {
  std::string why;
  if (!valid_params(params, why)) return fail(nullptr, KSTAP_EINVAL, "%s", why.c_str());
  if (!Y) return fail(nullptr, KSTAP_EINVAL, "Y is NULL");
  if (!factors || !factors->UA || !factors->UB_hi || !factors->UB_lo)
    return fail(nullptr, KSTAP_EINVAL, "factors (UA, UB_hi, UB_lo) must be non-NULL");
  if (H_in < 2 * params->ring_r + 1 || W_in < 2 * params->ring_a + params->q)
    return fail(nullptr, KSTAP_EINVAL, "frame %dx%d smaller than the training box plus window",
                H_in, W_in);
  const Geom g = noalloc_geom(*params, H_in, W_in);
  const size_t ncell = (size_t)g.H * g.W;
  if (ncell > KSTAP_NOALLOC_MAX_CELLS)
    return fail(nullptr, KSTAP_EINVAL,
                "frame has %zu cells; kstap_fit_project_noalloc handles at most %d cells "
                "(use kstap_fit_project, or split the frame into tiles)",
                ncell, KSTAP_NOALLOC_MAX_CELLS);
  const WsLayout L = ws_layout(g.p, g.q, g.H, g.W, false);
  if (L.total > KSTAP_NOALLOC_SCRATCH_BYTES)
    return fail(nullptr, KSTAP_EINVAL, "scratch layout %zu B exceeds the static %zu B", L.total,
                (size_t)KSTAP_NOALLOC_SCRATCH_BYTES);
  void* scratch = nullptr;
  kstap_status st = noalloc_scratch(&scratch);
  if (st != KSTAP_OK) return st;
  return dispatch_fit(nullptr, g, (const float2*)Y, (char*)scratch, L, false, factors,
                      (cudaStream_t)cuda_stream);
}
