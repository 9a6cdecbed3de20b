// Kernel launch sequences of the fit and detect passes, instantiated per
// class (p, q) and r_b by kstap_inst.cu.
#pragma once
#include "kstap_host.cuh"

namespace kh {

// Enqueues the fit (scale, moments, flip-flop, B / U_B) of all jobs of JL.
template <int P, int Q, int R>
kstap_status enqueue_fit(kstap_ctx* ctx, kstap_ctx* prof, const Geom& g, const JobList& JL,
                         char* scratch, const Layout& L, bool lag_store, int sm_count, int waves,
                         cudaStream_t s) {
  float2* Mw = (float2*)(scratch + L.Mw);
  float2* Sw = (float2*)(scratch + L.Sw);
  float2* aw = (float2*)(scratch + L.aw);
  float4* Lw = lag_store ? (float4*)(scratch + L.Lw) : nullptr;
  if (JL.njobs < 1) return KSTAP_OK;
  KSTAP_CUDA(ctx, cudaMemsetAsync(scratch + L.flags, 0, 8 * (size_t)JL.njobs, s));
  kstap_status st = enqueue_scan(ctx, prof, g, JL, sm_count, s);
  if (st != KSTAP_OK) return st;

  const size_t sm1 = smem_moments(g);
  KSTAP_CUDA(ctx, cudaFuncSetAttribute(kstap::k_moments<P, Q>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1));
  const int g1 = grid_for(kstap::k_moments<P, Q>, kstap::kMomThreads, sm1,
                          JL.ntiles[kstap::kKindMoments], sm_count, waves);
  prof_collect(prof, KSTAP_K_MOMENTS);
  prof_begin(prof, KSTAP_K_MOMENTS, s);
  kstap::k_moments<P, Q><<<g1, kstap::kMomThreads, sm1, s>>>(g, JL, Mw, Sw, Lw);
  prof_end(prof, KSTAP_K_MOMENTS, s);
  KSTAP_CUDA(ctx, cudaGetLastError());

  if constexpr (P <= 3) {
    const int g2 = grid_for(kstap::k_flipflop<P>, 128, 0, JL.ntiles[kstap::kKindFlip], sm_count,
                            waves);
    prof_collect(prof, KSTAP_K_FLIPFLOP);
    prof_begin(prof, KSTAP_K_FLIPFLOP, s);
    kstap::k_flipflop<P><<<g2, 128, 0, s>>>(g, JL, Mw, Sw, aw);
    // the classical filter refines u_a in FP64 (counted with the flip-flop)
    if (g.filter == KSTAP_FILTER_CLASSICAL && g.r_a == 1)
      kstap::k_refine_ua<P><<<g2, 128, 0, s>>>(g, JL, Mw, aw);
    prof_end(prof, KSTAP_K_FLIPFLOP, s);
    KSTAP_CUDA(ctx, cudaGetLastError());
  } else {
    // stacked passes: M and the block sums from the lag store (a warp per
    // cell), then Alg. 2 with a thread per cell
    if (!lag_store) return fail(ctx, KSTAP_EINVAL, "p > 3 needs the lag store");
    const size_t smg = smem_mgram(g);
    KSTAP_CUDA(ctx, cudaFuncSetAttribute(kstap::k_mgram<P, Q>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smg));
    const int gm = grid_for(kstap::k_mgram<P, Q>, 64, smg, JL.ntiles[kstap::kKindMgram],
                            sm_count, waves);
    prof_collect(prof, KSTAP_K_MGRAM);
    prof_begin(prof, KSTAP_K_MGRAM, s);
    kstap::k_mgram<P, Q><<<gm, 64, smg, s>>>(g, JL, Mw, Sw, Lw);
    prof_end(prof, KSTAP_K_MGRAM, s);
    KSTAP_CUDA(ctx, cudaGetLastError());
    const size_t smf = smem_flipt(g);
    KSTAP_CUDA(ctx, cudaFuncSetAttribute(kstap::k_flipflop_t<P>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smf));
    const int gf = grid_for(kstap::k_flipflop_t<P>, kstap::kFlipThreads, smf,
                            JL.ntiles[kstap::kKindFlip], sm_count, waves);
    prof_collect(prof, KSTAP_K_FLIPFLOP);
    prof_begin(prof, KSTAP_K_FLIPFLOP, s);
    kstap::k_flipflop_t<P><<<gf, kstap::kFlipThreads, smf, s>>>(g, JL, Mw, Sw, aw);
    prof_end(prof, KSTAP_K_FLIPFLOP, s);
    KSTAP_CUDA(ctx, cudaGetLastError());
  }

  const size_t sm3 = smem_bfit(g, lag_store);
  auto kb = kstap::k_bfit<P, Q, R, true>;
  if constexpr (P <= 3) {
    if (!lag_store) kb = kstap::k_bfit<P, Q, R, false>;
  }
  KSTAP_CUDA(ctx, cudaFuncSetAttribute(kb, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm3));
  constexpr int nt3 = kstap::bfit_threads(Q);
  const int g3 = grid_for(kb, nt3, sm3, JL.ntiles[kstap::kKindBfit], sm_count, waves);
  prof_collect(prof, KSTAP_K_BFIT);
  prof_begin(prof, KSTAP_K_BFIT, s);
  kb<<<g3, nt3, sm3, s>>>(g, JL, aw, Lw);
  prof_end(prof, KSTAP_K_BFIT, s);
  KSTAP_CUDA(ctx, cudaGetLastError());
  return KSTAP_OK;
}

template <int P, int Q, int R, bool BF16>
kstap_status enqueue_detect_tc(kstap_ctx* ctx, kstap_ctx* prof, const Geom& g, const JobList& JL,
                               int sm_count, int waves, cudaStream_t s) {
  auto k = kstap::k_detect_tc<P, Q, R, BF16>;
  const size_t sm = kstap::tc_smem_request(P, Q, R);
  KSTAP_CUDA(ctx, cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  constexpr int nt = kstap::tc_threads(Q);
  const int grid = grid_for(k, nt, sm, JL.ntiles[kstap::kKindDetect], sm_count, waves);
  prof_collect(prof, KSTAP_K_DETECT);
  prof_begin(prof, KSTAP_K_DETECT, s);
  k<<<grid, nt, sm, s>>>(g, JL, ctx->bank_op, ctx->bank_inv, ctx->bank_aT, ctx->bank_bT,
                         ctx->bank_n2, ctx->fault);
  prof_end(prof, KSTAP_K_DETECT, s);
  KSTAP_CUDA(ctx, cudaGetLastError());
  return KSTAP_OK;
}

template <int P, int Q, int R, int RA>
kstap_status enqueue_detect_fp32(kstap_ctx* ctx, kstap_ctx* prof, const Geom& g, const JobList& JL,
                                 int sm_count, int waves, cudaStream_t s);

template <int P, int Q, int R>
kstap_status enqueue_detect(kstap_ctx* ctx, kstap_ctx* prof, const Geom& g, const JobList& JL,
                            int sm_count, int waves, cudaStream_t s) {
  if (JL.njobs < 1) return KSTAP_OK;
  if (g.r_a == 2) return enqueue_detect_fp32<P, Q, R, 2>(ctx, prof, g, JL, sm_count, waves, s);
  if constexpr (P <= 3 && R <= kstap::kRbTc) {
    if (ctx->prm.precision == KSTAP_FP16X3)
      return enqueue_detect_tc<P, Q, R, false>(ctx, prof, g, JL, sm_count, waves, s);
    if (ctx->prm.precision == KSTAP_BF16X3)
      return enqueue_detect_tc<P, Q, R, true>(ctx, prof, g, JL, sm_count, waves, s);
  }
  return enqueue_detect_fp32<P, Q, R, 1>(ctx, prof, g, JL, sm_count, waves, s);
}

template <int P, int Q, int R, int RA>
kstap_status enqueue_detect_fp32(kstap_ctx* ctx, kstap_ctx* prof, const Geom& g, const JobList& JL,
                                 int sm_count, int waves, cudaStream_t s) {
  const size_t sm = smem_detect(g);
  KSTAP_CUDA(ctx, cudaFuncSetAttribute(kstap::k_detect<P, Q, R, RA>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  const int grid = grid_for(kstap::k_detect<P, Q, R, RA>, kstap::kThreads, sm,
                            JL.ntiles[kstap::kKindDetect], sm_count, waves);
  prof_collect(prof, KSTAP_K_DETECT);
  prof_begin(prof, KSTAP_K_DETECT, s);
  kstap::k_detect<P, Q, R, RA><<<grid, kstap::kThreads, sm, s>>>(g, JL, ctx->bank_aT,
                                                                   ctx->bank_bT, ctx->bank_n2);
  prof_end(prof, KSTAP_K_DETECT, s);
  KSTAP_CUDA(ctx, cudaGetLastError());
  return KSTAP_OK;
}

// r_b dispatch of one class: defines fit_P_Q / detect_P_Q (declared in
// kstap_host.cuh) for r_b in [1, 8] (p <= 3) or [1, 4] (stacked passes),
// r_b < q.
template <int P, int Q, int R = 1>
kstap_status fit_rb(kstap_ctx* ctx, kstap_ctx* prof, const Geom& g, const JobList& JL,
                    char* scratch, const Layout& L, bool lag_store, int sm_count, int waves,
                    cudaStream_t s) {
  if constexpr (R < Q && R <= (P <= 3 ? kstap::kRbMax : 4)) {
    if (g.r_b == R)
      return enqueue_fit<P, Q, R>(ctx, prof, g, JL, scratch, L, lag_store, sm_count, waves, s);
    return fit_rb<P, Q, R + 1>(ctx, prof, g, JL, scratch, L, lag_store, sm_count, waves, s);
  }
  return fail(ctx, KSTAP_EINVAL, "unsupported r_b %d", g.r_b);
}
template <int P, int Q, int R = 1>
kstap_status detect_rb(kstap_ctx* ctx, kstap_ctx* prof, const Geom& g, const JobList& JL,
                       int sm_count, int waves, cudaStream_t s) {
  if constexpr (R < Q && R <= (P <= 3 ? kstap::kRbMax : 4)) {
    if (g.r_b == R) return enqueue_detect<P, Q, R>(ctx, prof, g, JL, sm_count, waves, s);
    return detect_rb<P, Q, R + 1>(ctx, prof, g, JL, sm_count, waves, s);
  }
  return fail(ctx, KSTAP_EINVAL, "unsupported r_b %d", g.r_b);
}
#define KSTAP_DEFINE_FIT_(P, Q)                                                                \
  kstap_status fit_##P##_##Q(kstap_ctx* ctx, kstap_ctx* prof, const Geom& g, const JobList& JL, \
                             char* scratch, const Layout& L, bool lag_store, int sm_count,     \
                             int waves, cudaStream_t s) {                                       \
    return fit_rb<P, Q>(ctx, prof, g, JL, scratch, L, lag_store, sm_count, waves, s);          \
  }
#define KSTAP_DEFINE_DETECT_(P, Q)                                                             \
  kstap_status detect_##P##_##Q(kstap_ctx* ctx, kstap_ctx* prof, const Geom& g,               \
                                const JobList& JL, int sm_count, int waves, cudaStream_t s) {  \
    return detect_rb<P, Q>(ctx, prof, g, JL, sm_count, waves, s);                              \
  }
#define KSTAP_DEFINE_FIT(P, Q) KSTAP_DEFINE_FIT_(P, Q)
#define KSTAP_DEFINE_DETECT(P, Q) KSTAP_DEFINE_DETECT_(P, Q)

}  // namespace kh
