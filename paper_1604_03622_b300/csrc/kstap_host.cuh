// Host-side internals of libkstap shared by its translation units: the
// context, the workspace layout, shared-memory sizes of every pass, launch
// helpers, and the per-(p, q) class entry points that enqueue the kernels.
// Each class (p, q) is compiled in a translation unit of its own
// (kstap_inst.cu with KSTAP_INST_P / KSTAP_INST_Q / KSTAP_INST_PART), so the
// library builds in parallel.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/kstap.h"
#include "kstap_kernels.cuh"
#include "kstap_tc.cuh"
#include "kstap_mp.cuh"

using kstap::Geom;
using kstap::Job;
using kstap::JobList;

struct Server;
namespace kh {
struct Tuning {
  // grid = SMs x resident CTAs x waves, capped by the tile count.  64 leaves
  // one or two tiles per CTA on megapixel frames, so the block scheduler
  // balances the tail (1024^2 frame: 14.61 ms at 4 waves, 14.30 ms at 64)
  int waves = 64;
  int tc = 0;      // cells per tile in the B pass (0 = default: 32, or 16 for q = 32)
  int lag_store = 1;   // 1: the moments pass writes the lag store; 0: the B pass recomputes
};
}  // namespace kh

struct kstap_ctx {
  kstap_params prm;
  int V = 0;
  cudaStream_t stream = nullptr;
  size_t budget = 0;
  int device = 0;
  int sm_count = 148;
  // bank, transposed for the detect kernel: aT [p][V], bT [q][V], norms [2V]
  float2* bank_aT = nullptr;
  float2* bank_bT = nullptr;
  float* bank_n2 = nullptr;
  // tensor-core route: bank operand image (hi, lo; tcgen05 K-major layout)
  // and the inverse of its power-of-two scale
  uint4* bank_op = nullptr;
  float bank_inv = 1.f;
  // workspace and the device job table of kstap_run_batch
  void* ws = nullptr;
  size_t ws_bytes = 0;
  Job* jobs_dev = nullptr;
  size_t jobs_cap = 0;
  kh::Tuning tune;
  std::string err;
  // optional per-kernel timing: events around every launch on ctx->stream
  bool profile = false;
  cudaEvent_t ev[kstap_nkernels + 1][2] = {};
  float kernel_ms[kstap_nkernels] = {};
  int kernel_launches[kstap_nkernels] = {};
  bool ev_pending[kstap_nkernels] = {};
  struct Server* server = nullptr;   // created by the first kstap_submit
  // device words (kReportWords): the counters of the last fit ([0] cells at
  // max_iter, [1] non-finite cells, [2] cells whose B eigenspace was
  // recomputed by the ill-gapped path), then the frame scan of kstap_detect
  // (max bits, non-finite flag) and the tensor-core fault word
  unsigned* det_flags = nullptr;
  unsigned long long* report = nullptr;
  // device word of the tensor-core detect (bit 0: a completion wait gave up,
  // bit 1: tensor memory freed before the MMAs completed)
  unsigned* fault = nullptr;
};

struct kstap_graph {
  std::vector<void*> allocs;          // workspaces and job tables owned by the graph
  std::vector<cudaStream_t> streams;  // capture root and branches
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace kh {

constexpr int kReportCounters = 3;   // fit counters at the start of kstap_ctx::report
constexpr int kReportWords = 8;

// Records the message as ctx's last error (or, for ctx == NULL, as the
// calling thread's last context-free error) and returns st.
kstap_status fail(kstap_ctx* ctx, kstap_status st, const char* fmt, ...);
// Per-kernel launch timing on ctx's events (no-ops when ctx is NULL or
// profiling is off).
void prof_begin(kstap_ctx* ctx, int k, cudaStream_t s);
void prof_end(kstap_ctx* ctx, int k, cudaStream_t s);
void prof_collect(kstap_ctx* ctx, int k);

#define KSTAP_CUDA(ctx, call)                                                            \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return fail((ctx), KSTAP_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));   \
  } while (0)

inline size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

// Scratch layout of one launch over frames with cell grids H x W: per-job
// scale words, per-cell arrays (struct of arrays over all cells of all
// jobs), then the per-job lag stores.
struct Layout {
  size_t flags, Mw, Sw, aw, Lw, total;
  size_t NC;
  std::vector<size_t> cell0, lag0;   // per job (lag0 in float4 units)
};

inline int tiles_moments(int H, int W) {
  return ((W + kstap::kTileCells - 1) / kstap::kTileCells) *
         ((H + kstap::kMomRows - 1) / kstap::kMomRows);
}
inline int tiles_flip(int H, int W, int p = 3) {
  const size_t per = p <= 3 ? 128 : kstap::kFlipThreads;   // a thread per cell
  return (int)(((size_t)H * W + per - 1) / per);
}
inline int tiles_mgram(int H, int W, int p) {
  return p <= 3 ? 0 : ((W + kstap::kStrip - 1) / kstap::kStrip) * H;   // a CTA per strip
}
inline int tiles_bfit(int H, int W, int tc) { return ((W + tc - 1) / tc) * H; }
inline int cells_per_detect_block(int q) {
  return (kstap::kThreads / 32) * (32 / kstap::grp_lanes(q));
}
inline int tiles_detect(int H, int W, int q, int precision = KSTAP_FP32) {
  const int c = precision == KSTAP_FP32 ? cells_per_detect_block(q) : kstap::kTcCells;
  return (int)(((size_t)H * W + c - 1) / c);
}

inline size_t smem_moments(const Geom& g) {
  const int P = g.p, PP = P * P, TC = kstap::kTileCells, TR = kstap::kMomRows;
  const int NRT = 2 * g.Rr + TR, WT = TC + 2 * g.Ra + g.q - 1, NUmax = TC + g.q - 1;
  size_t b = (size_t)P * NRT * WT * 8;
  b += (b & 15);
  // box sums, then the row lags of the per-thread M; the TMA staging of the
  // frame tile reuses that region, which is grown if the tile is larger
  size_t region = 2 * (size_t)PP * WT * 16;
  if (P <= 3) region += (size_t)TR * PP * NUmax * 8;
  return b + std::max(region, (size_t)kstap::moments_stage_bytes(P, NRT, WT));
}

inline size_t smem_mgram(const Geom& g) {
  // the lag windows' ring (sum_g (q - g + 1) slots of PP entries), the fold
  // scratch and the block sums
  const size_t PP = (size_t)g.p * g.p, slots = (size_t)g.q * (g.q + 3) / 2;
  return (slots * PP + PP * PP + PP) * 8;
}

inline size_t smem_flipt(const Geom& g) {
  // a, y = M a and the two leading eigenvectors of each thread
  return (2 * (size_t)g.p * g.p + 2 * (size_t)g.p) * kstap::kFlipThreads * 8;
}

inline size_t smem_bfit(const Geom& g, bool from_store) {
  const int P = g.p, PP = P * P, Q = g.q, TC = g.tc, R = g.r_b;
  // the tile's B (float-float upper triangles) and a, then the lag / basis /
  // ill-gapped-cell region (kstap::bfit_region_bytes, shared with the kernel)
  return (size_t)TC * (Q * (Q + 1) / 2) * 16 + (size_t)TC * PP * 16 +
         (size_t)kstap::bfit_region_bytes(P, Q, R, TC, g.Ra, g.Rr, from_store);
}

inline size_t smem_detect(const Geom& g) {
  const int P = g.p, Q = g.q, V = g.V, R = g.r_b;
  const size_t CS = 2 * (size_t)P * Q + 2 * (size_t)Q * R + 2 * P + 4 * (size_t)P * R;
  const size_t cells = cells_per_detect_block(Q);
  const size_t QS = std::max(R, P + 1);   // near-blind queue entry (float2) per pair
  const size_t PF = (size_t)P * Q + 2 * (size_t)Q * R + 2 * P;   // prefetch buffer per cell
  return (size_t)(P + Q) * V * 8 + 2 * (size_t)V * 4 + cells * CS * 8 +
         (kstap::kThreads / 32) * kstap::kBlindQ * (QS * 8 + 4) + cells * PF * 8;
}

// Largest dynamic shared memory a CTA may opt into on sm_103a (227 KB).
constexpr size_t kSmemOptin = 232448;

// Persistent grid: SMs x resident CTAs x waves, capped by the tile count.
template <typename K>
int grid_for(K kernel, int threads, size_t smem, int tiles, int sm_count, int waves) {
  int occ = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, threads, smem) != cudaSuccess ||
      occ < 1)
    occ = 1;
  const long cap = (long)sm_count * occ * std::max(1, waves);
  return (int)std::max(1L, std::min<long>(tiles, cap));
}

// Frame scan of every job (k_frame_maxabs): max |component| and the
// non-finite flag, into each job's maxbits words (zeroed by the caller).
kstap_status enqueue_scan(kstap_ctx* ctx, kstap_ctx* prof, const Geom& g, const JobList& JL,
                          int sm_count, cudaStream_t s);

// Per-class entry points: fit (scale, moments, flip-flop, B / U_B) and
// detect (projection and bank) of every job of JL, for the r_b of g.
#define KSTAP_CLASSES(X) X(3, 8) X(3, 12) X(3, 16) X(3, 24) X(3, 32) X(6, 8) X(6, 16)
#define KSTAP_DECLARE_CLASS(P, Q)                                                              \
  kstap_status fit_##P##_##Q(kstap_ctx* ctx, kstap_ctx* prof, const Geom& g, const JobList& JL, \
                             char* scratch, const Layout& L, bool lag_store, int sm_count,     \
                             int waves, cudaStream_t s);                                        \
  kstap_status detect_##P##_##Q(kstap_ctx* ctx, kstap_ctx* prof, const Geom& g,               \
                                const JobList& JL, int sm_count, int waves, cudaStream_t s);
KSTAP_CLASSES(KSTAP_DECLARE_CLASS)

}  // namespace kh
