// libkstap: C ABI (include/kstap.h) over the Kron-STAP kernels.
//
// Every launch works on a job list: one frame passed by value (the per-frame
// calls) or a device table of frames (batches and CUDA graphs).  Kernels use
// persistent grids (occupancy x waves CTAs striding over all tiles of all
// jobs of the launch).  The launch sequences of each class (p, q) live in
// their own translation units (kstap_inst.cu); this file holds the host
// logic: validation, workspace layout, strips, batches, graphs, the
// autotuner, serving and the context-free entry points.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>

#include <cudaTypedefs.h>

#include "kstap_host.cuh"
#include "kstap_lrk.cuh"
#include "kstap_misc.cuh"

using namespace kh;

namespace {

thread_local std::string g_create_err;
// Set by the serving worker thread: failures it meets are recorded here
// instead of in the context, whose error string belongs to the caller's
// thread.
thread_local std::string* t_err_sink = nullptr;

}  // namespace

namespace kh {

void prof_begin(kstap_ctx* ctx, int k, cudaStream_t s) {
  if (!ctx || !ctx->profile) return;
  if (!ctx->ev[k][0]) {
    cudaEventCreate(&ctx->ev[k][0]);
    cudaEventCreate(&ctx->ev[k][1]);
  }
  cudaEventRecord(ctx->ev[k][0], s);
}

void prof_end(kstap_ctx* ctx, int k, cudaStream_t s) {
  if (!ctx || !ctx->profile) return;
  cudaEventRecord(ctx->ev[k][1], s);
  ctx->ev_pending[k] = true;
}

// Folds a finished launch into the per-kernel totals (waits for its end event;
// called before the next launch of the same kernel and by kstap_kernel_times).
void prof_collect(kstap_ctx* ctx, int k) {
  if (!ctx || !ctx->ev_pending[k]) return;
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
  if (t_err_sink)
    *t_err_sink = buf;
  else if (ctx)
    ctx->err = buf;
  else
    g_create_err = buf;
  return st;
}


// Frame scan of every job: max |component| (fixed-point scale) and the
// non-finite flag, into each job's maxbits words (zeroed by the caller).
kstap_status enqueue_scan(kstap_ctx* ctx, kstap_ctx* prof, const Geom& g, const JobList& JL,
                          int sm_count, cudaStream_t s) {
  const size_t maxf = JL.table ? 0 : 2 * (size_t)g.p * JL.one.H_in * JL.one.W_in;
  const int bx = JL.table ? sm_count * 2
                          : (int)std::min<size_t>((maxf + 1023) / 1024, (size_t)sm_count * 16);
  prof_collect(prof, KSTAP_K_SCALE);
  prof_begin(prof, KSTAP_K_SCALE, s);
  kstap::k_frame_maxabs<<<dim3(std::max(1, bx), JL.njobs), 256, 0, s>>>(g, JL);
  prof_end(prof, KSTAP_K_SCALE, s);
  KSTAP_CUDA(ctx, cudaGetLastError());
  return KSTAP_OK;
}

}  // namespace kh

namespace {

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
  if (p->p != 3 && p->p != 6) {
    why = "this build supports p == 3, or p == 6 (two stacked passes)";
    return false;
  }
  if (p->q != 8 && p->q != 12 && p->q != 16 && p->q != 24 && p->q != 32) {
    why = "q must be 8, 12, 16, 24 or 32";
    return false;
  }
  if (p->r_a < 1 || p->r_a > 2) {
    why = "r_a must be 1 (rank-one spatial clutter model) or 2";
    return false;
  }
  if (p->r_a == 2 && (p->precision != KSTAP_FP32 || p->filter != KSTAP_FILTER_KRON)) {
    why = "r_a == 2 runs on the KSTAP_FP32 bank with the Kron-STAP filter";
    return false;
  }
  if (p->p == 6 && (p->q > 16 || p->r_a < 1 || p->r_a > 2 || p->precision != KSTAP_FP32 ||
                    p->filter != KSTAP_FILTER_KRON)) {
    why = "p == 6 (stacked passes) needs q in {8, 16}, r_a in {1, 2}, KSTAP_FP32 and the Kron filter";
    return false;
  }
  if (p->r_b < 1 || p->r_b > kstap::kRbMax || p->r_b >= p->q) {
    why = "r_b must satisfy 1 <= r_b <= 8 and r_b < q";
    return false;
  }
  if (p->r_b > kstap::kRbTc && (p->p != 3 || p->precision != KSTAP_FP32)) {
    why = "r_b > 4 runs with p == 3 on the KSTAP_FP32 bank";
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
  if (p->precision != KSTAP_FP32 && p->precision != KSTAP_FP16X3 &&
      p->precision != KSTAP_BF16X3) {
    why = "precision must be KSTAP_FP32, KSTAP_FP16X3 or KSTAP_BF16X3";
    return false;
  }
  if (p->filter != KSTAP_FILTER_KRON && p->filter != KSTAP_FILTER_CLASSICAL) {
    why = "filter must be KSTAP_FILTER_KRON or KSTAP_FILTER_CLASSICAL";
    return false;
  }
  if (p->filter == KSTAP_FILTER_CLASSICAL && p->precision != KSTAP_FP32) {
    why = "the classical filter runs on the KSTAP_FP32 route only";
    return false;
  }
  return true;
}

// Class-wide geometry (per-frame sizes are filled per tile from the job).
// Cells per B-pass tile when the tuning leaves it open: the tile's B
// matrices (q (q + 1) / 2 float-float entries per cell) fill most of the
// CTA's shared memory at q >= 24.
int default_tc(const kstap_params& p) { return p.q >= 24 ? 16 : kstap::kTileCells; }

Geom make_geom(const kstap_params& p, int V, int tc) {
  Geom g;
  g.p = p.p;
  g.q = p.q;
  g.r_a = p.r_a;
  g.r_b = p.r_b;
  g.Rr = p.ring_r;
  g.Ra = p.ring_a;
  g.Gr = p.guard_r;
  g.Ga = p.guard_a;
  g.H_in = g.W_in = g.H = g.W = 0;
  const long nbox = (2L * p.ring_r + 1) * (2L * p.ring_a + 1);
  g.n = (int)(nbox - (2L * p.guard_r + 1) * (2L * p.guard_a + 1));
  g.V = V;
  // |Y| < 2^B per component keeps every box sum of products below 2^62:
  // 2B + 1 + ceil(log2(nbox)) <= 62.
  g.B = (61 - ceil_log2(nbox)) / 2;
  if (g.B > 26) g.B = 26;
  g.max_iter = p.max_iter > 0 ? p.max_iter : 64;
  g.eps = p.eps > 0 ? (float)p.eps : 2e-6f;
  g.tau = p.tau;
  g.tc = tc > 0 ? tc : default_tc(p);
  g.filter = p.filter;
  return g;
}

Layout make_layout(const kstap_params& p, const std::vector<std::pair<int, int>>& HW,
                   bool lag_store) {
  const size_t PP = (size_t)p.p * p.p, NE = PP * (PP + 1) / 2;
  Layout L;
  L.NC = 0;
  size_t lag = 0;
  for (auto& hw : HW) {
    L.cell0.push_back(L.NC);
    L.lag0.push_back(lag);
    L.NC += (size_t)hw.first * hw.second;
    if (lag_store) lag += (size_t)hw.first * p.q * PP * (hw.second + p.q - 1);
  }
  L.flags = 0;
  L.Mw = up256(8 * HW.size());
  L.Sw = up256(L.Mw + L.NC * NE * sizeof(float2));
  L.aw = up256(L.Sw + L.NC * PP * sizeof(float2));
  L.Lw = up256(L.aw + L.NC * PP * sizeof(float2));
  L.total = up256(L.Lw + lag * sizeof(float4));
  return L;
}

// A frame (or a row strip of one) as the library sees it (device pointers,
// caller-owned).  ch_stride: elements between channel planes (0 = H_in * W_in).
// A strip takes its own fixed-point scale (max over its rows), so its results
// agree with the whole frame's to rounding (within the parity tolerance), and
// a given split is deterministic.
struct Frame {
  const kstap_c64* Y;
  int H_in, W_in;
  kstap_factors f;
  float* Tmax;
  int32_t* vidx;
  uint8_t* map;
  float* T_all;
  long long ch_stride = 0;
};

// Row strips of at most `rows` cell rows.  Strip k covers cell rows
// [r0, r0 + nr) and reads input rows [r0, r0 + nr + 2 ring_r) of every
// channel; its factor and output pointers are offset to cell r0 * W.
std::vector<Frame> split_rows(const kstap_params& p, int V, const Frame& f, int rows) {
  std::vector<Frame> out;
  const int H = f.H_in - 2 * p.ring_r, W = f.W_in - 2 * p.ring_a - p.q + 1;
  const long long cs = f.ch_stride ? f.ch_stride : (long long)f.H_in * f.W_in;
  for (int r0 = 0; r0 < H; r0 += rows) {
    const int nr = std::min(rows, H - r0);
    const size_t c0 = (size_t)r0 * W;
    Frame s = f;
    s.Y = f.Y + (size_t)r0 * f.W_in;
    s.H_in = nr + 2 * p.ring_r;
    s.ch_stride = cs;
    auto off = [&](auto* ptr, size_t per) { return ptr ? ptr + c0 * per : ptr; };
    s.f.UA = off(f.f.UA, (size_t)p.p * p.r_a);
    s.f.UB_hi = off(f.f.UB_hi, (size_t)p.q * p.r_b);
    s.f.UB_lo = off(f.f.UB_lo, (size_t)p.q * p.r_b);
    s.f.lamA = off(f.f.lamA, (size_t)p.r_a);
    s.f.lamB = off(f.f.lamB, (size_t)p.r_b);
    s.f.iters = off(f.f.iters, 1);
    s.f.eta = off(f.f.eta, 1);
    s.Tmax = off(f.Tmax, 1);
    s.vidx = off(f.vidx, 1);
    s.map = off(f.map, 1);
    s.T_all = off(f.T_all, (size_t)V);
    out.push_back(s);
  }
  return out;
}

// cuTensorMapEncodeTiled from the driver, resolved once through the runtime
// (no link against the driver library).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)ptr;
  });
  return fn;
}

// The job's 1-D tensor map over its frame as float pairs, from Y to the end
// of the last channel's last row, with the moments pass's box (one tile row
// segment).  Left unset (ymap_ok = 0, plain loads) when Y is not 16-byte
// aligned or the extent does not fit the map's 32-bit signed coordinates.
void encode_ymap(Job& j, int P, int WT) {
  j.ymap_ok = 0;
  const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc || ((uintptr_t)j.Y & 15)) return;
  const unsigned long long nf =
      2ull * ((unsigned long long)(P - 1) * (unsigned long long)j.ch_stride +
              (unsigned long long)j.H_in * (unsigned long long)j.W_in);
  if (nf >= (1ull << 31)) return;
  cuuint64_t dim[1] = {nf};
  cuuint64_t stride[1] = {0};   // rank 1: no strides
  cuuint32_t box[1] = {(cuuint32_t)kstap::moments_box_floats(WT)};
  cuuint32_t es[1] = {1};
  if (enc(&j.ymap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 1, (void*)j.Y, dim, stride, box, es,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
          CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS)
    j.ymap_ok = 1;
}

// Fills the jobs of one launch; scratch and L may be null (detect-only).
void fill_jobs(const kstap_params& p, const Geom& g, const std::vector<Frame>& fr, char* scratch,
               const Layout* L, std::vector<Job>& jobs, JobList& JL) {
  jobs.clear();
  int t[kstap::kKinds] = {0, 0, 0, 0, 0};
  for (size_t k = 0; k < fr.size(); ++k) {
    Job j;
    memset(&j, 0, sizeof(j));
    j.Y = (const float2*)fr[k].Y;
    j.H_in = fr[k].H_in;
    j.W_in = fr[k].W_in;
    j.ch_stride = fr[k].ch_stride ? fr[k].ch_stride : (long long)fr[k].H_in * fr[k].W_in;
    j.H = fr[k].H_in - 2 * p.ring_r;
    j.W = fr[k].W_in - 2 * p.ring_a - p.q + 1;
    j.cell0 = L ? (long long)L->cell0[k] : 0;
    j.lag0 = L ? (long long)L->lag0[k] : 0;
    j.maxbits = (scratch && L) ? (unsigned*)(scratch + L->flags) + 2 * k : nullptr;
    j.UA = (float2*)fr[k].f.UA;
    j.UBh = (float2*)fr[k].f.UB_hi;
    j.UBl = (float2*)fr[k].f.UB_lo;
    j.lamA = fr[k].f.lamA;
    j.lamB = fr[k].f.lamB;
    j.iters = fr[k].f.iters;
    j.eta = fr[k].f.eta;
    j.Tmax = fr[k].Tmax;
    j.vidx = fr[k].vidx;
    j.map = fr[k].map;
    j.T_all = fr[k].T_all;
    if (scratch) encode_ymap(j, p.p, kstap::kTileCells + 2 * p.ring_a + p.q - 1);
    j.tile0[kstap::kKindMoments] = t[0];
    j.tile0[kstap::kKindFlip] = t[1];
    j.tile0[kstap::kKindBfit] = t[2];
    j.tile0[kstap::kKindDetect] = t[3];
    j.tile0[kstap::kKindMgram] = t[4];
    t[0] += tiles_moments(j.H, j.W);
    t[1] += tiles_flip(j.H, j.W, p.p);
    t[4] += tiles_mgram(j.H, j.W, p.p);
    t[2] += tiles_bfit(j.H, j.W, g.tc);
    t[3] += tiles_detect(j.H, j.W, p.q, p.precision);
    jobs.push_back(j);
  }
  memset(&JL, 0, sizeof(JL));
  if (!jobs.empty()) JL.one = jobs[0];
  JL.table = nullptr;
  JL.njobs = (int)jobs.size();
  for (int k = 0; k < kstap::kKinds; ++k) JL.ntiles[k] = t[k];
  JL.NC = L ? (long long)L->NC : 0;
}

// Checks every pass's shared-memory footprint for this geometry against the
// per-CTA limit (the ring box and p set them).
bool smem_fits(const Geom& g, bool lag_store, std::string& why) {
  struct { const char* name; size_t bytes; } use[] = {
      {"moments", smem_moments(g)},
      {"B fit", smem_bfit(g, lag_store)},
      {"detect", smem_detect(g)},
      {"M gram", g.p > 3 ? smem_mgram(g) : 0},
      {"flip-flop", g.p > 3 ? smem_flipt(g) : 0},
  };
  for (const auto& u : use)
    if (u.bytes > kSmemOptin) {
      char buf[160];
      snprintf(buf, sizeof buf, "the %s pass needs %zu B of shared memory per CTA (limit %zu B); "
               "use a smaller training ring", u.name, u.bytes, kSmemOptin);
      why = buf;
      return false;
    }
  return true;
}

// Whether this context's fits write the lag store (stacked passes always do:
// k_mgram reads it).
bool store_lags(const kstap_ctx* ctx) { return ctx->prm.p > 3 || ctx->tune.lag_store != 0; }

kstap_status dispatch_fit(kstap_ctx* ctx, kstap_ctx* prof, const Geom& g, const JobList& JL,
                          char* scratch, const Layout& L, bool lag_store, int sm_count, int waves,
                          cudaStream_t s) {
#define KSTAP_FIT_CLASS(P, Q) \
  if (g.p == P && g.q == Q) return fit_##P##_##Q(ctx, prof, g, JL, scratch, L, lag_store, sm_count, waves, s);
  KSTAP_CLASSES(KSTAP_FIT_CLASS)
#undef KSTAP_FIT_CLASS
  return fail(ctx, KSTAP_EINVAL, "unsupported (p, q) = (%d, %d)", g.p, g.q);
}

kstap_status dispatch_detect(kstap_ctx* ctx, kstap_ctx* prof, const Geom& g, const JobList& JL,
                             int sm_count, int waves, cudaStream_t s) {
  if (JL.njobs < 1) return KSTAP_OK;
#define KSTAP_DETECT_CLASS(P, Q) \
  if (g.p == P && g.q == Q) return detect_##P##_##Q(ctx, prof, g, JL, sm_count, waves, s);
  KSTAP_CLASSES(KSTAP_DETECT_CLASS)
#undef KSTAP_DETECT_CLASS
  return fail(ctx, KSTAP_EINVAL, "unsupported (p, q) = (%d, %d)", g.p, g.q);
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

kstap_status check_factors(kstap_ctx* ctx, const kstap_factors* f) {
  if (!f || !f->UA || !f->UB_hi || !f->UB_lo)
    return fail(ctx, KSTAP_EINVAL, "factors (UA, UB_hi, UB_lo) must be non-NULL");
  return KSTAP_OK;
}

// Grows ctx->ws to `bytes` within the budget (synchronises the stream when
// replacing a smaller workspace).
kstap_status ensure_ws(kstap_ctx* ctx, size_t bytes) {
  if (bytes <= ctx->ws_bytes) return KSTAP_OK;
  if (ctx->budget && bytes > ctx->budget)
    return fail(ctx, KSTAP_ENOMEM, "workspace %zu B exceeds the HBM budget %zu B", bytes,
                ctx->budget);
  if (ctx->ws) {
    KSTAP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    cudaFree(ctx->ws);
    ctx->ws = nullptr;
    ctx->ws_bytes = 0;
  }
  cudaError_t e = cudaMalloc(&ctx->ws, bytes);
  if (e != cudaSuccess)
    return fail(ctx, KSTAP_ENOMEM, "workspace cudaMalloc(%zu) failed: %s", bytes,
                cudaGetErrorString(e));
  ctx->ws_bytes = bytes;
  return KSTAP_OK;
}

kstap_status frames_from(kstap_ctx* ctx, const kstap_frame* frames, int n,
                         std::vector<Frame>& fr, std::vector<std::pair<int, int>>& HW) {
  if (n < 1 || !frames) return fail(ctx, KSTAP_EINVAL, "need at least one frame");
  fr.clear();
  HW.clear();
  const kstap_params& p = ctx->prm;
  for (int k = 0; k < n; ++k) {
    kstap_status st = check_frame(ctx, frames[k].Y, frames[k].H_in, frames[k].W_in);
    if (st != KSTAP_OK) return st;
    st = check_factors(ctx, &frames[k].factors);
    if (st != KSTAP_OK) return st;
    if (!frames[k].Tmax || !frames[k].vidx || !frames[k].map)
      return fail(ctx, KSTAP_EINVAL, "frame %d: Tmax, vidx and map are required", k);
    fr.push_back(Frame{frames[k].Y, frames[k].H_in, frames[k].W_in, frames[k].factors,
                       frames[k].Tmax, frames[k].vidx, frames[k].map, frames[k].T_all});
    HW.push_back({frames[k].H_in - 2 * p.ring_r, frames[k].W_in - 2 * p.ring_a - p.q + 1});
  }
  return KSTAP_OK;
}

// Enqueues fit + detect of all frames on stream s with the given scratch and
// device job table (unused for a single frame, whose job goes by value).
kstap_status enqueue_batch(kstap_ctx* ctx, kstap_ctx* prof, const std::vector<Frame>& fr,
                           const Layout& L, char* scratch, const Job* jobs_dev,
                           cudaStream_t s, unsigned long long* report = nullptr) {
  const Geom g = make_geom(ctx->prm, ctx->V, ctx->tune.tc);
  std::vector<Job> host;
  JobList JL;
  fill_jobs(ctx->prm, g, fr, scratch, &L, host, JL);
  if (fr.size() > 1) JL.table = jobs_dev;
  JL.report = report;
  JL.fault = ctx->fault;
  kstap_status st = dispatch_fit(ctx, prof, g, JL, scratch, L, store_lags(ctx), ctx->sm_count,
                                 ctx->tune.waves, s);
  if (st != KSTAP_OK) return st;
  return dispatch_detect(ctx, prof, g, JL, ctx->sm_count, ctx->tune.waves, s);
}

}  // namespace

extern "C" {

size_t kstap_workspace_bytes(const kstap_params* params, int H_in, int W_in) {
  std::string why;
  if (!valid_params(params, why)) return 0;
  const long H = H_in - 2L * params->ring_r;
  const long W = W_in - 2L * params->ring_a - params->q + 1;
  if (H < 1 || W < 1) return 0;
  return make_layout(*params, {{(int)H, (int)W}}, true).total;
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
  if (!smem_fits(make_geom(*params, V, 0), true, why))
    return fail(nullptr, KSTAP_EINVAL, "%s", why.c_str());
  kstap_ctx* ctx = new kstap_ctx();
  ctx->prm = *params;
  ctx->V = V;
  ctx->stream = (cudaStream_t)cuda_stream;
  ctx->budget = hbm_budget_bytes;
  cudaGetDevice(&ctx->device);
  cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, ctx->device);
  if (ctx->sm_count < 1) ctx->sm_count = 148;
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
  e = cudaMalloc(&ctx->report, kReportWords * sizeof(unsigned long long));
  if (e == cudaSuccess) {
    ctx->det_flags = (unsigned*)(ctx->report + 4);
    ctx->fault = (unsigned*)(ctx->report + 5);
    e = cudaMemset(ctx->report, 0, kReportWords * sizeof(unsigned long long));
  }
  if (e == cudaSuccess) e = cudaMalloc(&ctx->bank_aT, aT.size() * sizeof(float2));
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
  if (params->precision != KSTAP_FP32) {
    if (V > kstap::kTcM) {
      kstap_destroy(ctx);
      return fail(nullptr, KSTAP_EINVAL, "the tensor-core route needs V <= %d", kstap::kTcM);
    }
    // Bank operand of the tensor-core GEMM: row v = (Re b_v, Im b_v) scaled by a
    // power of two s (max |component| s in [0.5, 1)), split hi + lo into
    // 16-bit floats and laid out as the kernel's shared-memory image.
    float bmax = 0.f;
    for (const kstap_c64& z : hb) bmax = std::max(bmax, std::max(std::fabs(z.re), std::fabs(z.im)));
    const float sc = (bmax > 0.f && std::isfinite(bmax)) ? std::ldexp(1.f, -(std::ilogb(bmax) + 1)) : 1.f;
    ctx->bank_inv = 1.f / sc;
    const int K2 = kstap::tc_k2(q);   // 2 q columns (Re, Im), zero-padded to a multiple of 16
    const size_t half = (size_t)kstap::kTcM * K2 * 2;   // bytes of one 16-bit image
    std::vector<uint16_t> img(2 * half / 2, 0);
    const bool bf = params->precision == KSTAP_BF16X3;
    for (int v = 0; v < V; ++v)
      for (int k = 0; k < 2 * q; ++k) {
        const kstap_c64 z = hb[(size_t)v * q + (k % q)];
        const float x = (k < q ? z.re : z.im) * sc;
        uint16_t h, l;
        if (bf) {
          const __nv_bfloat16 hh = __float2bfloat16_rn(x);
          h = __bfloat16_as_ushort(hh);
          l = __bfloat16_as_ushort(__float2bfloat16_rn(x - __bfloat162float(hh)));
        } else {
          const __half hh = __float2half_rn(x);
          h = __half_as_ushort(hh);
          l = __half_as_ushort(__float2half_rn(x - __half2float(hh)));
        }
        const size_t off = kstap::tc_off(v, k, kstap::kTcM) / 2;
        img[off] = h;
        img[half / 2 + off] = l;
      }
    e = cudaMalloc(&ctx->bank_op, 2 * half);
    if (e == cudaSuccess)
      e = cudaMemcpy(ctx->bank_op, img.data(), 2 * half, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      kstap_destroy(ctx);
      return fail(nullptr, KSTAP_ECUDA, "bank operand upload failed: %s", cudaGetErrorString(e));
    }
  }
  *out = ctx;
  return KSTAP_OK;
}

kstap_status kstap_fit_project(kstap_ctx* ctx, const kstap_c64* Y, int H_in, int W_in,
                               const kstap_factors* factors) {
  kstap_status st = check_frame(ctx, Y, H_in, W_in);
  if (st != KSTAP_OK) return st;
  st = check_factors(ctx, factors);
  if (st != KSTAP_OK) return st;
  const kstap_params& p = ctx->prm;
  const int H = H_in - 2 * p.ring_r, W = W_in - 2 * p.ring_a - p.q + 1;
  const Geom g = make_geom(p, ctx->V, ctx->tune.tc);
  const Frame whole{Y, H_in, W_in, *factors, nullptr, nullptr, nullptr, nullptr};
  // A frame whose workspace exceeds the budget runs as row strips, one after
  // the other on the stream, in one strip-sized workspace.
  int rows = H;
  const bool store = store_lags(ctx);
  const size_t full = make_layout(p, {{H, W}}, store).total;
  if (ctx->budget && full > ctx->budget) {
    const size_t per_row = std::max<size_t>(1, make_layout(p, {{1, W}}, store).total);
    rows = (int)std::max<size_t>(kstap::kMomRows, ctx->budget / per_row);
    rows -= rows % kstap::kMomRows;
    if (make_layout(p, {{std::min(rows, H), W}}, store).total > ctx->budget)
      return fail(ctx, KSTAP_ENOMEM, "a %d-row strip of this frame exceeds the HBM budget %zu B",
                  kstap::kMomRows, ctx->budget);
  }
  const std::vector<Frame> strips = (rows >= H) ? std::vector<Frame>{whole}
                                                : split_rows(p, ctx->V, whole, rows);
  KSTAP_CUDA(ctx, cudaMemsetAsync(ctx->report, 0, kReportCounters * sizeof(unsigned long long), ctx->stream));
  for (const Frame& s : strips) {
    const int sh = s.H_in - 2 * p.ring_r;
    const Layout L = make_layout(p, {{sh, W}}, store);
    st = ensure_ws(ctx, L.total);
    if (st != KSTAP_OK) return st;
    std::vector<Frame> fr{s};
    std::vector<Job> jobs;
    JobList JL;
    fill_jobs(p, g, fr, (char*)ctx->ws, &L, jobs, JL);
    JL.report = ctx->report;
    JL.fault = ctx->fault;
    st = dispatch_fit(ctx, ctx, g, JL, (char*)ctx->ws, L, store, ctx->sm_count, ctx->tune.waves,
                      ctx->stream);
    if (st != KSTAP_OK) return st;
  }
  return KSTAP_OK;
}

kstap_status kstap_detect(kstap_ctx* ctx, const kstap_c64* Y, int H_in, int W_in,
                          const kstap_factors* factors, float* Tmax, int32_t* vidx, uint8_t* map,
                          float* T_all) {
  kstap_status st = check_frame(ctx, Y, H_in, W_in);
  if (st != KSTAP_OK) return st;
  st = check_factors(ctx, factors);
  if (st != KSTAP_OK) return st;
  if (!Tmax || !vidx || !map) return fail(ctx, KSTAP_EINVAL, "Tmax, vidx and map are required");
  const Geom g = make_geom(ctx->prm, ctx->V, ctx->tune.tc);
  std::vector<Frame> fr{Frame{Y, H_in, W_in, *factors, Tmax, vidx, map, T_all}};
  std::vector<Job> jobs;
  JobList JL;
  fill_jobs(ctx->prm, g, fr, nullptr, nullptr, jobs, JL);
  // this frame's own scan, for the per-cell non-finite flags
  JL.one.maxbits = ctx->det_flags;
  KSTAP_CUDA(ctx, cudaMemsetAsync(ctx->det_flags, 0, 2 * sizeof(unsigned), ctx->stream));
  st = enqueue_scan(ctx, ctx, g, JL, ctx->sm_count, ctx->stream);
  if (st != KSTAP_OK) return st;
  return dispatch_detect(ctx, ctx, g, JL, ctx->sm_count, ctx->tune.waves, ctx->stream);
}

kstap_status kstap_run_batch(kstap_ctx* ctx, const kstap_frame* frames, int n) {
  if (!ctx) return KSTAP_EINVAL;
  std::vector<Frame> fr;
  std::vector<std::pair<int, int>> HW;
  kstap_status st = frames_from(ctx, frames, n, fr, HW);
  if (st != KSTAP_OK) return st;
  const Layout L = make_layout(ctx->prm, HW, store_lags(ctx));
  st = ensure_ws(ctx, L.total);
  if (st != KSTAP_OK) return st;
  if (n > 1) {
    if ((size_t)n > ctx->jobs_cap) {
      if (ctx->jobs_dev) {
        KSTAP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        cudaFree(ctx->jobs_dev);
        ctx->jobs_dev = nullptr;
        ctx->jobs_cap = 0;
      }
      const size_t cap = std::max<size_t>(n, 64);
      KSTAP_CUDA(ctx, cudaMalloc(&ctx->jobs_dev, cap * sizeof(Job)));
      ctx->jobs_cap = cap;
    }
    const Geom g = make_geom(ctx->prm, ctx->V, ctx->tune.tc);
    std::vector<Job> host;
    JobList JL;
    fill_jobs(ctx->prm, g, fr, (char*)ctx->ws, &L, host, JL);
    // stream-ordered upload; pageable source, so the call returns once the
    // table has been staged and `host` may be released
    KSTAP_CUDA(ctx, cudaMemcpyAsync(ctx->jobs_dev, host.data(), n * sizeof(Job),
                                    cudaMemcpyHostToDevice, ctx->stream));
  }
  KSTAP_CUDA(ctx, cudaMemsetAsync(ctx->report, 0, kReportCounters * sizeof(unsigned long long), ctx->stream));
  return enqueue_batch(ctx, ctx, fr, L, (char*)ctx->ws, ctx->jobs_dev, ctx->stream, ctx->report);
}

kstap_status kstap_fit_report(kstap_ctx* ctx, long long* nonconverged, long long* nonfinite,
                              long long* eig_refined) {
  if (!ctx) return KSTAP_EINVAL;
  unsigned long long h[3] = {0, 0, 0};
  KSTAP_CUDA(ctx, cudaMemcpyAsync(h, ctx->report, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
  KSTAP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (nonconverged) *nonconverged = (long long)h[0];
  if (nonfinite) *nonfinite = (long long)h[1];
  if (eig_refined) *eig_refined = (long long)h[2];
  return h[0] ? KSTAP_WARN_NOCONV : KSTAP_OK;
}

kstap_status kstap_graph_create(kstap_ctx* const* ctxs, const kstap_frame* const* frames,
                                const int* nframes, int nctx, kstap_graph** out) {
  if (!out || !ctxs || !frames || !nframes || nctx < 1)
    return fail(nullptr, KSTAP_EINVAL, "kstap_graph_create: bad arguments");
  *out = nullptr;
  kstap_graph* G = new kstap_graph();
  auto bail = [&](kstap_status st) {
    kstap_graph_destroy(G);
    return st;
  };
  struct Plan {
    std::vector<Frame> fr;
    Layout L;
    char* ws = nullptr;
    Job* jobs = nullptr;
  };
  std::vector<Plan> plans(nctx);
  for (int c = 0; c < nctx; ++c) {
    kstap_ctx* ctx = ctxs[c];
    if (!ctx) return bail(fail(nullptr, KSTAP_EINVAL, "context %d is NULL", c));
    std::vector<std::pair<int, int>> HW;
    kstap_status st = frames_from(ctx, frames[c], nframes[c], plans[c].fr, HW);
    if (st != KSTAP_OK) return bail(fail(nullptr, st, "context %d: %s", c, ctx->err.c_str()));
    plans[c].L = make_layout(ctx->prm, HW, store_lags(ctx));
    void* ws = nullptr;
    cudaError_t e = cudaMalloc(&ws, plans[c].L.total);
    if (e != cudaSuccess)
      return bail(fail(nullptr, KSTAP_ENOMEM, "graph workspace cudaMalloc(%zu): %s",
                       plans[c].L.total, cudaGetErrorString(e)));
    G->allocs.push_back(ws);
    plans[c].ws = (char*)ws;
    void* jt = nullptr;
    e = cudaMalloc(&jt, plans[c].fr.size() * sizeof(Job));
    if (e != cudaSuccess)
      return bail(fail(nullptr, KSTAP_ENOMEM, "graph job table: %s", cudaGetErrorString(e)));
    G->allocs.push_back(jt);
    plans[c].jobs = (Job*)jt;
    const Geom g = make_geom(ctx->prm, ctx->V, ctx->tune.tc);
    std::vector<Job> host;
    JobList JL;
    fill_jobs(ctx->prm, g, plans[c].fr, plans[c].ws, &plans[c].L, host, JL);
    e = cudaMemcpy(jt, host.data(), host.size() * sizeof(Job), cudaMemcpyHostToDevice);
    if (e != cudaSuccess)
      return bail(fail(nullptr, KSTAP_ECUDA, "graph job table upload: %s", cudaGetErrorString(e)));
  }
  // capture: a root stream forks to one branch per context and joins back
  for (int c = 0; c <= nctx; ++c) {
    cudaStream_t s;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess)
      return bail(fail(nullptr, KSTAP_ECUDA, "cudaStreamCreate failed"));
    G->streams.push_back(s);
  }
  cudaStream_t root = G->streams[0];
  std::vector<cudaEvent_t> evs(nctx + 1);
  for (auto& ev : evs) cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  kstap_status st = KSTAP_OK;
  cudaError_t e = cudaStreamBeginCapture(root, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaEventRecord(evs[0], root);
    for (int c = 0; c < nctx; ++c) {
      cudaStream_t s = G->streams[c + 1];
      cudaStreamWaitEvent(s, evs[0], 0);
      if (st == KSTAP_OK) {
        st = enqueue_batch(ctxs[c], nullptr, plans[c].fr, plans[c].L, plans[c].ws, plans[c].jobs,
                           s);
        if (st != KSTAP_OK) fail(nullptr, st, "context %d: %s", c, ctxs[c]->err.c_str());
      }
      cudaEventRecord(evs[c + 1], s);
      cudaStreamWaitEvent(root, evs[c + 1], 0);
    }
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(root, &graph);
    G->graph = graph;
    if (st == KSTAP_OK && e2 != cudaSuccess)
      st = fail(nullptr, KSTAP_ECUDA, "stream capture failed: %s", cudaGetErrorString(e2));
  } else {
    st = fail(nullptr, KSTAP_ECUDA, "cudaStreamBeginCapture: %s", cudaGetErrorString(e));
  }
  for (auto& ev : evs) cudaEventDestroy(ev);
  if (st != KSTAP_OK) return bail(st);
  e = cudaGraphInstantiate(&G->exec, G->graph, 0);
  if (e != cudaSuccess)
    return bail(fail(nullptr, KSTAP_ECUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e)));
  *out = G;
  return KSTAP_OK;
}

kstap_status kstap_graph_launch(kstap_graph* G, void* cuda_stream) {
  if (!G || !G->exec) return fail(nullptr, KSTAP_EINVAL, "graph is NULL");
  cudaError_t e = cudaGraphLaunch(G->exec, (cudaStream_t)cuda_stream);
  if (e != cudaSuccess)
    return fail(nullptr, KSTAP_ECUDA, "cudaGraphLaunch: %s", cudaGetErrorString(e));
  return KSTAP_OK;
}

kstap_status kstap_graph_destroy(kstap_graph* G) {
  if (!G) return KSTAP_EINVAL;
  if (G->exec) {
    cudaDeviceSynchronize();
    cudaGraphExecDestroy(G->exec);
  }
  if (G->graph) cudaGraphDestroy(G->graph);
  for (auto s : G->streams) cudaStreamDestroy(s);
  for (auto p : G->allocs) cudaFree(p);
  delete G;
  return KSTAP_OK;
}

kstap_status kstap_autotune(kstap_ctx* ctx, const kstap_frame* frames, int n, int reps,
                            kstap_tuning* out) {
  if (!ctx) return KSTAP_EINVAL;
  if (reps < 1) reps = 3;
  const Tuning saved = ctx->tune;
  const bool prof = ctx->profile;
  ctx->profile = false;
  const std::vector<int> tcs =
      (ctx->prm.q >= 24) ? std::vector<int>{8, 16} : std::vector<int>{16, 32};
  const int wavesv[] = {1, 2, 4, 8, 16, 32, 64};
  std::vector<int> stores{1};
  if (ctx->prm.p <= 3) stores.push_back(0);
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  float best = 1e30f;
  Tuning bt = saved;
  kstap_status st = KSTAP_OK;
  for (size_t li = 0; li < stores.size() && st == KSTAP_OK; ++li)
  for (int tc : tcs) {
    const int ls = stores[li];
    std::string why;
    if (!smem_fits(make_geom(ctx->prm, ctx->V, tc), ls != 0, why)) continue;
    for (int w : wavesv) {
      ctx->tune.tc = tc;
      ctx->tune.waves = w;
      ctx->tune.lag_store = ls;
      st = kstap_run_batch(ctx, frames, n);   // warm-up (and workspace growth)
      if (st != KSTAP_OK) break;
      cudaEventRecord(a, ctx->stream);
      for (int r = 0; r < reps && st == KSTAP_OK; ++r) st = kstap_run_batch(ctx, frames, n);
      cudaEventRecord(b, ctx->stream);
      cudaEventSynchronize(b);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, a, b);
      ms /= reps;
      if (st == KSTAP_OK && ms < best) {
        best = ms;
        bt = ctx->tune;
      }
    }
    if (st != KSTAP_OK) break;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  ctx->profile = prof;
  if (st != KSTAP_OK) {
    ctx->tune = saved;
    return st;
  }
  ctx->tune = bt;
  if (out) {
    out->waves = bt.waves;
    out->tc = bt.tc > 0 ? bt.tc : default_tc(ctx->prm);
    out->lag_store = bt.lag_store;
    out->ms_per_batch = best;
  }
  return KSTAP_OK;
}

kstap_status kstap_set_tuning(kstap_ctx* ctx, const kstap_tuning* t) {
  if (!ctx || !t) return KSTAP_EINVAL;
  if (t->waves < 1 || t->waves > 64) return fail(ctx, KSTAP_EINVAL, "waves must be in [1, 64]");
  if (t->tc != 0 && t->tc != 8 && t->tc != 16 && t->tc != 32)
    return fail(ctx, KSTAP_EINVAL, "tc must be 0, 8, 16 or 32");
  if (t->lag_store != 0 && t->lag_store != 1)
    return fail(ctx, KSTAP_EINVAL, "lag_store must be 0 or 1");
  if (!t->lag_store && ctx->prm.p > 3)
    return fail(ctx, KSTAP_EINVAL, "stacked passes (p > 3) need the lag store");
  std::string why;
  if (!smem_fits(make_geom(ctx->prm, ctx->V, t->tc), t->lag_store != 0, why))
    return fail(ctx, KSTAP_EINVAL, "tc = %d: %s", t->tc, why.c_str());
  ctx->tune.waves = t->waves;
  ctx->tune.tc = t->tc;
  ctx->tune.lag_store = t->lag_store;
  return KSTAP_OK;
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

void server_shutdown(kstap_ctx* ctx);

kstap_status kstap_destroy(kstap_ctx* ctx) {
  if (!ctx) return KSTAP_EINVAL;
  server_shutdown(ctx);
  if (ctx->ws || ctx->bank_aT || ctx->jobs_dev || ctx->report)
    cudaStreamSynchronize(ctx->stream);
  for (int k = 0; k <= kstap_nkernels; ++k)
    if (ctx->ev[k][0]) {
      cudaEventDestroy(ctx->ev[k][0]);
      cudaEventDestroy(ctx->ev[k][1]);
    }
  cudaFree(ctx->ws);
  cudaFree(ctx->jobs_dev);
  cudaFree(ctx->bank_aT);
  cudaFree(ctx->bank_bT);
  cudaFree(ctx->bank_n2);
  cudaFree(ctx->report);
  cudaFree(ctx->bank_op);
  delete ctx;
  return KSTAP_OK;
}

kstap_status kstap_device_status(kstap_ctx* ctx) {
  if (!ctx) return KSTAP_EINVAL;
  KSTAP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  unsigned f = 0;
  KSTAP_CUDA(ctx, cudaMemcpy(&f, ctx->fault, sizeof(f), cudaMemcpyDeviceToHost));
  if (f) {
    KSTAP_CUDA(ctx, cudaMemset(ctx->fault, 0, sizeof(f)));
    if (f & 2u)
      return fail(ctx, KSTAP_ECUDA, "a tensor-core completion never arrived and the tile's tensor "
                  "memory was freed (fault word 0x%x): the device state is unknown", f);
    if (f & 4u)
      return fail(ctx, KSTAP_ECUDA, "a TMA tile load of the moments pass did not complete within "
                  "its bounded wait (fault word 0x%x)", f);
    return fail(ctx, KSTAP_ECUDA, "a tensor-core completion wait gave up (fault word 0x%x)", f);
  }
  return KSTAP_OK;
}

const char* kstap_last_error(const kstap_ctx* ctx) {
  return ctx ? ctx->err.c_str() : g_create_err.c_str();
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Serving: kstap_submit / kstap_poll / kstap_release.
//
// One worker thread per context admits pending requests in arrival order
// while their device memory fits the context's HBM budget, groups whatever is
// admissible into one batch (up to max_batch frames, same kernels as
// kstap_run_batch) and enqueues it on one of several streams, so that batches
// overlap on the device and requests arriving meanwhile join the next batch
// (continuous batching).  Scratch (workspace, factors, the device copy of a
// host frame, the job table) is allocated stream-ordered and freed right after
// the batch's kernels; results stay on the device until kstap_release.  A
// host callback on the stream stamps completion and returns the budget.
// ---------------------------------------------------------------------------
struct Server {
  struct Part {                     // one row strip of a request (or the whole frame)
    Frame fr;                       // Y view, outputs offset; factors filled at launch
    size_t scratch_bytes = 0;
    int state = 0;                  // 0 pending, 1 running, 2 done
  };
  struct Req {
    bool on_host = false;
    int H_in = 0, W_in = 0, H = 0, W = 0;
    int state = 0;                  // 0 pending, 1 running, 2 done, 3 error
    int remaining = 0;              // parts not yet done
    double t_submit = 0, t_admit = 0, t_done = 0;
    size_t out_bytes = 0;
    float* Tmax = nullptr;
    int32_t* vidx = nullptr;
    uint8_t* map = nullptr;
    void* out_mem = nullptr;
    std::vector<Part> parts;
  };
  struct Batch {
    Server* srv;
    std::vector<std::pair<uint64_t, int>> items;   // (ticket, part)
    size_t scratch_bytes = 0;
  };
  kstap_ctx* ctx = nullptr;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<std::pair<uint64_t, int>> pending;      // (ticket, part) in arrival order
  std::unordered_map<uint64_t, Req> reqs;
  std::thread worker;
  bool stop = false;
  size_t used = 0;
  int inflight = 0;
  int max_batch = 16;
  int max_inflight = 4;
  long long max_batch_cells = 1LL << 20;   // <= 0: no cap
  uint64_t next_ticket = 1;
  std::vector<cudaStream_t> streams;
  int rr = 0;
  int device = 0;
  std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
  std::string err;

  double now_us() const {
    return std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now() - t0)
        .count();
  }
};

namespace {

size_t factor_bytes(const kstap_params& p, size_t cells) {
  return cells * ((size_t)p.p * p.r_a * 8 + 2 * (size_t)p.q * p.r_b * 8 + (size_t)p.r_a * 4 +
                  (size_t)p.r_b * 4 + 4 + 4);
}

void CUDART_CB batch_done(void* arg) {
  Server::Batch* b = (Server::Batch*)arg;
  Server* s = b->srv;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    const double t = s->now_us();
    for (auto& it : b->items) {
      auto r = s->reqs.find(it.first);
      if (r == s->reqs.end()) continue;
      Server::Part& pt = r->second.parts[it.second];
      if (pt.state == 1) {
        pt.state = 2;
        if (--r->second.remaining == 0 && r->second.state == 1) {
          r->second.state = 2;
          r->second.t_done = t;
        }
      }
    }
    s->used -= b->scratch_bytes;
    s->inflight -= 1;
  }
  s->cv.notify_all();
  delete b;
}

// Enqueues one admitted batch (called by the worker without the lock held).
void launch_batch(Server* s, const std::vector<std::pair<uint64_t, int>>& items) {
  kstap_ctx* ctx = s->ctx;
  const kstap_params& p = ctx->prm;
  cudaStream_t st = s->streams[s->rr++ % s->streams.size()];
  std::vector<Frame> fr;
  std::vector<bool> host;
  Server::Batch* b = new Server::Batch{s, items, 0};
  {
    std::lock_guard<std::mutex> lock(s->mu);
    for (auto& it : items) {
      const Server::Req& r = s->reqs[it.first];
      fr.push_back(r.parts[it.second].fr);
      host.push_back(r.on_host);
      b->scratch_bytes += r.parts[it.second].scratch_bytes;
    }
  }
  std::vector<std::pair<int, int>> HW;
  size_t fbytes = 0, ybytes = 0;
  for (size_t k = 0; k < fr.size(); ++k) {
    const int H = fr[k].H_in - 2 * p.ring_r, W = fr[k].W_in - 2 * p.ring_a - p.q + 1;
    HW.push_back({H, W});
    fbytes += up256(factor_bytes(p, (size_t)H * W));
    if (host[k]) ybytes += up256((size_t)p.p * fr[k].H_in * fr[k].W_in * sizeof(kstap_c64));
  }
  const Layout L = make_layout(p, HW, store_lags(ctx));
  const size_t total = up256(L.total) + fbytes + ybytes + up256(fr.size() * sizeof(Job));
  char* mem = nullptr;
  kstap_status status = KSTAP_OK;
  if (cudaMallocAsync((void**)&mem, total, st) != cudaSuccess) {
    status = KSTAP_ENOMEM;
  } else {
    char* ws = mem;
    char* fac = mem + up256(L.total);
    char* yc = fac + fbytes;
    Job* jt = (Job*)(yc + ybytes);
    for (size_t k = 0; k < fr.size(); ++k) {
      const size_t cells = (size_t)HW[k].first * HW[k].second;
      char* q = fac;
      kstap_factors& f = fr[k].f;
      f.UA = (kstap_c64*)q;
      q += cells * p.p * p.r_a * 8;
      f.UB_hi = (kstap_c64*)q;
      q += cells * p.q * p.r_b * 8;
      f.UB_lo = (kstap_c64*)q;
      q += cells * p.q * p.r_b * 8;
      f.lamA = (float*)q;
      q += cells * p.r_a * 4;
      f.lamB = (float*)q;
      q += cells * p.r_b * 4;
      f.iters = (int32_t*)q;
      q += cells * 4;
      f.eta = (float*)q;
      fac += up256(factor_bytes(p, cells));
      if (host[k]) {
        // host frame: copy this part's rows of every channel to a dense device block
        const long long cs = fr[k].ch_stride ? fr[k].ch_stride
                                             : (long long)fr[k].H_in * fr[k].W_in;
        const size_t plane = (size_t)fr[k].H_in * fr[k].W_in;
        for (int i = 0; i < p.p; ++i)
          cudaMemcpyAsync(yc + i * plane * sizeof(kstap_c64), fr[k].Y + (size_t)i * cs,
                          plane * sizeof(kstap_c64), cudaMemcpyHostToDevice, st);
        fr[k].Y = (const kstap_c64*)yc;
        fr[k].ch_stride = (long long)plane;
        yc += up256(p.p * plane * sizeof(kstap_c64));
      }
    }
    if (fr.size() > 1) {
      const Geom g = make_geom(p, ctx->V, ctx->tune.tc);
      std::vector<Job> hj;
      JobList JL;
      fill_jobs(p, g, fr, ws, &L, hj, JL);
      cudaMemcpyAsync(jt, hj.data(), hj.size() * sizeof(Job), cudaMemcpyHostToDevice, st);
    }
    status = enqueue_batch(ctx, nullptr, fr, L, ws, jt, st);
    cudaFreeAsync(mem, st);
  }
  if (status != KSTAP_OK) {
    std::lock_guard<std::mutex> lock(s->mu);
    for (auto& it : items) s->reqs[it.first].state = 3;
    s->err = t_err_sink ? *t_err_sink : std::string("batch launch failed");
  }
  if (cudaLaunchHostFunc(st, batch_done, b) != cudaSuccess) {
    // could not register the completion callback: finish synchronously
    cudaStreamSynchronize(st);
    batch_done(b);
  }
}

void worker_loop(Server* s) {
  cudaSetDevice(s->device);
  std::string worker_err;
  t_err_sink = &worker_err;
  std::unique_lock<std::mutex> lock(s->mu);
  auto part_bytes = [&](const std::pair<uint64_t, int>& it) {
    return s->reqs[it.first].parts[it.second].scratch_bytes;
  };
  const kstap_params& p = s->ctx->prm;
  auto part_cells = [&](const std::pair<uint64_t, int>& it) {
    const Frame& f = s->reqs[it.first].parts[it.second].fr;
    return (long long)(f.H_in - 2 * p.ring_r) * (f.W_in - 2 * p.ring_a - p.q + 1);
  };
  while (true) {
    s->cv.wait(lock, [&] {
      if (s->stop) return true;
      if (s->pending.empty() || s->inflight >= s->max_inflight) return false;
      return !s->ctx->budget || s->used + part_bytes(s->pending.front()) <= s->ctx->budget ||
             s->inflight == 0;
    });
    if (s->stop) break;
    std::vector<std::pair<uint64_t, int>> batch;
    long long cells = 0;
    while (!s->pending.empty() && (int)batch.size() < s->max_batch) {
      const auto it = s->pending.front();
      const size_t need = part_bytes(it);
      if (s->ctx->budget && s->used + need > s->ctx->budget && !(batch.empty() && s->inflight == 0))
        break;
      const long long nc = part_cells(it);
      if (!batch.empty() && s->max_batch_cells > 0 && cells + nc > s->max_batch_cells) break;
      cells += nc;
      s->used += need;
      Server::Req& r = s->reqs[it.first];
      r.parts[it.second].state = 1;
      if (r.state == 0) {
        r.state = 1;
        r.t_admit = s->now_us();
      }
      batch.push_back(it);
      s->pending.pop_front();
    }
    if (batch.empty()) continue;
    s->inflight += 1;
    lock.unlock();
    launch_batch(s, batch);
    lock.lock();
  }
}

Server* get_server(kstap_ctx* ctx) {
  if (ctx->server) return ctx->server;
  Server* s = new Server();
  s->ctx = ctx;
  cudaGetDevice(&s->device);
  // keep freed stream-ordered allocations in the pool between batches
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, s->device) == cudaSuccess) {
    uint64_t thr = ~0ull;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  for (int k = 0; k < s->max_inflight; ++k) {
    cudaStream_t st;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    s->streams.push_back(st);
  }
  s->worker = std::thread(worker_loop, s);
  ctx->server = s;
  return s;
}

}  // namespace

void server_shutdown(kstap_ctx* ctx) {
  Server* s = ctx->server;
  if (!s) return;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  if (s->worker.joinable()) s->worker.join();
  for (auto st : s->streams) cudaStreamSynchronize(st);
  for (auto& kv : s->reqs)
    if (kv.second.out_mem) cudaFree(kv.second.out_mem);
  for (auto st : s->streams) cudaStreamDestroy(st);
  delete s;
  ctx->server = nullptr;
}

extern "C" {

kstap_status kstap_serve_batch_cells(kstap_ctx* ctx, long long cells) {
  if (!ctx) return KSTAP_EINVAL;
  Server* s = get_server(ctx);
  {
    std::lock_guard<std::mutex> lock(s->mu);
    if (s->next_ticket == 1) {   // nothing submitted yet
      s->max_batch_cells = cells;
      return KSTAP_OK;
    }
  }
  return fail(ctx, KSTAP_EINVAL, "configure serving before the first submit");
}

kstap_status kstap_serve_config(kstap_ctx* ctx, int max_batch, int max_inflight) {
  if (!ctx) return KSTAP_EINVAL;
  if (ctx->server) return fail(ctx, KSTAP_EINVAL, "configure serving before the first submit");
  if (max_batch < 1 || max_batch > 1024 || max_inflight < 1 || max_inflight > 16)
    return fail(ctx, KSTAP_EINVAL, "max_batch in [1, 1024], max_inflight in [1, 16]");
  Server* s = get_server(ctx);
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->max_batch = max_batch;
  }
  // rebuild the stream pool for the new in-flight limit
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  s->worker.join();
  for (auto st : s->streams) cudaStreamDestroy(st);
  s->streams.clear();
  s->stop = false;
  s->max_inflight = max_inflight;
  for (int k = 0; k < max_inflight; ++k) {
    cudaStream_t st;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    s->streams.push_back(st);
  }
  s->worker = std::thread(worker_loop, s);
  return KSTAP_OK;
}

kstap_status kstap_submit(kstap_ctx* ctx, const kstap_c64* Y, int H_in, int W_in, int flags,
                          uint64_t* ticket) {
  if (!ticket) return fail(ctx, KSTAP_EINVAL, "ticket is NULL");
  kstap_status st = check_frame(ctx, Y, H_in, W_in);
  if (st != KSTAP_OK) return st;
  const kstap_params& p = ctx->prm;
  Server::Req r;
  r.on_host = (flags & KSTAP_FRAME_ON_HOST) != 0;
  r.H_in = H_in;
  r.W_in = W_in;
  r.H = H_in - 2 * p.ring_r;
  r.W = W_in - 2 * p.ring_a - p.q + 1;
  const size_t cells = (size_t)r.H * r.W;
  r.out_bytes = up256(cells * 4) * 2 + up256(cells);
  auto part_scratch = [&](int rows) {
    return make_layout(p, {{rows, r.W}}, store_lags(ctx)).total + factor_bytes(p, (size_t)rows * r.W) +
           (r.on_host ? (size_t)p.p * (rows + 2 * p.ring_r) * W_in * sizeof(kstap_c64) : 0) +
           4096;
  };
  // frames whose scratch exceeds a quarter of the budget are served as row
  // strips admitted one by one (at least kMomRows rows each)
  int rows = r.H;
  if (ctx->budget && part_scratch(r.H) > ctx->budget / 4) {
    const size_t per_row = std::max<size_t>(1, part_scratch(1));
    rows = (int)std::max<size_t>(kstap::kMomRows, (ctx->budget / 4) / per_row);
    rows -= rows % kstap::kMomRows;
  }
  if (ctx->budget && part_scratch(std::min(rows, r.H)) + r.out_bytes > ctx->budget)
    return fail(ctx, KSTAP_ENOMEM, "frame needs %zu B per strip, more than the HBM budget %zu B",
                part_scratch(std::min(rows, r.H)) + r.out_bytes, ctx->budget);
  cudaError_t e = cudaMalloc(&r.out_mem, r.out_bytes);   // results, held until kstap_release
  if (e != cudaSuccess)
    return fail(ctx, KSTAP_ENOMEM, "result cudaMalloc(%zu): %s", r.out_bytes,
                cudaGetErrorString(e));
  r.Tmax = (float*)r.out_mem;
  r.vidx = (int32_t*)((char*)r.out_mem + up256(cells * 4));
  r.map = (uint8_t*)((char*)r.out_mem + 2 * up256(cells * 4));
  const Frame whole{Y, H_in, W_in, kstap_factors{}, r.Tmax, r.vidx, r.map, nullptr};
  const std::vector<Frame> strips =
      rows >= r.H ? std::vector<Frame>{whole} : split_rows(p, ctx->V, whole, rows);
  for (const Frame& f : strips) {
    Server::Part pt;
    pt.fr = f;
    pt.scratch_bytes = part_scratch(f.H_in - 2 * p.ring_r);
    r.parts.push_back(pt);
  }
  r.remaining = (int)r.parts.size();
  Server* s = get_server(ctx);
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->used += r.out_bytes;   // results count against the budget until released
    r.t_submit = s->now_us();
    const uint64_t tk = s->next_ticket++;
    const int np = (int)r.parts.size();
    s->reqs[tk] = std::move(r);
    for (int k = 0; k < np; ++k) s->pending.push_back({tk, k});
    *ticket = tk;
  }
  s->cv.notify_all();
  return KSTAP_OK;
}

kstap_status kstap_poll(kstap_ctx* ctx, uint64_t ticket, kstap_result* out, int timeout_us) {
  if (!ctx || !out) return KSTAP_EINVAL;
  Server* s = ctx->server;
  if (!s) return fail(ctx, KSTAP_ENOTFOUND, "no request was submitted");
  std::unique_lock<std::mutex> lock(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return fail(ctx, KSTAP_ENOTFOUND, "unknown ticket %llu",
                                       (unsigned long long)ticket);
  // a ticket released by another thread while this one waits counts as done
  auto ready = [&] {
    auto f = s->reqs.find(ticket);
    return f == s->reqs.end() || f->second.state >= 2;
  };
  if (!ready()) {
    if (timeout_us == 0) return KSTAP_EAGAIN;
    if (timeout_us < 0)
      s->cv.wait(lock, ready);
    else if (!s->cv.wait_for(lock, std::chrono::microseconds(timeout_us), ready))
      return KSTAP_ETIMEOUT;
  }
  it = s->reqs.find(ticket);
  if (it == s->reqs.end())
    return fail(ctx, KSTAP_ENOTFOUND, "ticket %llu was released while waiting",
                (unsigned long long)ticket);
  const Server::Req& r = it->second;
  if (r.state == 3) return fail(ctx, KSTAP_ECUDA, "request failed: %s", s->err.c_str());
  out->ticket = ticket;
  out->H = r.H;
  out->W = r.W;
  out->Tmax = r.Tmax;
  out->vidx = r.vidx;
  out->map = r.map;
  out->t_submit_us = r.t_submit;
  out->t_admit_us = r.t_admit;
  out->t_done_us = r.t_done;
  return KSTAP_OK;
}

kstap_status kstap_release(kstap_ctx* ctx, uint64_t ticket) {
  if (!ctx || !ctx->server) return KSTAP_EINVAL;
  Server* s = ctx->server;
  void* mem = nullptr;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end())
      return fail(ctx, KSTAP_ENOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
    if (it->second.state < 2) return fail(ctx, KSTAP_EAGAIN, "request still in flight");
    mem = it->second.out_mem;
    s->used -= it->second.out_bytes;
    s->reqs.erase(it);
  }
  s->cv.notify_all();
  if (mem) cudaFree(mem);
  return KSTAP_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free fit (kstap_fit_project_noalloc).  Its scratch -- the frame
// scale word and the per-cell moments M, block sums and flip-flop factor a --
// lives in this file-scope device array instead of a cudaMalloc'd workspace.
// Host code must not pass the array's name to a kernel: on the host it is only
// a stand-in symbol.  The device address is looked up with
// cudaGetSymbolAddress on the current device at every call (no caching, so a
// context torn down and recreated by cudaDeviceReset is picked up).  The B
// pass recomputes the lag sums (no lag store), which keeps the array at
// ~16.5 MB.
// ---------------------------------------------------------------------------
#define KSTAP_NOALLOC_MAX_CELLS 32768
#define KSTAP_NOALLOC_SCRATCH_BYTES (256 + (size_t)KSTAP_NOALLOC_MAX_CELLS * (45 + 9 + 9) * 8 + 1024)

static __device__ __align__(256) unsigned char g_noalloc_scratch[KSTAP_NOALLOC_SCRATCH_BYTES];

namespace {

// Device address of g_noalloc_scratch on the current device.
kstap_status noalloc_scratch(void** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p)
    return fail(nullptr, KSTAP_ECUDA, "cudaGetSymbolAddress(scratch) failed: %s",
                cudaGetErrorString(e));
  *out = p;
  return KSTAP_OK;
}

}  // namespace

extern "C" kstap_status kstap_fit_project_noalloc(const kstap_params* params, const kstap_c64* Y,
                                                  int H_in, int W_in,
                                                  const kstap_factors* factors,
                                                  void* cuda_stream) {
  std::string why;
  if (!valid_params(params, why)) return fail(nullptr, KSTAP_EINVAL, "%s", why.c_str());
  if (params->p != 3)
    return fail(nullptr, KSTAP_EINVAL, "kstap_fit_project_noalloc handles p == 3 only");
  if (!smem_fits(make_geom(*params, 1, 0), false, why))
    return fail(nullptr, KSTAP_EINVAL, "%s", why.c_str());
  if (!Y) return fail(nullptr, KSTAP_EINVAL, "Y is NULL");
  if (!factors || !factors->UA || !factors->UB_hi || !factors->UB_lo)
    return fail(nullptr, KSTAP_EINVAL, "factors (UA, UB_hi, UB_lo) must be non-NULL");
  if (H_in < 2 * params->ring_r + 1 || W_in < 2 * params->ring_a + params->q)
    return fail(nullptr, KSTAP_EINVAL, "frame %dx%d smaller than the training box plus window",
                H_in, W_in);
  const int H = H_in - 2 * params->ring_r, W = W_in - 2 * params->ring_a - params->q + 1;
  const size_t ncell = (size_t)H * W;
  if (ncell > KSTAP_NOALLOC_MAX_CELLS)
    return fail(nullptr, KSTAP_EINVAL,
                "frame has %zu cells; kstap_fit_project_noalloc handles at most %d cells "
                "(use kstap_fit_project, or split the frame into tiles)",
                ncell, KSTAP_NOALLOC_MAX_CELLS);
  const Layout L = make_layout(*params, {{H, W}}, false);
  if (L.total > KSTAP_NOALLOC_SCRATCH_BYTES)
    return fail(nullptr, KSTAP_EINVAL, "scratch layout %zu B exceeds the static %zu B", L.total,
                (size_t)KSTAP_NOALLOC_SCRATCH_BYTES);
  void* scratch = nullptr;
  kstap_status st = noalloc_scratch(&scratch);
  if (st != KSTAP_OK) return st;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const Geom g = make_geom(*params, 0, 0);
  std::vector<Frame> fr{Frame{Y, H_in, W_in, *factors, nullptr, nullptr, nullptr, nullptr}};
  std::vector<Job> jobs;
  JobList JL;
  fill_jobs(*params, g, fr, (char*)scratch, &L, jobs, JL);
  return dispatch_fit(nullptr, nullptr, g, JL, (char*)scratch, L, false, sms > 0 ? sms : 148, 4,
                      (cudaStream_t)cuda_stream);
}

// ------------------------------------------------ large-covariance fit -----
extern "C" kstap_status kstap_lrkron_fit(const kstap_c64* X, int n, int p, int q, int r_a,
                                         double eps, int max_iter, kstap_c64* A_out,
                                         kstap_c64* B_out, int32_t* iters, double* eta,
                                         void* cuda_stream) {
  if (!X || !B_out) return fail(nullptr, KSTAP_EINVAL, "X and B_out are required");
  if (n < 1 || n > kstap::kLrkMaxN || p < 1 || p > kstap::kLrkMaxP || q < 2 || q > 16384 ||
      r_a < 1 || r_a > p)
    return fail(nullptr, KSTAP_EINVAL,
                "need 1 <= n <= %d, 1 <= p <= %d, 2 <= q <= 16384, 1 <= r_a <= p",
                kstap::kLrkMaxN, kstap::kLrkMaxP);
  if (!(eps > 0.0)) eps = 1e-6;
  if (max_iter < 1) max_iter = 100;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const int np = n * p, p2 = p * p;
  const size_t nG = (size_t)np * np, nT = (size_t)p2 * p2;
  const size_t bytes = (nG + np + nT + 2 * (size_t)p2) * sizeof(double2) + 8 * sizeof(double);
  char* ws = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&ws, bytes, st);
  if (e != cudaSuccess)
    return fail(nullptr, KSTAP_ENOMEM, "cudaMallocAsync(%zu): %s", bytes, cudaGetErrorString(e));
  double2* G = (double2*)ws;
  double2* s = G + nG;
  double2* Tm = s + np;
  double2* Afin = Tm + nT;
  double2* Aprev = Afin + p2;
  double* info = (double*)(Aprev + p2);
  kstap_status res = KSTAP_OK;
  const size_t smem = 2 * (size_t)np * kstap::kLrkTile * sizeof(float2);
  double hinfo[5] = {0, 0, 0, 0, 0};
  do {
    kstap::k_lrk_gram<<<dim3(np, np + 1), 256, 0, st>>>((const float2*)X, np, q, G, s);
    kstap::k_lrk_tmat<<<(unsigned)((nT + 127) / 128), 128, 0, st>>>(G, n, p, Tm);
    kstap::k_lrk_iterate<<<1, 32, 0, st>>>(Tm, G, s, n, p, q, r_a, eps, max_iter, Afin, Aprev,
                                           info);
    if (A_out) kstap::k_lrk_aout<<<1, 64, 0, st>>>(Afin, info, p, (float2*)A_out);
    if ((e = cudaFuncSetAttribute(kstap::k_lrk_bout, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem)) != cudaSuccess)
      break;
    const unsigned nt = (unsigned)((q + kstap::kLrkTile - 1) / kstap::kLrkTile);
    kstap::k_lrk_bout<<<dim3(nt, nt), 256, smem, st>>>((const float2*)X, Aprev, info, n, p, q,
                                                       (float2*)B_out);
    if ((e = cudaGetLastError()) != cudaSuccess) break;
    if ((e = cudaMemcpyAsync(hinfo, info, sizeof(hinfo), cudaMemcpyDeviceToHost, st)) !=
        cudaSuccess)
      break;
  } while (0);
  cudaFreeAsync(ws, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess)
    return fail(nullptr, KSTAP_ECUDA, "kstap_lrkron_fit: %s", cudaGetErrorString(e));
  if (iters) *iters = (int32_t)hinfo[3];
  if (eta) *eta = hinfo[2];
  return res;
}

extern "C" kstap_status kstap_change_map(const float* T_all, long long ncell, int V, int K,
                                         float* Tmax_k, float* change, void* cuda_stream) {
  if (ncell < 0 || V < 1 || K < 1 || (ncell > 0 && !T_all))
    return fail(nullptr, KSTAP_EINVAL, "kstap_change_map: need ncell >= 0, V >= 1, K >= 1, T_all");
  if (ncell == 0) return KSTAP_OK;
  const unsigned blocks = (unsigned)std::min<long long>((ncell + 255) / 256, 148LL * 16);
  kstap::k_change<<<blocks, 256, 0, (cudaStream_t)cuda_stream>>>(T_all, ncell, V, K, Tmax_k,
                                                                 change);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    return fail(nullptr, KSTAP_ECUDA, "kstap_change_map: %s", cudaGetErrorString(e));
  return KSTAP_OK;
}
