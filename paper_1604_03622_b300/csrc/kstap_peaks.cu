// Throughput probes of the arithmetic pipes that bound the Kron-STAP kernels:
// FP32 fused multiply-add, packed f32x2 FMA (two lanes per instruction),
// 64-bit integer multiply-add (the exact lag sums) and FP64 FMA (the
// ill-gapped eigen path).  They are the measured denominators of the
// kernels' arithmetic roofline fractions; the paper has no counterpart.
//
// Each thread runs kChains independent dependency chains, so that the issue
// of one chain's next operation never waits for the previous result, and the
// grid holds SMs x kBlocksPerSm CTAs of 256 threads (64 warps per SM).  The
// chains' final values feed a comparison that is never true, which keeps the
// work from being eliminated.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/kstap.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreadsPerCta = 256;
constexpr int kBlocksPerSm = 8;

template <int OP>
__global__ void __launch_bounds__(kThreadsPerCta) k_alu_probe(int iters, float seed,
                                                              unsigned long long* sink) {
  const float s = seed + (float)threadIdx.x * 1e-7f;
  bool hit = false;
  if constexpr (OP == KSTAP_PROBE_FFMA) {
    float a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = s + (float)c;
    const float m = 0.9999999f, b = 1e-7f;
    for (int i = 0; i < iters; i += 4) {
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = __fmaf_rn(a[c], m, b);
    }
    float t = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) t += a[c];
    hit = (t == -1.f);
  } else if constexpr (OP == KSTAP_PROBE_FFMA2) {
    float2 a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = make_float2(s + (float)c, s - (float)c);
    const float2 m = make_float2(0.9999999f, 0.9999998f), b = make_float2(1e-7f, 2e-7f);
    for (int i = 0; i < iters; i += 4) {
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = __ffma2_rn(a[c], m, b);
    }
    float t = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) t += a[c].x + a[c].y;
    hit = (t == -1.f);
  } else if constexpr (OP == KSTAP_PROBE_IMAD64) {
    long long a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = (long long)threadIdx.x * 977 + c;
    const long long m = 6364136223846793005LL, b = 1442695040888963407LL;
    for (int i = 0; i < iters; i += 4) {
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = a[c] * m + b;
    }
    long long t = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) t ^= a[c];
    hit = (t == 0x7fffffffffffffffLL);
  } else {
    double a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = (double)s + (double)c;
    const double m = 0.9999999999, b = 1e-12;
    for (int i = 0; i < iters; i += 4) {
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = __fma_rn(a[c], m, b);
    }
    double t = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) t += a[c];
    hit = (t == -1.0);
  }
  if (hit) atomicAdd(sink, 1ull);
}

template <int OP>
cudaError_t launch(int blocks, int iters, unsigned long long* sink, cudaStream_t st) {
  k_alu_probe<OP><<<blocks, kThreadsPerCta, 0, st>>>(iters, 1.f, sink);
  return cudaGetLastError();
}

}  // namespace

extern "C" kstap_status kstap_alu_probe(int op, int iters, int reps, void* cuda_stream,
                                        double* ops_per_s) {
  if (op < KSTAP_PROBE_FFMA || op > KSTAP_PROBE_DFMA || iters < 4 || reps < 1 || !ops_per_s)
    return KSTAP_EINVAL;
  iters &= ~3;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
    return KSTAP_ECUDA;
  const int blocks = sms * kBlocksPerSm;
  unsigned long long* sink = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&sink, sizeof(*sink), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(sink, 0, sizeof(*sink), st);
  if (e == cudaSuccess) e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  auto run = [&]() -> cudaError_t {
    switch (op) {
      case KSTAP_PROBE_FFMA: return launch<KSTAP_PROBE_FFMA>(blocks, iters, sink, st);
      case KSTAP_PROBE_FFMA2: return launch<KSTAP_PROBE_FFMA2>(blocks, iters, sink, st);
      case KSTAP_PROBE_IMAD64: return launch<KSTAP_PROBE_IMAD64>(blocks, iters, sink, st);
      default: return launch<KSTAP_PROBE_DFMA>(blocks, iters, sink, st);
    }
  };
  if (e == cudaSuccess) e = run();   // warm-up
  if (e == cudaSuccess) e = cudaEventRecord(a, st);
  for (int r = 0; r < reps && e == cudaSuccess; ++r) e = run();
  if (e == cudaSuccess) e = cudaEventRecord(b, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(b);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
  if (sink) cudaFreeAsync(sink, st);
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (e != cudaSuccess || !(ms > 0.f)) return KSTAP_ECUDA;
  // one operation = one FMA (or multiply-add) per lane; packed f32x2 counts
  // both lanes
  const double lanes = (op == KSTAP_PROBE_FFMA2) ? 2.0 : 1.0;
  const double ops = (double)blocks * kThreadsPerCta * (double)iters * kChains * lanes * reps;
  *ops_per_s = ops / (ms * 1e-3);
  return KSTAP_OK;
}
