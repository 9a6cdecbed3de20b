// Non-template kernels of libkstap, compiled once (in kstap_api.cu): the
// frame scan that sets the fixed-point scale, and the noncoherent change map
// of stacked passes (Sec. 8).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "kstap_kernels.cuh"

namespace kstap {

// ------------------------------------------------------- frame scale -------
// max |component| of Y via the order-preserving bit pattern of non-negative
// floats; non-finite values are recorded in *nonfinite.
__global__ void k_frame_maxabs(Geom g0, JobList L) {
  const Job& J = L.table ? L.table[blockIdx.y] : L.one;
  const float* __restrict__ Y = reinterpret_cast<const float*>(J.Y);
  const size_t plane = 2 * (size_t)J.H_in * J.W_in;   // floats of one channel of this job
  const size_t nfloat = plane * g0.p;
  unsigned* maxbits = J.maxbits;
  unsigned* nonfinite = J.maxbits + 1;
  unsigned m = 0, bad = 0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nfloat;
       i += (size_t)gridDim.x * blockDim.x) {
    const size_t ch = i / plane;
    const float a = fabsf(__ldg(Y + ch * 2 * (size_t)J.ch_stride + (i - ch * plane)));
    if (a <= kFltMax) {
      m = max(m, __float_as_uint(a));
    } else {
      bad = 1;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    bad |= __shfl_xor_sync(0xffffffffu, bad, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(maxbits, m);
    if (bad) atomicOr(nonfinite, 1u);
  }
}

// Per cell: Tmax_k = max over the V velocities of pass k of T_all (K V per
// cell, pass-major), and change = Tmax_{K-1} - Tmax_0 (mission minus
// reference pixel magnitude after filtering).
__global__ void k_change(const float* __restrict__ T_all, long long ncell, int V, int K,
                         float* __restrict__ Tmax_k, float* __restrict__ change) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell;
       c += (long long)gridDim.x * blockDim.x) {
    const float* t = T_all + c * (long long)K * V;
    float first = 0.f, last = 0.f;
    for (int k = 0; k < K; ++k) {
      float m = t[(size_t)k * V];
      for (int v = 1; v < V; ++v) m = fmaxf(m, t[(size_t)k * V + v]);
      if (Tmax_k) Tmax_k[(size_t)k * ncell + c] = m;
      if (k == 0) first = m;
      last = m;
    }
    if (change) change[c] = last - first;
  }
}

}  // namespace kstap
