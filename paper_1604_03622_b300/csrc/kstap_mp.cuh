// Kernels for stacked passes (Sec. 3: K registered passes as K p channels,
// rank-K spatial factor).  With p = 6 the p^2 x p^2 Gram M = R R^H has 666
// complex entries, too many for one thread, so the two steps that hold it run
// a warp per cell: k_mgram forms M and the block sums of S(i, k) from the
// exact lag store the moments pass wrote, and k_flipflop_w runs Alg. 2 on M.
// The B / U_B pass (k_bfit) and the projection (k_detect) are the
// single-pass kernels instantiated for more channels.  k_change forms the
// per-pass maxima of the statistic and their difference (the noncoherent
// change detection of Sec. 8).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace kstap {

constexpr int kWarpCells = 8;   // cells per CTA (one warp each) in k_mgram and k_flipflop_w

// Row J of the Hermitian upper-triangle index: the J with
// tri_idx(n, J, J) <= e < tri_idx(n, J + 1, J + 1).
__device__ __forceinline__ void tri_rowcol(int n, int e, int& J, int& K) {
  J = 0;
  while (J + 1 < n && tri_idx(n, J + 1, J + 1) <= e) ++J;
  K = J + (e - tri_idx(n, J, J));
}

// CTA = one cell row x kWarpCells cells, a warp per cell.  Per lag
// g = Q-1 .. 0 the tile's lag sums (hi parts of the float-float store) are
// staged as [position][J]; each lane accumulates its entries of
// W = sum_j l_g(c + j) l_g(c + j)^H and of the block sums s.  Before lag 0
// the negative lags are folded in (M += conj(Pi M Pi^T), s += conj(Pi s),
// Pi swapping the channel pair (i, k) -> (k, i)), as in the single-pass
// moments kernel.
template <int P, int Q>
__global__ void __launch_bounds__(kWarpCells * 32)
k_mgram(Geom g0, JobList JL, float2* __restrict__ Mw, float2* __restrict__ Sw,
        const float4* __restrict__ Lw0) {
  constexpr int PP = P * P;
  constexpr int NE = PP * (PP + 1) / 2;
  constexpr int EPL = (NE + 31) / 32;   // M entries per lane
  constexpr int SPL = (PP + 31) / 32;   // block sums per lane
  constexpr int TCm = kWarpCells;
  constexpr int NUmax = TCm + Q - 1;
  extern __shared__ __align__(16) unsigned char smem[];
  float2* Ls = reinterpret_cast<float2*>(smem);                 // [NUmax][PP]
  float2* Ft = Ls + NUmax * PP;                                 // [warps][NE] fold scratch
  float2* Fs = Ft + kWarpCells * NE;                            // [warps][PP]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int ejk[EPL];                                                 // (J | K << 8) of each entry
#pragma unroll
  for (int t = 0; t < EPL; ++t) {
    const int e = lane + 32 * t;
    int J = 0, K = 0;
    if (e < NE) tri_rowcol(PP, e, J, K);
    ejk[t] = J | (K << 8);
  }
  for (int tile = blockIdx.x; tile < JL.ntiles[kKindMgram]; tile += gridDim.x) {
    int lt;
    const Job& JB = job_of(JL, kKindMgram, tile, lt);
    const Geom g = with_job(g0, JB);
    const float4* __restrict__ Lw = Lw0 + JB.lag0;
    const int ntx = (g.W + TCm - 1) / TCm;
    const int r = lt / ntx, c0 = (lt % ntx) * TCm;
    const int cl = warp;
    const bool live = c0 + cl < g.W;
    const int WL = g.W + Q - 1;
    float2 acc[EPL], sacc[SPL];
#pragma unroll
    for (int t = 0; t < EPL; ++t) acc[t] = make_float2(0.f, 0.f);
#pragma unroll
    for (int t = 0; t < SPL; ++t) sacc[t] = make_float2(0.f, 0.f);
    for (int lagg = Q - 1; lagg >= 0; --lagg) {
      const int NU = TCm + Q - 1 - lagg;
      const float4* src = Lw + ((size_t)r * Q + lagg) * PP * WL;
      for (int idx = threadIdx.x; idx < PP * NU; idx += blockDim.x) {
        const int u = idx / PP, J = idx - u * PP;
        const float4 v = (c0 + u < WL) ? __ldg(src + (size_t)J * WL + c0 + u)
                                        : make_float4(0.f, 0.f, 0.f, 0.f);
        Ls[u * PP + J] = make_float2(v.x, v.z);
      }
      __syncthreads();
      if (lagg == 0) {
        // fold the negative lags into the sums over g > 0
        float2* ft = Ft + warp * NE;
        float2* fs = Fs + warp * PP;
#pragma unroll
        for (int t = 0; t < EPL; ++t)
          if (lane + 32 * t < NE) ft[lane + 32 * t] = acc[t];
#pragma unroll
        for (int t = 0; t < SPL; ++t)
          if (lane + 32 * t < PP) fs[lane + 32 * t] = sacc[t];
        __syncwarp();
#pragma unroll
        for (int t = 0; t < EPL; ++t) {
          if (lane + 32 * t >= NE) continue;
          const int J = ejk[t] & 255, K = ejk[t] >> 8;
          const int a = (J % P) * P + J / P, b = (K % P) * P + K / P;   // Pi J, Pi K
          const float2 w = (a <= b) ? ft[tri_idx(PP, a, b)] : cconj(ft[tri_idx(PP, b, a)]);
          acc[t] = cadd(acc[t], cconj(w));
        }
#pragma unroll
        for (int t = 0; t < SPL; ++t) {
          const int J = lane + 32 * t;
          if (J >= PP) continue;
          sacc[t] = cadd(sacc[t], cconj(fs[(J % P) * P + J / P]));
        }
        __syncwarp();
      }
      if (live) {
        for (int j = 0; j < Q - lagg; ++j) {
          const float2* l = Ls + (cl + j) * PP;
#pragma unroll
          for (int t = 0; t < EPL; ++t) {
            if (lane + 32 * t >= NE) continue;
            const float2 x = l[ejk[t] & 255], y = l[ejk[t] >> 8];
            acc[t].x += x.x * y.x + x.y * y.y;   // l[J] conj(l[K])
            acc[t].y += x.y * y.x - x.x * y.y;
          }
#pragma unroll
          for (int t = 0; t < SPL; ++t)
            if (lane + 32 * t < PP) sacc[t] = cadd(sacc[t], l[lane + 32 * t]);
        }
      }
      __syncthreads();
    }
    if (live) {
      const size_t ncell = (size_t)JL.NC;
      const size_t cell = (size_t)JB.cell0 + (size_t)r * g.W + (c0 + cl);
#pragma unroll
      for (int t = 0; t < EPL; ++t)
        if (lane + 32 * t < NE) Mw[(size_t)(lane + 32 * t) * ncell + cell] = acc[t];
#pragma unroll
      for (int t = 0; t < SPL; ++t)
        if (lane + 32 * t < PP) Sw[(size_t)(lane + 32 * t) * ncell + cell] = sacc[t];
    }
  }
}

// Alg. 2 on M with a warp per cell (see k_flipflop for the single-pass form):
// y = M a by rows over the lanes, the rank-r_a truncation of the P x P
// Hermitian A~ by a Jacobi sweep in lane 0, the stop rule
// |a_k+1 - a_k| <= eps |a_k+1|, eta from the closed form with float-float sums.
template <int P>
__global__ void __launch_bounds__(kWarpCells * 32)
k_flipflop_w(Geom g0, JobList JL, const float2* __restrict__ Mw, const float2* __restrict__ Sw,
             float2* __restrict__ aw) {
  constexpr int PP = P * P;
  constexpr int NE = PP * (PP + 1) / 2;
  constexpr int RPL = (PP + 31) / 32;   // rows of M per lane
  extern __shared__ __align__(16) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float2* Mt = reinterpret_cast<float2*>(smem) + warp * (NE + 3 * PP);
  float2* as = Mt + NE;          // a
  float2* ys = as + PP;          // y = M a
  float2* an_ = ys + PP;         // next a
  __shared__ int done_w[kWarpCells];
  __shared__ float2 UAw[kWarpCells][P * P];
  __shared__ float dw[kWarpCells][P];
  const size_t ncell = (size_t)JL.NC;
  const Geom& g = g0;
  const int ra = g.r_a;
  for (int tile = blockIdx.x; tile < JL.ntiles[kKindFlip]; tile += gridDim.x) {
    int lt;
    const Job& JB = job_of(JL, kKindFlip, tile, lt);
    const size_t local = (size_t)lt * kWarpCells + warp;
    if (local >= (size_t)JB.H * JB.W) continue;   // warp-uniform
    const size_t cell = (size_t)JB.cell0 + local;
    for (int e = lane; e < NE; e += 32) Mt[e] = Mw[(size_t)e * ncell + cell];
    for (int J = lane; J < PP; J += 32) as[J] = Sw[(size_t)J * ncell + cell];
    __syncwarp();
    for (int J = lane; J < PP; J += 32) {   // a_0 ~ block sums of S, Hermitised
      const int i = J % P, k = J / P;
      const float2 x = as[i + P * k], y = as[k + P * i];
      an_[J] = make_float2(0.5f * (x.x + y.x), 0.5f * (x.y - y.y));
    }
    __syncwarp();
    for (int J = lane; J < PP; J += 32) as[J] = an_[J];
    __syncwarp();
    const float tol2 = g.eps * g.eps;
    int it = 0;
    if (lane == 0) {
      done_w[warp] = 0;
      for (int i = 0; i < P; ++i) {     // factors of a cell whose first iterate is degenerate
        dw[warp][i] = 0.f;
        for (int m = 0; m < P; ++m) UAw[warp][i * P + m] = make_float2(i == m ? 1.f : 0.f, 0.f);
      }
    }
    __syncwarp();
    for (it = 1; it <= g.max_iter; ++it) {
      float an = 0.f, aMa = 0.f;
#pragma unroll
      for (int t = 0; t < RPL; ++t) {
        const int J = lane + 32 * t;
        if (J >= PP) continue;
        float2 s = make_float2(0.f, 0.f);
        for (int K = 0; K < PP; ++K) {
          const float2 m = (J <= K) ? Mt[tri_idx(PP, J, K)] : cconj(Mt[tri_idx(PP, K, J)]);
          s = cadd(s, cmul(m, as[K]));
        }
        ys[J] = s;
        an += cabs2(as[J]);
        aMa += as[J].x * s.x + as[J].y * s.y;
      }
      an = warp_sum(an);
      aMa = warp_sum(aMa);
      if (!(aMa > 0.f) || !(an > 0.f)) break;   // warp-uniform
      __syncwarp();
      if (lane == 0) {
        const float f = an / aMa;
        float2 At[P][P], U[P][P];
        float d[P];
#pragma unroll
        for (int i = 0; i < P; ++i)
#pragma unroll
          for (int k = 0; k < P; ++k) {
            const float2 x = ys[i + P * k], z = ys[k + P * i];
            At[i][k] = make_float2(0.5f * f * (x.x + z.x), 0.5f * f * (x.y - z.y));
          }
        jacobi_small<P>(At, d, U);
        float dn = 0.f, nn = 0.f;
#pragma unroll
        for (int i = 0; i < P; ++i)
#pragma unroll
          for (int k = 0; k < P; ++k) {
            float2 s = make_float2(0.f, 0.f);
#pragma unroll
            for (int m = 0; m < P; ++m)
              if (m < ra) s = cadd(s, cscale(cmul(U[i][m], cconj(U[k][m])), d[m]));
            dn += cabs2(csub(s, as[i + P * k]));
            nn += cabs2(s);
            an_[i + P * k] = s;
          }
#pragma unroll
        for (int i = 0; i < P; ++i) {
          dw[warp][i] = d[i];
#pragma unroll
          for (int m = 0; m < P; ++m) UAw[warp][i * P + m] = U[i][m];
        }
        done_w[warp] = dn <= tol2 * nn;
      }
      __syncwarp();
      for (int J = lane; J < PP; J += 32) as[J] = an_[J];
      __syncwarp();
      if (done_w[warp]) break;
    }
    const bool noconv = it > g.max_iter;
    if (noconv) it = g.max_iter;
    if (JL.report && lane == 0) count_lanes(JL.report, noconv);
    // eta^2 = 1 - a^H M a / (|a|^2 tr M), float-float sums over the lanes' rows
    float trs = 0.f, trc = 0.f, ans = 0.f, anc = 0.f, qs = 0.f, qc = 0.f;
#pragma unroll
    for (int t = 0; t < RPL; ++t) {
      const int J = lane + 32 * t;
      if (J >= PP) continue;
      const float dM = Mt[tri_idx(PP, J, J)].x;
      float tt, e;
      two_sum(trs, dM, tt, e);
      trs = tt;
      trc = __fadd_rn(trc, e);
      float p1, pe;
      two_prod(as[J].x, as[J].x, p1, pe);
      acc_ffxf(ans, anc, p1, pe, 1.f);
      acc_ffxf(qs, qc, p1, pe, dM);
      two_prod(as[J].y, as[J].y, p1, pe);
      acc_ffxf(ans, anc, p1, pe, 1.f);
      acc_ffxf(qs, qc, p1, pe, dM);
      for (int K = J + 1; K < PP; ++K) {   // 2 Re(conj(a_J) M_JK a_K)
        const float2 m = Mt[tri_idx(PP, J, K)];
        float rs = 0.f, rc = 0.f, is = 0.f, ic = 0.f;
        acc_prod(rs, rc, m.x, as[K].x);
        acc_prod(rs, rc, -m.y, as[K].y);
        acc_prod(is, ic, m.x, as[K].y);
        acc_prod(is, ic, m.y, as[K].x);
        acc_ffxf(qs, qc, rs, rc, 2.f * as[J].x);
        acc_ffxf(qs, qc, is, ic, 2.f * as[J].y);
      }
    }
    const ff trf = ff_warp_sum(ff_make(trs, trc)), anf = ff_warp_sum(ff_make(ans, anc));
    const ff qf = ff_warp_sum(ff_make(qs, qc));
    for (int J = lane; J < PP; J += 32) aw[(size_t)J * ncell + cell] = as[J];
    // cells whose box holds a NaN / Inf sample: iters = -1, eta = NaN
    bool bad = false;
    if (JB.maxbits && JB.maxbits[1]) {
      const Geom gj = with_job(g0, JB);
      bad = box_nonfinite(JB.Y, gj, (int)(local / JB.W), (int)(local % JB.W), lane, 32);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) bad |= __shfl_xor_sync(0xffffffffu, bad, o);
      if (JL.report && lane == 0) count_lanes(JL.report + 1, bad);
    }
    if (lane == 0) {
      float trA = 0.f;
#pragma unroll
      for (int m = 0; m < P; ++m)
        if (m < ra) trA += dw[warp][m];
      const float sc = (trA != 0.f) ? (float)P / trA : 1.f;
      for (int i = 0; i < P; ++i)
        for (int m = 0; m < ra; ++m) JB.UA[(local * P + i) * ra + m] = UAw[warp][i * P + m];
      if (JB.lamA)
        for (int m = 0; m < ra; ++m) JB.lamA[local * ra + m] = dw[warp][m] * sc;
      if (JB.iters) JB.iters[local] = bad ? -1 : it;
      if (JB.eta) {
        const double tr = (double)trf.hi + trf.lo, an = (double)anf.hi + anf.lo;
        const double aMa = (double)qf.hi + qf.lo;
        const double e2 = (tr > 0.0 && an > 0.0) ? 1.0 - aMa / (an * tr) : 0.0;
        JB.eta[local] = bad ? __int_as_float(0x7fc00000) : (float)sqrt(e2 > 0.0 ? e2 : 0.0);
      }
    }
    __syncwarp();
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
