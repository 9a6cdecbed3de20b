// Kernels for stacked passes (Sec. 3: K registered passes as K p channels,
// rank-K spatial factor).  With p = 6 the p^2 x p^2 Gram M = R R^H has 666
// complex entries, too many for one thread's registers: k_mgram forms M and
// the block sums of S(i, k) from the exact lag store the moments pass wrote,
// a warp per strip of cells with sliding windows, and k_flipflop_t runs
// Alg. 2 with a thread per cell, streaming M from the per-cell arrays.
// The B / U_B pass (k_bfit) and the projection (k_detect) are the
// single-pass kernels instantiated for more channels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace kstap {

constexpr int kFlipThreads = 64;  // cells per CTA (one thread each) in k_flipflop_t

// Row J of the Hermitian upper-triangle index: the J with
// tri_idx(n, J, J) <= e < tri_idx(n, J + 1, J + 1).
__device__ __forceinline__ void tri_rowcol(int n, int e, int& J, int& K) {
  J = 0;
  while (J + 1 < n && tri_idx(n, J + 1, J + 1) <= e) ++J;
  K = J + (e - tri_idx(n, J, J));
}

// M = R R^H and the block sums of S(i, k) from the lag store, a CTA of two
// warps per strip of kStrip consecutive cells of one row.  With l_g(u) the
// PP-vector of lag-g sums at position u (hi parts of the float-float store),
//   M(c) = F(X(c)),  X(c) = sum_g w_g sum_{u = c}^{c+Q-1-g} l_g(u) l_g(u)^H,
// w_0 = 1/2, w_g = 1 otherwise, and F(X) = X + conj(Pi X Pi^T) (Pi swaps the
// channel pair (i, k) -> (k, i); the negative lags are the Pi-conjugates of
// the positive ones, and the lag-0 term is its own, hence the half weight).
// Neighbouring cells share all but two positions per lag, so the CTA forms
// X of its strip's first cell directly and then slides the windows:
//   X(c+1) = X(c) + sum_g w_g (l_g(c+Q-g) l_g(c+Q-g)^H - l_g(c) l_g(c)^H),
// 2Q outer products per cell instead of sum_g (Q - g) (restarting every
// kStrip cells bounds the rounding growth of the running sums).  Lane
// b < P(P+1)/2 of warp h holds rows P I + a, a in [hP/2, (h+1)P/2), of the
// P x P block (I, K), I <= K, of X (columns P K + b); lanes above that in
// warp 0 hold the block sums.  The current windows sit in a shared-memory
// ring per lag (Q - g + 1 slots: the position that enters at a step lands in
// the slot after the window), read by both warps; the next step's entering
// positions are loaded into registers while the warps compute.
constexpr int kStrip = 32;   // cells per CTA tile of k_mgram

template <int Q>
__host__ __device__ constexpr int ring_off(int g) {   // first ring slot of lag g
  return g * (Q + 1) - (g * (g - 1)) / 2;
}

template <int P, int Q>
__global__ void __launch_bounds__(64)
k_mgram(Geom g0, JobList JL, float2* __restrict__ Mw, float2* __restrict__ Sw,
        const float4* __restrict__ Lw0) {
  constexpr int PP = P * P;
  constexpr int NBP = P * (P + 1) / 2;   // blocks of M on and above the diagonal
  constexpr int HR = P / 2;              // block rows per warp
  static_assert(NBP < 32 && P % 2 == 0 && HR % 1 == 0, "a half block per lane");
  constexpr int NSL = 32 - NBP;          // lanes of warp 0 for the block sums
  constexpr int SPL = (PP + NSL - 1) / NSL;
  constexpr int NSLOT = ring_off<Q>(Q);  // ring slots of all lags
  constexpr int NEW = Q * PP;            // entries of one step's entering positions
  constexpr int NPL = (NEW + 63) / 64;   // of them per thread
  constexpr int NX = kStrip + Q;         // offsets u - c0 that occur
  extern __shared__ __align__(16) unsigned char smem[];
  float2* ring = reinterpret_cast<float2*>(smem);   // [NSLOT][PP]
  float2* ft = ring + NSLOT * PP;                   // [PP][PP] fold scratch
  float2* fs = ft + PP * PP;                        // [PP]
  __shared__ unsigned char slot_tab[Q][NX];         // (u - c0) mod (Q - g + 1)
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int e = tid; e < Q * NX; e += 64) slot_tab[e / NX][e % NX] = (unsigned char)((e % NX) % (Q - e / NX + 1));
  __syncthreads();
  const bool mlane = lane < NBP;
  const bool slane = warp == 0 && !mlane;
  const int a0 = warp * HR;
  int bI = 0, bK = 0;
  if (mlane) tri_rowcol(P, lane, bI, bK);
  const size_t ncell = (size_t)JL.NC;
  for (int tile = blockIdx.x; tile < JL.ntiles[kKindMgram]; tile += gridDim.x) {
    int lt;
    const Job& JB = job_of(JL, kKindMgram, tile, lt);
    const Geom g = with_job(g0, JB);
    const float4* __restrict__ Lw = Lw0 + JB.lag0;
    const int ntx = (g.W + kStrip - 1) / kStrip;
    const int r = lt / ntx, c0 = (lt % ntx) * kStrip;
    const int ncl = min(kStrip, g.W - c0);
    const int WL = g.W + Q - 1;
    const float4* __restrict__ rowL = Lw + (size_t)r * Q * PP * WL;
    // lag-g sum J at position u: rowL[(g PP + J) WL + u]; its ring slot is
    // ring_off(g) + (u - c0) mod (Q - g + 1)
    auto slot = [&](int lg, int u) { return ring_off<Q>(lg) + slot_tab[lg][u - c0]; };
    // the first cell's windows: positions c0 .. c0 + Q - 1 - g of every lag
    for (int e = tid; e < NSLOT * PP; e += 64) {
      const int sl = e / PP, J = e - sl * PP;
      int lg = 0;
      while (lg + 1 < Q && ring_off<Q>(lg + 1) <= sl) ++lg;
      const int k = sl - ring_off<Q>(lg);   // position c0 + k
      if (k < Q - lg) {
        ring[sl * PP + J] = __ldg(reinterpret_cast<const float2*>(rowL + ((size_t)lg * PP + J) * WL + c0 + k));
      }
    }
    __syncthreads();
    float2 acc[HR][P], sacc[SPL];
#pragma unroll
    for (int a = 0; a < HR; ++a)
#pragma unroll
      for (int b = 0; b < P; ++b) acc[a][b] = make_float2(0.f, 0.f);
#pragma unroll
    for (int t = 0; t < SPL; ++t) sacc[t] = make_float2(0.f, 0.f);
    // w l l^H into the thread's half block, or w l into the block sums
    // (w = +-1 folds into the multiply-adds; lag 0 passes its half weight)
    auto outer = [&](const float2* l, float w) {
      if (mlane) {
        float2 x[HR], y[P];
        const float2* lx = l + P * bI + a0;
        const float4* ly = reinterpret_cast<const float4*>(l + P * bK);
#pragma unroll
        for (int a = 0; a < HR; ++a) x[a] = w == 1.f ? lx[a] : make_float2(w * lx[a].x, w * lx[a].y);
#pragma unroll
        for (int h = 0; h < P / 2; ++h) {
          const float4 u = ly[h];
          y[2 * h] = make_float2(u.x, u.y);
          y[2 * h + 1] = make_float2(u.z, u.w);
        }
#pragma unroll
        for (int a = 0; a < HR; ++a)
#pragma unroll
          for (int b = 0; b < P; ++b) {   // x[a] conj(y[b])
            acc[a][b].x += x[a].x * y[b].x + x[a].y * y[b].y;
            acc[a][b].y += x[a].y * y[b].x - x[a].x * y[b].y;
          }
      } else if (slane) {
#pragma unroll
        for (int t = 0; t < SPL; ++t) {
          const int J = (lane - NBP) + NSL * t;
          if (J < PP) sacc[t] = make_float2(sacc[t].x + w * l[J].x, sacc[t].y + w * l[J].y);
        }
      }
    };
#pragma unroll 1
    for (int lg = 0; lg < Q; ++lg) {
      const float w = lg == 0 ? 0.5f : 1.f;
#pragma unroll 1
      for (int k = 0; k < Q - lg; ++k) outer(ring + (ring_off<Q>(lg) + k) * PP, w);
    }
    float2 nv[NPL];
    auto load_new = [&](int c) {   // positions c + Q - 1 - g entering the windows of cell c
#pragma unroll
      for (int t = 0; t < NPL; ++t) {
        const int e = tid + 64 * t;
        nv[t] = make_float2(0.f, 0.f);
        if (e < NEW) {
          const int lg = e / PP, J = e - lg * PP;
          nv[t] = __ldg(reinterpret_cast<const float2*>(rowL + ((size_t)lg * PP + J) * WL + c + Q - 1 - lg));
        }
      }
    };
    if (ncl > 1) load_new(c0 + 1);
#pragma unroll 1
    for (int cl = 0; cl < ncl; ++cl) {
      const int c = c0 + cl;
      if (cl > 0) {
        // slide every window from cell c - 1 to c: the positions c + Q - 1 - g
        // enter (from registers into their ring slots), c - 1 leaves
#pragma unroll
        for (int t = 0; t < NPL; ++t) {
          const int e = tid + 64 * t;
          if (e < NEW) {
            const int lg = e / PP, J = e - lg * PP;
            ring[slot(lg, c + Q - 1 - lg) * PP + J] = nv[t];
          }
        }
        __syncthreads();
        if (cl + 1 < ncl) load_new(c + 1);
#pragma unroll 1
        for (int lg = 0; lg < Q; ++lg) {
          const float w = lg == 0 ? 0.5f : 1.f;
          outer(ring + slot(lg, c + Q - 1 - lg) * PP, w);
          outer(ring + slot(lg, c - 1) * PP, -w);
        }
      }
      // M(c) = X + conj(Pi X Pi^T): the whole Hermitian X through shared
      // memory; Pi maps entry (a, b) of block (I, K) to entry (I, K) of
      // block (a, b), so each thread reads its partners at fixed offsets
      if (mlane) {
#pragma unroll
        for (int a = 0; a < HR; ++a)
#pragma unroll
          for (int b = 0; b < P; ++b) {
            if (bI == bK && a0 + a > b) continue;
            const int J = P * bI + a0 + a, K = P * bK + b;
            ft[J * PP + K] = acc[a][b];
            ft[K * PP + J] = cconj(acc[a][b]);
          }
      } else if (slane) {
#pragma unroll
        for (int t = 0; t < SPL; ++t) {
          const int J = (lane - NBP) + NSL * t;
          if (J < PP) fs[J] = sacc[t];
        }
      }
      __syncthreads();
      const size_t cell = (size_t)JB.cell0 + (size_t)r * g.W + c;
      if (mlane) {
        const float2* fp = ft + bI * PP + bK;   // X[P a + I][P b + K] = fp[a P PP + b P]
#pragma unroll
        for (int a = 0; a < HR; ++a)
#pragma unroll
          for (int b = 0; b < P; ++b) {
            if (bI == bK && a0 + a > b) continue;
            const int J = P * bI + a0 + a, K = P * bK + b;
            Mw[(size_t)tri_idx(PP, J, K) * ncell + cell] =
                cadd(acc[a][b], cconj(fp[(a0 + a) * P * PP + b * P]));
          }
      } else if (slane) {
#pragma unroll
        for (int t = 0; t < SPL; ++t) {
          const int J = (lane - NBP) + NSL * t;
          if (J < PP) Sw[(size_t)J * ncell + cell] = cadd(sacc[t], cconj(fs[(J % P) * P + J / P]));
        }
      }
    }
    __syncthreads();   // the next tile refills the ring
  }
}

// Alg. 2 on M with a thread per cell (the single-pass kernel k_flipflop holds
// M in registers; here the 666 entries of M are streamed from the per-cell
// arrays each iteration, coalesced over the cells of a warp, and each entry
// serves both y_J += M_JK a_K and y_K += conj(M_JK) a_J).  The thread's a, y
// and leading eigenvectors sit in shared memory ([entry][thread], so the
// lanes of a warp hit distinct banks) and the loops over them stay rolled:
// a fully unrolled 36 x 36 product does not fit the instruction cache.  The
// rank-r_a truncation of the P x P Hermitian A~ = vec^-1(y) |a|^2 / a^H M a
// is a cyclic Jacobi in registers whose off-diagonal entries below the
// rounding level of the matrix are dropped, not rotated (only the leading
// r_a eigenpairs are used).  Stop rule |a_k+1 - a_k| <= eps |a_k+1|; eta from
// the closed form with float-float sums, as in k_flipflop.
template <int P>
__global__ void __launch_bounds__(kFlipThreads)
k_flipflop_t(Geom g0, JobList JL, const float2* __restrict__ Mw, const float2* __restrict__ Sw,
             float2* __restrict__ aw) {
  constexpr int PP = P * P;
  constexpr int RA = 2;                             // largest r_a of this route
  constexpr int nt = kFlipThreads;
  extern __shared__ __align__(16) unsigned char smem[];
  float2* as = reinterpret_cast<float2*>(smem);     // [PP][nt] a
  float2* ys = as + PP * nt;                        // [PP][nt] y = M a
  float2* Ut = ys + PP * nt;                        // [P RA][nt] leading eigenvectors
  const size_t ncell = (size_t)JL.NC;
  const int tid = threadIdx.x;
  float2* a_ = as + tid;
  float2* y_ = ys + tid;
  for (int tile = blockIdx.x; tile < JL.ntiles[kKindFlip]; tile += gridDim.x) {
  int lt;
  const Job& JB = job_of(JL, kKindFlip, tile, lt);
  const Geom& g = g0;
  const size_t local = (size_t)lt * nt + tid;
  if (local >= (size_t)JB.H * JB.W) continue;
  const size_t cell = (size_t)JB.cell0 + local;
  const float2* __restrict__ Mc = Mw + cell;        // entry e at Mc[e ncell]
  // a_0 = R 1 / q^2 is proportional to the sum of S's block entries; Hermitise.
#pragma unroll 1
  for (int J = 0; J < PP; ++J) {
    const int i = J % P, k = J / P;
    const float2 x = Sw[J * ncell + cell], z = Sw[(k + P * i) * ncell + cell];
    a_[J * nt] = make_float2(0.5f * (x.x + z.x), 0.5f * (x.y - z.y));
  }
  const int ra = g.r_a;
  // the leading r_a eigenpairs of the last truncation (identity columns and
  // zeros for a cell whose first iterate is degenerate)
  float dt[RA];
#pragma unroll
  for (int m = 0; m < RA; ++m) {
    dt[m] = 0.f;
#pragma unroll
    for (int i = 0; i < P; ++i) Ut[(i * RA + m) * nt + tid] = make_float2(i == m ? 1.f : 0.f, 0.f);
  }
  int it = 0;
  const float tol2 = g.eps * g.eps;
  float dn_prev = kFltMax;
  for (it = 1; it <= g.max_iter; ++it) {
#pragma unroll 1
    for (int J = 0; J < PP; ++J) y_[J * nt] = make_float2(0.f, 0.f);
    const float2* mp = Mc;
    float an = 0.f, aMa = 0.f;
#pragma unroll 1
    for (int J = 0; J < PP; ++J) {
      const float2 aJ = a_[J * nt];
      float2 yJ = cadd(y_[J * nt], cmul(__ldg(mp), aJ));   // diagonal (real) entry
      mp += ncell;
#pragma unroll 4
      for (int K = J + 1; K < PP; ++K) {   // upper-triangle order
        const float2 m = __ldg(mp);
        mp += ncell;
        yJ = cadd(yJ, cmul(m, a_[K * nt]));
        y_[K * nt] = cadd(y_[K * nt], cmulc(m, aJ));
      }
      y_[J * nt] = yJ;
      an += cabs2(aJ);
      aMa += aJ.x * yJ.x + aJ.y * yJ.y;
    }
    if (!(aMa > 0.f) || !(an > 0.f)) break;
    const float f = an / aMa;
    float2 At[P][P];
    float tr = 0.f;
#pragma unroll
    for (int i = 0; i < P; ++i)
#pragma unroll
      for (int k = 0; k < P; ++k) {
        const float2 x = y_[(i + P * k) * nt], z = y_[(k + P * i) * nt];
        At[i][k] = make_float2(0.5f * f * (x.x + z.x), 0.5f * f * (x.y - z.y));
        if (i == k) tr += fabsf(At[i][i].x);
      }
    float d[P];
    float2 U[P][P];
    jacobi_small<P>(At, d, U, 1e-14f, 3e-8f * tr);
#pragma unroll
    for (int m = 0; m < RA; ++m) {
      dt[m] = d[m];
#pragma unroll
      for (int i = 0; i < P; ++i) Ut[(i * RA + m) * nt + tid] = U[i][m];
    }
    // a_k+1 = sum_{m < r_a} d_m u_m u_m^H over a_k in place, and the stop rule
    float dn = 0.f, nn = 0.f;
#pragma unroll 1
    for (int J = 0; J < PP; ++J) {
      const int i = J % P, k = J / P;
      float2 s = make_float2(0.f, 0.f);
#pragma unroll
      for (int m = 0; m < RA; ++m)
        if (m < ra)
          s = cadd(s, cscale(cmul(Ut[(i * RA + m) * nt + tid], cconj(Ut[(k * RA + m) * nt + tid])),
                             dt[m]));
      // exactly Hermitian (the B pass mirrors the upper triangle of B, which
      // is the Hermitian part of b only for a Hermitian a): entry (i, k) with
      // i < k is the conjugate of its mirror (k, i), already updated in this
      // loop (k + P i < i + P k), and the diagonal is real
      if (i < k) s = cconj(a_[(k + P * i) * nt]);
      if (i == k) s.y = 0.f;
      dn += cabs2(csub(s, a_[J * nt]));
      nn += cabs2(s);
      a_[J * nt] = s;
    }
    if (dn <= tol2 * nn) break;
    // rounding floor: once |a_k+1 - a_k| <= 1e-4 |a_k+1|, a step that no
    // longer shrinks means the single-precision truncation has stopped
    // improving the iterate (cells whose leading spatial eigenvalues are
    // close); further iterations only move it within that floor
    if (dn <= 1e-8f * nn && dn >= dn_prev) break;
    dn_prev = dn;
  }
  const bool noconv = it > g.max_iter;
  if (noconv) it = g.max_iter;
  if (JL.report) count_lanes(JL.report, noconv);
  // cells whose box holds a NaN / Inf sample: iters = -1, eta = NaN
  bool bad = false;
  if (JB.maxbits && JB.maxbits[1]) {
    Geom gj = with_job(g0, JB);
    bad = box_nonfinite(JB.Y, gj, (int)(local / JB.W), (int)(local % JB.W), 0, 1);
    if (JL.report) count_lanes(JL.report + 1, bad);
  }
  // eta^2 = 1 - a^H M a / (|a|^2 tr M), the three sums in float-float
  float trs = 0.f, trc = 0.f, ans = 0.f, anc = 0.f, qs = 0.f, qc = 0.f;
  {
    const float2* mp = Mc;
#pragma unroll 1
    for (int J = 0; J < PP; ++J) {
      const float2 aJ = a_[J * nt];
      aw[J * ncell + cell] = aJ;
      const float dM = __ldg(mp).x;
      mp += ncell;
      float t, e;
      two_sum(trs, dM, t, e);
      trs = t;
      trc = __fadd_rn(trc, e);
      float p1, pe;
      two_prod(aJ.x, aJ.x, p1, pe);
      acc_ffxf(ans, anc, p1, pe, 1.f);
      acc_ffxf(qs, qc, p1, pe, dM);
      two_prod(aJ.y, aJ.y, p1, pe);
      acc_ffxf(ans, anc, p1, pe, 1.f);
      acc_ffxf(qs, qc, p1, pe, dM);
#pragma unroll 2
      for (int K = J + 1; K < PP; ++K) {   // 2 Re(conj(a_J) M_JK a_K)
        const float2 m = __ldg(mp);
        const float2 aK = a_[K * nt];
        mp += ncell;
        float rs = 0.f, rc = 0.f, is = 0.f, ic = 0.f;
        acc_prod(rs, rc, m.x, aK.x);
        acc_prod(rs, rc, -m.y, aK.y);
        acc_prod(is, ic, m.x, aK.y);
        acc_prod(is, ic, m.y, aK.x);
        acc_ffxf(qs, qc, rs, rc, 2.f * aJ.x);
        acc_ffxf(qs, qc, is, ic, 2.f * aJ.y);
      }
    }
  }
  const double tr = (double)trs + (double)trc;
  const double an = (double)ans + (double)anc;
  const double aMa = (double)qs + (double)qc;
  float trA = 0.f;
#pragma unroll
  for (int m = 0; m < RA; ++m)
    if (m < ra) trA += dt[m];
  const float sc = (trA != 0.f) ? (float)P / trA : 1.f;
#pragma unroll
  for (int i = 0; i < P; ++i)
#pragma unroll
    for (int m = 0; m < RA; ++m)
      if (m < ra) JB.UA[(local * P + i) * ra + m] = Ut[(i * RA + m) * nt + tid];
  if (JB.lamA) {
#pragma unroll
    for (int m = 0; m < RA; ++m)
      if (m < ra) JB.lamA[local * ra + m] = dt[m] * sc;
  }
  if (JB.iters) JB.iters[local] = bad ? -1 : it;
  if (JB.eta) {
    const double e2 = (tr > 0.0 && an > 0.0) ? 1.0 - aMa / (an * tr) : 0.0;
    JB.eta[local] = bad ? __int_as_float(0x7fc00000) : (float)sqrt(e2 > 0.0 ? e2 : 0.0);
  }
  }  // tile loop
}

}  // namespace kstap
