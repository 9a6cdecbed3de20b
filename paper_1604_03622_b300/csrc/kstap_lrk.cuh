// One large-covariance LR-Kron fit (Alg. 2) from n snapshots X_m (p x q):
// the paper's timing workload (Sec. 7.1: rank-one A, B = I so r_b = q, n = 5,
// q up to 2500).  R = R(S) (p^2 x q^2, Alg. 1) is never formed.  With
// G_mm' = X_m X_m'^H (p x p) every quantity of Alg. 2 is a small expression:
//   B   = vec^-1(b) = (1 / (n |a|^2)) sum_m X_m^T conj(A) conj(X_m)      (q x q)
//   |b|^2 = Re <A, T(A)> / (n^2 |a|^2^2),  T(A) = sum_mm' G_mm' A G_m'm
//   A~  = vec^-1(R conj(b) / |b|^2) = T(A) / (n^2 |a|^2 |b|^2)
//   |R|^2 = |S|_F^2 = sum_mm' |tr G_m'm|^2 / n^2
//   A_0 = vec^-1(R 1 / q^2) = sum_m s_m s_m^H / (n q^2),  s_m = X_m 1
//   eta^2 = (|R|^2 - 2 |b|^2 Re <a', a~> + |a'|^2 |b|^2) / |R|^2
// T is linear in A: vec(T(A)) = Tm vec(A) with the p^2 x p^2 matrix
// Tm = sum_mm' G_m'm^T (x) G_mm' (vec column-major, a[i + p k] = A[i][k]).
// The Grams and the iteration run in FP64 (the loop test |eta_k - eta_k-1|
// <= eps resolves differences of 1e-6 and below); only B^, the one q x q
// output, is formed, in FP32 by a tiled kernel.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace kstap {

constexpr int kLrkMaxP = 8;
constexpr int kLrkMaxN = 16;

__device__ __forceinline__ double2 zadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 zconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double zabs2(double2 a) { return a.x * a.x + a.y * a.y; }

// Block-wide FP64 sum over blockDim.x (a multiple of 32, <= 1024) threads.
__device__ __forceinline__ double block_sum_d(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  for (int k = 0; k < nw; ++k) t += red[k];   // same order in every thread
  return t;
}

// Grid (n p, n p + 1): block (r1, r2) forms sum_j X_r1[j] conj(X_r2[j]) over
// the rows r = m p + i of X (n p rows of q), i.e. G_big[r1][r2] with
// G_mm'[i][k] = G_big[m p + i][m' p + k]; column n p gives the row sums s_r1.
__global__ void k_lrk_gram(const float2* __restrict__ X, int np, int q, double2* __restrict__ G,
                           double2* __restrict__ s) {
  __shared__ double red[32];
  const int r1 = blockIdx.x, r2 = blockIdx.y;
  const bool ones = r2 == np;
  const float2* x1 = X + (size_t)r1 * q;
  const float2* x2 = X + (size_t)(ones ? r1 : r2) * q;
  double sr = 0.0, si = 0.0;
  for (int j = threadIdx.x; j < q; j += blockDim.x) {
    const float2 a = x1[j];
    if (ones) {
      sr += a.x;
      si += a.y;
    } else {
      const float2 b = x2[j];
      sr += (double)a.x * b.x + (double)a.y * b.y;
      si += (double)a.y * b.x - (double)a.x * b.y;
    }
  }
  sr = block_sum_d(sr, red);
  si = block_sum_d(si, red);
  if (threadIdx.x == 0) {
    if (ones)
      s[r1] = make_double2(sr, si);
    else
      G[(size_t)r1 * np + r2] = make_double2(sr, si);
  }
}

// Tm[(i + p k)][(i2 + p k2)] = sum_mm' G_m'm[k2][k] G_mm'[i][i2]; one thread
// per entry (p^4 of them).
__global__ void k_lrk_tmat(const double2* __restrict__ G, int n, int p, double2* __restrict__ Tm) {
  const int p2 = p * p, np = n * p;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= p2 * p2) return;
  const int row = e / p2, col = e % p2;
  const int i = row % p, k = row / p, i2 = col % p, k2 = col / p;
  double2 acc = make_double2(0.0, 0.0);
  for (int m = 0; m < n; ++m)
    for (int mp = 0; mp < n; ++mp) {
      const double2 g1 = G[(size_t)(mp * p + k2) * np + (m * p + k)];   // G_m'm[k2][k]
      const double2 g2 = G[(size_t)(m * p + i) * np + (mp * p + i2)];   // G_mm'[i][i2]
      acc = zadd(acc, zmul(g1, g2));
    }
  Tm[e] = acc;
}

// Cyclic Jacobi on a Hermitian p x p matrix (FP64, row-major in `A`, shared
// memory), run by the 32 lanes of one warp: each sweep visits the p(p-1)/2
// pairs in n - 1 rounds of n/2 disjoint pairs (n = p rounded up to even; the
// round-robin tournament order), so a round's rotation angles are computed
// side by side (one lane per pair) and its updates of A = G^H A G and U = U G
// run one lane per (row or column, pair).  On return w holds the eigenvalues
// in decreasing order and the columns of U (row-major) the eigenvectors.
// Off-diagonal entries at or below the matrix's rounding level (1e-16 of
// sum |A_ii|) are set to zero instead of rotated: without that floor the
// entries between eigenvalues near zero (a rank-one A has p - 1 of them)
// keep the sweeps going to the cap.  Every lane returns with the same w and U.
__device__ void lrk_jacobi_warp(double2* A, int p, double* w, double2* U, int lane) {
  __shared__ double rc[kLrkMaxP / 2], rs[kLrkMaxP / 2];
  __shared__ double2 rph[kLrkMaxP / 2];
  __shared__ int ra[kLrkMaxP / 2], rb[kLrkMaxP / 2], rk[kLrkMaxP / 2];   // pair, kind
  const int n = p + (p & 1), np2 = n / 2;
  for (int e = lane; e < p * p; e += 32) U[e] = make_double2(e / p == e % p ? 1.0 : 0.0, 0.0);
  __syncwarp();
  for (int sweep = 0; sweep < 30; ++sweep) {
    double off = 0.0, diag = 0.0, tr = 0.0;
    for (int e = lane; e < p * p; e += 32) {
      const int i = e / p, j = e % p;
      if (i == j) {
        diag += A[e].x * A[e].x;
        tr += fabs(A[e].x);
      } else if (j > i) {
        off += zabs2(A[e]);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_xor_sync(0xffffffffu, off, o);
      diag += __shfl_xor_sync(0xffffffffu, diag, o);
      tr += __shfl_xor_sync(0xffffffffu, tr, o);
    }
    if (off <= 1e-30 * diag || off == 0.0) break;   // warp-uniform
    const double floor_ab = 1e-16 * tr;
    for (int round = 0; round < n - 1; ++round) {
      if (lane < np2) {
        // pair `lane` of the round: player 0 fixed, the others rotate
        auto pos = [&](int i) { return i == 0 ? 0 : 1 + (i - 1 + round) % (n - 1); };
        int a = pos(lane), b = pos(n - 1 - lane);
        if (a > b) {
          const int tmp = a;
          a = b;
          b = tmp;
        }
        int kind = 0;   // 0 none (dummy player), 1 rotate, 2 drop the entry
        if (b < p) {
          const double2 apq = A[a * p + b];
          const double ab = hypot(apq.x, apq.y);   // no squaring: no underflow for tiny entries
          const double App = A[a * p + a].x, Aqq = A[b * p + b].x;
          if (!(ab > fmax(1e-20 * (fabs(App) + fabs(Aqq)), floor_ab))) {
            kind = 2;
          } else {
            kind = 1;
            double2 ph = make_double2(apq.x / ab, apq.y / ab);
            const double pn = 1.0 / sqrt(zabs2(ph));
            ph = make_double2(ph.x * pn, ph.y * pn);
            const double tau = (Aqq - App) / (2.0 * ab);
            const double t = copysign(1.0, tau) / (fabs(tau) + sqrt(1.0 + tau * tau));
            const double c = 1.0 / sqrt(1.0 + t * t);
            rc[lane] = c;
            rs[lane] = t * c;
            rph[lane] = zconj(ph);
          }
        }
        ra[lane] = a;
        rb[lane] = b;
        rk[lane] = kind;
      }
      __syncwarp();
      // columns a, b of every row (A G, and U G)
      for (int L = lane; L < p * np2; L += 32) {
        const int k = L / np2, j = L % np2;
        if (rk[j] != 1) continue;
        const int a = ra[j], b = rb[j];
        const double c = rc[j], sn = rs[j];
        const double2 cph = rph[j];
        const double2 xa = A[k * p + a], yb = zmul(cph, A[k * p + b]);
        A[k * p + a] = make_double2(c * xa.x - sn * yb.x, c * xa.y - sn * yb.y);
        A[k * p + b] = make_double2(sn * xa.x + c * yb.x, sn * xa.y + c * yb.y);
        const double2 ua = U[k * p + a], ub = zmul(cph, U[k * p + b]);
        U[k * p + a] = make_double2(c * ua.x - sn * ub.x, c * ua.y - sn * ub.y);
        U[k * p + b] = make_double2(sn * ua.x + c * ub.x, sn * ua.y + c * ub.y);
      }
      __syncwarp();
      // rows a, b of every column (G^H (A G))
      for (int L = lane; L < p * np2; L += 32) {
        const int k = L / np2, j = L % np2;
        if (rk[j] != 1) continue;
        const int a = ra[j], b = rb[j];
        const double c = rc[j], sn = rs[j];
        const double2 ph = zconj(rph[j]);
        const double2 xa = A[a * p + k], yb = zmul(ph, A[b * p + k]);
        A[a * p + k] = make_double2(c * xa.x - sn * yb.x, c * xa.y - sn * yb.y);
        A[b * p + k] = make_double2(sn * xa.x + c * yb.x, sn * xa.y + c * yb.y);
      }
      __syncwarp();
      if (lane < np2 && rk[lane] != 0) {   // the rotated (or dropped) entry is zero
        const int a = ra[lane], b = rb[lane];
        A[a * p + b] = A[b * p + a] = make_double2(0.0, 0.0);
        A[a * p + a].y = 0.0;
        A[b * p + b].y = 0.0;
      }
      __syncwarp();
    }
  }
  if (lane == 0) {
    for (int i = 0; i < p; ++i) w[i] = A[i * p + i].x;
    for (int i = 0; i < p - 1; ++i)
      for (int j = i + 1; j < p; ++j)
        if (w[j] > w[i]) {
          const double tw = w[i];
          w[i] = w[j];
          w[j] = tw;
          for (int k = 0; k < p; ++k) {
            const double2 u = U[k * p + i];
            U[k * p + i] = U[k * p + j];
            U[k * p + j] = u;
          }
        }
  }
  __syncwarp();
}

__global__ void k_lrk_aout(const double2* __restrict__ A_fin, const double* __restrict__ info,
                           int p, float2* __restrict__ Aout) {
  const int e = threadIdx.x;
  if (e >= p * p) return;
  const double sc = (info[1] != 0.0) ? (double)p / info[1] : 1.0;
  const int i = e / p, k = e % p;
  const double2 v = A_fin[i + p * k];
  Aout[e] = make_float2((float)(v.x * sc), (float)(v.y * sc));
}

// Alg. 2 on the p^2 x p^2 operator Tm: one warp, FP64.  Writes the final a
// (vec, column-major) to A_fin, the a that produced the last b to A_prev, and
// info = {|a_prev|^2, tr A_fin, eta, iterations, |R|^2}.
__global__ void k_lrk_iterate(const double2* __restrict__ Tm, const double2* __restrict__ G,
                              const double2* __restrict__ s, int n, int p, int q, int r_a,
                              double eps, int max_iter, double2* __restrict__ A_fin,
                              double2* __restrict__ A_prev, double* __restrict__ info) {
  constexpr int PP = kLrkMaxP * kLrkMaxP;
  __shared__ double2 a[PP], t[PP], Am[PP], U[PP], Ub[PP], Tt[PP];
  __shared__ double w[kLrkMaxP];
  __shared__ int done, ok;
  __shared__ double sh_f, sh_an, sh_bn;
  const int lane = threadIdx.x, p2 = p * p, np = n * p;
  double Rn2 = 0.0;
  if (lane == 0) {
    for (int m = 0; m < n; ++m)       // |R|^2 = sum_mm' |tr G_m'm|^2 / n^2
      for (int mp = 0; mp < n; ++mp) {
        double2 tr = make_double2(0.0, 0.0);
        for (int i = 0; i < p; ++i) tr = zadd(tr, G[(size_t)(mp * p + i) * np + (m * p + i)]);
        Rn2 += zabs2(tr);
      }
    Rn2 /= (double)n * n;
    for (int i = 0; i < p; ++i)       // A_0[i][k] = sum_m s_m[i] conj(s_m[k]) / (n q^2)
      for (int k = 0; k < p; ++k) {
        double2 acc = make_double2(0.0, 0.0);
        for (int m = 0; m < n; ++m) acc = zadd(acc, zmul(s[m * p + i], zconj(s[m * p + k])));
        a[i + p * k] = make_double2(acc.x / ((double)n * q * q), acc.y / ((double)n * q * q));
      }
    done = 0;
  }
  for (int e = lane; e < p2; e += 32)   // eigenbasis of the previous iterate: I
    Ub[e] = make_double2(e / p == e % p ? 1.0 : 0.0, 0.0);
  __syncwarp();
  double eta_prev = 1.0 / 0.0, an_prev = 0.0, eta = 0.0;
  int it = 0;
  while (true) {
    for (int r = lane; r < p2; r += 32) {   // t = Tm vec(A)
      double2 acc = make_double2(0.0, 0.0);
      for (int c = 0; c < p2; ++c) acc = zadd(acc, zmul(Tm[(size_t)r * p2 + c], a[c]));
      t[r] = acc;
    }
    __syncwarp();
    if (lane == 0) {
      double an = 0.0, ip = 0.0;
      for (int J = 0; J < p2; ++J) {
        an += zabs2(a[J]);
        ip += a[J].x * t[J].x + a[J].y * t[J].y;   // Re <A, T(A)>
      }
      const double nn = (double)n * n;
      const double bn = (an > 0.0) ? ip / (nn * an * an) : 0.0;
      ok = (an > 0.0) && (bn > 0.0);
      if (!ok) {
        done = 1;
      } else {
        const double f = 1.0 / (nn * an * bn);
        sh_f = f;
        sh_an = an;
        sh_bn = bn;
        for (int i = 0; i < p; ++i)        // herm(vec^-1 a~), row-major
          for (int k = 0; k < p; ++k) {
            const double2 x = t[i + p * k], y = t[k + p * i];
            Am[i * p + k] = make_double2(0.5 * f * (x.x + y.x), 0.5 * f * (x.y - y.y));
          }
      }
    }
    __syncwarp();
    if (!ok) break;
    // EIG of A~ warm-started in the previous iterate's eigenbasis Ub: B =
    // Ub^H A~ Ub is nearly diagonal, so the Jacobi below needs a sweep or two
    // (the iterates change little from one step to the next); U = Ub W.
    for (int e = lane; e < p2; e += 32) {   // Tt = A~ Ub
      const int i = e / p, m = e % p;
      double2 acc = make_double2(0.0, 0.0);
      for (int k = 0; k < p; ++k) acc = zadd(acc, zmul(Am[i * p + k], Ub[k * p + m]));
      Tt[e] = acc;
    }
    __syncwarp();
    for (int e = lane; e < p2; e += 32) {   // B = Ub^H Tt (into Am, now free)
      const int m = e / p, k2 = e % p;
      double2 acc = make_double2(0.0, 0.0);
      for (int i = 0; i < p; ++i) acc = zadd(acc, zmul(zconj(Ub[i * p + m]), Tt[i * p + k2]));
      Am[e] = acc;
    }
    __syncwarp();
    if (lane == 0) {
      for (int m = 0; m < p; ++m)           // Hermitian part, pairwise in place
        for (int k2 = m; k2 < p; ++k2) {
          const double2 x = Am[m * p + k2], y = Am[k2 * p + m];
          const double2 h = make_double2(0.5 * (x.x + y.x), 0.5 * (x.y - y.y));
          Am[m * p + k2] = h;
          Am[k2 * p + m] = zconj(h);
        }
    }
    __syncwarp();
    lrk_jacobi_warp(Am, p, w, U, lane);
    for (int e = lane; e < p2; e += 32) {   // U = Ub W
      const int i = e / p, m = e % p;
      double2 acc = make_double2(0.0, 0.0);
      for (int k = 0; k < p; ++k) acc = zadd(acc, zmul(Ub[i * p + k], U[k * p + m]));
      Tt[e] = acc;
    }
    __syncwarp();
    for (int e = lane; e < p2; e += 32) U[e] = Ub[e] = Tt[e];
    __syncwarp();
    if (lane == 0) {
      {
        const double f = sh_f, an = sh_an, bn = sh_bn;
        double anew = 0.0, re = 0.0;
        for (int i = 0; i < p; ++i)
          for (int k = 0; k < p; ++k) {
            double2 acc = make_double2(0.0, 0.0);   // EIG_{r_a}: sum_m w_m u_m u_m^H
            for (int m = 0; m < r_a; ++m) {
              const double2 uu = zmul(U[i * p + m], zconj(U[k * p + m]));
              acc = make_double2(acc.x + w[m] * uu.x, acc.y + w[m] * uu.y);
            }
            const double2 at = make_double2(f * t[i + p * k].x, f * t[i + p * k].y);   // a~
            anew += zabs2(acc);
            re += acc.x * at.x + acc.y * at.y;                                         // Re <a', a~>
            A_prev[i + p * k] = a[i + p * k];
            a[i + p * k] = acc;
          }
        an_prev = an;
        const double e2 = (Rn2 > 0.0) ? (Rn2 - 2.0 * bn * re + anew * bn) / Rn2 : 0.0;
        eta = sqrt(e2 > 0.0 ? e2 : 0.0);
        ++it;
        done = (fabs(eta - eta_prev) <= eps) || (it >= max_iter);
        eta_prev = eta;
      }
    }
    __syncwarp();
    if (done) break;
  }
  if (lane == 0) {
    double tr = 0.0;
    for (int i = 0; i < p; ++i) tr += a[i + p * i].x;
    for (int J = 0; J < p2; ++J) A_fin[J] = a[J];
    info[0] = an_prev;
    info[1] = tr;
    info[2] = eta;
    info[3] = (double)it;
    info[4] = Rn2;
  }
}

// B^[j][l] = coef sum_m sum_i X_m[i][j] Y_m[i][l], Y_m[i][l] = sum_k conj(A[i][k])
// conj(X_m[k][l]) (A = the a that produced the last b, vec column-major),
// coef = 1 / (n |a|^2 sc) with sc = p / tr A^ (tr A^ = p normalisation), read
// from info; q x q row-major complex64 output.  Block = 32 x 32 tile of
// (j, l), 256 threads, 4 outputs each; dynamic shared memory 2 n p 32 x 8 B.
constexpr int kLrkTile = 32;
__global__ void __launch_bounds__(256)
k_lrk_bout(const float2* __restrict__ X, const double2* __restrict__ Aprev,
           const double* __restrict__ info, int n, int p, int q, float2* __restrict__ Bout) {
  constexpr int TB = kLrkTile;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ float2 Ac[kLrkMaxP * kLrkMaxP];   // conj(A), row-major
  const int np = n * p;
  float2 (*Xj)[TB] = reinterpret_cast<float2 (*)[TB]>(smem);
  float2 (*Yl)[TB] = reinterpret_cast<float2 (*)[TB]>(smem + (size_t)np * TB * sizeof(float2));
  const float coef = (float)(info[1] / ((double)n * info[0] * (double)p));
  const int j0 = blockIdx.y * TB, l0 = blockIdx.x * TB;
  for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
    const int i = e / p, k = e % p;
    const double2 v = Aprev[i + p * k];
    Ac[e] = make_float2((float)v.x, (float)-v.y);
  }
  for (int e = threadIdx.x; e < np * TB; e += blockDim.x) {
    const int r = e / TB, c = e % TB;
    Xj[r][c] = (j0 + c < q) ? X[(size_t)r * q + j0 + c] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < np * TB; e += blockDim.x) {
    const int r = e / TB, c = e % TB, m = r / p, i = r % p;
    float2 acc = make_float2(0.f, 0.f);
    if (l0 + c < q)
      for (int k = 0; k < p; ++k) {
        const float2 x = X[(size_t)(m * p + k) * q + l0 + c];
        acc = cadd(acc, cmul(Ac[i * p + k], cconj(x)));
      }
    Yl[r][c] = acc;
  }
  __syncthreads();
  const int c = threadIdx.x % TB;
  for (int rr = threadIdx.x / TB; rr < TB; rr += blockDim.x / TB) {
    const int j = j0 + rr, l = l0 + c;
    float2 acc = make_float2(0.f, 0.f);
    for (int r = 0; r < np; ++r) acc = cadd(acc, cmul(Xj[r][rr], Yl[r][c]));
    if (j < q && l < q) Bout[(size_t)j * q + l] = cscale(acc, coef);
  }
}

}  // namespace kstap
