// Kron-STAP CUDA kernels for sm_103a (B300).
//
// Per test cell (r, c) (paper notation, Sec. 2-5):
//   S = (1/n) sum_m x_m x_m^H over the training ring        (Eq. SCM)
//   R = R(S): row J = i + p k holds vec(S(i, k))             (Alg. 1 / Eq. SVD)
//   Alg. 2 flip-flop: b = R^T conj(a)/|a|^2, a~ = R conj(b)/|b|^2,
//                     a = vec(EIG_{r_a}(vec^-1 a~))
//   B^ = EIG_{r_b}(vec^-1 b) -> U_B;  U_A from A^
//   T_v = |d_v^H (F_A (x) F_B) x|^2 / (d_v^H (F_A (x) F_B) d_v) (Eq. KronSTAP)
//
// How the GPU path computes it (same result in exact arithmetic):
//  * Lag sums.  S(i,k)_{j,l} = L_{ik, l-j}(r, c + j) / n with
//      L_{ik,g}(r, u) = sum_{(rho, kappa) in ring(u)} Y_i(rho, kappa) conj(Y_k(rho, kappa + g)),
//    a box-filtered product image shared by all cells whose windows overlap.
//    The box sums run in exact 64-bit integer arithmetic on a fixed-point copy
//    of Y (power-of-two scale per frame, 2^B full scale), so S carries no
//    accumulation rounding at all.
//  * Flip-flop on M = R R^H (p^2 x p^2).  With a~ = R R^H a |a|^2 / (a^H R R^H a),
//    every Alg. 2 iterate is a function of the 9 x 9 matrix M only, so the
//    p^2 q^2 contractions per iteration become one p^4 q^2 / 2 pass.
//    M = sum_g W_g + conj(Pi (sum_{g>0} W_g) Pi^T), W_g = sum_j l_g(c+j) l_g(c+j)^H,
//    l_g(u)[J] = L_{ik,g}(u), Pi swapping (i,k) <-> (k,i): lags -g are the
//    conjugate transposes of lags +g.
//  * B (upper triangle, diagonal g) = sum_J conj(a_J) L_{J,g}(c + j), float-float.
//  * U_B: subspace iteration in FP32, then float-float subspace steps with
//    Cholesky-QR; U_B is kept as hi + lo.
//  * X F_B^T in float-float, then F_A and the bank in FP32.  Steering
//    vectors that keep < 1e-2 of their energy after projection are
//    re-projected with the float-float U_B.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "kstap_ff.cuh"

namespace kstap {

constexpr int kTileCells = 32;      // cells of one range row per CTA (moments / B passes)
constexpr int kThreads = 256;
constexpr int kRbMax = 4;
constexpr float kBlind = 1e-2f;     // relative projected energy below which T_v is re-projected in FF
constexpr float kLagNorm = 8.673617379884035e-19f;   // 2^-60: integer lag sums -> O(1) floats

struct Geom {
  int p, q, r_a, r_b;
  int Rr, Ra, Gr, Ga;
  int H_in, W_in, H, W;
  int n;
  int V;
  int B;          // fixed-point bits of |Y| components
  int max_iter;
  float eps;
  float tau;
  int tc;         // cells per tile in the B pass
};

// ------------------------------------------------------------- helpers -----
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) * b
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float cabs2(float2 a) { return a.x * a.x + a.y * a.y; }

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float2 warp_sum2(float2 v) {
  return make_float2(warp_sum(v.x), warp_sum(v.y));
}

// Frame fixed-point shift: maxabs * 2^sh < 2^B.
__device__ __forceinline__ int frame_shift(unsigned maxbits, int B) {
  const float m = __uint_as_float(maxbits);
  if (!(m > 0.f) || !(m < 3.0e38f)) return 0;
  return B - 1 - ilogbf(m);
}

__device__ __forceinline__ int quantise(float y, float scale) {
  const float v = y * scale;   // exact: scale is a power of two
  if (!(fabsf(v) < 2147483520.f)) return 0;   // non-finite or out of range
  return __float2int_rn(v);
}

// Upper-triangle index (row-major over J <= J') of an n x n Hermitian matrix.
__host__ __device__ constexpr int tri_idx(int n, int J, int Jp) {
  return J * n - (J * (J - 1)) / 2 + (Jp - J);
}

// ------------------------------------------------------- frame scale -------
// max |component| of Y via the order-preserving bit pattern of non-negative
// floats; non-finite values are recorded in *nonfinite.
__global__ void k_frame_maxabs(const float* __restrict__ Y, size_t nfloat,
                               unsigned* __restrict__ maxbits, unsigned* __restrict__ nonfinite) {
  unsigned m = 0, bad = 0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nfloat;
       i += (size_t)gridDim.x * blockDim.x) {
    const float a = fabsf(__ldg(Y + i));
    if (a < 3.4e38f) {
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

// ------------------------------------------------ shared lag-sum stage -----
// Loads the fixed-point tile of rows [r, r + 2Rr] and columns [c0, c0 + WT)
// of all channels: Yq[(i * NR + rho) * WT + col].
template <int P>
__device__ void load_tile_q(const float2* __restrict__ Y, const Geom& g, int r, int c0, int WT,
                            float scale, int2* __restrict__ Yq) {
  const int NR = 2 * g.Rr + 1;
  const int total = P * NR * WT;
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    const int col = idx % WT;
    const int rho = (idx / WT) % NR;
    const int i = idx / (WT * NR);
    const int gc = c0 + col;
    int2 v = make_int2(0, 0);
    if (gc < g.W_in) {
      const float2 y = __ldg(Y + ((size_t)i * g.H_in + (r + rho)) * g.W_in + gc);
      v.x = quantise(y.x, scale);
      v.y = quantise(y.y, scale);
    }
    Yq[idx] = v;
  }
}

// Vertical ring sums for lag g of all P*P ordered channel pairs:
//   Vo[J][kappa] = sum_{rho in [0, NR)}          Yq_i(rho, kappa) conj(Yq_k(rho, kappa + g))
//   Vg[J][kappa] = sum_{rho in guard rows}       (same product)
// for kappa in [0, KW).  J = i + P k.
template <int P>
__device__ void vertical_sums(const int2* __restrict__ Yq, const Geom& g, int WT, int lag, int KW,
                              longlong2* __restrict__ Vo, longlong2* __restrict__ Vg) {
  const int NR = 2 * g.Rr + 1;
  const int g0 = g.Rr - g.Gr, g1 = g.Rr + g.Gr;
  const int total = P * P * KW;
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    const int kap = idx % KW;
    const int J = idx / KW;
    const int i = J % P, k = J / P;
    const int2* yi = Yq + (size_t)i * NR * WT + kap;
    const int2* yk = Yq + (size_t)k * NR * WT + kap + lag;
    long long vr = 0, vi = 0, gr = 0, gi = 0;
    for (int rho = 0; rho < NR; ++rho) {
      const int2 a = yi[rho * WT];
      const int2 b = yk[rho * WT];
      const long long pr = (long long)a.x * b.x + (long long)a.y * b.y;
      const long long pi = (long long)a.y * b.x - (long long)a.x * b.y;
      vr += pr;
      vi += pi;
      if (rho >= g0 && rho <= g1) {
        gr += pr;
        gi += pi;
      }
    }
    Vo[idx] = make_longlong2(vr, vi);
    Vg[idx] = make_longlong2(gr, gi);
  }
}

// Horizontal box sums: L(u) = sum_{kappa=u}^{u+2Ra} Vo - sum_{kappa=u+Ra-Ga}^{u+Ra+Ga} Vg.
__device__ __forceinline__ longlong2 ring_sum(const longlong2* __restrict__ Vo,
                                              const longlong2* __restrict__ Vg, const Geom& g,
                                              int u) {
  long long lr = 0, li = 0;
  for (int t = 0; t <= 2 * g.Ra; ++t) {
    const longlong2 v = Vo[u + t];
    lr += v.x;
    li += v.y;
  }
  for (int t = g.Ra - g.Ga; t <= g.Ra + g.Ga; ++t) {
    const longlong2 v = Vg[u + t];
    lr -= v.x;
    li -= v.y;
  }
  return make_longlong2(lr, li);
}

// Exact split of a 64-bit integer into a float-float pair, scaled by 2^-60.
__device__ __forceinline__ void ll_to_ff(long long v, float& hi, float& lo) {
  const float h = __ll2float_rn(v);
  const long long rest = v - __float2ll_rn(h);
  hi = h * kLagNorm;
  lo = __ll2float_rn(rest) * kLagNorm;
}

// ------------------------------------------------ K1a: lag moments ---------
// CTA = (cell row r, tile of kTileCells cells).  Output per cell:
//   Mw[cell][tri(J, J')]  (PP(PP+1)/2 complex) : M = R R^H, in 2^-60 L units
//   Sw[cell][J]                                : sum of all S(i,k) entries (A_0 ~ this)
template <int P, int Q>
__global__ void __launch_bounds__(kThreads)
k_moments(const float2* __restrict__ Y, Geom g, const unsigned* __restrict__ maxbits,
          float2* __restrict__ Mw, float2* __restrict__ Sw) {
  constexpr int PP = P * P;
  constexpr int NE = PP * (PP + 1) / 2;
  constexpr int TC = kTileCells;
  constexpr int TPC = kThreads / TC;   // threads per cell
  extern __shared__ __align__(16) unsigned char smem[];
  const int r = blockIdx.y;
  const int c0 = blockIdx.x * TC;
  const int WT = TC + 2 * g.Ra + Q - 1;
  const int NR = 2 * g.Rr + 1;
  const int NUmax = TC + Q - 1;
  int2* Yq = reinterpret_cast<int2*>(smem);
  longlong2* Vo = reinterpret_cast<longlong2*>(Yq + P * NR * WT + (P * NR * WT & 1));
  longlong2* Vg = Vo + PP * WT;
  float2* lag = reinterpret_cast<float2*>(Vg + PP * WT);
  float2* W0s = lag + PP * NUmax;          // [TC][NE]
  float2* S0s = W0s + TC * NE;             // [TC][PP]

  const int sh = frame_shift(*maxbits, g.B);
  const float scale = ldexpf(1.f, sh);
  load_tile_q<P>(Y, g, r, c0, WT, scale, Yq);
  __syncthreads();

  const int cl = threadIdx.x / TPC;
  const int t = threadIdx.x % TPC;
  const bool live = (c0 + cl) < g.W;

  float wr[NE], wi[NE], sr[PP], si[PP];
#pragma unroll
  for (int e = 0; e < NE; ++e) wr[e] = wi[e] = 0.f;
#pragma unroll
  for (int J = 0; J < PP; ++J) sr[J] = si[J] = 0.f;

  for (int lagg = 0; lagg < Q; ++lagg) {
    const int NU = TC + Q - 1 - lagg;
    const int KW = NU + 2 * g.Ra;
    vertical_sums<P>(Yq, g, WT, lagg, KW, Vo, Vg);
    __syncthreads();
    for (int idx = threadIdx.x; idx < PP * NU; idx += blockDim.x) {
      const int u = idx % NU, J = idx / NU;
      const longlong2 L = ring_sum(Vo + J * KW, Vg + J * KW, g, u);
      lag[J * NUmax + u] = make_float2(__ll2float_rn(L.x) * kLagNorm, __ll2float_rn(L.y) * kLagNorm);
    }
    __syncthreads();
    if (live) {
      for (int j = t; j < Q - lagg; j += TPC) {
        float2 l[PP];
#pragma unroll
        for (int J = 0; J < PP; ++J) l[J] = lag[J * NUmax + cl + j];
#pragma unroll
        for (int J = 0; J < PP; ++J) {
          sr[J] += l[J].x;
          si[J] += l[J].y;
#pragma unroll
          for (int Jp = J; Jp < PP; ++Jp) {
            const int e = tri_idx(PP, J, Jp);
            // l[J] conj(l[Jp])
            wr[e] += l[J].x * l[Jp].x + l[J].y * l[Jp].y;
            wi[e] += l[J].y * l[Jp].x - l[J].x * l[Jp].y;
          }
        }
      }
    }
    if (lagg == 0) {
      // reduce W_0 over the TPC threads of the cell, park it in shared memory
#pragma unroll
      for (int e = 0; e < NE; ++e) {
#pragma unroll
        for (int o = TPC / 2; o > 0; o >>= 1) {
          wr[e] += __shfl_xor_sync(0xffffffffu, wr[e], o);
          wi[e] += __shfl_xor_sync(0xffffffffu, wi[e], o);
        }
      }
#pragma unroll
      for (int J = 0; J < PP; ++J) {
#pragma unroll
        for (int o = TPC / 2; o > 0; o >>= 1) {
          sr[J] += __shfl_xor_sync(0xffffffffu, sr[J], o);
          si[J] += __shfl_xor_sync(0xffffffffu, si[J], o);
        }
      }
      if (t == 0) {
#pragma unroll
        for (int e = 0; e < NE; ++e) W0s[cl * NE + e] = make_float2(wr[e], wi[e]);
#pragma unroll
        for (int J = 0; J < PP; ++J) S0s[cl * PP + J] = make_float2(sr[J], si[J]);
      }
#pragma unroll
      for (int e = 0; e < NE; ++e) wr[e] = wi[e] = 0.f;
#pragma unroll
      for (int J = 0; J < PP; ++J) sr[J] = si[J] = 0.f;
    }
    __syncthreads();
  }
  // reduce W_{>0}
#pragma unroll
  for (int e = 0; e < NE; ++e) {
#pragma unroll
    for (int o = TPC / 2; o > 0; o >>= 1) {
      wr[e] += __shfl_xor_sync(0xffffffffu, wr[e], o);
      wi[e] += __shfl_xor_sync(0xffffffffu, wi[e], o);
    }
  }
#pragma unroll
  for (int J = 0; J < PP; ++J) {
#pragma unroll
    for (int o = TPC / 2; o > 0; o >>= 1) {
      sr[J] += __shfl_xor_sync(0xffffffffu, sr[J], o);
      si[J] += __shfl_xor_sync(0xffffffffu, si[J], o);
    }
  }
  if (t == 0 && live) {
    const size_t cell = (size_t)r * g.W + (c0 + cl);
    // M[J,J'] = W0 + Wp + conj(Wp[pi J, pi J'])
#pragma unroll
    for (int J = 0; J < PP; ++J) {
#pragma unroll
      for (int Jp = J; Jp < PP; ++Jp) {
        const int e = tri_idx(PP, J, Jp);
        const int a = (J % P) * P + (J / P);     // pi(J): (i,k) -> (k,i)
        const int b = (Jp % P) * P + (Jp / P);
        float pr, pim;                           // Wp[a, b]
        if (a <= b) {
          pr = wr[tri_idx(PP, a, b)];
          pim = wi[tri_idx(PP, a, b)];
        } else {
          pr = wr[tri_idx(PP, b, a)];
          pim = -wi[tri_idx(PP, b, a)];
        }
        const float2 w0 = W0s[cl * NE + e];
        Mw[cell * NE + e] = make_float2(w0.x + wr[e] + pr, w0.y + wi[e] - pim);
      }
    }
#pragma unroll
    for (int J = 0; J < PP; ++J) {
      const int a = (J % P) * P + (J / P);
      const float2 s0 = S0s[cl * PP + J];
      Sw[cell * PP + J] = make_float2(s0.x + sr[J] + sr[a], s0.y + si[J] - si[a]);
    }
  }
}

// ------------------------------------------------ small Hermitian Jacobi ---
// Cyclic Jacobi on an N x N Hermitian matrix held in registers (FP32).  On
// return d[] holds the eigenvalues and the columns of U the eigenvectors,
// sorted by decreasing eigenvalue.
template <int N>
__device__ void jacobi_small(float2 (&A)[N][N], float (&d)[N], float2 (&U)[N][N]) {
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = 0; j < N; ++j) U[i][j] = make_float2(i == j ? 1.f : 0.f, 0.f);
  for (int sweep = 0; sweep < 12; ++sweep) {
    float off = 0.f, diag = 0.f;
#pragma unroll
    for (int i = 0; i < N; ++i) {
      diag += A[i][i].x * A[i][i].x;
#pragma unroll
      for (int j = i + 1; j < N; ++j) off += cabs2(A[i][j]);
    }
    if (off <= 1e-14f * diag) break;
#pragma unroll
    for (int p = 0; p < N - 1; ++p) {
#pragma unroll
      for (int q = p + 1; q < N; ++q) {
        const float2 b = A[p][q];
        const float ab = sqrtf(cabs2(b));
        if (ab == 0.f) continue;
        const float2 ph = make_float2(b.x / ab, b.y / ab);          // e^{i phi}
        const float tau = (A[q][q].x - A[p][p].x) / (2.f * ab);
        const float tt = copysignf(1.f, tau) / (fabsf(tau) + sqrtf(1.f + tau * tau));
        const float c = rsqrtf(1.f + tt * tt);
        const float s = tt * c;
        // G = diag(1, conj(ph)) [[c, s], [-s, c]]
        const float2 gpp = make_float2(c, 0.f), gpq = make_float2(s, 0.f);
        const float2 gqp = cscale(cconj(ph), -s), gqq = cscale(cconj(ph), c);
#pragma unroll
        for (int k = 0; k < N; ++k) {   // A <- A G
          const float2 ap = A[k][p], aq = A[k][q];
          A[k][p] = cadd(cmul(ap, gpp), cmul(aq, gqp));
          A[k][q] = cadd(cmul(ap, gpq), cmul(aq, gqq));
        }
#pragma unroll
        for (int k = 0; k < N; ++k) {   // A <- G^H A
          const float2 ap = A[p][k], aq = A[q][k];
          A[p][k] = cadd(cmulc(gpp, ap), cmulc(gqp, aq));
          A[q][k] = cadd(cmulc(gpq, ap), cmulc(gqq, aq));
        }
        A[p][q] = make_float2(0.f, 0.f);
        A[q][p] = make_float2(0.f, 0.f);
        A[p][p].y = 0.f;
        A[q][q].y = 0.f;
#pragma unroll
        for (int k = 0; k < N; ++k) {   // U <- U G
          const float2 up = U[k][p], uq = U[k][q];
          U[k][p] = cadd(cmul(up, gpp), cmul(uq, gqp));
          U[k][q] = cadd(cmul(up, gpq), cmul(uq, gqq));
        }
      }
    }
  }
#pragma unroll
  for (int i = 0; i < N; ++i) d[i] = A[i][i].x;
  // selection sort, decreasing
#pragma unroll
  for (int i = 0; i < N - 1; ++i) {
#pragma unroll
    for (int j = i + 1; j < N; ++j) {
      if (d[j] > d[i]) {
        const float tmp = d[i];
        d[i] = d[j];
        d[j] = tmp;
#pragma unroll
        for (int k = 0; k < N; ++k) {
          const float2 u = U[k][i];
          U[k][i] = U[k][j];
          U[k][j] = u;
        }
      }
    }
  }
}

// ------------------------------------------------ K2: flip-flop ------------
// One thread per cell: Alg. 2 on M = R R^H.  Writes a = vec(A^) (FP32),
// U_A, lamA (tr A^ = p), iterations and eta.
template <int P>
__global__ void __launch_bounds__(128)
k_flipflop(const float2* __restrict__ Mw, const float2* __restrict__ Sw, Geom g, size_t ncell,
           float2* __restrict__ aw, float2* __restrict__ UA, float* __restrict__ lamA,
           int32_t* __restrict__ iters, float* __restrict__ eta) {
  constexpr int PP = P * P;
  constexpr int NE = PP * (PP + 1) / 2;
  const size_t cell = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (cell >= ncell) return;
  float2 M[NE];
#pragma unroll
  for (int e = 0; e < NE; ++e) M[e] = Mw[cell * NE + e];
  float2 a[PP];
#pragma unroll
  for (int J = 0; J < PP; ++J) a[J] = Sw[cell * PP + J];
  // a_0 = R 1 / q^2 is proportional to the sum of S's block entries; Hermitise.
#pragma unroll
  for (int i = 0; i < P; ++i)
#pragma unroll
    for (int k = i; k < P; ++k) {
      const float2 x = a[i + P * k], y = a[k + P * i];
      const float2 h = make_float2(0.5f * (x.x + y.x), 0.5f * (x.y - y.y));
      a[i + P * k] = h;
      a[k + P * i] = cconj(h);
    }
  const int ra = g.r_a;
  float d[P];
  float2 U[P][P];
#pragma unroll
  for (int i = 0; i < P; ++i) {
    d[i] = 0.f;
#pragma unroll
    for (int k = 0; k < P; ++k) U[i][k] = make_float2(i == k ? 1.f : 0.f, 0.f);
  }
  int it = 0;
  const float tol2 = g.eps * g.eps;
  for (it = 1; it <= g.max_iter; ++it) {
    // y = M a
    float2 y[PP];
    float an = 0.f;
#pragma unroll
    for (int J = 0; J < PP; ++J) {
      an += cabs2(a[J]);
      float2 s = make_float2(0.f, 0.f);
#pragma unroll
      for (int Jp = 0; Jp < PP; ++Jp) {
        const float2 m = (J <= Jp) ? M[tri_idx(PP, J, Jp)] : cconj(M[tri_idx(PP, Jp, J)]);
        s = cadd(s, cmul(m, a[Jp]));
      }
      y[J] = s;
    }
    float aMa = 0.f;
#pragma unroll
    for (int J = 0; J < PP; ++J) aMa += a[J].x * y[J].x + a[J].y * y[J].y;
    if (!(aMa > 0.f) || !(an > 0.f)) break;
    const float f = an / aMa;
    // A~ = vec^-1(y f), Hermitised; EIG_{r_a}
    float2 At[P][P];
#pragma unroll
    for (int i = 0; i < P; ++i)
#pragma unroll
      for (int k = 0; k < P; ++k) {
        const float2 x = y[i + P * k], z = y[k + P * i];
        At[i][k] = make_float2(0.5f * f * (x.x + z.x), 0.5f * f * (x.y - z.y));
      }
    jacobi_small<P>(At, d, U);
    float2 an_new[PP];
    float dn = 0.f, nn = 0.f;
#pragma unroll
    for (int i = 0; i < P; ++i)
#pragma unroll
      for (int k = 0; k < P; ++k) {
        float2 s = make_float2(0.f, 0.f);
#pragma unroll
        for (int m = 0; m < P; ++m)
          if (m < ra) s = cadd(s, cscale(cmul(U[i][m], cconj(U[k][m])), d[m]));
        an_new[i + P * k] = s;
      }
#pragma unroll
    for (int J = 0; J < PP; ++J) {
      dn += cabs2(csub(an_new[J], a[J]));
      nn += cabs2(an_new[J]);
      a[J] = an_new[J];
    }
    if (dn <= tol2 * nn) break;
  }
  if (it > g.max_iter) it = g.max_iter;
  // eta^2 = 1 - a^H M a / (|a|^2 tr M) for b matched to the final a
  double tr = 0.0, aMa = 0.0, an = 0.0;
#pragma unroll
  for (int J = 0; J < PP; ++J) {
    tr += (double)M[tri_idx(PP, J, J)].x;
    an += (double)cabs2(a[J]);
    double sr = 0.0, si = 0.0;
#pragma unroll
    for (int Jp = 0; Jp < PP; ++Jp) {
      const float2 m = (J <= Jp) ? M[tri_idx(PP, J, Jp)] : cconj(M[tri_idx(PP, Jp, J)]);
      sr += (double)m.x * a[Jp].x - (double)m.y * a[Jp].y;
      si += (double)m.x * a[Jp].y + (double)m.y * a[Jp].x;
    }
    aMa += (double)a[J].x * sr + (double)a[J].y * si;
  }
#pragma unroll
  for (int J = 0; J < PP; ++J) aw[cell * PP + J] = a[J];
  float trA = 0.f;
#pragma unroll
  for (int m = 0; m < P; ++m)
    if (m < ra) trA += d[m];
  const float sc = (trA != 0.f) ? (float)P / trA : 1.f;
#pragma unroll
  for (int i = 0; i < P; ++i)
#pragma unroll
    for (int m = 0; m < P; ++m)
      if (m < ra) UA[(cell * P + i) * ra + m] = U[i][m];
  if (lamA) {
#pragma unroll
    for (int m = 0; m < P; ++m)
      if (m < ra) lamA[cell * ra + m] = d[m] * sc;
  }
  if (iters) iters[cell] = it;
  if (eta) {
    double e2 = (tr > 0.0 && an > 0.0) ? 1.0 - aMa / (an * tr) : 0.0;
    eta[cell] = (float)sqrt(e2 > 0.0 ? e2 : 0.0);
  }
}

// ------------------------------------------------ K3: B and U_B ------------
// Reads B(j, l) of one cell from the float-float upper triangle (by diagonal).
template <int Q>
__device__ __forceinline__ float4 b_at(const float4* __restrict__ Bc, int j, int l) {
  // Bc layout: diagonal d = l - j >= 0 at offset d*Q - d(d-1)/2, entry j
  if (l >= j) {
    const int d = l - j;
    return Bc[d * Q - (d * (d - 1)) / 2 + j];
  }
  const int d = j - l;
  const float4 v = Bc[d * Q - (d * (d - 1)) / 2 + l];
  return make_float4(v.x, v.y, -v.z, -v.w);   // conj: (re_hi, re_lo, im_hi, im_lo)
}

template <int P, int Q>
__device__ void eig_top_subspace(const float4* __restrict__ Bc, const Geom& g, int lane,
                                 float2 (&uh)[kRbMax], float2 (&ul)[kRbMax], float (&lam)[kRbMax],
                                 float2* __restrict__ Vs);

template <int P, int Q>
__global__ void __launch_bounds__(kThreads)
k_bfit(const float2* __restrict__ Y, Geom g, const unsigned* __restrict__ maxbits,
       const float2* __restrict__ aw, float2* __restrict__ UBh, float2* __restrict__ UBl,
       float* __restrict__ lamB) {
  constexpr int PP = P * P;
  constexpr int NB = Q * (Q + 1) / 2;
  extern __shared__ __align__(16) unsigned char smem[];
  const int TC = g.tc;
  const int r = blockIdx.y;
  const int c0 = blockIdx.x * TC;
  const int WT = TC + 2 * g.Ra + Q - 1;
  const int NR = 2 * g.Rr + 1;
  const int NUmax = TC + Q - 1;
  float4* Bs = reinterpret_cast<float4*>(smem);                 // [TC][NB]
  float2* as = reinterpret_cast<float2*>(Bs + TC * NB);         // [TC][PP]
  float2* Vs = as + TC * PP;                                    // [warps][Q][kRbMax]
  float4* lag = reinterpret_cast<float4*>(Vs + (kThreads / 32) * Q * kRbMax);   // [PP][NUmax]
  longlong2* Vo = reinterpret_cast<longlong2*>(lag + PP * NUmax);
  longlong2* Vg = Vo + PP * WT;
  int2* Yq = reinterpret_cast<int2*>(Vg + PP * WT);

  const int sh = frame_shift(*maxbits, g.B);
  const float scale = ldexpf(1.f, sh);
  load_tile_q<P>(Y, g, r, c0, WT, scale, Yq);
  for (int idx = threadIdx.x; idx < TC * PP; idx += blockDim.x) {
    const int cl = idx / PP, J = idx % PP;
    const int c = c0 + cl;
    as[idx] = (c < g.W) ? aw[((size_t)r * g.W + c) * PP + J] : make_float2(0.f, 0.f);
  }
  __syncthreads();

  for (int lagg = 0; lagg < Q; ++lagg) {
    const int NU = TC + Q - 1 - lagg;
    const int KW = NU + 2 * g.Ra;
    vertical_sums<P>(Yq, g, WT, lagg, KW, Vo, Vg);
    __syncthreads();
    for (int idx = threadIdx.x; idx < PP * NU; idx += blockDim.x) {
      const int u = idx % NU, J = idx / NU;
      const longlong2 L = ring_sum(Vo + J * KW, Vg + J * KW, g, u);
      float4 v;
      ll_to_ff(L.x, v.x, v.y);
      ll_to_ff(L.y, v.z, v.w);
      lag[J * NUmax + u] = v;
    }
    __syncthreads();
    // B(j, j + lag) = sum_J conj(a_J) l_lag(c + j)[J], float-float
    const int nj = Q - lagg;
    for (int idx = threadIdx.x; idx < TC * nj; idx += blockDim.x) {
      const int cl = idx / nj, j = idx % nj;
      float sr = 0.f, cr = 0.f, si = 0.f, ci = 0.f;
#pragma unroll
      for (int J = 0; J < PP; ++J) {
        const float2 a = as[cl * PP + J];
        const float4 L = lag[J * NUmax + cl + j];
        // conj(a) * L = (a.x L.re + a.y L.im) + i (a.x L.im - a.y L.re)
        acc_ffxf(sr, cr, L.x, L.y, a.x);
        acc_ffxf(sr, cr, L.z, L.w, a.y);
        acc_ffxf(si, ci, L.z, L.w, a.x);
        acc_ffxf(si, ci, L.x, L.y, -a.y);
      }
      const ff re = ff_make(sr, cr), im = ff_make(si, ci);
      Bs[cl * NB + lagg * Q - (lagg * (lagg - 1)) / 2 + j] = make_float4(re.hi, re.lo, im.hi, im.lo);
    }
    __syncthreads();
  }

  // eigen phase: one warp per cell
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int cl = warp; cl < TC; cl += kThreads / 32) {
    const int c = c0 + cl;
    if (c >= g.W) break;
    float2 uh[kRbMax], ul[kRbMax];
    float lam[kRbMax];
    eig_top_subspace<P, Q>(Bs + cl * NB, g, lane, uh, ul, lam, Vs + warp * Q * kRbMax);
    const size_t cell = (size_t)r * g.W + c;
    if (lane < Q) {
      for (int m = 0; m < g.r_b; ++m) {
        UBh[(cell * Q + lane) * g.r_b + m] = uh[m];
        UBl[(cell * Q + lane) * g.r_b + m] = ul[m];
      }
    }
    if (lane == 0 && lamB) {
      // B^ = b / |a|^2 in S units, then tr A^ = p normalisation
      float an = 0.f, tr = 0.f;
      for (int J = 0; J < PP; ++J) an += cabs2(as[cl * PP + J]);
      for (int i = 0; i < P; ++i) tr += as[cl * PP + i * (P + 1)].x;
      const float unit = ldexpf(1.f, 60 - 2 * frame_shift(*maxbits, g.B)) / (float)g.n;
      const float f = (an > 0.f) ? unit / an * tr / (float)P : 0.f;
      for (int m = 0; m < g.r_b; ++m) lamB[cell * g.r_b + m] = lam[m] * f;
    }
  }
}

// FP32 subspace iteration on B_hi, then float-float steps (Cholesky-QR) on
// the full B.  Lane j < Q owns row j of the q x r_b basis.
template <int P, int Q>
__device__ void eig_top_subspace(const float4* __restrict__ Bc, const Geom& g, int lane,
                                 float2 (&uh)[kRbMax], float2 (&ul)[kRbMax], float (&lam)[kRbMax],
                                 float2* __restrict__ Vs) {
  const int R = g.r_b;
  const bool row = lane < Q;
  float2 v[kRbMax], y[kRbMax];
  // start: r_b columns of B spread over the window
#pragma unroll
  for (int m = 0; m < kRbMax; ++m) {
    v[m] = make_float2(0.f, 0.f);
    if (m < R && row) {
      const float4 b = b_at<Q>(Bc, lane, ((2 * m + 1) * Q) / (2 * R));
      v[m] = make_float2(b.x, b.z);
    }
  }
  auto orthonormalise = [&](float2 (&x)[kRbMax]) {
#pragma unroll
    for (int m = 0; m < kRbMax; ++m) {
      if (m >= R) break;
#pragma unroll
      for (int mp = 0; mp < kRbMax; ++mp) {
        if (mp >= m) break;
        const float2 cc = warp_sum2(cmulc(x[mp], x[m]));
        x[m] = csub(x[m], cmul(x[mp], cc));
      }
      const float nrm = sqrtf(warp_sum(cabs2(x[m])));
      const float inv = (nrm > 0.f) ? 1.f / nrm : 0.f;
      x[m] = cscale(x[m], inv);
    }
  };
  orthonormalise(v);
  // FP32 subspace iteration until the residual |BV - V V^H B V| / |BV| is small
  for (int it = 0; it < 64; ++it) {
#pragma unroll
    for (int m = 0; m < kRbMax; ++m)
      if (row) Vs[lane * kRbMax + m] = v[m];
    __syncwarp();
#pragma unroll
    for (int m = 0; m < kRbMax; ++m) y[m] = make_float2(0.f, 0.f);
    if (row) {
      for (int l = 0; l < Q; ++l) {
        const float4 b = b_at<Q>(Bc, lane, l);
        const float2 bh = make_float2(b.x, b.z);
#pragma unroll
        for (int m = 0; m < kRbMax; ++m) y[m] = cadd(y[m], cmul(bh, Vs[l * kRbMax + m]));
      }
    }
    __syncwarp();
    // residual
    float ry = 0.f, re = 0.f;
    float2 e[kRbMax];
#pragma unroll
    for (int m = 0; m < kRbMax; ++m) e[m] = y[m];
#pragma unroll
    for (int m = 0; m < kRbMax; ++m) {
      if (m >= R) break;
#pragma unroll
      for (int mp = 0; mp < kRbMax; ++mp) {
        if (mp >= R) break;
        const float2 gmm = warp_sum2(cmulc(v[mp], y[m]));
        e[m] = csub(e[m], cmul(v[mp], gmm));
      }
      ry += cabs2(y[m]);
      re += cabs2(e[m]);
    }
    ry = warp_sum(ry);
    re = warp_sum(re);
    orthonormalise(y);
#pragma unroll
    for (int m = 0; m < kRbMax; ++m) v[m] = y[m];
    if (re <= 1e-12f * ry) break;
  }
  // Rayleigh-Ritz values (FP32) for reporting: eigenvalues of V^H B V
  {
#pragma unroll
    for (int m = 0; m < kRbMax; ++m)
      if (row) Vs[lane * kRbMax + m] = v[m];
    __syncwarp();
    float2 G[kRbMax][kRbMax];
    float2 bv[kRbMax];
#pragma unroll
    for (int m = 0; m < kRbMax; ++m) bv[m] = make_float2(0.f, 0.f);
    if (row) {
      for (int l = 0; l < Q; ++l) {
        const float4 b = b_at<Q>(Bc, lane, l);
        const float2 bh = make_float2(b.x, b.z);
#pragma unroll
        for (int m = 0; m < kRbMax; ++m) bv[m] = cadd(bv[m], cmul(bh, Vs[l * kRbMax + m]));
      }
    }
    __syncwarp();
#pragma unroll
    for (int m = 0; m < kRbMax; ++m)
#pragma unroll
      for (int mp = 0; mp < kRbMax; ++mp)
        G[m][mp] = (m < R && mp < R) ? warp_sum2(cmulc(v[m], bv[mp]))
                                     : make_float2(0.f, 0.f);
    float dd[kRbMax];
    float2 UU[kRbMax][kRbMax];
    jacobi_small<kRbMax>(G, dd, UU);
#pragma unroll
    for (int m = 0; m < kRbMax; ++m) lam[m] = dd[m];
  }
  // float-float subspace steps: Y = B V (FF), Cholesky-QR in FF
  cff U[kRbMax];
  for (int step = 0; step < 3; ++step) {
#pragma unroll
    for (int m = 0; m < kRbMax; ++m)
      if (row) Vs[lane * kRbMax + m] = v[m];
    __syncwarp();
    float s[kRbMax][4];
#pragma unroll
    for (int m = 0; m < kRbMax; ++m) s[m][0] = s[m][1] = s[m][2] = s[m][3] = 0.f;
    if (row) {
      for (int l = 0; l < Q; ++l) {
        const float4 b = b_at<Q>(Bc, lane, l);
#pragma unroll
        for (int m = 0; m < kRbMax; ++m) {
          const float2 x = Vs[l * kRbMax + m];
          // (br + i bi)(xr + i xi): re = br xr - bi xi, im = br xi + bi xr
          acc_ffxf(s[m][0], s[m][1], b.x, b.y, x.x);
          acc_ffxf(s[m][0], s[m][1], b.z, b.w, -x.y);
          acc_ffxf(s[m][2], s[m][3], b.x, b.y, x.y);
          acc_ffxf(s[m][2], s[m][3], b.z, b.w, x.x);
        }
      }
    }
    __syncwarp();
    cff Yf[kRbMax];
#pragma unroll
    for (int m = 0; m < kRbMax; ++m) Yf[m] = cff{ff_make(s[m][0], s[m][1]), ff_make(s[m][2], s[m][3])};
    // Gram G = Y^H Y (FF), Cholesky G = L L^H, U = Y L^-H
    cff G[kRbMax][kRbMax];
#pragma unroll
    for (int m = 0; m < kRbMax; ++m)
#pragma unroll
      for (int mp = m; mp < kRbMax; ++mp) {
        if (m < R && mp < R) {
          const cff pr = cff_cmul(Yf[m], Yf[mp]);
          G[m][mp] = cff{ff_warp_sum(pr.re), ff_warp_sum(pr.im)};
        } else {
          G[m][mp] = cff_zero();
        }
      }
    cff L[kRbMax][kRbMax];
#pragma unroll
    for (int m = 0; m < kRbMax; ++m) {
      if (m >= R) break;
      ff dsum = G[m][m].re;
#pragma unroll
      for (int k = 0; k < kRbMax; ++k) {
        if (k >= m) break;
        dsum = ff_sub(dsum, ff_add(ff_mul(L[m][k].re, L[m][k].re), ff_mul(L[m][k].im, L[m][k].im)));
      }
      const ff lmm = ff_sqrt(dsum);
      L[m][m] = cff{lmm, {0.f, 0.f}};
#pragma unroll
      for (int i = 0; i < kRbMax; ++i) {
        if (i <= m || i >= R) continue;
        // L[i][m] = (G[i][m] - sum_k L[i][k] conj(L[m][k])) / L[m][m];  G[i][m] = conj(G[m][i])
        cff t = cff{G[m][i].re, ff_neg(G[m][i].im)};
#pragma unroll
        for (int k = 0; k < kRbMax; ++k) {
          if (k >= m) break;
          t = cff_sub(t, cff_mul(L[i][k], cff{L[m][k].re, ff_neg(L[m][k].im)}));
        }
        L[i][m] = cff{ff_div(t.re, lmm), ff_div(t.im, lmm)};
      }
    }
    float change = 0.f;
#pragma unroll
    for (int m = 0; m < kRbMax; ++m) {
      if (m >= R) {
        U[m] = cff_zero();
        continue;
      }
      cff t = Yf[m];
#pragma unroll
      for (int k = 0; k < kRbMax; ++k) {
        if (k >= m) break;
        // Y[:, m] = sum_{k <= m} U[:, k] conj(L[m][k])
        t = cff_sub(t, cff_mul(U[k], cff{L[m][k].re, ff_neg(L[m][k].im)}));
      }
      const ff lmm = L[m][m].re;
      U[m] = cff{ff_div(t.re, lmm), ff_div(t.im, lmm)};
      if (!row) U[m] = cff_zero();
    }
    // change of the subspace: |U - V V^H U|_F (single precision estimate)
#pragma unroll
    for (int m = 0; m < kRbMax; ++m) {
      if (m >= R) break;
      float2 um = make_float2(U[m].re.hi, U[m].im.hi);
      float2 e = um;
#pragma unroll
      for (int mp = 0; mp < kRbMax; ++mp) {
        if (mp >= R) break;
        const float2 cc = warp_sum2(cmulc(v[mp], um));
        e = csub(e, cmul(v[mp], cc));
      }
      change += cabs2(e);
    }
    change = warp_sum(change);
#pragma unroll
    for (int m = 0; m < kRbMax; ++m) v[m] = make_float2(U[m].re.hi, U[m].im.hi);
    if (step >= 1 && change < 1e-12f) break;
  }
#pragma unroll
  for (int m = 0; m < kRbMax; ++m) {
    uh[m] = make_float2(U[m].re.hi, U[m].im.hi);
    ul[m] = make_float2(U[m].re.lo, U[m].im.lo);
  }
}

// ------------------------------------------------ K4: detect ---------------
// One warp per cell.  Bank in shared memory, transposed: bT[j * V + v].
template <int P, int Q>
__global__ void __launch_bounds__(kThreads)
k_detect(const float2* __restrict__ Y, Geom g, const float2* __restrict__ bank_aT,
         const float2* __restrict__ bank_bT, const float* __restrict__ bank_n2,
         const float2* __restrict__ UA, const float2* __restrict__ UBh,
         const float2* __restrict__ UBl, float* __restrict__ Tmax, int32_t* __restrict__ vidx,
         uint8_t* __restrict__ map, float* __restrict__ T_all) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int V = g.V;
  float2* aT = reinterpret_cast<float2*>(smem);       // [P][V]
  float2* bT = aT + P * V;                             // [Q][V]
  float* na = reinterpret_cast<float*>(bT + Q * V);    // [V]
  float* nb = na + V;                                  // [V]
  constexpr int WS = P * Q + 2 * Q * kRbMax + P * 2;   // per-warp float2 scratch
  float2* wsp = reinterpret_cast<float2*>(na + 2 * V);  // 8V bytes past an 8-aligned start
  for (int i = threadIdx.x; i < P * V; i += blockDim.x) aT[i] = bank_aT[i];
  for (int i = threadIdx.x; i < Q * V; i += blockDim.x) bT[i] = bank_bT[i];
  for (int i = threadIdx.x; i < 2 * V; i += blockDim.x) na[i] = bank_n2[i];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const size_t cell = (size_t)blockIdx.x * (kThreads / 32) + warp;
  const size_t ncell = (size_t)g.H * g.W;
  if (cell >= ncell) return;
  float2* Zs = wsp + warp * WS;              // [P][Q]
  float2* Us = Zs + P * Q;                   // [Q][kRbMax] hi
  float2* Ul = Us + Q * kRbMax;              // [Q][kRbMax] lo
  float2* Uas = Ul + Q * kRbMax;             // [P] (r_a = 1 columns; P * r_a <= 2P)
  const int r = (int)(cell / g.W), c = (int)(cell % g.W);
  const int R = g.r_b;
  const bool row = lane < Q;
  // X column `lane`, U_B row `lane`
  float2 x[P];
  float2 uh[kRbMax], ul[kRbMax];
#pragma unroll
  for (int i = 0; i < P; ++i)
    x[i] = row ? __ldg(Y + ((size_t)i * g.H_in + (r + g.Rr)) * g.W_in + (c + g.Ra + lane))
               : make_float2(0.f, 0.f);
#pragma unroll
  for (int m = 0; m < kRbMax; ++m) {
    uh[m] = (row && m < R) ? UBh[(cell * Q + lane) * R + m] : make_float2(0.f, 0.f);
    ul[m] = (row && m < R) ? UBl[(cell * Q + lane) * R + m] : make_float2(0.f, 0.f);
    if (row) {
      Us[lane * kRbMax + m] = uh[m];
      Ul[lane * kRbMax + m] = ul[m];
    }
  }
  if (lane < P * g.r_a) Uas[lane] = UA[cell * P * g.r_a + lane];
  // C[i][m] = sum_j X[i][j] conj(U_B[j][m])  (float-float)
  cff Cm[P][kRbMax];
#pragma unroll
  for (int i = 0; i < P; ++i)
#pragma unroll
    for (int m = 0; m < kRbMax; ++m) {
      float sr = 0.f, cr = 0.f, si = 0.f, ci = 0.f;
      // x * conj(u): re = xr ur + xi ui, im = xi ur - xr ui
      acc_ffxf(sr, cr, uh[m].x, ul[m].x, x[i].x);
      acc_ffxf(sr, cr, uh[m].y, ul[m].y, x[i].y);
      acc_ffxf(si, ci, uh[m].x, ul[m].x, x[i].y);
      acc_ffxf(si, ci, uh[m].y, ul[m].y, -x[i].x);
      Cm[i][m] = cff{ff_warp_sum(ff_make(sr, cr)), ff_warp_sum(ff_make(si, ci))};
    }
  // Z1 = X - C U_B^T (float-float), then Z = Z1 - U_A U_A^H Z1 (FP32)
  float2 z[P];
#pragma unroll
  for (int i = 0; i < P; ++i) {
    cff t = cff{{x[i].x, 0.f}, {x[i].y, 0.f}};
#pragma unroll
    for (int m = 0; m < kRbMax; ++m) {
      if (m >= R) break;
      const cff u = cff{{uh[m].x, ul[m].x}, {uh[m].y, ul[m].y}};
      t = cff_sub(t, cff_mul(Cm[i][m], u));
    }
    z[i] = make_float2(__fadd_rn(t.re.hi, t.re.lo), __fadd_rn(t.im.hi, t.im.lo));
  }
  __syncwarp();
  for (int m = 0; m < g.r_a; ++m) {
    float2 tm = make_float2(0.f, 0.f);
#pragma unroll
    for (int i = 0; i < P; ++i) tm = cadd(tm, cmulc(Uas[i * g.r_a + m], z[i]));
#pragma unroll
    for (int i = 0; i < P; ++i) z[i] = csub(z[i], cmul(Uas[i * g.r_a + m], tm));
  }
  if (row)
#pragma unroll
    for (int i = 0; i < P; ++i) Zs[i * Q + lane] = row ? z[i] : make_float2(0.f, 0.f);
  __syncwarp();
  // bank: lane handles v = lane, lane + 32, ...
  float best = -1.f;
  int bestv = 0;
  for (int v = lane; v < V; v += 32) {
    // num = a_v^H Z conj(b_v)
    float2 num = make_float2(0.f, 0.f);
#pragma unroll
    for (int i = 0; i < P; ++i) {
      float2 zi = make_float2(0.f, 0.f);
#pragma unroll
      for (int j = 0; j < Q; ++j) zi = cadd(zi, cmul(Zs[i * Q + j], cconj(bT[j * V + v])));
      num = cadd(num, cmulc(aT[i * V + v], zi));
    }
    // den_B = |b|^2 - sum_m |U_B[:,m]^H b|^2, den_A likewise
    float pb = 0.f;
    for (int m = 0; m < R; ++m) {
      float2 t = make_float2(0.f, 0.f);
#pragma unroll
      for (int j = 0; j < Q; ++j) t = cadd(t, cmulc(Us[j * kRbMax + m], bT[j * V + v]));
      pb += cabs2(t);
    }
    float pa = 0.f;
    for (int m = 0; m < g.r_a; ++m) {
      float2 t = make_float2(0.f, 0.f);
#pragma unroll
      for (int i = 0; i < P; ++i) t = cadd(t, cmulc(Uas[i * g.r_a + m], aT[i * V + v]));
      pa += cabs2(t);
    }
    const float nav = na[v], nbv = nb[v];
    float denA = nav - pa, denB = nbv - pb;
    float nm = cabs2(num);
    if (denB < kBlind * nbv || denA < kBlind * nav) {
      // re-project the steering factors: w_b = F_B b in float-float, w_a = F_A a
      float2 wa[P];
#pragma unroll
      for (int i = 0; i < P; ++i) wa[i] = aT[i * V + v];
      for (int m = 0; m < g.r_a; ++m) {
        float2 t = make_float2(0.f, 0.f);
#pragma unroll
        for (int i = 0; i < P; ++i) t = cadd(t, cmulc(Uas[i * g.r_a + m], aT[i * V + v]));
#pragma unroll
        for (int i = 0; i < P; ++i) wa[i] = csub(wa[i], cmul(Uas[i * g.r_a + m], t));
      }
      cff tb[kRbMax];
#pragma unroll
      for (int m = 0; m < kRbMax; ++m) {
        float sr = 0.f, cr = 0.f, si = 0.f, ci = 0.f;
        if (m < R) {
#pragma unroll
          for (int j = 0; j < Q; ++j) {
            const float2 b = bT[j * V + v];
            const float2 h = Us[j * kRbMax + m], l = Ul[j * kRbMax + m];
            // conj(u) b: re = ur br + ui bi, im = ur bi - ui br
            acc_ffxf(sr, cr, h.x, l.x, b.x);
            acc_ffxf(sr, cr, h.y, l.y, b.y);
            acc_ffxf(si, ci, h.x, l.x, b.y);
            acc_ffxf(si, ci, h.y, l.y, -b.x);
          }
        }
        tb[m] = cff{ff_make(sr, cr), ff_make(si, ci)};
      }
      float2 numw = make_float2(0.f, 0.f);
      float dB = 0.f;
      float2 zi[P];
#pragma unroll
      for (int i = 0; i < P; ++i) zi[i] = make_float2(0.f, 0.f);
#pragma unroll
      for (int j = 0; j < Q; ++j) {
        const float2 b = bT[j * V + v];
        cff w = cff{{b.x, 0.f}, {b.y, 0.f}};
#pragma unroll
        for (int m = 0; m < kRbMax; ++m) {
          if (m >= R) break;
          const cff u = cff{{Us[j * kRbMax + m].x, Ul[j * kRbMax + m].x},
                            {Us[j * kRbMax + m].y, Ul[j * kRbMax + m].y}};
          w = cff_sub(w, cff_mul(u, tb[m]));
        }
        const float2 wb = make_float2(__fadd_rn(w.re.hi, w.re.lo), __fadd_rn(w.im.hi, w.im.lo));
        dB += cabs2(wb);
#pragma unroll
        for (int i = 0; i < P; ++i) zi[i] = cadd(zi[i], cmul(Zs[i * Q + j], cconj(wb)));
      }
      float dA = 0.f;
#pragma unroll
      for (int i = 0; i < P; ++i) {
        dA += cabs2(wa[i]);
        numw = cadd(numw, cmulc(wa[i], zi[i]));
      }
      nm = cabs2(numw);
      denA = dA;
      denB = dB;
    }
    const float den = denA * denB;
    const float T = (den < 1e-12f * nav * nbv) ? 0.f : nm / den;
    if (T_all) T_all[cell * V + v] = T;
    if (T > best) {
      best = T;
      bestv = v;
    }
  }
  // warp argmax, lowest v on ties
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float ob = __shfl_xor_sync(0xffffffffu, best, o);
    const int ov = __shfl_xor_sync(0xffffffffu, bestv, o);
    if (ob > best || (ob == best && ov < bestv)) {
      best = ob;
      bestv = ov;
    }
  }
  if (lane == 0) {
    Tmax[cell] = best;
    vidx[cell] = bestv;
    map[cell] = (best > g.tau) ? 1 : 0;
  }
}

}  // namespace kstap
