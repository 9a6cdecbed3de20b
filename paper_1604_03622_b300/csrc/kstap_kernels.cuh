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
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "kstap_ff.cuh"

namespace kstap {

constexpr int kTileCells = 32;      // cells of one range row per CTA (moments / B passes)
constexpr int kThreads = 256;
constexpr int kRbMax = 8;    // largest r_b
constexpr int kRbTc = 4;     // largest r_b of the tensor-core bank (2 (p + r_b) <= 16 operand rows)

// Lanes of the group that holds one cell wherever a cell's q rows map onto
// lanes (q <= 32): the next power of two, so that groups tile a warp; lanes
// j >= q of a group hold no row and contribute zeros to the group sums.
__host__ __device__ constexpr int grp_lanes(int q) { return q <= 8 ? 8 : q <= 16 ? 16 : 32; }
constexpr float kBlindRefine = 1e-3f;   // |F_B b|^2 / |b|^2 below which w_b is refined in float-float
constexpr int kBlindQ = 32;             // near-blind (cell, velocity) pairs queued per warp and pass
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
  int filter;     // 0: F_A (x) F_B (Eq. KronSTAP); 1: I - (U_A (x) U_B)(U_A (x) U_B)^H (Sec. 5)
  long long ch_stride;   // elements between channel planes of Y (>= H_in * W_in)
};

// One frame of a batch.  Per-cell workspace arrays of a launch are
// struct-of-arrays over all cells of all jobs (stride NC), this job's cells
// starting at cell0; its lag store starts at lag0 (float4 units).
enum { kKindMoments = 0, kKindFlip = 1, kKindBfit = 2, kKindDetect = 3, kKindMgram = 4,
       kKinds = 5 };
struct Job {
  // 1-D tiled tensor map over this job's frame, as float pairs from Y to the
  // end of the last channel's last row (TMA tile loads of the moments pass);
  // ymap_ok = 0 when Y is not 16-byte aligned or the frame exceeds the map's
  // extent, and that pass then loads its tiles with plain loads
  CUtensorMap ymap;
  int ymap_ok;
  const float2* Y;              // first row of this job's rows, channel 0
  int H_in, W_in, H, W;         // rows / columns of this job (a frame or a row strip of one)
  long long ch_stride;          // elements between channel planes
  long long cell0, lag0;
  unsigned* maxbits;            // 2 words: max |component| bits, non-finite flag
  float2* UA;
  float2* UBh;
  float2* UBl;
  float* lamA;
  float* lamB;
  int32_t* iters;
  float* eta;
  float* Tmax;
  int32_t* vidx;
  uint8_t* map;
  float* T_all;
  int tile0[kKinds];            // first tile of this job in each kernel's tile space
};

// A launch's jobs: one job passed by value (table == nullptr), or a device
// table sorted by tile0.  ntiles = total tiles of each kernel kind.
struct JobList {
  Job one;
  const Job* table;
  int njobs;
  int ntiles[kKinds];
  long long NC;                 // total cells (stride of the per-cell workspace arrays)
  unsigned long long* report;   // optional counters: [0] cells at max_iter, [1] cells flagged
                                // non-finite, [2] cells of the ill-gapped EIG_{r_b} path
  unsigned* fault;              // optional device word: bit 2 = a TMA tile wait gave up
};

__device__ __forceinline__ const Job& job_of(const JobList& L, int kind, int tile, int& local) {
  if (!L.table) {
    local = tile;
    return L.one;
  }
  int lo = 0, hi = L.njobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (L.table[mid].tile0[kind] <= tile)
      lo = mid;
    else
      hi = mid - 1;
  }
  local = tile - L.table[lo].tile0[kind];
  return L.table[lo];
}

__device__ __forceinline__ Geom with_job(const Geom& g0, const Job& J) {
  Geom g = g0;
  g.H_in = J.H_in;
  g.W_in = J.W_in;
  g.ch_stride = J.ch_stride;
  g.H = J.H;
  g.W = J.W;
  return g;
}

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

constexpr float kFltMax = 3.4028234663852886e38f;

// Frame fixed-point shift: maxabs * 2^sh < 2^B.
__device__ __forceinline__ int frame_shift(unsigned maxbits, int B) {
  const float m = __uint_as_float(maxbits);
  if (!(m > 0.f) || !(m <= kFltMax)) return 0;
  return B - 1 - ilogbf(m);
}

// True if any sample of cell (r, c)'s box is NaN or infinite: rows
// [r, r + 2 Rr] and columns [c, c + 2 Ra + q - 1] of every channel (the union
// of its training windows, its guard and its test window).  Lanes `lane` of
// `nl` share the scan; the caller combines their answers.  Only run when the
// frame scan found a non-finite value, so the finite path never pays for it.
__device__ __forceinline__ bool box_nonfinite(const float2* __restrict__ Y, const Geom& g, int r,
                                              int c, int lane, int nl) {
  const int NR = 2 * g.Rr + 1, NK = 2 * g.Ra + g.q;
  const int tot = g.p * NR * NK;
  bool bad = false;
  for (int idx = lane; idx < tot; idx += nl) {
    const int kap = idx % NK, rho = (idx / NK) % NR, i = idx / (NK * NR);
    const float2 y = __ldg(Y + (size_t)i * g.ch_stride + (size_t)(r + rho) * g.W_in + c + kap);
    bad |= !(fabsf(y.x) <= kFltMax) || !(fabsf(y.y) <= kFltMax);
  }
  return bad;
}

// Adds the number of lanes of the calling (converged) warp subset with
// `flag` set to *ctr: one atomic per warp.
__device__ __forceinline__ void count_lanes(unsigned long long* ctr, bool flag) {
  const unsigned mask = __activemask();
  const unsigned b = __ballot_sync(mask, flag);
  if (b && (threadIdx.x & 31) == __ffs(mask) - 1) atomicAdd(ctr, (unsigned long long)__popc(b));
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
      const float2 y = __ldg(Y + (size_t)i * g.ch_stride + (size_t)(r + rho) * g.W_in + gc);
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

// Exact integer < 2^23 as a float: OR it into the mantissa of 2^23 and
// subtract 2^23 (bit-level construction, no conversion instruction).
__device__ __forceinline__ float small_u2f(unsigned t) {
  return __fsub_rn(__uint_as_float(0x4B000000u | t), 8388608.f);
}

// A 64-bit integer |v| < 2^62 as a float-float pair scaled by 2^-60, to
// ~2^-48 relative.  v = t2 2^42 + t1 2^21 + t0 with 21-bit pieces, each
// converted exactly; the pieces are then summed error-free (two_sum).  Only
// 32-bit integer and single-precision operations: 64-bit integer <-> float
// conversions would run on the (narrow) FP64 pipe.
__device__ __forceinline__ void ll_to_ff(long long v, float& hi, float& lo) {
  const int t2 = (int)(v >> 42);                                   // in [-2^20, 2^20)
  const unsigned t1 = (unsigned)((unsigned long long)v >> 21) & 0x1FFFFFu;
  const unsigned t0 = (unsigned)v & 0x1FFFFFu;
  const float f2 = __fmul_rn(__fsub_rn(small_u2f((unsigned)(t2 + 0x400000)), 4194304.f),
                             3.814697265625e-06f);                 // 2^-18
  const float f1 = __fmul_rn(small_u2f(t1), 1.8189894035458565e-12f);   // 2^-39
  const float f0 = __fmul_rn(small_u2f(t0), kLagNorm);                  // 2^-60
  float s, e;
  two_sum(f2, f1, s, e);
  quick_two_sum(s, __fadd_rn(e, f0), hi, lo);
}

// Plane groups of the single-pass lag planes (p <= 3): group gi < P is the
// diagonal plane J = i + P i alone (j2 = -1); the others are the pairs
// (j1 = i + P k, j2 = k + P i), i < k.  The B pass replaces a pair's planes
// in its tile buffers by S = L_j1 + L_j2 at j1 and D = L_j1 - L_j2 at j2,
// because with a Hermitian a (a_j2 = conj(a_j1)) the pair's part of
// B = sum_J conj(a_J) L_J is Re(a_j1) S - i Im(a_j1) D: two real-coefficient
// float-float products per entry instead of two complex ones.
template <int P>
__device__ __forceinline__ void plane_group(int gi, int& j1, int& j2) {
  if (gi < P) {
    j1 = gi * (P + 1);
    j2 = -1;
    return;
  }
  int idx = gi - P;
  j1 = 0;
  j2 = -1;
#pragma unroll
  for (int i = 0; i < P; ++i)
#pragma unroll
    for (int k = i + 1; k < P; ++k) {
      if (idx == 0) {
        j1 = i + P * k;
        j2 = k + P * i;
      }
      --idx;
    }
}

constexpr int kMomRows = 4;                         // cell rows per CTA in the moments pass
constexpr int kMomThreads = kTileCells * kMomRows;  // one thread per cell
constexpr int kHChunk = 3;                          // positions per item in the running ring sums

// TMA staging of the moments pass's frame tile.  Each (channel, row) segment
// of WT complex samples is one load of the job's 1-D tensor map (float
// elements); a TMA start coordinate must be 16-byte aligned, so a load starts
// at the even sample at or before the segment and covers WT + 1 samples,
// rounded up to whole 16-byte units.  A tensor copy's shared-memory
// destination must be 128-byte aligned: the staging area starts at the first
// 128-byte boundary of its region and its rows are 128-byte multiples apart.
// Host and device size the box and the staging area with these functions.
__host__ __device__ constexpr int moments_box_floats(int WT) { return ((2 * (WT + 1) + 3) / 4) * 4; }
__host__ __device__ constexpr int moments_stage_row_floats(int WT) {
  return ((moments_box_floats(WT) + 31) / 32) * 32;
}
__host__ __device__ constexpr int moments_stage_bytes(int P, int NRT, int WT) {
  return P * NRT * moments_stage_row_floats(WT) * 4 + 128;
}
constexpr long long kTmaWaitCycles = 1ll << 30;   // ~0.5 s at 2 GHz: bound of one tile wait

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// One 1-D tiled TMA load of the map's box at element x into shared memory,
// completing on the mbarrier's transaction count.
__device__ __forceinline__ void tma_load_1d(void* dst, const CUtensorMap* map, int x,
                                            uint64_t* mbar) {
  asm volatile(
      "cp.async.bulk.tensor.1d.shared::cluster.global.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2}], [%3];\n" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(smem_addr(mbar))
      : "memory");
}

// Polls the mbarrier for phase `parity` for at most `cycles` SM cycles.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* mbar, uint32_t parity,
                                                  long long cycles) {
  uint32_t done = 0;
  const long long t0 = clock64();
  while (!done && clock64() - t0 < cycles) {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_addr(mbar)), "r"(parity)
        : "memory");
  }
  return done != 0;
}

// ------------------------------------------------ K1a: lag moments ---------
// CTA = kMomRows cell rows x kTileCells cells, one thread per cell.  The
// vertical box sums run down the kMomRows rows as exact int64 running sums.
// Output per cell (struct of arrays, element-major: X[e * ncell + cell]):
//   Mw[e]  e < PP(PP+1)/2 : M = R R^H upper triangle, in 2^-60 L units
//   Sw[J]                 : sum of the entries of block S(i, k) (A_0 ~ this)
// Lags run g = Q-1 .. 0.  Before lag 0 each thread folds in the negative lags:
// W <- W + conj(Pi W Pi^T), s <- s + conj(Pi s) (linear, so per-thread partial
// sums may be folded before they are complete).
// Lag store (optional, Lw != nullptr): the exact lag sums of every cell row,
// as float-float complex (re_hi, im_hi, re_lo, im_lo), laid out
// Lw[((row * Q + g) * PP + J) * WL + u], WL = W + Q - 1, so that the B pass
// reads them instead of recomputing them.  Each tile writes positions
// u in [c0, c0 + TC) (the last tile also its halo).
template <int P, int Q>
__global__ void __launch_bounds__(kMomThreads)
k_moments(const __grid_constant__ Geom g0, const __grid_constant__ JobList JL,
          float2* __restrict__ Mw, float2* __restrict__ Sw, float4* __restrict__ Lw0) {
  constexpr int PP = P * P;
  // the per-thread Gram M (and the block sums) only for P <= 3; for more
  // channels (stacked passes) this pass writes the lag store and k_mgram forms
  // M and the block sums from it with a warp per cell
  constexpr bool kThreadM = P <= 3;
  constexpr int NE = kThreadM ? PP * (PP + 1) / 2 : 1;
  constexpr int NS = kThreadM ? PP : 1;
  constexpr int TC = kTileCells;
  constexpr int TR = kMomRows;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t ymbar;   // completion of a tile's TMA loads
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(&ymbar)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  uint32_t yphase = 0;
  for (int tile = blockIdx.x; tile < JL.ntiles[kKindMoments]; tile += gridDim.x) {
  int lt;
  const Job& JB = job_of(JL, kKindMoments, tile, lt);
  const Geom g = with_job(g0, JB);
  const float2* __restrict__ Y = JB.Y;
  const unsigned* __restrict__ maxbits = JB.maxbits;
  float4* __restrict__ Lw = Lw0 ? Lw0 + JB.lag0 : nullptr;
  const int ntx = (g.W + TC - 1) / TC;
  const int r0 = (lt / ntx) * TR;
  const int c0 = (lt % ntx) * TC;
  const int WT = TC + 2 * g.Ra + Q - 1;
  const int NR = 2 * g.Rr + 1;
  const int NRT = NR + TR - 1;
  const int NUmax = TC + Q - 1;
  int2* Yq = reinterpret_cast<int2*>(smem);                                  // [P][NRT][WT]
  longlong2* Vo = reinterpret_cast<longlong2*>(Yq + P * NRT * WT + (P * NRT * WT & 1));
  longlong2* Vg = Vo + PP * WT;                                             // [PP][WT]
  float2* lag = reinterpret_cast<float2*>(Vg + PP * WT);                    // [TR][PP][NUmax]

  const int sh = frame_shift(*maxbits, g.B);
  const float scale = ldexpf(1.f, sh);
  // a tensor map must sit on a 64-byte boundary (it does in the kernel
  // parameters and in the device job table; plain loads otherwise)
  if (JB.ymap_ok && (reinterpret_cast<uintptr_t>(&JB.ymap) & 63) == 0) {
    // TMA: warp 0 arms the mbarrier with the tile's bytes and issues one load
    // per (channel, row) segment inside the frame into the staging area (the
    // box-sum buffers, dead until the lag loop); every thread then waits and
    // converts its samples from the staging rows (offset by the odd start)
    float* stg = reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(Vo) +
                                          ((128u - (smem_addr(Vo) & 127u)) & 127u));
    const int BF = moments_stage_row_floats(WT);   // row stride; the box is moments_box_floats
    const int nin = min(NRT, g.H_in - r0);   // rows inside the frame
    if (threadIdx.x < 32) {
      if (threadIdx.x == 0) {
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(
                         smem_addr(&ymbar)),
                     "r"((unsigned)(P * nin * moments_box_floats(WT) * 4))
                     : "memory");
      }
      __syncwarp();
      for (int s = threadIdx.x; s < P * nin; s += 32) {
        const int i = s / nin, rho = s - i * nin;
        const long long e = (long long)i * g.ch_stride + (long long)(r0 + rho) * g.W_in + c0;
        tma_load_1d(stg + (i * NRT + rho) * BF, &JB.ymap, (int)((e & ~1ll) * 2), &ymbar);
      }
    }
    if (!mbar_wait_bounded(&ymbar, yphase, kTmaWaitCycles)) {
      if (JL.fault) atomicOr(JL.fault, 4u);
      mbar_wait_bounded(&ymbar, yphase, kTmaWaitCycles);
    }
    yphase ^= 1u;
    const int total = P * NRT * WT;
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
      const int col = idx % WT;
      const int rho = (idx / WT) % NRT;
      const int i = idx / (WT * NRT);
      const int gr = r0 + rho, gc = c0 + col;
      int2 v = make_int2(0, 0);
      if (gc < g.W_in && gr < g.H_in) {
        const long long e = (long long)i * g.ch_stride + (long long)gr * g.W_in + c0;
        const float2 y = *reinterpret_cast<const float2*>(
            stg + (i * NRT + rho) * BF + 2 * (col + (int)(e & 1)));
        v.x = quantise(y.x, scale);
        v.y = quantise(y.y, scale);
      }
      Yq[idx] = v;
    }
  } else {
    const int total = P * NRT * WT;
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
      const int col = idx % WT;
      const int rho = (idx / WT) % NRT;
      const int i = idx / (WT * NRT);
      const int gr = r0 + rho, gc = c0 + col;
      int2 v = make_int2(0, 0);
      if (gc < g.W_in && gr < g.H_in) {
        const float2 y = __ldg(Y + (size_t)i * g.ch_stride + (size_t)gr * g.W_in + gc);
        v.x = quantise(y.x, scale);
        v.y = quantise(y.y, scale);
      }
      Yq[idx] = v;
    }
  }
  __syncthreads();

  const int tr = threadIdx.x / TC, cl = threadIdx.x % TC;
  const bool live = (c0 + cl) < g.W && (r0 + tr) < g.H;
  float2 W[NE];   // entries of M (re, im), packed pairs
  float sr[NS], si[NS];
#pragma unroll
  for (int e = 0; e < NE; ++e) W[e] = make_float2(0.f, 0.f);
#pragma unroll
  for (int J = 0; J < NS; ++J) sr[J] = si[J] = 0.f;

  const int g0 = g.Rr - g.Gr, g1 = g.Rr + g.Gr;
  for (int lagg = Q - 1; lagg >= 0; --lagg) {
    const int NU = TC + Q - 1 - lagg;
    const int KW = NU + 2 * g.Ra;
    const bool last_tile = c0 + TC >= g.W;
    const int WL = g.W + Q - 1;
    const int nch = (NU + kHChunk - 1) / kHChunk;
#pragma unroll 1
    for (int t = 0; t < TR; ++t) {
      // (1) vertical ring sums of cell row t, one item per (channel i, column
      // kap) covering the P pairs J = i + P k (one load of channel i per row
      // serves them all): direct for t = 0, running (rows entering and leaving
      // the box and the guard band) after
      for (int item = threadIdx.x; item < P * KW; item += blockDim.x) {
        const int i = item / KW, kap = item - i * KW;
        if (t == 0) {
          longlong2 vo[P], vg[P];
#pragma unroll
          for (int k = 0; k < P; ++k) vo[k] = vg[k] = make_longlong2(0, 0);
          for (int rho = 0; rho < NR; ++rho) {
            const int2 a = Yq[(i * NRT + rho) * WT + kap];
            const bool guard = rho >= g0 && rho <= g1;
#pragma unroll
            for (int k = 0; k < P; ++k) {
              const int2 b = Yq[(k * NRT + rho) * WT + kap + lagg];
              const long long pr = (long long)a.x * b.x + (long long)a.y * b.y;
              const long long pim = (long long)a.y * b.x - (long long)a.x * b.y;
              vo[k].x += pr;
              vo[k].y += pim;
              if (guard) {
                vg[k].x += pr;
                vg[k].y += pim;
              }
            }
          }
#pragma unroll
          for (int k = 0; k < P; ++k) {
            Vo[(i + P * k) * WT + kap] = vo[k];
            Vg[(i + P * k) * WT + kap] = vg[k];
          }
        } else {
          const int2 ai = Yq[(i * NRT + t - 1 + NR) * WT + kap];   // entering the box
          const int2 ao = Yq[(i * NRT + t - 1) * WT + kap];        // leaving it
          const int2 gi = Yq[(i * NRT + t + g1) * WT + kap];       // entering the guard band
          const int2 go = Yq[(i * NRT + t - 1 + g0) * WT + kap];   // leaving it
#pragma unroll 1
          for (int k = 0; k < P; ++k) {
            const int J = i + P * k;
            const int2* yk = Yq + (size_t)k * NRT * WT + kap + lagg;
            const int2 bi = yk[(t - 1 + NR) * WT], bo = yk[(t - 1) * WT];
            const int2 hi = yk[(t + g1) * WT], ho = yk[(t - 1 + g0) * WT];
            longlong2 vo = Vo[J * WT + kap], vg = Vg[J * WT + kap];
            vo.x += (long long)ai.x * bi.x + (long long)ai.y * bi.y -
                    (long long)ao.x * bo.x - (long long)ao.y * bo.y;
            vo.y += (long long)ai.y * bi.x - (long long)ai.x * bi.y -
                    (long long)ao.y * bo.x + (long long)ao.x * bo.y;
            vg.x += (long long)gi.x * hi.x + (long long)gi.y * hi.y -
                    (long long)go.x * ho.x - (long long)go.y * ho.y;
            vg.y += (long long)gi.y * hi.x - (long long)gi.x * hi.y -
                    (long long)go.y * ho.x + (long long)go.x * ho.y;
            Vo[J * WT + kap] = vo;
            Vg[J * WT + kap] = vg;
          }
        }
      }
      __syncthreads();
      // (2) horizontal ring sums, exact int64, one item per (plane, chunk of
      // kHChunk positions): the chunk's first sum direct, the rest running
      // (L(u + 1) = L(u) + Vo[u + 1 + 2Ra] - Vo[u] - Vg[u + 1 + Ra + Ga] +
      // Vg[u + Ra - Ga]); kHChunk is odd, so the lanes of a warp start in
      // different 16-byte bank groups.  Each sum goes straight to
      // float-float: row t's hi parts for the M products, and the lag store
      // (positions of this tile; the last tile also its halo).
      for (int item = threadIdx.x; item < PP * nch; item += blockDim.x) {
        const int J = item / nch, u0 = (item - J * nch) * kHChunk;
        const int u1 = min(u0 + kHChunk, NU);
        const longlong2* vo = Vo + J * WT;
        const longlong2* vg = Vg + J * WT;
        longlong2 L = ring_sum(vo, vg, g, u0);
        for (int u = u0; u < u1; ++u) {
          if (u > u0) {
            const longlong2 a = vo[u + 2 * g.Ra], b = vo[u - 1];
            const longlong2 c = vg[u + g.Ra + g.Ga], d = vg[u - 1 + g.Ra - g.Ga];
            L.x += a.x - b.x - c.x + d.x;
            L.y += a.y - b.y - c.y + d.y;
          }
          float4 v;
          ll_to_ff(L.x, v.x, v.z);
          ll_to_ff(L.y, v.y, v.w);
          if constexpr (kThreadM) lag[((size_t)t * PP + J) * NUmax + u] = make_float2(v.x, v.y);
          if (Lw && (u < TC || last_tile) && c0 + u < WL && r0 + t < g.H)
            Lw[(((size_t)(r0 + t) * Q + lagg) * PP + J) * WL + c0 + u] = v;
        }
      }
      __syncthreads();
    }
    if constexpr (kThreadM) {
    if (lagg == 0) {
      // fold the negative lags: W += conj(Pi W Pi^T), s += conj(Pi s)
#pragma unroll
      for (int J = 0; J < PP; ++J) {
#pragma unroll
        for (int Jp = J; Jp < PP; ++Jp) {
          const int a = (J % P) * P + (J / P), b = (Jp % P) * P + (Jp / P);
          const int e = tri_idx(PP, J, Jp);
          const int ep = (a <= b) ? tri_idx(PP, a, b) : tri_idx(PP, b, a);
          if (ep < e) continue;                 // each pair once
          if (ep == e) {
            // conj(W[pi J, pi J']) with the same storage slot
            const float xr = W[e].x, xi = (a <= b) ? W[e].y : -W[e].y;
            W[e].x += xr;
            W[e].y -= xi;
          } else {
            // slot e receives conj(W[a,b]); slot ep receives conj(W[pi a, pi b]) = conj(W[J,J'] or its conj)
            const float er = W[e].x, ei = W[e].y, fr = W[ep].x, fi = W[ep].y;
            const float abr = fr, abi = (a <= b) ? fi : -fi;    // W[a, b]
            W[e].x = er + abr;
            W[e].y = ei - abi;
            // slot ep holds W[min(a,b), max(a,b)]; pi maps (a,b) back to (J,J')
            const float jr = er, ji = (a <= b) ? ei : -ei;      // W[pi a, pi b] in ep's orientation
            W[ep].x = fr + jr;
            W[ep].y = fi - ji;
          }
        }
      }
#pragma unroll
      for (int J = 0; J < PP; ++J) {
        const int a = (J % P) * P + (J / P);
        if (a < J) continue;
        if (a == J) {
          si[J] = 0.f;                             // s_J + conj(s_J) is real
          sr[J] *= 2.f;
        } else {
          const float xr = sr[J], xi = si[J], yr = sr[a], yi = si[a];
          sr[J] = xr + yr;
          si[J] = xi - yi;
          sr[a] = yr + xr;
          si[a] = yi - xi;
        }
      }
    }
    }
    if constexpr (kThreadM) {
    if (live) {
      const float2* lt = lag + (size_t)tr * PP * NUmax;
      for (int j = 0; j < Q - lagg; ++j) {
        float2 l[PP], lb[PP];
#pragma unroll
        for (int J = 0; J < PP; ++J) {
          l[J] = lt[J * NUmax + cl + j];
          lb[J] = make_float2(l[J].y, -l[J].x);
          sr[J] += l[J].x;
          si[J] += l[J].y;
        }
        // W[J][J'] += l[J] conj(l[J']) = (lr, li) l'r + (li, -lr) l'i, column
        // by column so that only one column's broadcast pairs are live
#pragma unroll
        for (int Jp = 0; Jp < PP; ++Jp) {
          const float2 xr = make_float2(l[Jp].x, l[Jp].x), xi = make_float2(l[Jp].y, l[Jp].y);
#pragma unroll
          for (int J = 0; J <= Jp; ++J) {
            const int e = tri_idx(PP, J, Jp);
            W[e] = f2_fma(lb[J], xi, f2_fma(l[J], xr, W[e]));
          }
        }
      }
    }
    }
    __syncthreads();
  }
  if constexpr (kThreadM) {
  if (live) {
    const size_t ncell = (size_t)JL.NC;
    const size_t cell = (size_t)JB.cell0 + (size_t)(r0 + tr) * g.W + (c0 + cl);
#pragma unroll
    for (int e = 0; e < NE; ++e) Mw[e * ncell + cell] = W[e];
#pragma unroll
    for (int J = 0; J < PP; ++J) Sw[J * ncell + cell] = make_float2(sr[J], si[J]);
  }
  }
  // this tile's generic-proxy writes to the staging area (box sums, row
  // lags) are ordered before the next tile's TMA writes into it
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  __syncthreads();
  }  // tile loop
}

// ------------------------------------------------ small Hermitian Jacobi ---
// Cyclic Jacobi on an N x N Hermitian matrix held in registers (FP32).  On
// return d[] holds the eigenvalues and the columns of U the eigenvectors,
// sorted by decreasing eigenvalue.
// WANT_U = false skips the eigenvector accumulation (eigenvalues only);
// sweeps stop once sum_{i<j} |A_ij|^2 <= tol * sum_i A_ii^2.  Off-diagonal
// entries at or below max(1e-10 (|A_pp| + |A_qq|), abs_skip) are set to zero
// instead of rotated (abs_skip: an absolute floor, e.g. the rounding level of
// the matrix when only its leading eigenpairs are wanted).
template <int N, bool WANT_U = true>
__device__ void jacobi_small(float2 (&A)[N][N], float (&d)[N], float2 (&U)[N][N],
                             float tol = 1e-14f, float abs_skip = 0.f) {
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
    if (off <= tol * diag) break;
#pragma unroll
    for (int p = 0; p < N - 1; ++p) {
#pragma unroll
      for (int q = p + 1; q < N; ++q) {
        const float2 b = A[p][q];
        // |b| without squaring (|b|^2 of a small off-diagonal entry falls
        // into the subnormal range and loses its digits); an entry below
        // 1e-10 of the diagonal pair is dropped: a rotation that small
        // changes nothing at single precision
        const float ab = hypotf(b.x, b.y);
        if (!(ab > fmaxf(1e-10f * (fabsf(A[p][p].x) + fabsf(A[q][q].x)), abs_skip))) {
          A[p][q] = A[q][p] = make_float2(0.f, 0.f);
          continue;
        }
        float2 ph = make_float2(b.x / ab, b.y / ab);                // e^{i phi}
        const float pn = rsqrtf(cabs2(ph));                          // |ph| = 1 to rounding
        ph = make_float2(ph.x * pn, ph.y * pn);
        const float tau = (A[q][q].x - A[p][p].x) / (2.f * ab);
        const float tt = copysignf(1.f, tau) / (fabsf(tau) + sqrtf(1.f + tau * tau));
        const float c = rsqrtf(1.f + tt * tt);
        const float s = tt * c;
        // G = diag(1, conj(ph)) [[c, s], [-s, c]]; A <- G^H A G touches only
        // rows / columns p and q: the 2 x 2 block closes analytically
        // (A_pp -= t |A_pq|, A_qq += t |A_pq|, A_pq = 0), the other entries
        // of columns p, q rotate and are mirrored to keep A Hermitian
        const float2 cph = cconj(ph);
#pragma unroll
        for (int k = 0; k < N; ++k) {
          if (k == p || k == q) continue;
          const float2 akp = A[k][p];
          const float2 x = cmul(cph, A[k][q]);
          const float2 nkp = make_float2(c * akp.x - s * x.x, c * akp.y - s * x.y);
          const float2 nkq = make_float2(s * akp.x + c * x.x, s * akp.y + c * x.y);
          A[k][p] = nkp;
          A[p][k] = cconj(nkp);
          A[k][q] = nkq;
          A[q][k] = cconj(nkq);
        }
        A[p][p] = make_float2(A[p][p].x - tt * ab, 0.f);
        A[q][q] = make_float2(A[q][q].x + tt * ab, 0.f);
        A[p][q] = make_float2(0.f, 0.f);
        A[q][p] = make_float2(0.f, 0.f);
        if (WANT_U) {
#pragma unroll
          for (int k = 0; k < N; ++k) {   // U <- U G
            const float2 up = U[k][p];
            const float2 x = cmul(cph, U[k][q]);
            U[k][p] = make_float2(c * up.x - s * x.x, c * up.y - s * x.y);
            U[k][q] = make_float2(s * up.x + c * x.x, s * up.y + c * x.y);
          }
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

// Classical filter (Sec. 5): its projector keeps the clutter orthogonal to
// u_a, so the statistic needs U_A beyond the single-precision flip-flop's
// ~1e-7.  After the flip-flop, one Alg. 2 update in FP64 from the final a (a
// thread per cell): a~ = M a (M as accumulated), u_a = the leading
// eigenvector of herm(vec^-1 a~) by FP64 power iteration from the
// single-precision U_A (the spatial eigenvalue ratio is ~0.1, so six steps
// take 1e-7 below double rounding).  A kernel of its own, launched for that
// filter only, so the FP64 registers stay out of the flip-flop.
template <int P>
__global__ void __launch_bounds__(128)
k_refine_ua(Geom g0, JobList JL, const float2* __restrict__ Mw, const float2* __restrict__ aw) {
  constexpr int PP = P * P;
  constexpr int NE = PP * (PP + 1) / 2;
  const size_t ncell = (size_t)JL.NC;
  for (int tile = blockIdx.x; tile < JL.ntiles[kKindFlip]; tile += gridDim.x) {
  int lt;
  const Job& JB = job_of(JL, kKindFlip, tile, lt);
  const size_t local = (size_t)lt * blockDim.x + threadIdx.x;
  if (local >= (size_t)JB.H * JB.W) continue;
  const size_t cell = (size_t)JB.cell0 + local;
  float2 M[NE], a[PP];
#pragma unroll
  for (int e = 0; e < NE; ++e) M[e] = Mw[e * ncell + cell];
#pragma unroll
  for (int J = 0; J < PP; ++J) a[J] = aw[J * ncell + cell];
  float2 u[P];
#pragma unroll
  for (int i = 0; i < P; ++i) u[i] = JB.UA[local * P + i];
  double yr[PP], yi[PP];
#pragma unroll
  for (int J = 0; J < PP; ++J) {
    double sr = 0.0, si = 0.0;
#pragma unroll
    for (int Jp = 0; Jp < PP; ++Jp) {
      const float2 m = (J <= Jp) ? M[tri_idx(PP, J, Jp)] : cconj(M[tri_idx(PP, Jp, J)]);
      sr += (double)m.x * a[Jp].x - (double)m.y * a[Jp].y;
      si += (double)m.x * a[Jp].y + (double)m.y * a[Jp].x;
    }
    yr[J] = sr;
    yi[J] = si;
  }
  double ur[P], ui[P];
#pragma unroll
  for (int i = 0; i < P; ++i) {
    ur[i] = u[i].x;
    ui[i] = u[i].y;
  }
  for (int step = 0; step < 6; ++step) {
    double vr[P], vi[P], n2 = 0.0;
#pragma unroll
    for (int i = 0; i < P; ++i) {
      vr[i] = vi[i] = 0.0;
#pragma unroll
      for (int kk = 0; kk < P; ++kk) {
        // herm(vec^-1 y)[i][kk] = (y[i + P kk] + conj(y[kk + P i])) / 2
        const double hr = 0.5 * (yr[i + P * kk] + yr[kk + P * i]);
        const double hi = 0.5 * (yi[i + P * kk] - yi[kk + P * i]);
        vr[i] += hr * ur[kk] - hi * ui[kk];
        vi[i] += hr * ui[kk] + hi * ur[kk];
      }
      n2 += vr[i] * vr[i] + vi[i] * vi[i];
    }
    const double inv = n2 > 0.0 ? 1.0 / sqrt(n2) : 0.0;
#pragma unroll
    for (int i = 0; i < P; ++i) {
      ur[i] = vr[i] * inv;
      vi[i] *= inv;
      ui[i] = vi[i];
    }
  }
#pragma unroll
  for (int i = 0; i < P; ++i) JB.UA[local * P + i] = make_float2((float)ur[i], (float)ui[i]);
  }  // tile loop
}

// ------------------------------------------------ K2: flip-flop ------------
// One thread per cell: Alg. 2 on M = R R^H.  Writes a = vec(A^) (FP32),
// U_A, lamA (tr A^ = p), iterations and eta.
template <int P>
__global__ void __launch_bounds__(128)
k_flipflop(Geom g0, JobList JL, const float2* __restrict__ Mw, const float2* __restrict__ Sw,
           float2* __restrict__ aw) {
  constexpr int PP = P * P;
  constexpr int NE = PP * (PP + 1) / 2;
  const size_t ncell = (size_t)JL.NC;
  for (int tile = blockIdx.x; tile < JL.ntiles[kKindFlip]; tile += gridDim.x) {
  int lt;
  const Job& JB = job_of(JL, kKindFlip, tile, lt);
  const Geom& g = g0;
  const size_t local = (size_t)lt * blockDim.x + threadIdx.x;
  if (local >= (size_t)JB.H * JB.W) continue;
  const size_t cell = (size_t)JB.cell0 + local;
  float2* __restrict__ UA = JB.UA;
  float* __restrict__ lamA = JB.lamA;
  int32_t* __restrict__ iters = JB.iters;
  float* __restrict__ eta = JB.eta;
  float2 M[NE];
#pragma unroll
  for (int e = 0; e < NE; ++e) M[e] = Mw[e * ncell + cell];
  float2 a[PP];
#pragma unroll
  for (int J = 0; J < PP; ++J) a[J] = Sw[J * ncell + cell];
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
    // exactly Hermitian (the two roundings of u_i conj(u_k) and u_k conj(u_i)
    // differ): the B pass forms only the upper triangle of B = sum_J
    // conj(a_J) L_J and mirrors it, which equals the Hermitian part of b only
    // for a Hermitian a; the anti-Hermitian rounding residue would move the
    // ill-gapped eigenvectors of B by ~1e-7 lambda_1 / gap
#pragma unroll
    for (int i = 0; i < P; ++i) {
      an_new[i + P * i].y = 0.f;
#pragma unroll
      for (int k = 0; k < i; ++k) an_new[i + P * k] = cconj(an_new[k + P * i]);
    }
#pragma unroll
    for (int J = 0; J < PP; ++J) {
      dn += cabs2(csub(an_new[J], a[J]));
      nn += cabs2(an_new[J]);
      a[J] = an_new[J];
    }
    if (dn <= tol2 * nn) break;
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
  // eta^2 = 1 - a^H M a / (|a|^2 tr M) for b matched to the final a, with the
  // three sums in float-float (the ratio is 1 - eta^2, so eta << 1 cancels):
  // a^H M a = sum_J M_JJ |a_J|^2 + 2 Re sum_{J<J'} conj(a_J) M_JJ' a_J'
  float trs = 0.f, trc = 0.f, ans = 0.f, anc = 0.f, qs = 0.f, qc = 0.f;
#pragma unroll
  for (int J = 0; J < PP; ++J) {
    const float d = M[tri_idx(PP, J, J)].x;
    float t, e;
    two_sum(trs, d, t, e);
    trs = t;
    trc = __fadd_rn(trc, e);
    float p, pe;
    two_prod(a[J].x, a[J].x, p, pe);            // |a_J|^2 exactly, as two pairs
    acc_ffxf(ans, anc, p, pe, 1.f);
    acc_ffxf(qs, qc, p, pe, d);
    two_prod(a[J].y, a[J].y, p, pe);
    acc_ffxf(ans, anc, p, pe, 1.f);
    acc_ffxf(qs, qc, p, pe, d);
#pragma unroll
    for (int Jp = J + 1; Jp < PP; ++Jp) {
      // 2 Re(conj(a_J) m a_J') with m = M_JJ': m a_J' in float-float first
      const float2 m = M[tri_idx(PP, J, Jp)];
      float rs = 0.f, rc = 0.f, is = 0.f, ic = 0.f;
      acc_prod(rs, rc, m.x, a[Jp].x);
      acc_prod(rs, rc, -m.y, a[Jp].y);
      acc_prod(is, ic, m.x, a[Jp].y);
      acc_prod(is, ic, m.y, a[Jp].x);
      acc_ffxf(qs, qc, rs, rc, 2.f * a[J].x);
      acc_ffxf(qs, qc, is, ic, 2.f * a[J].y);
    }
  }
  const double tr = (double)trs + (double)trc;
  const double an = (double)ans + (double)anc;
  const double aMa = (double)qs + (double)qc;
#pragma unroll
  for (int J = 0; J < PP; ++J) aw[J * ncell + cell] = a[J];
  float trA = 0.f;
#pragma unroll
  for (int m = 0; m < P; ++m)
    if (m < ra) trA += d[m];
  const float sc = (trA != 0.f) ? (float)P / trA : 1.f;
#pragma unroll
  for (int i = 0; i < P; ++i)
#pragma unroll
    for (int m = 0; m < P; ++m)
      if (m < ra) UA[(local * P + i) * ra + m] = U[i][m];
  if (lamA) {
#pragma unroll
    for (int m = 0; m < P; ++m)
      if (m < ra) lamA[local * ra + m] = d[m] * sc;
  }
  if (iters) iters[local] = bad ? -1 : it;
  if (eta) {
    double e2 = (tr > 0.0 && an > 0.0) ? 1.0 - aMa / (an * tr) : 0.0;
    eta[local] = bad ? __int_as_float(0x7fc00000) : (float)sqrt(e2 > 0.0 ? e2 : 0.0);
  }
  }  // tile loop
}

// ------------------------------------------------ K3: B and U_B ------------
// B(j, l) of one cell, float-float upper triangle stored by diagonal:
// diagonal d = l - j >= 0 at offset d*Q - d(d-1)/2, entry j.  float4 =
// (re_hi, im_hi, re_lo, im_lo).  Lower entries are conjugates.
template <int Q>
__host__ __device__ constexpr int diag_off(int d) { return d * Q - (d * (d - 1)) / 2; }

template <int Q>
__device__ __forceinline__ float4 b_at(const float4* __restrict__ Bc, int j, int l) {
  if (l >= j) return Bc[diag_off<Q>(l - j) + j];
  const float4 v = Bc[diag_off<Q>(j - l) + l];
  return make_float4(v.x, -v.y, v.z, -v.w);
}

// Row j of B times the q x R matrix Vs (column-major, [m][l]: lanes read
// consecutive words), visiting l = (j + t) mod Q so that the Q lanes of a
// group also read consecutive entries of B.
template <int Q, int R>
__device__ __forceinline__ void b_times_v_fp32(const float4* __restrict__ Bc, int j,
                                               const float2* __restrict__ Vs, float2 (&y)[R]) {
#pragma unroll
  for (int m = 0; m < R; ++m) y[m] = make_float2(0.f, 0.f);
#pragma unroll 4
  for (int t = 0; t < Q; ++t) {
    const int l = (j + t < Q) ? j + t : j + t - Q;
    const float4 b = b_at<Q>(Bc, j, l);
    const float2 bh = make_float2(b.x, b.y);
#pragma unroll
    for (int m = 0; m < R; ++m) y[m] = cadd(y[m], cmul(bh, Vs[m * Q + l]));
  }
}

template <int G>
__device__ __forceinline__ float grp_sum(float v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <int G>
__device__ __forceinline__ float2 grp_sum2(float2 v) {
  return make_float2(grp_sum<G>(v.x), grp_sum<G>(v.y));
}
template <int G>
__device__ __forceinline__ ff grp_sum_ff(ff v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) {
    ff w;
    w.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
    w.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
    v = ff_add(v, w);
  }
  return v;
}

// Modified Gram-Schmidt of R columns over a group of G lanes holding RP
// rows each (FP32; rows that do not exist are zeros).
template <int G, int RP, int R>
__device__ __forceinline__ void orthonormalise_g(float2 (&x)[RP][R]) {
#pragma unroll
  for (int m = 0; m < R; ++m) {
#pragma unroll
    for (int mp = 0; mp < m; ++mp) {
      float2 d = make_float2(0.f, 0.f);
#pragma unroll
      for (int k = 0; k < RP; ++k) d = cadd(d, cmulc(x[k][mp], x[k][m]));
      const float2 cc = grp_sum2<G>(d);
#pragma unroll
      for (int k = 0; k < RP; ++k) x[k][m] = csub(x[k][m], cmul(x[k][mp], cc));
    }
    float n2 = 0.f;
#pragma unroll
    for (int k = 0; k < RP; ++k) n2 += cabs2(x[k][m]);
    const float nrm = sqrtf(grp_sum<G>(n2));
#pragma unroll
    for (int k = 0; k < RP; ++k) x[k][m] = cscale(x[k][m], nrm > 0.f ? 1.f / nrm : 0.f);
  }
}

// Ritz values of a subspace step: the eigenvalues of the Hermitian part of
// the R x R matrix H = V^H B V (FP32), in decreasing order.
template <int R>
__device__ __forceinline__ void ritz_values(const float2 (&H)[R][R], float (&lam)[R]) {
  {
    float2 Hh[R][R];   // Hermitian part of V^H B V (the Jacobi below assumes it)
#pragma unroll
    for (int m = 0; m < R; ++m)
#pragma unroll
      for (int mp = 0; mp < R; ++mp)
        Hh[m][mp] = make_float2(0.5f * (H[m][mp].x + H[mp][m].x), 0.5f * (H[m][mp].y - H[mp][m].y));
    if constexpr (R == 1) {
      lam[0] = Hh[0][0].x;
    } else if constexpr (R == 2) {
      // the larger root directly, the smaller as det / larger (no cancellation)
      const float a = Hh[0][0].x, d = Hh[1][1].x, h = 0.5f * (a - d), m = 0.5f * (a + d);
      const float r = sqrtf(h * h + cabs2(Hh[0][1]));
      const float det = a * d - cabs2(Hh[0][1]);
      lam[0] = m + r;
      lam[1] = (m + r != 0.f) ? det / (m + r) : m - r;
    } else if constexpr (R == 3) {
      // closed form (trigonometric solution of the characteristic cubic of
      // the shifted, scaled matrix (H - q I) / p, q = tr H / 3): the three
      // Ritz values are well separated relative to the largest here, so its
      // single-precision rounding is far inside the tolerance of lambda_B
      const float a11 = Hh[0][0].x, a22 = Hh[1][1].x, a33 = Hh[2][2].x;
      const float2 a12 = Hh[0][1], a13 = Hh[0][2], a23 = Hh[1][2];
      const float q = (a11 + a22 + a33) * (1.f / 3.f);
      const float b11 = a11 - q, b22 = a22 - q, b33 = a33 - q;
      const float s12 = cabs2(a12), s13 = cabs2(a13), s23 = cabs2(a23);
      const float p2 = b11 * b11 + b22 * b22 + b33 * b33 + 2.f * (s12 + s13 + s23);
      if (!(p2 > 0.f)) {
        lam[0] = lam[1] = lam[2] = q;
      } else {
        const float p = sqrtf(p2 * (1.f / 6.f));
        const float2 t = cmul(a12, a23);
        const float det = b11 * b22 * b33 + 2.f * (t.x * a13.x + t.y * a13.y) - b11 * s23 -
                          b22 * s13 - b33 * s12;   // det(H - q I)
        const float r = fminf(1.f, fmaxf(-1.f, det / (2.f * p * p * p)));
        const float phi = acosf(r) * (1.f / 3.f);
        const float l1 = q + 2.f * p * cosf(phi);
        const float l3 = q + 2.f * p * cosf(phi + 2.0943951f);   // + 2 pi / 3
        lam[0] = l1;
        lam[1] = 3.f * q - l1 - l3;
        lam[2] = l3;
      }
    } else {
      float dd[R];
      float2 UU[R][R];
      // eigenvalues only; an off-diagonal remainder of 1e-5 |diag| moves them
      // by ~1e-10 lambda_1^2 / gap
      jacobi_small<R, false>(Hh, dd, UU, 1e-10f);
#pragma unroll
      for (int m = 0; m < R; ++m) lam[m] = dd[m];
    }
  }
}

// Rows of one cell per lane in the eigen phase of the B pass: two for
// 12 <= q <= 24, so that a cell takes a group of eig_lanes(q) lanes (8 at
// q = 12 and 16, 16 at q = 24) and the r_b x r_b work that every lane of a
// group repeats (Cholesky factor, Ritz values, convergence bound) serves twice
// as many cells per warp; lane jl of a group holds rows jl + k q / 2, k < 2.
// At q = 32 a 16-cell tile already fills the 16 warps of its CTA with one row
// per lane (two rows per lane left half of them idle: B pass 128 -> 179 ms
// on the 2048^2 frame).
__host__ __device__ constexpr int eig_rpl(int q) { return (q >= 12 && q <= 24) ? 2 : 1; }
__host__ __device__ constexpr int eig_lanes(int q) { return grp_lanes(q / eig_rpl(q)); }

constexpr float kSubTol = 1e-8f;   // accepted error of the leading subspace of B
constexpr int kSubSteps = 4;       // float-float subspace steps before a cell is handed on

// Leading R-dimensional eigenspace of one cell's B (a group of eig_lanes(Q)
// lanes, eig_rpl(Q) rows per lane).  Start: R columns of B (they lie mostly in the clutter subspace),
// orthonormalised; one FP32 subspace step on B_hi; then float-float subspace
// steps Y = B V with Cholesky-QR, U = Y L^-H.  Each step measures how far it
// moved the subspace, c_k = |U - V V^H U|_F = |(Y - V H) L^-H|_F with
// H = V^H Y (the Ritz matrix of V).  Subspace iteration contracts the error
// by rho = lambda_{R+1} / lambda_R per step; an upper bound is
// (tr B - sum of the Ritz values) / (smallest Ritz value), since the
// remaining trace bounds lambda_{R+1} and Ritz values never exceed the
// eigenvalues.  The error left after step k is then at most about
// c_k rho / (1 - rho), and the loop stops once that is below kSubTol.
// Returns false if it is not after kSubSteps steps (an ill-gapped cell:
// lambda_{R+1} close to lambda_R, e.g. clutter tones closer than a Doppler
// bin), whose subspace the caller recomputes with eig_block_rr.  lam = the
// Ritz values of the last step.  Loop exits are warp-uniform because several
// cells share a warp; `live` = this group's cell exists (dead groups compute
// on zeros).
template <int Q, int R>
__device__ bool eig_top_subspace(const float4* __restrict__ Bc, int jl, bool live,
                                 float2* __restrict__ Vs, float2 (&uh)[eig_rpl(Q)][R],
                                 float2 (&ul)[eig_rpl(Q)][R], float (&lam)[R]) {
  constexpr int RP = eig_rpl(Q), QL = Q / RP, G = eig_lanes(Q);
  // rows j[k] = jl + k QL of lane jl; lanes jl >= QL (q / RP not a power of
  // two) hold zeros and compute on row 0 without keeping the result
  bool row[RP];
  int j[RP];
#pragma unroll
  for (int k = 0; k < RP; ++k) {
    row[k] = jl < QL;
    j[k] = row[k] ? jl + k * QL : 0;
  }
  float2 v[RP][R], y[RP][R];
#pragma unroll
  for (int k = 0; k < RP; ++k)
#pragma unroll
    for (int m = 0; m < R; ++m) {
      const float4 b = b_at<Q>(Bc, j[k], ((2 * m + 1) * Q) / (2 * R));
      v[k][m] = row[k] ? make_float2(b.x, b.y) : make_float2(0.f, 0.f);
    }
  orthonormalise_g<G, RP, R>(v);
#pragma unroll
  for (int k = 0; k < RP; ++k)
    if (row[k]) {
#pragma unroll
      for (int m = 0; m < R; ++m) Vs[m * Q + j[k]] = v[k][m];
    }
  __syncwarp();
#pragma unroll
  for (int k = 0; k < RP; ++k) {
    b_times_v_fp32<Q, R>(Bc, j[k], Vs, y[k]);
    if (!row[k]) {
#pragma unroll
      for (int m = 0; m < R; ++m) y[k][m] = make_float2(0.f, 0.f);
    }
  }
  __syncwarp();
  // Gram-Schmidt keeps orthonormality to ~eps cond(B V), which the change
  // measure of the float-float step below relies on (a one-pass Cholesky-QR
  // of the unnormalised start would leave ~eps cond^2)
  orthonormalise_g<G, RP, R>(y);
  // tr B (for the bound on lambda_{R+1})
  float trl = 0.f;
#pragma unroll
  for (int k = 0; k < RP; ++k) trl += row[k] ? b_at<Q>(Bc, j[k], j[k]).x : 0.f;
  const float trB = grp_sum<G>(trl);
#pragma unroll
  for (int k = 0; k < RP; ++k)
#pragma unroll
    for (int m = 0; m < R; ++m) v[k][m] = y[k][m];

  cff U[RP][R];
  float2 H[R][R];
  bool converged = !live;
  for (int step = 0; step < kSubSteps; ++step) {
#pragma unroll
    for (int k = 0; k < RP; ++k)
      if (row[k]) {
#pragma unroll
        for (int m = 0; m < R; ++m) Vs[m * Q + j[k]] = v[k][m];
      }
    __syncwarp();
    cff Yf[RP][R];
#pragma unroll
    for (int k = 0; k < RP; ++k) {
      // packed pairs: (re, im) += (br, bi) xr and (x, y) += (br, bi) (xi, -xi),
      // then re = re1 + y, im = im1 + x (error-free merge)
      float2 s1[R], c1[R], s2[R], c2[R];
#pragma unroll
      for (int m = 0; m < R; ++m) s1[m] = c1[m] = s2[m] = c2[m] = make_float2(0.f, 0.f);
      const int jj = j[k];
#pragma unroll 2
      for (int t = 0; t < Q; ++t) {
        const int l = (jj + t < Q) ? jj + t : jj + t - Q;
        const float4 b = b_at<Q>(Bc, jj, l);
        const float2 xh = make_float2(b.x, b.y), xl = make_float2(b.z, b.w);
        const float2 nxh = f2_mul(xh, make_float2(-1.f, -1.f));
#pragma unroll
        for (int m = 0; m < R; ++m) {
          const float2 x = Vs[m * Q + l];
          acc_ffxf2(s1[m], c1[m], xh, nxh, xl, make_float2(x.x, x.x));
          acc_ffxf2(s2[m], c2[m], xh, nxh, xl, make_float2(x.y, -x.y));
        }
      }
#pragma unroll
      for (int m = 0; m < R; ++m) {
        float sr, er, si, ei;
        two_sum(s1[m].x, s2[m].y, sr, er);
        two_sum(s1[m].y, s2[m].x, si, ei);
        Yf[k][m] = row[k] ? cff{ff_make(sr, __fadd_rn(er, __fadd_rn(c1[m].x, c2[m].y))),
                                ff_make(si, __fadd_rn(ei, __fadd_rn(c1[m].y, c2[m].x)))}
                          : cff_zero();
      }
    }
    __syncwarp();
    // H = V^H Y (FP32), Gram G = Y^H Y (float-float)
#pragma unroll
    for (int m = 0; m < R; ++m)
#pragma unroll
      for (int mp = 0; mp < R; ++mp) {
        float2 d = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < RP; ++k)
          d = cadd(d, cmulc(v[k][m], make_float2(Yf[k][mp].re.hi, Yf[k][mp].im.hi)));
        H[m][mp] = grp_sum2<G>(d);
      }
    cff Gm[R][R];
#pragma unroll
    for (int m = 0; m < R; ++m)
#pragma unroll
      for (int mp = m; mp < R; ++mp) {
        cff pr = cff_cmul(Yf[0][m], Yf[0][mp]);
#pragma unroll
        for (int k = 1; k < RP; ++k) pr = cff_add(pr, cff_cmul(Yf[k][m], Yf[k][mp]));
        Gm[m][mp] = cff{grp_sum_ff<G>(pr.re), grp_sum_ff<G>(pr.im)};
      }
    // Cholesky G = L L^H
    cff L[R][R];
#pragma unroll
    for (int m = 0; m < R; ++m) {
      ff dsum = Gm[m][m].re;
#pragma unroll
      for (int k = 0; k < m; ++k)
        dsum = ff_sub(dsum, ff_add(ff_mul(L[m][k].re, L[m][k].re), ff_mul(L[m][k].im, L[m][k].im)));
      const ff lmm = ff_sqrt(dsum);
      L[m][m] = cff{lmm, {0.f, 0.f}};
#pragma unroll
      for (int i = m + 1; i < R; ++i) {
        cff t = cff{Gm[m][i].re, ff_neg(Gm[m][i].im)};
#pragma unroll
        for (int k = 0; k < m; ++k) t = cff_sub(t, cff_mul(L[i][k], cff{L[m][k].re, ff_neg(L[m][k].im)}));
        L[i][m] = (lmm.hi > 0.f) ? cff{ff_div(t.re, lmm), ff_div(t.im, lmm)} : cff_zero();
      }
    }
    // U = Y L^-H (rows j[k])
#pragma unroll
    for (int k = 0; k < RP; ++k)
#pragma unroll
      for (int m = 0; m < R; ++m) {
        cff t = Yf[k][m];
#pragma unroll
        for (int i = 0; i < m; ++i)
          t = cff_sub(t, cff_mul(U[k][i], cff{L[m][i].re, ff_neg(L[m][i].im)}));
        const ff lmm = L[m][m].re;
        U[k][m] = (lmm.hi > 0.f) ? cff{ff_div(t.re, lmm), ff_div(t.im, lmm)} : cff_zero();
      }
    // change of the subspace: (I - V V^H) U = (Y - V H) L^-H, rows j[k]
    // (FP32; the residual is formed directly, so small changes do not cancel)
    float local = 0.f;
#pragma unroll
    for (int k = 0; k < RP; ++k) {
      float2 X[R];
#pragma unroll
      for (int m = 0; m < R; ++m) {
        float2 t = make_float2(Yf[k][m].re.hi, Yf[k][m].im.hi);
#pragma unroll
        for (int mp = 0; mp < R; ++mp) t = csub(t, cmul(v[k][mp], H[mp][m]));
#pragma unroll
        for (int i = 0; i < m; ++i) t = csub(t, cmul(X[i], make_float2(L[m][i].re.hi, -L[m][i].im.hi)));
        const float lmm = L[m][m].re.hi;
        X[m] = (lmm > 0.f) ? cscale(t, 1.f / lmm) : make_float2(0.f, 0.f);
        local += cabs2(X[m]);
      }
    }
    const float change = grp_sum<G>(local);
#pragma unroll
    for (int k = 0; k < RP; ++k)
#pragma unroll
      for (int m = 0; m < R; ++m) v[k][m] = make_float2(U[k][m].re.hi, U[k][m].im.hi);
    ritz_values<R>(H, lam);
    float rs = 0.f;
#pragma unroll
    for (int m = 0; m < R; ++m) rs += lam[m];
    const float c = sqrtf(change);
    const float rho = (lam[R - 1] > 0.f) ? fminf(fmaxf(trB - rs, 0.f) / lam[R - 1], 0.99f)
                                         : (c > 0.f ? 0.99f : 0.f);
    converged = converged || c * rho < kSubTol * (1.f - rho);
    if (__all_sync(0xffffffffu, converged)) break;
  }
#pragma unroll
  for (int k = 0; k < RP; ++k)
#pragma unroll
    for (int m = 0; m < R; ++m) {
      uh[k][m] = make_float2(U[k][m].re.hi, U[k][m].im.hi);
      ul[k][m] = make_float2(U[k][m].re.lo, U[k][m].im.lo);
    }
  return converged;
}

// ------------------------------------------------ ill-gapped B -------------
// EIG_{r_b} (Sec. 4) of a cell whose eigenvalue lambda_{R+1} lies close to
// lambda_R, where subspace iteration on R vectors crawls: block subspace
// iteration with K = min(Q, max(8, R + 4)) vectors in float-float (kRrSteps steps; the
// error of the leading R directions contracts by lambda_{K+1} / lambda_R per
// step, and for Q <= 8 the block is the whole space), then Rayleigh-Ritz: the
// K x K matrix V^H B V, diagonalised by a single-precision Jacobi (warm
// start) and FP64 Jacobi sweeps on the rotated matrix, so that nearly equal
// Ritz values are separated at double precision.  One warp per cell, lane j
// < Q = row j.
constexpr int kRrMinK = 8;
constexpr int kRrSteps = 4;
__host__ __device__ constexpr int rr_k(int q, int r) {
  return q < (r + 4 > kRrMinK ? r + 4 : kRrMinK) ? q : (r + 4 > kRrMinK ? r + 4 : kRrMinK);
}
// shared memory of one warp: the bases V and Y = B V [K][Q] float-float
// complex (16 B), and four K x K matrices (FP64 H and Z1, FP32 H and Z0, 16 B
// slots)
__host__ __device__ constexpr int rr_bytes(int q, int r) {
  return 2 * rr_k(q, r) * q * 16 + 4 * rr_k(q, r) * rr_k(q, r) * 16;
}

template <typename T>
struct cpx {
  T re, im;
};
template <typename T>
__device__ __forceinline__ cpx<T> cpx_mul(cpx<T> a, cpx<T> b) {
  return cpx<T>{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename T>
__device__ __forceinline__ cpx<T> cpx_conj(cpx<T> a) { return cpx<T>{a.re, -a.im}; }

template <typename T>
__device__ __forceinline__ T warp_sum_t(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Cyclic Jacobi on a K x K Hermitian matrix A (shared memory, row-major, full
// storage) by one warp.  Every lane computes each rotation's parameters from
// the same 2 x 2 block, so all branches are uniform; lane k < K then rotates
// entries (k, p), (k, q) and mirrors them, and row k of Z.  On return
// A = Z^H A_in Z (Z = I at entry if init_z, else Z is right-multiplied).
// Stops when sum_{i<j} |A_ij|^2 <= tol2 sum_i A_ii^2, or after max_sweeps;
// an entry |A_pq| <= skip (|A_pp| + |A_qq|) is set to zero, not rotated.
template <typename T, int K>
__device__ void jacobi_warp(cpx<T>* A, cpx<T>* Z, int lane, T tol2, T skip, int max_sweeps,
                            bool init_z) {
  if (init_z) {
    for (int e = lane; e < K * K; e += 32) Z[e] = cpx<T>{(e / K == e % K) ? T(1) : T(0), T(0)};
  }
  __syncwarp();
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    T off = T(0), diag = T(0);
    for (int e = lane; e < K * K; e += 32) {
      const int r = e / K, c = e % K;
      if (r == c) diag += A[e].re * A[e].re;
      if (r < c) off += A[e].re * A[e].re + A[e].im * A[e].im;
    }
    off = warp_sum_t(off);
    diag = warp_sum_t(diag);
    if (off <= tol2 * diag) break;
    for (int p = 0; p < K - 1; ++p) {
      for (int q = p + 1; q < K; ++q) {
        const cpx<T> b = A[p * K + q];
        const T app = A[p * K + p].re, aqq = A[q * K + q].re;
        const T ab = hypot(b.re, b.im);
        __syncwarp();
        if (!(ab > skip * (fabs(app) + fabs(aqq)))) {
          if (lane == 0) A[p * K + q] = A[q * K + p] = cpx<T>{T(0), T(0)};
          __syncwarp();
          continue;
        }
        const cpx<T> ph = cpx<T>{b.re / ab, b.im / ab};
        const T tau = (aqq - app) / (T(2) * ab);
        const T t = copysign(T(1), tau) / (fabs(tau) + sqrt(T(1) + tau * tau));
        const T c = T(1) / sqrt(T(1) + t * t);
        const T s = t * c;
        const cpx<T> cph = cpx_conj(ph);
        if (lane < K) {
          const int k = lane;
          if (k != p && k != q) {
            const cpx<T> akp = A[k * K + p];
            const cpx<T> x = cpx_mul(cph, A[k * K + q]);
            const cpx<T> nkp{c * akp.re - s * x.re, c * akp.im - s * x.im};
            const cpx<T> nkq{s * akp.re + c * x.re, s * akp.im + c * x.im};
            A[k * K + p] = nkp;
            A[p * K + k] = cpx_conj(nkp);
            A[k * K + q] = nkq;
            A[q * K + k] = cpx_conj(nkq);
          }
          const cpx<T> up = Z[k * K + p];
          const cpx<T> x = cpx_mul(cph, Z[k * K + q]);
          Z[k * K + p] = cpx<T>{c * up.re - s * x.re, c * up.im - s * x.im};
          Z[k * K + q] = cpx<T>{s * up.re + c * x.re, s * up.im + c * x.im};
        }
        __syncwarp();
        if (lane == 0) {
          A[p * K + p] = cpx<T>{app - t * ab, T(0)};
          A[q * K + q] = cpx<T>{aqq + t * ab, T(0)};
          A[p * K + q] = A[q * K + p] = cpx<T>{T(0), T(0)};
        }
        __syncwarp();
      }
    }
  }
}

__device__ __forceinline__ cff cff_warp_sum(cff v) { return cff{ff_warp_sum(v.re), ff_warp_sum(v.im)}; }

// Modified Gram-Schmidt, applied twice, on the K float-float columns of
// X [K][Q] (shared memory; lane j < Q holds row j, other lanes contribute
// zeros to the warp sums).
template <int Q, int K>
__device__ void mgs2_ff(cff* __restrict__ X, int lane) {
  const bool row = lane < Q;
  for (int m = 0; m < K; ++m) {
    cff x = row ? X[m * Q + lane] : cff_zero();
    for (int pass = 0; pass < 2; ++pass) {
      for (int mp = 0; mp < m; ++mp) {
        const cff u = row ? X[mp * Q + lane] : cff_zero();
        const cff c = cff_warp_sum(cff_cmul(u, x));
        x = cff_sub(x, cff_mul(u, c));
      }
    }
    const ff n2 = ff_warp_sum(ff_add(ff_mul(x.re, x.re), ff_mul(x.im, x.im)));
    const ff nrm = ff_sqrt(n2);
    const ff inv = (nrm.hi > 0.f) ? ff_div(ff{1.f, 0.f}, nrm) : ff{0.f, 0.f};
    if (row) X[m * Q + lane] = cff_scale(x, inv);
    __syncwarp();
  }
}

// Y[:, m] = B X[:, m] for m < K, float-float (lane j < Q computes row j).
template <int Q, int K>
__device__ void b_times_block_ff(const float4* __restrict__ Bc, const cff* __restrict__ X,
                                 cff* __restrict__ Y, int lane) {
  if (lane < Q) {
    for (int m = 0; m < K; ++m) {
      cff s = cff_zero();
      for (int l = 0; l < Q; ++l) {
        const float4 b = b_at<Q>(Bc, lane, l);
        s = cff_add(s, cff_mul(cff{ff_make(b.x, b.z), ff_make(b.y, b.w)}, X[m * Q + l]));
      }
      Y[m * Q + lane] = s;
    }
  }
  __syncwarp();
}

// Noinline: its registers and spills stay out of the B pass's main path.
template <int Q, int R>
__device__ __noinline__ void eig_block_rr(const float4* __restrict__ Bc,
                                          unsigned char* __restrict__ scr, int lane,
                                          float2 (&uh)[R], float2 (&ul)[R], float (&lam)[R]) {
  constexpr int K = rr_k(Q, R);
  cff* Vs = reinterpret_cast<cff*>(scr);                                   // [K][Q]
  cff* Ys = Vs + K * Q;                                                    // [K][Q]
  cpx<double>* Hd = reinterpret_cast<cpx<double>*>(Ys + K * Q);            // [K][K]
  cpx<double>* Z1 = Hd + K * K;                                            // [K][K]
  cpx<float>* Hf = reinterpret_cast<cpx<float>*>(Z1 + K * K);              // [K][K]
  cpx<float>* Z0 = reinterpret_cast<cpx<float>*>(reinterpret_cast<cpx<double>*>(Hf) + K * K);
  const bool row = lane < Q;
  const int j = row ? lane : 0;
  if constexpr (K == Q) {
    // the block is the whole space: V = I, V^H B V = B
    for (int e = lane; e < K * K; e += 32) {
      const float4 b = b_at<Q>(Bc, e / K, e % K);
      Hd[e] = cpx<double>{(double)b.x + (double)b.z,
                          (e / K == e % K) ? 0.0 : (double)b.y + (double)b.w};
    }
  } else {
    // start: K columns of B spread over the window, orthonormalised
    if (row) {
      for (int m = 0; m < K; ++m) {
        const float4 b = b_at<Q>(Bc, j, (m * Q) / K);
        Vs[m * Q + j] = cff{ff_make(b.x, b.z), ff_make(b.y, b.w)};
      }
    }
    __syncwarp();
    mgs2_ff<Q, K>(Vs, lane);
    for (int step = 0; step < kRrSteps; ++step) {
      b_times_block_ff<Q, K>(Bc, Vs, Ys, lane);
      mgs2_ff<Q, K>(Ys, lane);
      cff* t = Vs;
      Vs = Ys;
      Ys = t;
    }
    b_times_block_ff<Q, K>(Bc, Vs, Ys, lane);   // Y = B V of the final basis
    // Ritz matrix H = V^H B V (float-float sums, stored as FP64)
    for (int m = 0; m < K; ++m)
      for (int n = m; n < K; ++n) {
        const cff vm = row ? Vs[m * Q + j] : cff_zero();
        const cff yn = row ? Ys[n * Q + j] : cff_zero();
        const cff h = cff_warp_sum(cff_cmul(vm, yn));
        if (lane == 0) {
          const double hr = (double)h.re.hi + (double)h.re.lo;
          const double hi = (double)h.im.hi + (double)h.im.lo;
          Hd[m * K + n] = cpx<double>{hr, m == n ? 0.0 : hi};
          if (n != m) Hd[n * K + m] = cpx<double>{hr, -hi};
        }
      }
  }
  __syncwarp();
  // single-precision warm start, then FP64 sweeps on Z0^H H Z0.  The
  // single-precision rotations are unitary only to ~1e-7, which would make
  // Z0^H H Z0 a congruence rather than a similarity (errors ~1e-7 lambda_1
  // in the Ritz vectors): Z0 is re-orthonormalised in FP64 first (Zd, in
  // the then dead FP32 H's slots).
  for (int e = lane; e < K * K; e += 32)
    Hf[e] = cpx<float>{(float)Hd[e].re, (float)Hd[e].im};
  __syncwarp();
  jacobi_warp<float, K>(Hf, Z0, lane, 1e-12f, 1e-9f, 10, true);
  cpx<double>* Zd = reinterpret_cast<cpx<double>*>(Hf);   // [K][K], FP64 unitary warm start
  {
    // lane k < K holds row k; modified Gram-Schmidt twice over the columns
    const bool zr = lane < K;
    cpx<double> z[K];
#pragma unroll
    for (int m = 0; m < K; ++m)
      z[m] = zr ? cpx<double>{(double)Z0[lane * K + m].re, (double)Z0[lane * K + m].im}
                : cpx<double>{0.0, 0.0};
#pragma unroll
    for (int m = 0; m < K; ++m) {
#pragma unroll
      for (int pass = 0; pass < 2; ++pass) {
#pragma unroll
        for (int mp = 0; mp < m; ++mp) {
          // c = z_mp^H z_m
          const double cr = warp_sum_t(z[mp].re * z[m].re + z[mp].im * z[m].im);
          const double ci = warp_sum_t(z[mp].re * z[m].im - z[mp].im * z[m].re);
          z[m].re -= z[mp].re * cr - z[mp].im * ci;
          z[m].im -= z[mp].re * ci + z[mp].im * cr;
        }
      }
      const double n2 = warp_sum_t(z[m].re * z[m].re + z[m].im * z[m].im);
      const double inv = n2 > 0.0 ? 1.0 / sqrt(n2) : 0.0;
      z[m].re *= inv;
      z[m].im *= inv;
    }
    __syncwarp();
    if (zr) {
#pragma unroll
      for (int m = 0; m < K; ++m) Zd[lane * K + m] = z[m];
    }
  }
  __syncwarp();
  // Z1 <- H Zd, then Hd <- Zd^H Z1 (FP64)
  for (int e = lane; e < K * K; e += 32) {
    const int r = e / K, c = e % K;
    cpx<double> s{0.0, 0.0};
    for (int m = 0; m < K; ++m) {
      const cpx<double> t = cpx_mul(Hd[r * K + m], Zd[m * K + c]);
      s.re += t.re;
      s.im += t.im;
    }
    Z1[e] = s;
  }
  __syncwarp();
  for (int e = lane; e < K * K; e += 32) {
    const int r = e / K, c = e % K;
    cpx<double> s{0.0, 0.0};
    for (int m = 0; m < K; ++m) {
      const cpx<double> t = cpx_mul(cpx_conj(Zd[m * K + r]), Z1[m * K + c]);
      s.re += t.re;
      s.im += t.im;
    }
    s.im = (r == c) ? 0.0 : s.im;
    Hd[e] = s;   // no lane reads Hd in this loop
  }
  __syncwarp();
  // Hermitise (the two triangles of Z0^H H Z0 differ by rounding)
  for (int e = lane; e < K * K; e += 32) {
    const int r = e / K, c = e % K;
    if (r < c) {
      const cpx<double> a = Hd[r * K + c], b = Hd[c * K + r];
      const cpx<double> h{0.5 * (a.re + b.re), 0.5 * (a.im - b.im)};
      Hd[r * K + c] = h;
      Hd[c * K + r] = cpx_conj(h);
    }
  }
  __syncwarp();
  jacobi_warp<double, K>(Hd, Z1, lane, 1e-30, 1e-20, 6, true);
  // leading R Ritz values (every lane ranks the same diagonal)
  int sel[R];
  {
    double d[K];
#pragma unroll
    for (int m = 0; m < K; ++m) d[m] = Hd[m * K + m].re;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      int best = 0;
      double bv = -1e300;
#pragma unroll
      for (int m = 0; m < K; ++m) {
        bool taken = false;
#pragma unroll
        for (int rr = 0; rr < r; ++rr) taken |= (sel[rr] == m);
        if (!taken && d[m] > bv) {
          bv = d[m];
          best = m;
        }
      }
      sel[r] = best;
      lam[r] = (float)bv;
    }
  }
  // U[:, r] = V Zd Z1[:, sel[r]]: w = Zd Z1[:, sel r] (K, FP64), then row j of V w
#pragma unroll
  for (int r = 0; r < R; ++r) {
    double ur = 0.0, ui = 0.0;
#pragma unroll
    for (int m = 0; m < K; ++m) {
      cpx<double> w{0.0, 0.0};
      for (int n = 0; n < K; ++n) {
        const cpx<double> t = cpx_mul(Zd[m * K + n], Z1[n * K + sel[r]]);
        w.re += t.re;
        w.im += t.im;
      }
      double vr, vi;
      if constexpr (K == Q) {
        vr = (m == j) ? 1.0 : 0.0;
        vi = 0.0;
      } else {
        const cff v = Vs[m * Q + j];
        vr = (double)v.re.hi + (double)v.re.lo;
        vi = (double)v.im.hi + (double)v.im.lo;
      }
      ur += vr * w.re - vi * w.im;
      ui += vr * w.im + vi * w.re;
    }
    const float hr = (float)ur, hi = (float)ui;
    uh[r] = make_float2(hr, hi);
    ul[r] = make_float2((float)(ur - (double)hr), (float)(ui - (double)hi));
  }
}

// Threads of a B-pass CTA: 512 at q = 32, where the tile's B matrices fill
// most of shared memory and one CTA per SM must bring its own 16 warps.
__host__ __device__ constexpr int bfit_threads(int q) { return q >= 32 ? 512 : kThreads; }


constexpr int kLagStages = 4;   // lag-store prefetch depth of the B pass



// Shared memory of the B pass after the tile's B and a: the lag buffers
// (and, when the lags are recomputed, the box-sum buffers and the
// fixed-point tile), reused by the eigen phase's bases and then by the block
// Rayleigh-Ritz scratch of ill-gapped cells (at least one warp's worth).
// Host and device size it with the same functions.
__host__ __device__ constexpr int bfit_lag_bytes(int P, int Q, int TC, int Ra, bool from_store) {
  return (from_store ? kLagStages : 1) * P * P * (TC + Q - 1) * 16 +
         (from_store ? 0 : 2 * P * P * (TC + 2 * Ra + Q - 1) * 16);
}
__host__ __device__ constexpr int bfit_basis_bytes(int Q, int R) {
  return (bfit_threads(Q) / 32) * (32 / eig_lanes(Q)) * Q * R * 8;
}
__host__ __device__ constexpr int imax3(int a, int b, int c) {
  return a > b ? (a > c ? a : c) : (b > c ? b : c);
}
// The region from the lag buffers' start: lags or bases or fallback scratch,
// then (recompute variant only) the fixed-point tile, which is dead by the
// eigen phase and counts toward the fallback scratch.
__host__ __device__ constexpr int bfit_region_bytes(int P, int Q, int R, int TC, int Ra, int Rr,
                                                     bool from_store) {
  return imax3(bfit_lag_bytes(P, Q, TC, Ra, from_store), bfit_basis_bytes(Q, R), rr_bytes(Q, R)) +
         (from_store ? 0 : P * (2 * Rr + 1) * (TC + 2 * Ra + Q - 1) * 8);
}

// 16-byte asynchronous global -> shared copy; valid == false zero-fills the
// destination (src is then not read but must still be a mapped address).
__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src),
               "r"(valid ? 16 : 0)
               : "memory");
}
// 8-byte asynchronous global -> shared copy (one complex64 sample).
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// One B entry, float-float: sum_J conj(a_J) L_J with a single precision and L
// float-float (re_hi, im_hi, re_lo, im_lo), on packed pairs: (re, im) +=
// (Lr, Li) ar and (x, y) += (Lr, Li) (-ai, ai) run as two compensated pair
// sums (two independent dependency chains), merged at the end with an
// error-free two_sum: re = re1 + y, im = im1 + x.  ya = (ar, ar, -ai, ai).
struct BAcc {
  float2 s1 = {0.f, 0.f}, c1 = {0.f, 0.f}, s2 = {0.f, 0.f}, c2 = {0.f, 0.f};
  __device__ __forceinline__ void add(float4 ya, float4 L) {
    const float2 xh = make_float2(L.x, L.y), xl = make_float2(L.z, L.w);
    const float2 nxh = f2_mul(xh, make_float2(-1.f, -1.f));
    acc_ffxf2(s1, c1, xh, nxh, xl, make_float2(ya.x, ya.y));
    acc_ffxf2(s2, c2, xh, nxh, xl, make_float2(ya.z, ya.w));
  }
  // a term with a real coefficient ar: only the (re, im) += L ar chain (the
  // diagonal J = i + P i of the Hermitian a, stored with a zero imaginary
  // part, and a pair's S plane)
  __device__ __forceinline__ void add_real(float4 ya, float4 L) {
    const float2 xh = make_float2(L.x, L.y), xl = make_float2(L.z, L.w);
    const float2 nxh = f2_mul(xh, make_float2(-1.f, -1.f));
    acc_ffxf2(s1, c1, xh, nxh, xl, make_float2(ya.x, ya.y));
  }
  // -i ai L (a pair's D plane, ya of the pair's upper a): only the second
  // chain, (x, y) += (Lr, Li) (-ai, ai)
  __device__ __forceinline__ void add_imag(float4 ya, float4 L) {
    const float2 xh = make_float2(L.x, L.y), xl = make_float2(L.z, L.w);
    const float2 nxh = f2_mul(xh, make_float2(-1.f, -1.f));
    acc_ffxf2(s2, c2, xh, nxh, xl, make_float2(ya.z, ya.w));
  }
  // (re_hi, im_hi, re_lo, im_lo), the layout of the tile's B entries
  __device__ __forceinline__ float4 get() const {
    float s, e;
    two_sum(s1.x, s2.y, s, e);
    const ff re = ff_make(s, __fadd_rn(e, __fadd_rn(c1.x, c2.y)));
    two_sum(s1.y, s2.x, s, e);
    const ff im = ff_make(s, __fadd_rn(e, __fadd_rn(c1.y, c2.x)));
    return make_float4(re.hi, im.hi, re.lo, im.lo);
  }
};

// CTA = one row of tc cells.  B phase: for each lag, the tile's lag sums
// (read from the lag store with a double-buffered cp.async prefetch of the
// next lag, or recomputed from Y) are contracted with each cell's a into the
// diagonal of B, two entries per thread at a time (independent float-float
// chains).  Eigen phase: one group of Q lanes per cell.
template <int P, int Q, int R, bool FROM_STORE>
__global__ void __launch_bounds__(bfit_threads(Q), 65536 / 128 / bfit_threads(Q))
k_bfit(Geom g0, JobList JL, const float2* __restrict__ aw, const float4* __restrict__ Lw0) {
  constexpr int PP = P * P;
  constexpr int NB = Q * (Q + 1) / 2;
  constexpr bool kPairs = P <= 3;    // the single-pass lag planes hold pair sums / differences
  constexpr int GL = eig_lanes(Q);   // lanes per cell in the eigen phase
  constexpr int RP = eig_rpl(Q);     // rows per lane in the eigen phase
  constexpr int CPW = 32 / GL;       // cells per warp in the eigen phase
  constexpr int NT = bfit_threads(Q);
  extern __shared__ __align__(16) unsigned char smem[];
  for (int tile = blockIdx.x; tile < JL.ntiles[kKindBfit]; tile += gridDim.x) {
  int lt;
  const Job& JB = job_of(JL, kKindBfit, tile, lt);
  const Geom g = with_job(g0, JB);
  const float2* __restrict__ Y = JB.Y;
  const unsigned* __restrict__ maxbits = JB.maxbits;
  const float4* __restrict__ Lw = Lw0 ? Lw0 + JB.lag0 : nullptr;
  float2* __restrict__ UBh = JB.UBh;
  float2* __restrict__ UBl = JB.UBl;
  float* __restrict__ lamB = JB.lamB;
  const int TC = g.tc;
  const int ntx = (g.W + TC - 1) / TC;
  const int r = lt / ntx;
  const int c0 = (lt % ntx) * TC;
  const int WT = TC + 2 * g.Ra + Q - 1;
  const int NUmax = TC + Q - 1;
  const size_t ncell = (size_t)JL.NC;
  float4* Bs = reinterpret_cast<float4*>(smem);                 // [TC][NB]
  float4* as = Bs + TC * NB;                                    // [TC][PP] (ar, ar, -ai, ai)
  float4* lag = as + TC * PP;                                   // [kLagStages or 1][PP][NUmax]
  float2* Vs = reinterpret_cast<float2*>(lag);                  // eigen phase: [warps * CPW][Q][R]
  longlong2* Vo = reinterpret_cast<longlong2*>(lag + PP * NUmax);   // recompute only
  longlong2* Vg = Vo + PP * WT;
  int2* Yq = reinterpret_cast<int2*>(Vg + PP * WT);

  const int sh = frame_shift(*maxbits, g.B);
  const float scale = ldexpf(1.f, sh);
  const int WL = g.W + Q - 1;
  // prefetch of lag lg into buffer buf: rows J of the store are contiguous
  // in u, positions past the row end are zero-filled
  auto prefetch = [&](int lg, int buf) {
    const int NU = TC + Q - 1 - lg;
    const float4* src = Lw + ((size_t)r * Q + lg) * PP * WL;
    float4* dst = lag + buf * PP * NUmax;
    for (int idx = threadIdx.x; idx < PP * NU; idx += NT) {
      const int u = idx % NU, J = idx / NU;
      const bool ok = c0 + u < WL;
      cp_async16(dst + J * NUmax + u, ok ? src + (size_t)J * WL + c0 + u : src, ok);
    }
    cp_async_commit();
  };
  // lag of load position pos in the B-phase order 0, 1, Q-1, 2, Q-2, ..,
  // Q/2: lags g and Q - g are contracted together, TC * Q entries per pair
  auto lag_at = [](int pos) { return pos == 0 ? 0 : pos == Q - 1 ? Q / 2 : (pos & 1) ? (pos + 1) / 2 : Q - pos / 2; };
  int issued = 0;
  if (FROM_STORE) {
    for (; issued < kLagStages && issued < Q; ++issued) prefetch(lag_at(issued), issued);
  } else {
    load_tile_q<P>(Y, g, r, c0, WT, scale, Yq);
  }
  for (int idx = threadIdx.x; idx < TC * PP; idx += NT) {
    const int cl = idx / PP, J = idx % PP;
    const int c = c0 + cl;
    const float2 a = (c < g.W) ? aw[J * ncell + (size_t)JB.cell0 + (size_t)r * g.W + c]
                               : make_float2(0.f, 0.f);
    as[idx] = make_float4(a.x, a.x, -a.y, a.y);
  }
  __syncthreads();

  // B(j, j + lag) = sum_J conj(a_J) l_lag(c + j)[J], float-float, for entry
  // e = cl * (Q - lag) + j of one lag.  Positions the prefetch zero-filled
  // are read only by cells past the frame edge.
  auto b_entry = [&](int lagg, const float4* lb, int e) {
    const int nj = Q - lagg;
    const int cl = e / nj, j = e - cl * nj;
    BAcc b;
#pragma unroll
    for (int J = 0; J < PP; ++J) {
      // the flip-flop stores a exactly Hermitian with a real diagonal, so the
      // diagonal terms' imaginary chain would add exact zeros.  Single pass:
      // the off-diagonal planes hold a pair's S (at i + P k, i < k) and D (at
      // k + P i), taken with Re(a_{i + P k}) and -i Im(a_{i + P k})
      // (plane_group); stacked passes: every plane is L_J itself
      const int i = J % P, k = J / P;
      if (J % (P + 1) == 0 || (kPairs && i < k))
        b.add_real(as[cl * PP + J], lb[J * NUmax + cl + j]);
      else if (kPairs)
        b.add_imag(as[cl * PP + k + P * i], lb[J * NUmax + cl + j]);
      else
        b.add(as[cl * PP + J], lb[J * NUmax + cl + j]);
    }
    Bs[cl * NB + diag_off<Q>(lagg) + j] = b.get();
  };
  if (FROM_STORE) {
    // Q / 2 + 1 steps: {0}, {1, Q-1}, .., {Q/2-1, Q/2+1}, {Q/2}.  A pair has
    // TC * Q entries (whole rounds of the CTA where a lag alone leaves most
    // threads idle at the long lags).  Load positions [p0, p1) of a step sit
    // in buffers pos % kLagStages; after the step they are refilled with the
    // next positions, so at most kLagStages - (p1 - p0) groups are in flight.
    for (int step = 0; step <= Q / 2; ++step) {
      const int p0 = (step == 0) ? 0 : 2 * step - 1;
      const int p1 = (step == 0) ? 1 : (step == Q / 2) ? Q : 2 * step + 1;
      const int ahead = issued - p1;   // groups allowed to stay outstanding, 0 .. 3
      if (ahead >= 3)
        cp_async_wait<3>();
      else if (ahead == 2)
        cp_async_wait<2>();
      else if (ahead == 1)
        cp_async_wait<1>();
      else
        cp_async_wait<0>();
      __syncthreads();
      const int la = lag_at(p0), lb_ = lag_at(p1 - 1);
      const int na = TC * (Q - la);
      const int tot = (p1 - p0 == 2) ? na + TC * (Q - lb_) : na;
      float4* bufa = lag + (p0 % kLagStages) * PP * NUmax;
      float4* bufb = lag + ((p1 - 1) % kLagStages) * PP * NUmax;
      if constexpr (kPairs) {
        // each pair's planes -> S, D (float-float sums of the stored sums;
        // their rounding, 2^-48 of the terms, is that of the stored sums)
        constexpr int NPR = P * (P - 1) / 2;
        const int nua = TC + Q - 1 - la, nub = TC + Q - 1 - lb_;
        const int nitem = NPR * (nua + ((p1 - p0 == 2) ? nub : 0));
        for (int idx = threadIdx.x; idx < nitem; idx += NT) {
          const bool first = idx < NPR * nua;
          const int r2 = first ? idx : idx - NPR * nua;
          const int nu = first ? nua : nub;
          const int pr = r2 / nu, u = r2 - pr * nu;
          int J1, J2;
          plane_group<P>(P + pr, J1, J2);
          float4* bf = first ? bufa : bufb;
          const float4 x = bf[J1 * NUmax + u], y = bf[J2 * NUmax + u];
          const ff sr = ff_add(ff{x.x, x.z}, ff{y.x, y.z}), si = ff_add(ff{x.y, x.w}, ff{y.y, y.w});
          const ff dr = ff_sub(ff{x.x, x.z}, ff{y.x, y.z}), di = ff_sub(ff{x.y, x.w}, ff{y.y, y.w});
          bf[J1 * NUmax + u] = make_float4(sr.hi, si.hi, sr.lo, si.lo);
          bf[J2 * NUmax + u] = make_float4(dr.hi, di.hi, dr.lo, di.lo);
        }
        __syncthreads();
      }
      for (int idx = threadIdx.x; idx < tot; idx += NT) {
        const bool first = idx < na;
        b_entry(first ? la : lb_, first ? bufa : bufb, first ? idx : idx - na);
      }
      __syncthreads();
      for (; issued < Q && issued < p1 + kLagStages; ++issued)
        prefetch(lag_at(issued), issued % kLagStages);
    }
  } else {
    for (int lagg = 0; lagg < Q; ++lagg) {
      const int NU = TC + Q - 1 - lagg;
      const int KW = NU + 2 * g.Ra;
      vertical_sums<P>(Yq, g, WT, lagg, KW, Vo, Vg);
      __syncthreads();
      for (int idx = threadIdx.x; idx < PP * NU; idx += NT) {
        const int u = idx % NU, J = idx / NU;
        const longlong2 L = ring_sum(Vo + J * KW, Vg + J * KW, g, u);
        const int i = J % P, k = J / P;
        float4 v;
        ll_to_ff(L.x, v.x, v.z);
        ll_to_ff(L.y, v.y, v.w);
        if (kPairs && i != k) {
          // the pair's S (at i + P k, i < k) or D (at k + P i), formed from
          // the two planes' float-float values exactly as the lag-store
          // branch forms them from the stored planes (plane_group), so the
          // two branches stay bit-identical
          const int Jm = k + P * i;
          const longlong2 Lm = ring_sum(Vo + Jm * KW, Vg + Jm * KW, g, u);
          float4 w;
          ll_to_ff(Lm.x, w.x, w.z);
          ll_to_ff(Lm.y, w.y, w.w);
          const float4 x = (i < k) ? v : w, y = (i < k) ? w : v;   // planes j1, j2
          const ff re = (i < k) ? ff_add(ff{x.x, x.z}, ff{y.x, y.z}) : ff_sub(ff{x.x, x.z}, ff{y.x, y.z});
          const ff im = (i < k) ? ff_add(ff{x.y, x.w}, ff{y.y, y.w}) : ff_sub(ff{x.y, x.w}, ff{y.y, y.w});
          v = make_float4(re.hi, im.hi, re.lo, im.lo);
        }
        lag[J * NUmax + u] = v;
      }
      __syncthreads();
      for (int idx = threadIdx.x; idx < TC * (Q - lagg); idx += NT) b_entry(lagg, lag, idx);
      __syncthreads();
    }
  }

  // eigen phase: a group of GL lanes per cell; cells whose subspace
  // iteration does not converge (ill-gapped B) are queued for the block
  // Rayleigh-Ritz phase below
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int sub = lane / GL, j = lane % GL;
  const int slot = warp * CPW + sub;
  const int per_pass = (NT / 32) * CPW;
  // writes U_B (row j of cell cl) and, from lane j == 0, lambda_B
  auto store = [&](int cl, int jj, const float2 (&uh)[R], const float2 (&ul)[R],
                   const float (&lam)[R]) {
    const size_t cell = (size_t)r * g.W + (c0 + cl);   // this job's cell index
#pragma unroll
    for (int m = 0; m < R; ++m) {
      UBh[(cell * Q + jj) * R + m] = uh[m];
      UBl[(cell * Q + jj) * R + m] = ul[m];
    }
    if (jj == 0 && lamB) {
      // B^ = b / |a|^2 in S units, then tr A^ = p normalisation
      float an = 0.f, tr = 0.f;
      for (int J = 0; J < PP; ++J) an += cabs2(make_float2(as[cl * PP + J].x, as[cl * PP + J].w));
      for (int i = 0; i < P; ++i) tr += as[cl * PP + i * (P + 1)].x;
      const float unit = ldexpf(1.f, 60 - 2 * sh) / (float)g.n;
      const float f = (an > 0.f) ? unit / an * tr / (float)P : 0.f;
#pragma unroll
      for (int m = 0; m < R; ++m) lamB[cell * R + m] = lam[m] * f;
    }
  };
  __shared__ int fb_n;
  __shared__ int fb_cell[kTileCells];
  if (threadIdx.x == 0) fb_n = 0;
  __syncthreads();
  for (int base = 0; base < TC; base += per_pass) {
    const int cl = base + slot;
    const bool live = cl < TC && (c0 + cl) < g.W;
    const int clc = live ? cl : 0;
    float2 uh[RP][R], ul[RP][R];
    float lam[R];
    const bool conv =
        eig_top_subspace<Q, R>(Bs + clc * NB, j, live, Vs + slot * Q * R, uh, ul, lam);
    if (live && conv && j < Q / RP) {
#pragma unroll
      for (int k = 0; k < RP; ++k) store(cl, j + k * (Q / RP), uh[k], ul[k], lam);
    }
    if (live && !conv && j == 0) fb_cell[atomicAdd(&fb_n, 1)] = cl;
  }
  __syncthreads();
  const int nfb = fb_n;
  if (nfb > 0) {
    // one warp per queued cell, each with rr_bytes of the (now dead) lag and
    // basis scratch
    constexpr int RB = rr_bytes(Q, R);
    const int slots = min(NT / 32, bfit_region_bytes(P, Q, R, TC, g.Ra, g.Rr, FROM_STORE) / RB);
    if (warp < slots) {
      for (int e = warp; e < nfb; e += slots) {
        const int cl = fb_cell[e];
        float2 uh[R], ul[R];
        float lam[R];
        eig_block_rr<Q, R>(Bs + cl * NB, reinterpret_cast<unsigned char*>(lag) + warp * RB, lane,
                           uh, ul, lam);
        if (lane < Q) store(cl, lane, uh, ul, lam);
        __syncwarp();
      }
    }
    if (threadIdx.x == 0 && JL.report) atomicAdd(JL.report + 2, (unsigned long long)nfb);
  }
  __syncthreads();
  }  // tile loop
}


// ------------------------------------------------ projection helpers -------
// Splits of the j sum of a per-cell contraction over a group of G lanes with
// NI outputs: the largest power of two S with S NI <= G that divides q (so
// that S NI lanes work where NI would, the rest of the group idle).
__host__ __device__ constexpr int split_j(int q, int g, int ni) {
  int s = 1;
  while (2 * s * ni <= g && q % (2 * s) == 0) s *= 2;
  return s;
}

// C[i][m] = sum_j X[i][j] conj(U[j][m]) of one cell, float-float (U = hi +
// lo), into Cs[i R + m] as (re_hi, re_lo, im_hi, im_lo).  With S =
// split_j(Q, G, P R) > 1, lane gl of the group takes output gl % (P R) over
// the j range of split gl / (P R), and the S compensated partial sums are
// merged by shuffles.  Every lane of the warp calls it (the merge shuffles
// over the whole warp); live = this group's cell exists.
template <int P, int Q, int R, int G>
__device__ __forceinline__ void xconj_u_ff(const float2* __restrict__ Xs,
                                           const float2* __restrict__ Uh,
                                           const float2* __restrict__ Ul, float4* __restrict__ Cs,
                                           int gl, bool live) {
  constexpr int NI = P * R, S = split_j(Q, G, NI), QS = Q / S;
  auto partial = [&](int it, int j0, int j1, float& sr, float& cr, float& si, float& ci) {
    const int i = it / R, m = it % R;
#pragma unroll 4
    for (int j = j0; j < j1; ++j) {
      const float2 x = Xs[i * Q + j];
      const float2 uh = Uh[j * R + m], ul = Ul[j * R + m];
      acc_ffxf(sr, cr, uh.x, ul.x, x.x);    // re += ur xr + ui xi
      acc_ffxf(sr, cr, uh.y, ul.y, x.y);
      acc_ffxf(si, ci, uh.x, ul.x, x.y);    // im += ur xi - ui xr
      acc_ffxf(si, ci, uh.y, ul.y, -x.x);
    }
  };
  if constexpr (S == 1) {
    if (live) {
      for (int it = gl; it < NI; it += G) {
        float sr = 0.f, cr = 0.f, si = 0.f, ci = 0.f;
        partial(it, 0, Q, sr, cr, si, ci);
        const ff re = ff_make(sr, cr), im = ff_make(si, ci);
        Cs[it] = make_float4(re.hi, re.lo, im.hi, im.lo);
      }
    }
  } else {
    const int sp = gl / NI, it = gl - sp * NI;
    const bool act = live && sp < S;
    float sr = 0.f, cr = 0.f, si = 0.f, ci = 0.f;
    if (act) partial(it, sp * QS, sp * QS + QS, sr, cr, si, ci);
    // split sp receives split sp + h (lane + h NI, inside the group)
#pragma unroll
    for (int h = S / 2; h >= 1; h >>= 1) {
      const float a = __shfl_down_sync(0xffffffffu, sr, h * NI);
      const float b = __shfl_down_sync(0xffffffffu, cr, h * NI);
      const float c = __shfl_down_sync(0xffffffffu, si, h * NI);
      const float d = __shfl_down_sync(0xffffffffu, ci, h * NI);
      float t, e;
      two_sum(sr, a, t, e);
      sr = t;
      cr = __fadd_rn(cr, __fadd_rn(b, e));
      two_sum(si, c, t, e);
      si = t;
      ci = __fadd_rn(ci, __fadd_rn(d, e));
    }
    if (act && sp == 0) {
      const ff re = ff_make(sr, cr), im = ff_make(si, ci);
      Cs[it] = make_float4(re.hi, re.lo, im.hi, im.lo);
    }
  }
}

// ------------------------------------------------ K4: detect ---------------
// A group of Q lanes per cell (32/Q cells per warp).  Per cell:
//   C  = X conj(U_B)                 (P x R, float-float; one lane per (i, m))
//   Z1 = X - C U_B^T = X F_B^T       (float-float, rounded; lane j owns column j)
//   Z  = F_A Z1                      (FP32)
// Bank (lanes over v, 4 velocities per pass):
//   w_b = F_B b_v = b_v - U_B (U_B^H b_v),  w_a = F_A a_v     (FP32)
//   T_v = |w_a^H Z conj(w_b)|^2 / (|w_a|^2 |w_b|^2)
// which equals |d^H P x|^2 / (d^H P d) since P Z = Z.  Computing the
// numerator with the projected steering factors keeps it well conditioned
// when d_v lies close to the clutter subspace; with Z float-float accurate,
// the error of T_v is ~2 eps sqrt(q) / sqrt(d^H P d / |d|^2).
template <int P, int Q, int R, int RA = 1>
__global__ void __launch_bounds__(kThreads)
k_detect(Geom g0, JobList JL, const float2* __restrict__ bank_aT,
         const float2* __restrict__ bank_bT, const float* __restrict__ bank_n2) {
  constexpr int G = grp_lanes(Q);              // lanes per cell (lanes >= Q hold no column)
  constexpr int CPW = 32 / G;                  // cells per warp
  constexpr int CPB = (kThreads / 32) * CPW;   // cells per block
  constexpr int VB = R > 4 ? 2 : 4;            // velocities per lane per pass
  // float2 scratch per cell (even, so every cell's float4 blocks stay
  // 16-byte aligned)
  constexpr int CS = 2 * P * Q + 2 * Q * R + 2 * P + 4 * P * R;
  extern __shared__ __align__(16) unsigned char smem[];
  const int V = g0.V;
  float2* aT = reinterpret_cast<float2*>(smem);       // [P][V]
  float2* bT = aT + P * V;                             // [Q][V]
  float* na = reinterpret_cast<float*>(bT + Q * V);    // [V]
  float* nb = na + V;                                  // [V]
  float2* scr = reinterpret_cast<float2*>(na + 2 * V);
  // near-blind queue of each warp: per pair, G in (R entries) then y (P
  // entries) and |w_b|^2 out, and the packed (velocity, cell slot)
  constexpr int QS = (R > P + 1) ? R : P + 1;
  float2* qd_all = scr + CPB * CS;                                  // [warps][kBlindQ][QS]
  int* qi_all = reinterpret_cast<int*>(qd_all + (kThreads / 32) * kBlindQ * QS);
  // per-slot prefetch buffer of the next tile's inputs: X [P][Q], U_B hi and
  // lo [Q][R], U_A [P][RA] (2P slots)
  constexpr int PF = P * Q + 2 * Q * R + 2 * P;
  float2* pf_all = reinterpret_cast<float2*>(qi_all + (kThreads / 32) * kBlindQ);
  for (int i = threadIdx.x; i < P * V; i += blockDim.x) aT[i] = bank_aT[i];
  for (int i = threadIdx.x; i < Q * V; i += blockDim.x) bT[i] = bank_bT[i];
  for (int i = threadIdx.x; i < 2 * V; i += blockDim.x) na[i] = bank_n2[i];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int sub = lane / G, gl = lane % G;
  const int slot = warp * CPW + sub;
  float2* pf = pf_all + slot * PF;
  // the group of slot `slot` prefetches its cell of tile t (X, U_B hi / lo,
  // U_A) with 8-byte cp.async into its own buffer while the CTA works on the
  // previous tile; every lane copies exactly the elements it later reads
  // back, so a wait on its own copies and a warp barrier order the data
  auto prefetch = [&](int t) {
    if (t < JL.ntiles[kKindDetect]) {
      int ltn;
      const Job& JN = job_of(JL, kKindDetect, t, ltn);
      const size_t cn = (size_t)ltn * CPB + slot;
      if (cn < (size_t)JN.H * JN.W) {
        const int r = (int)(cn / JN.W), c = (int)(cn % JN.W);
        if (gl < Q) {
#pragma unroll
          for (int i = 0; i < P; ++i)
            cp_async8(pf + i * Q + gl, JN.Y + (size_t)i * JN.ch_stride +
                                           (size_t)(r + g0.Rr) * JN.W_in + (c + g0.Ra + gl));
#pragma unroll
          for (int m = 0; m < R; ++m) {
            cp_async8(pf + P * Q + gl * R + m, JN.UBh + (cn * Q + gl) * R + m);
            cp_async8(pf + P * Q + Q * R + gl * R + m, JN.UBl + (cn * Q + gl) * R + m);
          }
        }
        for (int e = gl; e < P * RA; e += G)
          cp_async8(pf + P * Q + 2 * Q * R + e, JN.UA + cn * P * RA + e);
      }
    }
    cp_async_commit();
  };
  prefetch(blockIdx.x);
  for (int tile = blockIdx.x; tile < JL.ntiles[kKindDetect]; tile += gridDim.x) {
  int lt;
  const Job& JB = job_of(JL, kKindDetect, tile, lt);
  const Geom g = with_job(g0, JB);
  const float2* __restrict__ Y = JB.Y;
  float* __restrict__ T_all = JB.T_all;
  const size_t cell = (size_t)lt * CPB + slot;
  const size_t ncell = (size_t)g.H * g.W;
  const bool live = cell < ncell;
  float2* Xs = scr + slot * CS;        // [P][Q]
  float2* Zs = Xs + P * Q;             // [P][Q]
  float2* Uh = Zs + P * Q;             // [Q][R]
  float2* Ul = Uh + Q * R;             // [Q][R]
  static_assert(RA >= 1 && RA <= 2, "the scratch holds U_A for r_a <= 2");
  float2* Ua = Ul + Q * R;             // [P][RA] (2P slots)
  float4* Cs = reinterpret_cast<float4*>(Ua + 2 * P);   // [P][R] float-float complex
  float4* Es = Cs + P * R;                               // [P][R] F_A C, float-float (classical)
  cp_async_wait<0>();
  if (live) {
    if (gl < Q) {
#pragma unroll
      for (int i = 0; i < P; ++i) Xs[i * Q + gl] = pf[i * Q + gl];
#pragma unroll
      for (int m = 0; m < R; ++m) {
        Uh[gl * R + m] = pf[P * Q + gl * R + m];
        Ul[gl * R + m] = pf[P * Q + Q * R + gl * R + m];
      }
    }
    for (int e = gl; e < P * RA; e += G) Ua[e] = pf[P * Q + 2 * Q * R + e];   // [i][m]
  }
  __syncwarp();
  prefetch(tile + gridDim.x);
  // C[i][m] = sum_j X[i][j] conj(U[j][m]), float-float
  xconj_u_ff<P, Q, R, G>(Xs, Uh, Ul, Cs, gl, live);
  __syncwarp();
  const bool classical = g.filter == 1;
  if (classical && live) {
    // classical projector (W = u_a (x) U_B): d^H (I - W W^H) x splits into
    // a^H Z1 conj(F_B b) + sum_m (a^H E[:, m]) conj(G_m), Z1 = X F_B^T,
    // E = F_A C, G = U_B^H b.  The first term is the Kron path's product; E
    // keeps clutter that a^H E can cancel, so E stays float-float here and
    // a^H E is accumulated in float-float per velocity
    for (int it = gl; it < P * R; it += G) {
      const int i = it / R, m = it % R;
      float sr = 0.f, cr = 0.f, si = 0.f, ci = 0.f;   // c_m = u_a^H C[:, m]
#pragma unroll
      for (int k2 = 0; k2 < P; ++k2) {
        const float4 C = Cs[k2 * R + m];
        const float2 u = Ua[k2];
        acc_ffxf(sr, cr, C.x, C.y, u.x);
        acc_ffxf(sr, cr, C.z, C.w, u.y);
        acc_ffxf(si, ci, C.z, C.w, u.x);
        acc_ffxf(si, ci, C.x, C.y, -u.y);
      }
      // c_m / |u_a|^2 (float-float): u_a is stored in single precision, so
      // |u_a|^2 differs from 1 by ~1e-7, which would leave that fraction of
      // u_a's clutter in E
      float ns = 0.f, nc = 0.f;
#pragma unroll
      for (int k2 = 0; k2 < P; ++k2) {
        acc_prod(ns, nc, Ua[k2].x, Ua[k2].x);
        acc_prod(ns, nc, Ua[k2].y, Ua[k2].y);
      }
      const ff nu2 = ff_make(ns, nc);
      const ff cre = ff_div(ff_make(sr, cr), nu2), cim = ff_div(ff_make(si, ci), nu2);
      const float4 C = Cs[i * R + m];
      const float2 u = Ua[i];
      float r1 = C.x, r2 = C.y, i1 = C.z, i2 = C.w;   // C[i][m] - u_a[i] c_m
      acc_ffxf(r1, r2, cre.hi, cre.lo, -u.x);
      acc_ffxf(r1, r2, cim.hi, cim.lo, u.y);
      acc_ffxf(i1, i2, cim.hi, cim.lo, -u.x);
      acc_ffxf(i1, i2, cre.hi, cre.lo, -u.y);
      const ff er = ff_make(r1, r2), ei = ff_make(i1, i2);
      Es[i * R + m] = make_float4(er.hi, er.lo, ei.hi, ei.lo);
    }
  }
  // Z1 = X - C U^T (float-float) then Z = F_A Z1 (Kron) or Z = Z1 (classical);
  // lane gl owns column j = gl
  if (live && gl < Q) {
    const int j = gl;
    float2 uh[R], ul[R];
#pragma unroll
    for (int m = 0; m < R; ++m) {
      uh[m] = Uh[j * R + m];
      ul[m] = Ul[j * R + m];
    }
    float2 z[P];
#pragma unroll
    for (int i = 0; i < P; ++i) {
      const float2 x = Xs[i * Q + j];
      float sr = x.x, cr = 0.f, si = x.y, ci = 0.f;
#pragma unroll
      for (int m = 0; m < R; ++m) {
        const float4 C = Cs[i * R + m];   // (re_hi, re_lo, im_hi, im_lo)
        // re -= Cr Ur - Ci Ui ; im -= Cr Ui + Ci Ur
        acc_ffxff(sr, cr, C.x, C.y, -uh[m].x, -ul[m].x);
        acc_ffxff(sr, cr, C.z, C.w, uh[m].y, ul[m].y);
        acc_ffxff(si, ci, C.x, C.y, -uh[m].y, -ul[m].y);
        acc_ffxff(si, ci, C.z, C.w, -uh[m].x, -ul[m].x);
      }
      z[i] = make_float2(__fadd_rn(sr, cr), __fadd_rn(si, ci));
    }
    float2 t[RA];   // U_A^H z: F_A z = z - U_A t (none for the classical filter)
#pragma unroll
    for (int m = 0; m < RA; ++m) {
      t[m] = make_float2(0.f, 0.f);
      if (!classical) {
#pragma unroll
        for (int i = 0; i < P; ++i) t[m] = cadd(t[m], cmulc(Ua[i * RA + m], z[i]));
      }
    }
#pragma unroll
    for (int i = 0; i < P; ++i) {
      float2 zi = z[i];
#pragma unroll
      for (int m = 0; m < RA; ++m) zi = csub(zi, cmul(Ua[i * RA + m], t[m]));
      Zs[i * Q + j] = zi;
    }
  }
  __syncwarp();
  float best = -1.f;
  int bestv = 0x7fffffff;
  float2* qd = qd_all + warp * kBlindQ * QS;
  int* qi = qi_all + warp * kBlindQ;
  {
    // every lane of the warp runs the bank loop (a dead cell's group computes
    // on its stale scratch and writes nothing), so the near-blind queue below
    // can use warp-wide votes and shuffles.
    // lane gl takes velocities base + k G + gl: the lanes of a group read
    // consecutive bank words, and each lane still visits its v in increasing
    // order (lowest v wins ties)
    for (int base = 0; base < V; base += G * VB) {
      float2 Gm[VB][R];
#pragma unroll
      for (int k = 0; k < VB; ++k)
#pragma unroll
        for (int m = 0; m < R; ++m) Gm[k][m] = make_float2(0.f, 0.f);
      // G = U_B^H b_v, on packed pairs: G += (br, bi) ur + (bi, br) (ui, -ui)
#pragma unroll 4
      for (int j = 0; j < Q; ++j) {
        float2 ur[R], ui[R];
#pragma unroll
        for (int m = 0; m < R; ++m) {
          const float2 u = Uh[j * R + m];
          ur[m] = make_float2(u.x, u.x);
          ui[m] = make_float2(u.y, -u.y);
        }
#pragma unroll
        for (int k = 0; k < VB; ++k) {
          if (base + k * G + gl < V) {
            const float2 b = bT[j * V + base + k * G + gl];
            const float2 bs = make_float2(b.y, b.x);
#pragma unroll
            for (int m = 0; m < R; ++m) Gm[k][m] = f2_fma(bs, ui[m], f2_fma(b, ur[m], Gm[k][m]));
          }
        }
      }
      // w_b = b - U G ; y_i = sum_j Z[i][j] conj(w_b[j]) ; dB = |w_b|^2
      float2 y[VB][P];
      float dB[VB];
#pragma unroll
      for (int k = 0; k < VB; ++k) {
        dB[k] = 0.f;
#pragma unroll
        for (int i = 0; i < P; ++i) y[k][i] = make_float2(0.f, 0.f);
      }
      // on packed pairs: w = b - U G as (br, bi) - G ur and (x, y) = G (-ui, ui),
      // w = (re + y, im + x); y_i += (zr, zi) wr + (zi, zr) (wi, -wi)
#pragma unroll 4
      for (int j = 0; j < Q; ++j) {
        float2 nur[R], nui[R], zz[P], zs[P];
#pragma unroll
        for (int m = 0; m < R; ++m) {
          const float2 u = Uh[j * R + m];
          nur[m] = make_float2(-u.x, -u.x);
          nui[m] = make_float2(-u.y, u.y);
        }
#pragma unroll
        for (int i = 0; i < P; ++i) {
          zz[i] = Zs[i * Q + j];
          zs[i] = make_float2(zz[i].y, zz[i].x);
        }
#pragma unroll
        for (int k = 0; k < VB; ++k) {
          if (base + k * G + gl < V) {
            float2 w1 = bT[j * V + base + k * G + gl], w2 = make_float2(0.f, 0.f);
#pragma unroll
            for (int m = 0; m < R; ++m) {
              w1 = f2_fma(Gm[k][m], nur[m], w1);
              w2 = f2_fma(Gm[k][m], nui[m], w2);
            }
            const float wr = w1.x + w2.y, wi = w1.y + w2.x;
            dB[k] += cabs2(make_float2(wr, wi));
            const float2 WR = make_float2(wr, wr), WI = make_float2(wi, -wi);
#pragma unroll
            for (int i = 0; i < P; ++i) y[k][i] = f2_fma(zs[i], WI, f2_fma(zz[i], WR, y[k][i]));
          }
        }
      }
      // Nearly blind velocities (|F_B b|^2 < 1e-3 |b|^2): redo w_b = b - U G with
      // the subtraction in float-float and the low part of U_B included.  Errors
      // of G itself lie in span(U_B), which Z annihilates, so G stays FP32.
      // The warp queues its (cell, velocity) pairs and refines each with a
      // group of G lanes (lane j owns w_b[j]) instead of one lane looping over
      // j while the others wait; pairs past the queue's capacity are refined
      // by their own lane.
      auto refine_serial = [&](int k) {
        const int v = base + k * G + gl;
        float dBn = 0.f;
#pragma unroll
        for (int i = 0; i < P; ++i) y[k][i] = make_float2(0.f, 0.f);
        for (int j = 0; j < Q; ++j) {
          const float2 b = bT[j * V + v];
          float sr = b.x, cr = 0.f, si = b.y, ci = 0.f;
#pragma unroll
          for (int m = 0; m < R; ++m) {
            const float2 u = Uh[j * R + m], ul = Ul[j * R + m], G_ = Gm[k][m];
            acc_prod(sr, cr, -u.x, G_.x);   // re -= ur Gr - ui Gi
            acc_prod(sr, cr, u.y, G_.y);
            acc_prod(si, ci, -u.x, G_.y);   // im -= ur Gi + ui Gr
            acc_prod(si, ci, -u.y, G_.x);
            cr = __fmaf_rn(-ul.x, G_.x, cr);
            cr = __fmaf_rn(ul.y, G_.y, cr);
            ci = __fmaf_rn(-ul.x, G_.y, ci);
            ci = __fmaf_rn(-ul.y, G_.x, ci);
          }
          const float2 w = make_float2(__fadd_rn(sr, cr), __fadd_rn(si, ci));
          dBn += cabs2(w);
#pragma unroll
          for (int i = 0; i < P; ++i) y[k][i] = cadd(y[k][i], cmul(Zs[i * Q + j], cconj(w)));
        }
        dB[k] = dBn;
      };
      int qpos[VB];
      int nq = 0;
#pragma unroll
      for (int k = 0; k < VB; ++k) {
        const int v = base + k * G + gl;
        const bool fl = live && v < V && dB[k] < kBlindRefine * nb[v];
        const unsigned bal = __ballot_sync(0xffffffffu, fl);
        qpos[k] = -1;
        if (fl) {
          const int pos = nq + __popc(bal & ((1u << lane) - 1u));
          if (pos < kBlindQ) {
            qpos[k] = pos;
            qi[pos] = v | (sub << 16);
#pragma unroll
            for (int m = 0; m < R; ++m) qd[pos * QS + m] = Gm[k][m];
          } else {
            qpos[k] = -2;
          }
        }
        nq += __popc(bal);
      }
      nq = min(nq, kBlindQ);
      __syncwarp();
      for (int i0 = 0; i0 < nq; i0 += CPW) {   // warp-uniform
        const int it = i0 + sub;
        const bool act = it < nq;
        float2 yv[P];
#pragma unroll
        for (int i = 0; i < P; ++i) yv[i] = make_float2(0.f, 0.f);
        float dBn = 0.f;
        if (act && gl < Q) {
          const int v = qi[it] & 0xffff, cs = qi[it] >> 16;
          const float2* sc = scr + (warp * CPW + cs) * CS;
          const float2* Zc = sc + P * Q;
          const float2* Uhc = sc + 2 * P * Q;
          const float2* Ulc = Uhc + Q * R;
          const int j = gl;
          const float2 b = bT[j * V + v];
          float sr = b.x, cr = 0.f, si = b.y, ci = 0.f;
#pragma unroll
          for (int m = 0; m < R; ++m) {
            const float2 u = Uhc[j * R + m], ul = Ulc[j * R + m], G_ = qd[it * QS + m];
            acc_prod(sr, cr, -u.x, G_.x);
            acc_prod(sr, cr, u.y, G_.y);
            acc_prod(si, ci, -u.x, G_.y);
            acc_prod(si, ci, -u.y, G_.x);
            cr = __fmaf_rn(-ul.x, G_.x, cr);
            cr = __fmaf_rn(ul.y, G_.y, cr);
            ci = __fmaf_rn(-ul.x, G_.y, ci);
            ci = __fmaf_rn(-ul.y, G_.x, ci);
          }
          const float2 w = make_float2(__fadd_rn(sr, cr), __fadd_rn(si, ci));
          dBn = cabs2(w);
#pragma unroll
          for (int i = 0; i < P; ++i) yv[i] = cmul(Zc[i * Q + j], cconj(w));
        }
        dBn = grp_sum<G>(dBn);
#pragma unroll
        for (int i = 0; i < P; ++i) yv[i] = grp_sum2<G>(yv[i]);
        if (act && gl == 0) {
#pragma unroll
          for (int i = 0; i < P; ++i) qd[it * QS + i] = yv[i];
          qd[it * QS + P] = make_float2(dBn, 0.f);
        }
      }
      __syncwarp();
#pragma unroll
      for (int k = 0; k < VB; ++k) {
        if (qpos[k] >= 0) {
#pragma unroll
          for (int i = 0; i < P; ++i) y[k][i] = qd[qpos[k] * QS + i];
          dB[k] = qd[qpos[k] * QS + P].x;
        } else if (qpos[k] == -2) {
          refine_serial(k);
        }
      }
      __syncwarp();

#pragma unroll
      for (int k = 0; k < VB; ++k) {
        if (base + k * G + gl >= V) break;
        const int v = base + k * G + gl;
        float2 t[RA];   // U_A^H a_v
#pragma unroll
        for (int m = 0; m < RA; ++m) {
          t[m] = make_float2(0.f, 0.f);
#pragma unroll
          for (int i = 0; i < P; ++i) t[m] = cadd(t[m], cmulc(Ua[i * RA + m], aT[i * V + v]));
        }
        float dA = 0.f;
        float2 num = make_float2(0.f, 0.f);
#pragma unroll
        for (int i = 0; i < P; ++i) {
          float2 wa = aT[i * V + v];
#pragma unroll
          for (int m = 0; m < RA; ++m) wa = csub(wa, cmul(Ua[i * RA + m], t[m]));
          dA += cabs2(wa);
          num = cadd(num, cmulc(classical ? aT[i * V + v] : wa, y[k][i]));
        }
        if (classical) {   // + sum_m (a^H E[:, m]) conj(G_m), a^H E in float-float
#pragma unroll
          for (int m = 0; m < R; ++m) {
            float sr = 0.f, cr = 0.f, si = 0.f, ci = 0.f;
#pragma unroll
            for (int i = 0; i < P; ++i) {
              const float4 E = Es[i * R + m];
              const float2 a = aT[i * V + v];
              acc_ffxf(sr, cr, E.x, E.y, a.x);     // conj(a) E
              acc_ffxf(sr, cr, E.z, E.w, a.y);
              acc_ffxf(si, ci, E.z, E.w, a.x);
              acc_ffxf(si, ci, E.x, E.y, -a.y);
            }
            num = cadd(num, cmul(make_float2(__fadd_rn(sr, cr), __fadd_rn(si, ci)),
                                 cconj(Gm[k][m])));
          }
        }
        // Kron: d^H P d = |F_A a|^2 |F_B b|^2.  Classical: |d|^2 - |W^H d|^2
        // = |a|^2 |F_B b|^2 + |F_A a|^2 (|b|^2 - |F_B b|^2), a sum of
        // non-negative terms (no cancellation)
        const float den = classical ? na[v] * dB[k] + dA * fmaxf(nb[v] - dB[k], 0.f) : dA * dB[k];
        const float T = (den < 1e-12f * na[v] * nb[v]) ? 0.f : cabs2(num) / den;
        if (T_all && live) T_all[cell * V + v] = T;
        if (T > best) {
          best = T;
          bestv = v;
        }
      }
    }
  }
  // group argmax, lowest v on ties
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) {
    const float ob = __shfl_xor_sync(0xffffffffu, best, o);
    const int ov = __shfl_xor_sync(0xffffffffu, bestv, o);
    if (ob > best || (ob == best && ov < bestv)) {
      best = ob;
      bestv = ov;
    }
  }
  // cells whose box holds a NaN / Inf sample: Tmax = NaN, vidx = -1, map = 0
  // (the frame flag is per job, so the branch is uniform over the warp)
  if (JB.maxbits && JB.maxbits[1]) {
    bool bad = live && box_nonfinite(Y, g, (int)(cell / g.W), (int)(cell % g.W), gl, G);
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) bad |= __shfl_xor_sync(0xffffffffu, bad, o);
    if (bad) {
      best = __int_as_float(0x7fc00000);
      bestv = -1;
      if (T_all)
        for (int v = gl; v < V; v += G) T_all[cell * V + v] = best;
    }
  }
  if (live && gl == 0) {
    JB.Tmax[cell] = best;
    JB.vidx[cell] = bestv;
    JB.map[cell] = (best > g.tau) ? 1 : 0;
  }
  __syncwarp();
  }  // tile loop
}

}  // namespace kstap
