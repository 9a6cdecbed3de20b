// Tensor-core route of the detection statistic (Eq. KronSTAP, velocity bank)
// on the 5th-generation tensor cores: tcgen05.mma with the accumulator in
// tensor memory (TMEM), operands in shared memory, FP16 (or BF16) hi/lo
// splitting with FP32 accumulation.
//
// Per cell the bank enters the statistic only through the contractions
//   Zb_i(v) = sum_j Z[i][j] conj(b_v[j])      i < p     (Z = F_A X F_B^T)
//   Gc_m(v) = sum_j U_B[j][m] conj(b_v[j])     m < r_b   (= conj(U_B^H b_v))
// which share the bank across cells: one GEMM
//   D[v][n] = sum_k Bank[v][k] Cells[n][k]
// with k over (Re, Im) x q, v over the bank (M = 128, zero-padded) and n over
// two real rows (Re, Im) per complex row of 16 cells (N = 256).  Each factor
// x is split x = hi + lo in 16-bit floats; three MMAs (hi hi, hi lo, lo hi)
// accumulate in FP32, dropping only lo lo (~2^-22 relative for FP16).
// The epilogue then forms, per (cell, v),
//   y = Zb - E conj(G),  E = Z conj(U_B)   (so y = Z conj(F_B b_v))
//   num = (F_A a_v)^H y,  dB = |b_v|^2 - |G|^2,  dA = |F_A a_v|^2
//   T_v = |num|^2 / (dA dB)
// Velocities with dB < kTcRefine |b_v|^2 (close to the clutter subspace,
// where the cancellation in dB costs accuracy) are queued and recomputed
// afterwards on the CUDA cores, one group of q lanes per (cell, v), with the
// float-float F_B of the single-precision path.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace kstap {

constexpr int kTcCells = 16;        // cells per tile
constexpr int kTcRowsPerCell = 16;  // operand rows per cell: 2 (p + r_b) <= 16 used
constexpr int kTcN = kTcCells * kTcRowsPerCell;   // 256 = MMA N
constexpr int kTcM = 128;           // bank rows (velocities), zero-padded = MMA M
constexpr float kTcRefine = 1e-2f;  // dB / |b|^2 below which v is recomputed
constexpr long long kTcWaitCycles = 1ll << 30;   // ~0.5 s at 2 GHz: bound of one completion wait

__host__ __device__ constexpr int tc_threads(int q) { return q >= 32 ? 512 : 256; }

// Contraction length of the bank GEMM: (Re, Im) x q real columns, padded
// with zero columns to whole MMA K steps of 16 (q = 12: 24 -> 32).
__host__ __device__ constexpr int tc_k2(int q) { return ((2 * q + 15) / 16) * 16; }

// K-major, no-swizzle core-matrix layout of a 16-bit operand with `rows`
// rows: a core matrix is 8 rows x 16 bytes (8 elements) stored contiguously.
// K advances in blocks of 16 elements (one MMA step); inside a block, row
// group g = row / 8 sits at g * 256 bytes (the stride-dimension offset) and
// its two 8-element halves of K 128 bytes apart (the leading-dimension
// offset).  Byte offset of element (row, k):
__host__ __device__ constexpr uint32_t tc_off(int row, int k, int rows) {
  return (uint32_t)((k >> 4) * rows * 32 + (row >> 3) * 256 + ((k >> 3) & 1) * 128 +
                    (row & 7) * 16 + (k & 7) * 2);
}

// Shared-memory matrix descriptor of one K block at byte address `addr`:
// start >> 4 (bits 0-13), leading-dimension offset 128 B (bits 16-29),
// stride-dimension offset 256 B (bits 32-45), fixed 0b001 (bits 46-48),
// base offset 0, relative offsets, no swizzle (bits 61-63 = 0).
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr) {
  uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)(128u >> 4) << 16;
  d |= (uint64_t)(256u >> 4) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor, kind::f16: D = FP32 (bits 4-5 = 1), A and B FP16 (0)
// or BF16 (1) in bits 7-9 / 10-12, both K-major, N >> 3 (bits 17-22),
// M >> 4 (bits 24-28).
__host__ __device__ constexpr uint32_t tc_idesc(bool bf16, int M, int N) {
  return (1u << 4) | ((bf16 ? 1u : 0u) << 7) | ((bf16 ? 1u : 0u) << 10) |
         ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

template <bool BF16>
__device__ __forceinline__ void split16(float x, uint16_t& hi, uint16_t& lo) {
  if (BF16) {
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    hi = __bfloat16_as_ushort(h);
    lo = __bfloat16_as_ushort(__float2bfloat16_rn(x - __bfloat162float(h)));
  } else {
    const __half h = __float2half_rn(x);
    hi = __half_as_ushort(h);
    lo = __half_as_ushort(__float2half_rn(x - __half2float(h)));
  }
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                       bool accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate ? 1 : 0));
}

// Polls the mbarrier for phase `parity` for at most kTcWaitCycles SM cycles.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  uint32_t done = 0;
  const long long t0 = clock64();
  while (!done && clock64() - t0 < kTcWaitCycles) {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
  }
  return done != 0;
}

__device__ __forceinline__ void tmem_ld16(uint32_t addr, float (&f)[16]) {
  uint32_t v[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15}, [%16];\n"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15])
      : "r"(addr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) f[i] = __uint_as_float(v[i]);
}

// Per-cell scratch of the projection phase, in float2: X, Z [p][q]; U_B hi,
// lo [q][r_b]; U_A [2p]; C [p][r_b] float4; E [p][r_b]; scale.  Even, so
// every cell's float4 block stays 16-byte aligned.
__host__ __device__ constexpr int tc_scratch(int P, int Q, int R) {
  return (2 * P * Q + 2 * Q * R + 2 * P + 3 * P * R + 2 + 1) & ~1;
}

// Dynamic shared memory of k_detect_tc (host and device agree on it).
__host__ __device__ constexpr size_t tc_smem_bytes(int P, int Q, int R) {
  return 2 * (size_t)kTcM * tc_k2(Q) * 2       // bank operand, hi and lo
         + 2 * (size_t)kTcN * tc_k2(Q) * 2     // cell operand, hi and lo
         + (size_t)kTcCells * tc_scratch(P, Q, R) * 8
         + (size_t)kTcCells * kTcM * 4         // T of the tile, for the argmax
         + (size_t)kTcCells * kTcM * 4;        // queue of (cell, v) to recompute
}

// Requested dynamic shared memory: at least 80 KB, so that at most two CTAs
// (2 x 256 TMEM columns = the SM's 512) are resident per SM.
__host__ __device__ constexpr size_t tc_smem_request(int P, int Q, int R) {
  return tc_smem_bytes(P, Q, R) > 81920 ? tc_smem_bytes(P, Q, R) : 81920;
}

// CTA = tc_threads(Q) threads; tiles of kTcCells cells over all jobs.
// bank_op: the bank operand image (hi block then lo block, tc_off layout),
// bank_inv = 1 / (power-of-two bank scale).  fault: a device word the host
// reads back; bit 0 = a completion wait gave up (the launch's results are
// not valid), bit 1 = the MMAs had still not completed when the CTA freed
// its tensor memory (the device's state is unknown).
template <int P, int Q, int R, bool BF16>
__global__ void __launch_bounds__(tc_threads(Q), tc_threads(Q) >= 512 ? 1 : 2)
k_detect_tc(Geom g0, JobList JL, const uint4* __restrict__ bank_op, float bank_inv,
            const float2* __restrict__ bank_aT, const float2* __restrict__ bank_bT,
            const float* __restrict__ bank_n2, unsigned* __restrict__ fault) {
  constexpr int NT = tc_threads(Q);
  constexpr int G = grp_lanes(Q);            // lanes per cell in the projection phase
  constexpr int K2 = tc_k2(Q);               // real contraction length (zero-padded)
  constexpr int ROWS = 2 * (P + R);          // operand rows used per cell
  static_assert(ROWS <= kTcRowsPerCell, "p + r_b > 8");
  constexpr int SCR = tc_scratch(P, Q, R);   // float2 per cell (even: float4 alignment)
  constexpr uint32_t kOpA = (uint32_t)kTcM * K2 * 2;   // bytes of one bank operand half
  constexpr uint32_t kOpB = (uint32_t)kTcN * K2 * 2;   // bytes of one cell operand half
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned char* sA = smem;                            // [hi | lo]
  unsigned char* sB = smem + 2 * kOpA;                 // [hi | lo]
  float2* scr = reinterpret_cast<float2*>(sB + 2 * kOpB);
  float* Tsm = reinterpret_cast<float*>(scr + kTcCells * SCR);
  uint32_t* rq = reinterpret_cast<uint32_t*>(Tsm + kTcCells * kTcM);   // (cell << 8) | v
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_slot;
  __shared__ uint32_t rq_n;

  const int V = g0.V;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // bank operand into shared memory; cell operand zeroed (padding rows stay 0)
  for (int i = tid; i < (int)(2 * kOpA / 16); i += NT)
    reinterpret_cast<uint4*>(sA)[i] = __ldg(bank_op + i);
  for (int i = tid; i < (int)(2 * kOpB / 16); i += NT)
    reinterpret_cast<uint4*>(sB)[i] = make_uint4(0u, 0u, 0u, 0u);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(kTcN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(&mbar)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tmem_slot;

  // epilogue identity: TMEM lane quarter (warp % 4) = velocities, the
  // NT / 128 warp sets share the cells of a tile
  const int v = 32 * (warp & 3) + lane;
  const int cset = warp >> 2, nsets = NT / 128;
  const bool vlive = v < V;
  float2 av[P];
  float na = 0.f, nb = 0.f;
#pragma unroll
  for (int i = 0; i < P; ++i) av[i] = vlive ? bank_aT[i * V + v] : make_float2(0.f, 0.f);
  if (vlive) {
    na = bank_n2[v];
    nb = bank_n2[V + v];
  }

  const int sub = lane / G, gl = lane % G;
  const int gslot = warp * (32 / G) + sub;   // cell slot of this lane group (projection phase)
  constexpr int GPP = (NT / 32) * (32 / G);  // cell groups per pass
  uint32_t phase = 0;
  bool abort = false;
  for (int tile = blockIdx.x; tile < JL.ntiles[kKindDetect] && !abort; tile += gridDim.x) {
    int lt;
    const Job& JB = job_of(JL, kKindDetect, tile, lt);
    const Geom g = with_job(g0, JB);
    const size_t ncell = (size_t)g.H * g.W;
    const size_t cbase = (size_t)lt * kTcCells;
    if (tid == 0) rq_n = 0;   // read after the barrier before the MMA

    // ---- projection: Z = F_A X F_B^T per cell (float-float F_B), E, scale,
    //      operand rows
    for (int c = gslot; c < kTcCells; c += GPP) {
      const size_t cell = cbase + c;
      const bool live = cell < ncell;
      float2* Xs = scr + c * SCR;          // [P][Q]
      float2* Zs = Xs + P * Q;             // [P][Q]
      float2* Uh = Zs + P * Q;             // [Q][R]
      float2* Ul = Uh + Q * R;             // [Q][R]
      float2* Ua = Ul + Q * R;             // [P] (+ pad)
      float4* Cs = reinterpret_cast<float4*>(Ua + 2 * P);   // [P][R]
      float2* Es = reinterpret_cast<float2*>(Cs + P * R);   // [P][R]
      float* scl = reinterpret_cast<float*>(Es + P * R);
      if (live) {
        const int r = (int)(cell / g.W), cc = (int)(cell % g.W);
        if (gl < Q) {
#pragma unroll
          for (int i = 0; i < P; ++i)
            Xs[i * Q + gl] = __ldg(JB.Y + (size_t)i * g.ch_stride + (size_t)(r + g.Rr) * g.W_in +
                                   (cc + g.Ra + gl));
#pragma unroll
          for (int m = 0; m < R; ++m) {
            Uh[gl * R + m] = JB.UBh[(cell * Q + gl) * R + m];
            Ul[gl * R + m] = JB.UBl[(cell * Q + gl) * R + m];
          }
        }
        if (gl < P) Ua[gl] = JB.UA[cell * P + gl];
      }
      __syncwarp();
      // C = X conj(U_B), float-float
      xconj_u_ff<P, Q, R, G>(Xs, Uh, Ul, Cs, gl, live);
      __syncwarp();
      float2 z[P];
      float zmax = 0.f;
      if (live && gl < Q) {
        const int j = gl;
        float2 uh[R], ul[R];
#pragma unroll
        for (int m = 0; m < R; ++m) {
          uh[m] = Uh[j * R + m];
          ul[m] = Ul[j * R + m];
        }
#pragma unroll
        for (int i = 0; i < P; ++i) {
          const float2 x = Xs[i * Q + j];
          float sr = x.x, cr = 0.f, si = x.y, ci = 0.f;
#pragma unroll
          for (int m = 0; m < R; ++m) {
            const float4 C = Cs[i * R + m];
            acc_ffxff(sr, cr, C.x, C.y, -uh[m].x, -ul[m].x);
            acc_ffxff(sr, cr, C.z, C.w, uh[m].y, ul[m].y);
            acc_ffxff(si, ci, C.x, C.y, -uh[m].y, -ul[m].y);
            acc_ffxff(si, ci, C.z, C.w, -uh[m].x, -ul[m].x);
          }
          z[i] = make_float2(__fadd_rn(sr, cr), __fadd_rn(si, ci));
        }
        float2 t = make_float2(0.f, 0.f);
#pragma unroll
        for (int i = 0; i < P; ++i) t = cadd(t, cmulc(Ua[i], z[i]));
#pragma unroll
        for (int i = 0; i < P; ++i) {
          z[i] = csub(z[i], cmul(Ua[i], t));
          Zs[i * Q + j] = z[i];
          zmax = fmaxf(zmax, fmaxf(fabsf(z[i].x), fabsf(z[i].y)));
        }
      }
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) zmax = fmaxf(zmax, __shfl_xor_sync(0xffffffffu, zmax, o));
      __syncwarp();
      // E = Z conj(U_hi): the part of Z left in span(conj U_B) by rounding;
      // the j sum split over the group's otherwise idle lanes as for C
      {
        constexpr int NI = P * R, S = split_j(Q, G, NI), QS = Q / S;
        const int sp = gl / NI, it = gl - sp * NI;
        const bool act = live && sp < S;
        float2 e = make_float2(0.f, 0.f);
        if (act) {
          const int i = it / R, m = it % R;
#pragma unroll 4
          for (int j = sp * QS; j < sp * QS + QS; ++j)
            e = cadd(e, cmul(Zs[i * Q + j], cconj(Uh[j * R + m])));
        }
#pragma unroll
        for (int h = S / 2; h >= 1; h >>= 1) {
          e.x += __shfl_down_sync(0xffffffffu, e.x, h * NI);
          e.y += __shfl_down_sync(0xffffffffu, e.y, h * NI);
        }
        if (act && sp == 0) Es[it] = e;
        if constexpr (S == 1) {
          // more outputs than lanes: the rest, one lane each
          if (live) {
            for (int it2 = gl + G; it2 < NI; it2 += G) {
              const int i = it2 / R, m = it2 % R;
              float2 e2 = make_float2(0.f, 0.f);
#pragma unroll 4
              for (int j = 0; j < Q; ++j) e2 = cadd(e2, cmul(Zs[i * Q + j], cconj(Uh[j * R + m])));
              Es[it2] = e2;
            }
          }
        }
      }
      // power-of-two scale putting max |Z| in [0.5, 1): FP16 range and
      // precision independent of the frame's amplitude
      const float sc = (zmax > 0.f && zmax <= kFltMax) ? ldexpf(1.f, -(ilogbf(zmax) + 1)) : 1.f;
      if (live && gl == 0) *scl = sc;
      if (live && gl < Q) {
        // complex row t: Z[t] * sc (t < P), U_hi[:, t - P] (t < P + R); real
        // rows n = 2t: (Re | Im), n = 2t + 1: (Im | -Re)
        const int j = gl;
#pragma unroll
        for (int t = 0; t < P + R; ++t) {
          const float2 x = (t < P) ? cscale(z[t], sc) : Uh[j * R + (t - P)];
          const int n = c * kTcRowsPerCell + 2 * t;
          uint16_t h, l;
          split16<BF16>(x.x, h, l);
          *reinterpret_cast<uint16_t*>(sB + tc_off(n, j, kTcN)) = h;
          *reinterpret_cast<uint16_t*>(sB + kOpB + tc_off(n, j, kTcN)) = l;
          *reinterpret_cast<uint16_t*>(sB + tc_off(n + 1, Q + j, kTcN)) = h ^ 0x8000u;   // -Re
          *reinterpret_cast<uint16_t*>(sB + kOpB + tc_off(n + 1, Q + j, kTcN)) = l ^ 0x8000u;
          split16<BF16>(x.y, h, l);
          *reinterpret_cast<uint16_t*>(sB + tc_off(n, Q + j, kTcN)) = h;
          *reinterpret_cast<uint16_t*>(sB + kOpB + tc_off(n, Q + j, kTcN)) = l;
          *reinterpret_cast<uint16_t*>(sB + tc_off(n + 1, j, kTcN)) = h;
          *reinterpret_cast<uint16_t*>(sB + kOpB + tc_off(n + 1, j, kTcN)) = l;
        }
      }
      __syncwarp();
    }

    // ---- GEMM on the tensor cores (one thread issues, all wait)
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const uint32_t idesc = tc_idesc(BF16, kTcM, kTcN);
      const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
#pragma unroll
      for (int kk = 0; kk < K2 / 16; ++kk) {
        const uint32_t ao = kk * kTcM * 32, bo = kk * kTcN * 32;
        tc_mma(tmem, tc_desc(a0 + ao), tc_desc(b0 + bo), idesc, kk > 0);              // hi hi
        tc_mma(tmem, tc_desc(a0 + ao), tc_desc(b0 + kOpB + bo), idesc, true);          // hi lo
        tc_mma(tmem, tc_desc(a0 + kOpA + ao), tc_desc(b0 + bo), idesc, true);          // lo hi
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
              smem_u32(&mbar))
          : "memory");
    }
    bool ok = mbar_wait(smem_u32(&mbar), phase);
    if (!ok) {
      atomicOr(fault, 1u);
      ok = mbar_wait(smem_u32(&mbar), phase);   // the MMAs may still complete
    }
    if (__syncthreads_or(!ok)) {
      // the tile is abandoned; the tensor memory is freed below, so the MMAs
      // get one last bounded wait first, and a commit that never arrives is
      // reported as an unknown device state
      if (!ok && !mbar_wait(smem_u32(&mbar), phase)) atomicOr(fault, 2u);
      abort = true;
      break;
    }
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");

    // ---- epilogue: thread = velocity v, cells of its set
    for (int c = cset; c < kTcCells; c += nsets) {
      const size_t cell = cbase + c;
      float f[16];
      tmem_ld16(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(c * kTcRowsPerCell), f);
      if (cell >= ncell || !vlive) continue;
      const float2* Zs = scr + c * SCR + P * Q;
      const float2* Uh = Zs + P * Q;
      const float2* Ul = Uh + Q * R;
      const float2* Ua = Ul + Q * R;
      const float2* Es = reinterpret_cast<const float2*>(reinterpret_cast<const float4*>(Ua + 2 * P) + P * R);
      const float sc = *reinterpret_cast<const float*>(Es + P * R);
      const float zs = bank_inv / sc;
      float2 Gc[R], y[P];
      float gg = 0.f;
#pragma unroll
      for (int m = 0; m < R; ++m) {
        Gc[m] = make_float2(f[2 * (P + m)] * bank_inv, f[2 * (P + m) + 1] * bank_inv);
        gg += cabs2(Gc[m]);
      }
#pragma unroll
      for (int i = 0; i < P; ++i) {
        float2 t = make_float2(f[2 * i] * zs, f[2 * i + 1] * zs);
#pragma unroll
        for (int m = 0; m < R; ++m) t = csub(t, cmul(Es[i * R + m], Gc[m]));
        y[i] = t;
      }
      const float dB = nb - gg;
      if (dB < kTcRefine * nb) {   // near-blind: recomputed below
        rq[atomicAdd(&rq_n, 1u)] = ((uint32_t)c << 8) | (uint32_t)v;
        continue;
      }
      float2 t = make_float2(0.f, 0.f);
#pragma unroll
      for (int i = 0; i < P; ++i) t = cadd(t, cmulc(Ua[i], av[i]));
      float dA = 0.f;
      float2 num = make_float2(0.f, 0.f);
#pragma unroll
      for (int i = 0; i < P; ++i) {
        const float2 wa = csub(av[i], cmul(Ua[i], t));
        dA += cabs2(wa);
        num = cadd(num, cmulc(wa, y[i]));
      }
      const float den = dA * dB;
      const float T = (den < 1e-12f * na * nb) ? 0.f : cabs2(num) / den;
      if (JB.T_all) JB.T_all[cell * V + v] = T;
      Tsm[c * kTcM + v] = T;
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();

    // ---- queued near-blind (cell, v): a group of Q lanes each, lane j = pulse j.
    //   G = U_hi^H b_v (FP32; its error lies in span(U_B), which Z annihilates),
    //   w_b = b_v - U_B G with the float-float U_B, y = Z conj(w_b), dB = |w_b|^2
    {
      const uint32_t nq = rq_n;
      // warp-uniform trip count (the group reductions shuffle over the whole
      // warp); groups past the end of the queue recompute entry 0 and discard it
      for (uint32_t e0 = (uint32_t)(gslot - sub); e0 < nq; e0 += GPP) {
        const uint32_t e = e0 + sub;
        const bool act = e < nq;
        const uint32_t ent = rq[act ? e : 0];
        const int c = (int)(ent >> 8), vq = (int)(ent & 255u);
        const size_t cell = cbase + c;
        const float2* Zs = scr + c * SCR + P * Q;
        const float2* Uh = Zs + P * Q;
        const float2* Ul = Uh + Q * R;
        const float2* Ua = Ul + Q * R;
        // lane gl = pulse j; lanes gl >= Q (no pulse) read row 0 and add zeros
        const bool prow = gl < Q;
        const int j = prow ? gl : 0;
        const float2 b = prow ? __ldg(bank_bT + j * V + vq) : make_float2(0.f, 0.f);
        float2 Gm[R];
#pragma unroll
        for (int m = 0; m < R; ++m) Gm[m] = grp_sum2<G>(cmulc(Uh[j * R + m], b));
        float sr = b.x, cr = 0.f, si = b.y, ci = 0.f;
#pragma unroll
        for (int m = 0; m < R; ++m) {
          const float2 u = Uh[j * R + m], ul = Ul[j * R + m];
          acc_prod(sr, cr, -u.x, Gm[m].x);   // re -= ur Gr - ui Gi
          acc_prod(sr, cr, u.y, Gm[m].y);
          acc_prod(si, ci, -u.x, Gm[m].y);   // im -= ur Gi + ui Gr
          acc_prod(si, ci, -u.y, Gm[m].x);
          cr = __fmaf_rn(-ul.x, Gm[m].x, cr);
          cr = __fmaf_rn(ul.y, Gm[m].y, cr);
          ci = __fmaf_rn(-ul.x, Gm[m].y, ci);
          ci = __fmaf_rn(-ul.y, Gm[m].x, ci);
        }
        const float2 w = prow ? make_float2(__fadd_rn(sr, cr), __fadd_rn(si, ci))
                              : make_float2(0.f, 0.f);
        const float dB = grp_sum<G>(cabs2(w));
        float2 y[P];
#pragma unroll
        for (int i = 0; i < P; ++i) y[i] = grp_sum2<G>(cmul(Zs[i * Q + j], cconj(w)));
        if (gl == 0 && act) {
          float2 a[P];
#pragma unroll
          for (int i = 0; i < P; ++i) a[i] = bank_aT[i * V + vq];
          const float nav = bank_n2[vq], nbv = bank_n2[V + vq];
          float2 t = make_float2(0.f, 0.f);
#pragma unroll
          for (int i = 0; i < P; ++i) t = cadd(t, cmulc(Ua[i], a[i]));
          float dA = 0.f;
          float2 num = make_float2(0.f, 0.f);
#pragma unroll
          for (int i = 0; i < P; ++i) {
            const float2 wa = csub(a[i], cmul(Ua[i], t));
            dA += cabs2(wa);
            num = cadd(num, cmulc(wa, y[i]));
          }
          const float den = dA * dB;
          const float T = (den < 1e-12f * nav * nbv) ? 0.f : cabs2(num) / den;
          if (JB.T_all) JB.T_all[cell * V + vq] = T;
          Tsm[c * kTcM + vq] = T;
        }
      }
    }
    __syncthreads();

    // ---- argmax over v (lowest v on ties), threshold, non-finite flags
    for (int c = warp; c < kTcCells; c += NT / 32) {
      const size_t cell = cbase + c;
      if (cell >= ncell) continue;
      float best = -1.f;
      int bestv = 0x7fffffff;
      for (int vv = lane; vv < V; vv += 32) {
        const float T = Tsm[c * kTcM + vv];
        if (T > best) {
          best = T;
          bestv = vv;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int ov = __shfl_xor_sync(0xffffffffu, bestv, o);
        if (ob > best || (ob == best && ov < bestv)) {
          best = ob;
          bestv = ov;
        }
      }
      if (JB.maxbits && JB.maxbits[1]) {
        bool bad = box_nonfinite(JB.Y, g, (int)(cell / g.W), (int)(cell % g.W), lane, 32);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) bad |= __shfl_xor_sync(0xffffffffu, bad, o);
        if (bad) {
          best = __int_as_float(0x7fc00000);
          bestv = -1;
          if (JB.T_all)
            for (int vv = lane; vv < V; vv += 32) JB.T_all[cell * V + vv] = best;
        }
      }
      if (lane == 0) {
        JB.Tmax[cell] = best;
        JB.vidx[cell] = bestv;
        JB.map[cell] = (best > g.tau) ? 1 : 0;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kTcN));
}

}  // namespace kstap
