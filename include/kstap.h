/*
 * kstap.h -- C ABI of libkstap, the B300 (sm_103a) Kronecker STAP hot path.
 *
 * Method: Greenewald, Zelnio and Hero, "Kronecker STAP and SAR GMTI".
 * For every test cell (pixel) of a p-channel SAR frame the library
 *   1. assembles the p x q space-time snapshot X (x = vec(X^T), Sec. 2) and
 *      the n training snapshots of the cells in a range x azimuth box around
 *      it minus a guard box, and forms their sample covariance S (Eq. SCM);
 *   2. fits S ~ A (x) B with rank(A) <= r_a, rank(B) <= r_b by LR-Kron
 *      (Alg. 2 on the rearrangement R = R(S) of Alg. 1 / Eq. SVD);
 *   3. projects X with F_KSTAP = (I - U_A U_A^H) (x) (I - U_B U_B^H)
 *      (Eq. KronSTAP);
 *   4. evaluates T_v = |d_v^H P x|^2 / (d_v^H P d_v) over a bank of velocity
 *      steering vectors d_v = a_v (x) b_v (Eq. Moving, Sec. 6 image
 *      formation), and reports Tmax = max_v T_v, its argmax and Tmax > tau.
 *
 * Frame layout (all calls): Y holds p channel images, each H_in x W_in
 * complex64 (interleaved re, im), row = range, column = azimuth, channel
 * planes contiguous: Y[(i * H_in + row) * W_in + col].  The cell grid is
 * H x W with H = H_in - 2 ring_r and W = W_in - 2 ring_a - q + 1; cell (r, c)
 * owns X[i][j] = Y_i(r + ring_r, c + ring_a + j), and its training cells are
 * (r + dr, c + dc) with |dr| <= ring_r, |dc| <= ring_a, excluding
 * |dr| <= guard_r && |dc| <= guard_a, so n = (2 ring_r + 1)(2 ring_a + 1)
 * - (2 guard_r + 1)(2 guard_a + 1).  Per-cell outputs are indexed
 * k = r * W + c.
 *
 * Memory: every pointer argument named "device" is a CUDA device pointer
 * owned by the caller (e.g. a torch tensor's data_ptr()).  The library owns
 * only its context and the workspace it allocates inside kstap_fit_project
 * (bounded by the context's HBM budget).  All work is enqueued on the
 * context's stream; the calls return after enqueueing, without a device
 * synchronisation, except where stated.
 *
 * Errors: every call returns a kstap_status; nothing throws across the ABI.
 * kstap_last_error(ctx) describes the last failure of that context.
 */
#ifndef KSTAP_H_
#define KSTAP_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  float re, im;
} kstap_c64; /* interleaved complex64 */

typedef enum {
  KSTAP_WARN_NOCONV = 1, /* kstap_fit_report: some cells stopped at max_iter (results valid) */
  KSTAP_OK = 0,
  KSTAP_EINVAL = -1,   /* bad argument; nothing was enqueued */
  KSTAP_ENOMEM = -2,   /* workspace would exceed the HBM budget, or cudaMalloc failed */
  KSTAP_ECUDA = -3,    /* a CUDA runtime call failed (see kstap_last_error) */
  KSTAP_EAGAIN = -4,   /* serving: result not ready / not admitted yet */
  KSTAP_ETIMEOUT = -5, /* serving: poll timed out */
  KSTAP_ENOTFOUND = -6 /* serving: unknown ticket */
} kstap_status;

/* Model and detector parameters.  Notation of the paper: p channels, q
 * pulses (azimuth window), ranks r_a, r_b of A and B (Eq. SparseOpt), Alg. 2
 * tolerance eps and iteration cap, detection threshold tau on Tmax.
 * Limits of this build: p == 3 with q in {8, 12, 16, 24, 32} and r_a == 1
 * (the paper's rank-one spatial model, Eq. KronCov) or r_a == 2 (KSTAP_FP32
 * bank and Kron-STAP filter); or p == 6 -- K = 2 registered passes of 3
 * channels stacked as one frame (Sec. 3), spatial rank r_a in {1, 2} -- with
 * q in {8, 16}, the KSTAP_FP32 bank and the Kron-STAP filter.
 * 1 <= r_b <= min(q - 1, 8) (Sec. 5 warns against r_b close to q); r_b > 4
 * needs p == 3 and the KSTAP_FP32 bank (the B pass's r_b x r_b Gram and
 * Cholesky factors then exceed the registers, and it runs 10-30 times slower
 * than at r_b = 3).  ring >= guard >= 0, n >= 1, (2 ring_r + 1)(2 ring_a + 1)
 * <= 1024, and a training box whose tiles fit shared memory.  Other values
 * give KSTAP_EINVAL. */
typedef struct {
  int p, q, r_a, r_b;
  int ring_r, ring_a, guard_r, guard_a;
  /* Alg. 2 stopping rule on the GPU: stop when the relative change of the
   * spatial factor a between iterations is <= eps (eps <= 0 selects 2e-6,
   * i.e. single-precision stagnation), or after max_iter iterations
   * (max_iter <= 0 selects 64). */
  double eps;
  int max_iter;
  float tau;
  /* Arithmetic of the velocity-bank contraction (Eq. KronSTAP statistic):
   * KSTAP_FP32 (CUDA cores; T within 1e-4 of FP64), or the tensor-core route
   * KSTAP_FP16X3 / KSTAP_BF16X3 (tcgen05 MMA on hi + lo 16-bit splits of
   * the projected snapshot and the bank, FP32 accumulation; near-blind
   * velocities fall back to the CUDA-core arithmetic).  The tensor-core
   * route needs V <= 128.  The fit (steps 1-2) is the same for all three. */
  int precision;
  /* Projector of the statistic: KSTAP_FILTER_KRON, F_A (x) F_B with
   * F = I - U U^H (Eq. KronSTAP), or KSTAP_FILTER_CLASSICAL,
   * I - (U_A (x) U_B)(U_A (x) U_B)^H, the rank r_a r_b projector that Sec. 5
   * compares it with.  The classical filter needs precision KSTAP_FP32. */
  int filter;
} kstap_params;

enum { KSTAP_FP32 = 0, KSTAP_FP16X3 = 1, KSTAP_BF16X3 = 2 };
enum { KSTAP_FILTER_KRON = 0, KSTAP_FILTER_CLASSICAL = 1 };

/* Per-cell LR-Kron factors, caller-owned device arrays of H * W cells each.
 *   UA    : [k][p][r_a]  complex64, orthonormal columns (U_A of Eq. KronSTAP)
 *   UB_hi : [k][q][r_b]  complex64, U_B rounded to single precision
 *   UB_lo : [k][q][r_b]  complex64, U_B - UB_hi (float-float low part; the
 *                        projection of X needs U_B to ~2^-40, Sec. 5)
 *   lamA  : [k][r_a]     float, eigenvalues of A^ (tr A^ = p normalisation)
 *   lamB  : [k][r_b]     float, eigenvalues of B^ (same normalisation)
 *   iters : [k]          int32, Alg. 2 iterations taken
 *   eta   : [k]          float, |R - a b^T|_F / |R|_F at the final a (Alg. 2)
 * lamA, lamB, iters and eta may be NULL. */
typedef struct {
  kstap_c64* UA;
  kstap_c64* UB_hi;
  kstap_c64* UB_lo;
  float* lamA;
  float* lamB;
  int32_t* iters;
  float* eta;
} kstap_factors;

typedef struct kstap_ctx kstap_ctx;

/* Create a context.  bank_a (V x p) and bank_b (V x q) are device arrays of
 * complex64 steering factors a_v, b_v (Eq. Moving: d_v = a_v (x) b_v, up to
 * normalisation, which T_v does not depend on); the library copies them.
 * 1 <= V <= 256.  hbm_budget_bytes bounds the workspace (0 = unlimited).
 * cuda_stream is a cudaStream_t (NULL = legacy default stream).
 * Returns KSTAP_EINVAL for unsupported parameters (see kstap_params). */
kstap_status kstap_create(const kstap_params* params, const kstap_c64* bank_a,
                          const kstap_c64* bank_b, int V, size_t hbm_budget_bytes,
                          void* cuda_stream, kstap_ctx** out);

/* Steps 1-2 above (Eq. SCM, Alg. 1 as an index map, Alg. 2, EIG_{r_b} of
 * B^): fits every cell of the frame Y (device, p x H_in x W_in complex64)
 * and writes the factors.  Requires H_in >= 2 ring_r + 1 and
 * W_in >= 2 ring_a + q.  Grows the workspace when needed; a frame whose
 * workspace exceeds the budget runs as row strips (KSTAP_ENOMEM if even a
 * 4-row strip does not fit).  The call is asynchronous on the context stream.
 * Non-finite input: NaN / Inf samples enter the sums as 0, and every cell
 * whose box (rows r .. r + 2 ring_r, columns c .. c + 2 ring_a + q - 1 of
 * every channel, i.e. its training windows, guard and test window) holds one
 * gets iters = -1 and eta = NaN; its factors are not meaningful. */
kstap_status kstap_fit_project(kstap_ctx* ctx, const kstap_c64* Y, int H_in, int W_in,
                               const kstap_factors* factors);

/* Waits for the context stream, then reports the last kstap_fit_project or
 * kstap_run_batch: cells whose Alg. 2 loop stopped at max_iter, cells flagged
 * for non-finite input, and cells whose EIG_{r_b} (Sec. 4) took the
 * ill-gapped path: their leading r_b eigenvalues of B were not separated
 * from the next one well enough for subspace iteration on r_b vectors (the
 * rate estimate left more than ~2e-7 of subspace error after 4 steps), so
 * U_B and lambda_B were recomputed by block subspace iteration on
 * min(q, max(8, r_b + 4)) vectors with a Rayleigh-Ritz step solved by FP64
 * Jacobi sweeps.  Any pointer may be NULL.  Returns KSTAP_WARN_NOCONV if any cell stopped at
 * max_iter (its factors are the last iterate, valid but not converged to
 * eps), else KSTAP_OK. */
kstap_status kstap_fit_report(kstap_ctx* ctx, long long* nonconverged, long long* nonfinite,
                              long long* eig_refined);

/* Steps 3-4 above (Eq. KronSTAP and the velocity bank) with the factors of a
 * previous kstap_fit_project on the same frame.  Outputs (device, H * W):
 * Tmax float, vidx int32 (lowest maximising v), map uint8 (Tmax > tau);
 * T_all (device, [k][V] float) may be NULL.  Velocities whose steering
 * vector keeps less than 1e-12 of its energy after projection get T_v = 0.
 * Cells whose box (see kstap_fit_project) holds a NaN / Inf sample of this Y
 * get Tmax = NaN, vidx = -1, map = 0 and T_all = NaN. */
kstap_status kstap_detect(kstap_ctx* ctx, const kstap_c64* Y, int H_in, int W_in,
                          const kstap_factors* factors, float* Tmax, int32_t* vidx, uint8_t* map,
                          float* T_all);

/* Waits for the context stream, then reports whether a kernel of this
 * context gave up a bounded wait -- a tensor-core kernel waiting for its MMAs,
 * or the moments pass waiting for a TMA tile load -- (KSTAP_ECUDA, with the
 * reason in kstap_last_error; the word is cleared) or not (KSTAP_OK).
 * Results of a launch that gave up are not valid; if the message says the
 * device state is unknown, the MMAs had not completed when the kernel freed
 * their tensor memory, and the process should reset the device
 * (cudaDeviceReset) before further work. */
kstap_status kstap_device_status(kstap_ctx* ctx);

/* Free the context, its workspace and its copies of the bank. */
kstap_status kstap_destroy(kstap_ctx* ctx);

/* Text of the last error of this context ("" if none).  ctx may be NULL, in
 * which case the last error of kstap_create on this thread is returned. */
const char* kstap_last_error(const kstap_ctx* ctx);

/* Kernel identifiers for kstap_kernel_times (launch order within one frame). */
enum {
  KSTAP_K_SCALE = 0,    /* frame fixed-point scale (max |component| of Y) */
  KSTAP_K_MOMENTS = 1,  /* exact lag box sums -> M = R R^H and A_0 (Eq. SCM, Sec. 4 init) */
  KSTAP_K_FLIPFLOP = 2, /* Alg. 2 iterations on M, EIG_{r_a} (one thread per cell) */
  KSTAP_K_BFIT = 3,     /* exact lag sums -> B (float-float) -> EIG_{r_b} -> U_B */
  KSTAP_K_DETECT = 4,   /* Eq. KronSTAP projection and the velocity bank */
  KSTAP_K_MGRAM = 5,    /* p = 6 (stacked passes): M = R R^H and A_0 from the lag store */
  kstap_nkernels = 6
};

/* Per-kernel timing for measurement.  When enabled, every launch is
 * bracketed by CUDA events on the context's stream; kstap_kernel_times
 * synchronises on the pending events and returns, per kernel id, the summed
 * milliseconds and launch counts since profiling was (re)enabled.  Enabling
 * or disabling resets the totals. n = number of entries in the arrays. */
kstap_status kstap_set_profiling(kstap_ctx* ctx, int enable);
kstap_status kstap_kernel_times(kstap_ctx* ctx, float* total_ms, int32_t* launches, int n);

/* Throughput probe of one arithmetic pipe, the measured denominator of the
 * kernels' roofline fractions (the paper has no counterpart): op
 * KSTAP_PROBE_FFMA (FP32 fused multiply-add), KSTAP_PROBE_FFMA2 (packed
 * f32x2 FMA, both lanes counted), KSTAP_PROBE_IMAD64 (64-bit integer
 * multiply-add, the arithmetic of the exact lag sums) or KSTAP_PROBE_DFMA
 * (FP64 FMA).  Every thread of SMs x 8 CTAs x 256 threads runs 8 independent
 * chains of `iters` operations (rounded down to a multiple of 4); one warm-up
 * launch, then `reps` launches timed with CUDA events on cuda_stream.
 * *ops_per_s = operations per second (one FMA or multiply-add per lane = one
 * operation; a flop rate is twice that).  Allocates an 8-byte counter
 * stream-ordered; synchronises the stream.  iters < 4, reps < 1, an unknown
 * op or a NULL ops_per_s give KSTAP_EINVAL. */
enum { KSTAP_PROBE_FFMA = 0, KSTAP_PROBE_FFMA2 = 1, KSTAP_PROBE_IMAD64 = 2, KSTAP_PROBE_DFMA = 3 };
kstap_status kstap_alu_probe(int op, int iters, int reps, void* cuda_stream, double* ops_per_s);

/* ------------------------------------------------------------ batches ----
 * One frame of a batch: the frame Y (device, p x H_in x W_in complex64), its
 * caller-owned factor arrays and outputs (device, H * W cells; layouts as in
 * kstap_factors / kstap_detect; T_all may be NULL). */
typedef struct {
  const kstap_c64* Y;
  int H_in, W_in;
  kstap_factors factors;
  float* Tmax;
  int32_t* vidx;
  uint8_t* map;
  float* T_all;
} kstap_frame;

/* Batched fit + detect of n frames of different sizes that share the
 * context's parameters and bank.  Every kernel of the path is launched once
 * for the whole batch (persistent grids over the tiles of all frames), so
 * many small tiles cost five launches, not five per tile.  The workspace
 * grows to the batch's needs (KSTAP_ENOMEM over budget); the device job table
 * is uploaded on the context stream.  Results are identical to per-frame
 * kstap_fit_project + kstap_detect calls (same kernels, same tiling of each
 * frame). */
kstap_status kstap_run_batch(kstap_ctx* ctx, const kstap_frame* frames, int n);

/* A CUDA graph over batches of several contexts (e.g. one per (q, r_b)
 * class of a mixed batch): ctxs[c] processes frames[c][0 .. nframes[c]-1].
 * The graph owns its own workspaces and job tables (allocated here, outside
 * the capture), captures each context's batch on its own branch stream
 * (fork / join), and is instantiated once; kstap_graph_launch replays it on
 * cuda_stream (a cudaStream_t).  Frame pointers and sizes are baked in: to
 * process new data, write it into the same device buffers and relaunch.  The
 * contexts must outlive the graph.  Errors: kstap_last_error(NULL). */
typedef struct kstap_graph kstap_graph;
kstap_status kstap_graph_create(kstap_ctx* const* ctxs, const kstap_frame* const* frames,
                                const int* nframes, int nctx, kstap_graph** out);
kstap_status kstap_graph_launch(kstap_graph* graph, void* cuda_stream);
kstap_status kstap_graph_destroy(kstap_graph* graph);

/* Launch tuning of a context.  waves: grid size in multiples of (SMs x
 * resident CTAs), 1..64, capped by the tile count (default 64: one or two
 * tiles per CTA on a megapixel frame; smaller values make each CTA stride
 * over more tiles); tc: cells per tile of the B / U_B pass
 * (0 = default: 32, or 16 at q = 32; allowed 8, 16, 32 with tc = 32 only for
 * q <= 16); lag_store: 1 = the moments pass writes the exact lag sums to a
 * workspace store that the B pass reads (9 q (W + q - 1) x 16 B per cell row,
 * e.g. 2.4 GB for a 1024^2 frame at q = 16), 0 = the B pass recomputes them
 * from its frame tile and the store is not allocated (p = 3 only; stacked
 * passes need the store).  Tuning changes only the schedule and memory, not
 * the arithmetic of any cell: results are bit-identical. */
typedef struct {
  int waves;
  int tc;
  int lag_store;
  float ms_per_batch; /* measured by kstap_autotune */
} kstap_tuning;

/* Autotuner: times kstap_run_batch on these frames (reps repetitions after a
 * warm-up) for every candidate (waves in {1,2,4,8,16,32,64}) x (tc in {16,32}, or
 * {8,16} at q = 32) x (lag_store in {1, 0} for p = 3), keeps the fastest in
 * the context and reports it.  Synchronises the context stream. */
kstap_status kstap_autotune(kstap_ctx* ctx, const kstap_frame* frames, int n, int reps,
                            kstap_tuning* out);
kstap_status kstap_set_tuning(kstap_ctx* ctx, const kstap_tuning* tuning);

/* ------------------------------------------------------------ serving ----
 * A request loop over the context: kstap_submit queues a frame and returns a
 * ticket at once; a worker thread admits queued frames in arrival order while
 * their device memory (workspace, factors and, for host frames, a device copy)
 * fits the context's HBM budget, groups whatever is admissible into one
 * batch (same kernels and results as kstap_run_batch) and enqueues it on one
 * of max_inflight streams, so batches overlap on the device and frames that
 * arrive meanwhile join the next batch.  Device frames are borrowed until
 * their request completes; host frames are copied at admission.  Results
 * (Tmax, vidx, map on the device, H * W cells) are held until kstap_release.
 * Results count against the budget from submit until release, so unreleased
 * results throttle admission.  Budget 0 = unlimited; a frame larger than the
 * budget is refused at submit (KSTAP_ENOMEM).  While a context serves, do not
 * call its other entry points from other threads. */
#define KSTAP_FRAME_ON_HOST 1
typedef struct {
  uint64_t ticket;
  int H, W;                 /* cell grid */
  const float* Tmax;        /* device, library-owned until kstap_release */
  const int32_t* vidx;
  const uint8_t* map;
  double t_submit_us;       /* microseconds since the context's first submit */
  double t_admit_us;
  double t_done_us;         /* completion (host callback after the last kernel) */
} kstap_result;

/* Serving limits: frames per batch (1..1024, default 16) and batches in
 * flight (1..16, default 4).  Call before the first kstap_submit. */
kstap_status kstap_serve_config(kstap_ctx* ctx, int max_batch, int max_inflight);
/* Work cap of one served batch in cells (H * W summed over its frames and
 * strips; a single frame or strip above the cap still forms a batch of its
 * own).  Every frame of a batch completes when the batch does, so the cap
 * bounds how long a small frame waits for the large ones batched with it.
 * cells <= 0 removes the cap; the default is 1 << 20.  Call before the first
 * kstap_submit. */
kstap_status kstap_serve_batch_cells(kstap_ctx* ctx, long long cells);
/* flags: KSTAP_FRAME_ON_HOST when Y is in host memory (pinned for overlap). */
kstap_status kstap_submit(kstap_ctx* ctx, const kstap_c64* Y, int H_in, int W_in, int flags,
                          uint64_t* ticket);
/* timeout_us: 0 = non-blocking (KSTAP_EAGAIN if not done), < 0 = wait,
 * > 0 = wait at most that long (KSTAP_ETIMEOUT). */
kstap_status kstap_poll(kstap_ctx* ctx, uint64_t ticket, kstap_result* out, int timeout_us);
/* Frees a completed request's results (KSTAP_EAGAIN while in flight). */
kstap_status kstap_release(kstap_ctx* ctx, uint64_t ticket);

/* Allocation-free variant of kstap_fit_project.  The paper has no
 * counterpart: this exists for callers that must not allocate device memory
 * while they run -- for example a real-time processing loop, where cudaMalloc
 * may synchronise the device and has unbounded latency, or a host whose
 * device memory is entirely owned by another allocator.  It needs no context
 * and calls no cudaMalloc, cudaFree or other allocating routine; the caller
 * passes the frame Y (device) and the factor arrays exactly as for
 * kstap_fit_project, and cuda_stream is a cudaStream_t (NULL = legacy default
 * stream).
 *
 * Scratch (frame scale, per-cell moments and flip-flop factors, 504 B per
 * cell) lives in one statically allocated device array of about 16.5 MB that
 * every GPU which loads the library holds until the process exits.  Frames
 * with more than 32768 cells (H * W), and parameters with p != 3, are
 * rejected with KSTAP_EINVAL and a message from kstap_last_error(NULL); other
 * errors are reported the same way.
 *
 * Every call looks up the array's address on the current device
 * (cudaGetSymbolAddress, which allocates nothing); the first lookup on a
 * device also loads the library's device code there, so make the first call
 * on each device before any stream capture.  Every call shares the one array: calls that overlap on the GPU
 * (different streams, or different host threads, on the same device) race
 * and corrupt each other's results, so serialise them.  The array keeps the
 * last call's contents; the call clears what it needs zeroed itself. */
kstap_status kstap_fit_project_noalloc(const kstap_params* params, const kstap_c64* Y, int H_in,
                                       int W_in, const kstap_factors* factors, void* cuda_stream);

/* Noncoherent change detection over stacked passes (Sec. 8): from T_all of a
 * kstap_detect whose bank lists every velocity once per pass (K V entries
 * per cell, pass-major: entry k V + v = velocity v steered on pass k's
 * channels), writes per cell Tmax_k = max_v T_all[cell][k V + v] (device,
 * K x ncell, pass-major; may be NULL) and change = Tmax_{K-1} - Tmax_0
 * (device, ncell; may be NULL): the difference of the filtered pixel
 * magnitudes of the last and the first pass.  Asynchronous on cuda_stream.
 * ncell = 0 is a no-op; ncell < 0, V < 1, K < 1 or a NULL T_all with
 * ncell > 0 give KSTAP_EINVAL (message from kstap_last_error(NULL)). */
kstap_status kstap_change_map(const float* T_all, long long ncell, int V, int K, float* Tmax_k,
                              float* change, void* cuda_stream);

/* One large-covariance LR-Kron fit (Alg. 2), the paper's timing workload
 * (Sec. 7.1): S = (1/n) sum_m x_m x_m^H from n snapshots x_m = vec(X_m^T),
 * fitted as A (x) B with rank(A) <= r_a and B untruncated (r_b = q, as in
 * that experiment), Alg. 2 from A_0 = vec^-1(R 1 / q^2), stopping when
 * |eta_k - eta_k-1| <= eps (eps <= 0 selects 1e-6) or after max_iter
 * iterations (<= 0 selects 100).  R = R(S) is never formed: every step is
 * evaluated through the n^2 p x p Grams X_m X_m'^H (FP64).
 *   X     : device, n x p x q complex64, X[m][i][j] (channel i, pulse j)
 *   A_out : device, p x p complex64 row-major, A^ with tr A^ = p (may be NULL)
 *   B_out : device, q x q complex64 row-major, B^ = vec^-1(b) of the last b
 *           (scaled by the same normalisation), Hermitian
 *   iters, eta (host, may be NULL): iterations taken and the final
 *           |R - a b^T|_F / |R|_F
 * Limits: 1 <= n <= 16, 1 <= p <= 8, 2 <= q <= 16384, 1 <= r_a <= p.  Needs no
 * context; allocates its ~KB of scratch stream-ordered on cuda_stream and
 * synchronises that stream before returning.  Errors: kstap_last_error(NULL). */
kstap_status kstap_lrkron_fit(const kstap_c64* X, int n, int p, int q, int r_a, double eps,
                              int max_iter, kstap_c64* A_out, kstap_c64* B_out, int32_t* iters,
                              double* eta, void* cuda_stream);

/* Bytes of workspace kstap_fit_project needs for an H_in x W_in frame with
 * these parameters (0 on invalid input). */
size_t kstap_workspace_bytes(const kstap_params* params, int H_in, int W_in);

#ifdef __cplusplus
}
#endif

#endif /* KSTAP_H_ */
