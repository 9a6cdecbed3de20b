"""Seeded synthetic SAR GMTI frames for Kronecker STAP.

This module only draws inputs: channel images, the velocity steering bank and
target truth.  It holds none of the estimation or detection arithmetic, so the
FP64 oracle and the CUDA path consume the same bytes.

Data model (Sec. 2 of the paper, SIRV clutter model, texture tau = 1):
  * p channel images Y_i, i = 0..p-1, each H_in x W_in complex64; row = range,
    column = azimuth (contiguous).
  * Test cell (r, c) of the H x W cell grid owns the snapshot
    X[i, j] = Y_i(r + ring_r, c + ring_a + j), j = 0..q-1, x = vec(X^T)
    (channel-major, pulse-minor, Sec. 2).
  * The frame carries a halo so every cell has its whole training ring:
    H_in = H + 2 ring_r, W_in = W + 2 ring_a + q - 1.
  * Clutter covariance A (x) B_c (Eq. KronCov) with B_c of rank r_b:
    C(row, col) = sum_k sqrt(mu_k) L_A g_k(row) exp(j 2 pi nu_k col),
    L_A L_A^H = A, g_k(row) ~ CN(0, I_p) per range row, mu_k proportional to
    2^-k with sum mu_k = sigma^2 10^(CNR/10).  Every q-window is then
    CN(0, A (x) B_c + sigma^2 I), B_c = sum_k mu_k e_k e_k^H,
    e_k[j] = exp(j 2 pi nu_k j).
  * Clutter tones nu_k are spaced 1.25 / q cycles/sample apart (+-10% jitter,
    common offset U(-0.02, 0.02)), so the r_b temporal clutter directions are
    resolvable inside one q-window.  With tone_band = w (make_frame) they are
    instead drawn independently and uniformly in [-w, w] cycles/sample (w =
    0.05: the narrow clutter band of a slow platform); tones closer than a
    Doppler bin make the trailing clutter eigenvalues of B small, so the
    eigengap of B at rank r_b spans many decades over the cells of a frame.
  * A_ij = 0.9^|i-j| exp(j phi (i-j)), one phi ~ U(-pi, pi) per frame: a
    modulated AR(1) covariance, Hermitian Toeplitz and positive definite.
  * Noise is CN(0, sigma^2) per pixel and channel, sigma^2 = 1.
  * Moving targets follow Eq. (Moving), x = alpha a(f) (x) b(f): a target at
    cell (r0, c0) with bank index v adds beta a_v[i] b_v[j] to
    Y_i(r0 + ring_r, c0 + ring_a + j), j < q.  Target velocities lie outside
    the clutter band: |nu_v| >= max(0.15, band + 1/q).
  * Steering bank: nu_v = (v - V/2) / V, a_v[i] = exp(j 2 pi nu_v i),
    b_v[j] = exp(j 2 pi nu_v j).

Random streams: numpy default_rng([seed, stream]), stream 0 = clutter,
1 = noise, 2 = targets, 3 = sizes / arrivals / samples, 4 = SIRV texture,
5 = targets inside training rings.

Robustness options of make_frame (Sec. 2 SIRV model, Sec. 5 robustness):
  * texture_nu: each input range row's clutter is scaled by tau_row with
    tau_row^2 ~ Gamma(nu, 1/nu) (mean 1): K-distributed clutter amplitude,
    heavier-tailed for small nu; snapshots of one row share their texture,
    as the SIRV model's per-snapshot tau does.
  * training_targets: every target gets this many copies (same velocity and
    amplitude) at random cells of its own training ring, which contaminates
    its training set.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional, Tuple

import numpy as np

SEED_BASE = 160403622

STREAM_CLUTTER = 0
STREAM_NOISE = 1
STREAM_TARGETS = 2
STREAM_SIZES = 3
STREAM_TEXTURE = 4
STREAM_CONTAM = 5


@dataclasses.dataclass
class Workload:
    """One synthetic Kron-STAP workload (frame geometry and model parameters)."""

    name: str
    p: int
    H: int                # cell-grid rows (range)
    W: int                # cell-grid columns (azimuth)
    q: int                # azimuth (pulse) window
    r_a: int              # spatial rank (1 in the paper's model, Eq. KronCov)
    r_b: int              # temporal rank
    ring_r: int           # outer training box half-height (range)
    ring_a: int           # outer training box half-width (azimuth)
    guard_r: int          # guard box half-height
    guard_a: int          # guard box half-width
    V: int                # steering-bank size
    cnr_db: float
    n_targets: int
    snr_db: Tuple[float, float]   # uniform range, per element
    seed: int
    sigma2: float = 1.0
    pfa: float = 1e-3

    @property
    def n(self) -> int:
        return ((2 * self.ring_r + 1) * (2 * self.ring_a + 1)
                - (2 * self.guard_r + 1) * (2 * self.guard_a + 1))

    @property
    def H_in(self) -> int:
        return self.H + 2 * self.ring_r

    @property
    def W_in(self) -> int:
        return self.W + 2 * self.ring_a + self.q - 1

    @property
    def cells(self) -> int:
        return self.H * self.W

    @property
    def tau(self) -> float:
        # Clutter-free white noise gives T_v ~ sigma^2 Exp(1); a per-cell
        # false-alarm rate pfa over V velocities gives tau = sigma^2 ln(V/pfa).
        return float(self.sigma2 * math.log(self.V / self.pfa))

    def with_size(self, H: int, W: int, name: Optional[str] = None) -> "Workload":
        """Same model on an H x W cell grid, keeping the target density."""
        nt = int(round(self.n_targets * H * W / float(self.H * self.W)))
        nt = max(1, nt) if self.n_targets > 0 else 0
        return dataclasses.replace(self, H=H, W=W, n_targets=nt,
                                   name=name or f"{self.name}_{H}x{W}")


# Training geometry per n = 2pq (p = 3): a centred range x azimuth box minus a
# centred guard box, (ring_r, ring_a, guard_r, guard_a).
RING_FOR_N = {48: (3, 4, 1, 2), 72: (4, 4, 1, 1), 96: (3, 7, 1, 1), 120: (4, 7, 1, 2),
              144: (4, 8, 1, 1), 192: (4, 11, 1, 2)}


def make_workload(name, H, W, q, r_b, n, V, cnr_db, n_targets, snr_db, seed_off, p=3, r_a=1):
    rr, ra, gr, ga = RING_FOR_N[n]
    return Workload(name=name, p=p, H=H, W=W, q=q, r_a=r_a, r_b=r_b, ring_r=rr, ring_a=ra,
                    guard_r=gr, guard_a=ga, V=V, cnr_db=cnr_db, n_targets=n_targets,
                    snr_db=snr_db, seed=SEED_BASE + seed_off)


WORKLOADS: Dict[str, Workload] = {
    # 64x64 cells, q=8, r_b=2, n=48 (7x9 box minus 3x5 guard), V=32,
    # 30 dB CNR, 5 targets at 10 dB.
    "small64": make_workload("small64", 64, 64, 8, 2, 48, 32, 30.0, 5, (10.0, 10.0), 0),
    # 1024x1024 cells, q=16, r_b=3, n=120 (9x15 minus 3x5), V=64, 40 dB CNR,
    # 200 targets at SNR U(0, 15) dB.
    "frame1024": make_workload("frame1024", 1024, 1024, 16, 3, 120, 64, 40.0, 200,
                               (0.0, 15.0), 1),
    # 2048x2048 cells, q=32, r_b=4, n=192 (9x23 minus 3x5), V=128, 40 dB CNR.
    "precision2048": make_workload("precision2048", 2048, 2048, 32, 4, 192, 128, 40.0, 200,
                                   (0.0, 15.0), 3),
    # the windows between the configurations' q values: q = 12 (n = 72, the
    # literal 9x9 box minus 3x3 guard) and q = 24 (n = 144, 9x17 minus 3x3),
    # 256x256 cells, 40 dB CNR, targets at the 1024^2 frame's density
    "frame_q12": make_workload("frame_q12", 256, 256, 12, 3, 72, 48, 40.0, 13, (0.0, 15.0), 7),
    "frame_q24": make_workload("frame_q24", 256, 256, 24, 4, 144, 96, 40.0, 13, (0.0, 15.0), 8),
}


def spatial_cov(p: int, phi: float) -> np.ndarray:
    idx = np.arange(p)
    d = idx[:, None] - idx[None, :]
    return (0.9 ** np.abs(d)) * np.exp(1j * phi * d)


def steering_bank(p: int, q: int, V: int) -> Tuple[np.ndarray, np.ndarray]:
    """Velocity bank a_v (V x p) and b_v (V x q), complex64, unit-modulus entries."""
    nu = (np.arange(V) - V / 2.0) / V
    a = np.exp(2j * np.pi * nu[:, None] * np.arange(p)[None, :])
    b = np.exp(2j * np.pi * nu[:, None] * np.arange(q)[None, :])
    return a.astype(np.complex64), b.astype(np.complex64)


def clutter_tones(q: int, r_b: int, rng: np.random.Generator,
                  band: Optional[float] = None) -> Tuple[np.ndarray, float]:
    """Clutter tones (cycles/sample) 1.25 bins apart -- or, with `band`, drawn
    uniformly in [-band, band] -- and the band half-width."""
    if band is not None:
        nu = np.sort(rng.uniform(-band, band, size=r_b))
        return nu, float(band)
    s = 1.25 / q
    off = rng.uniform(-0.02, 0.02)
    jit = rng.uniform(-0.1 * s, 0.1 * s, size=r_b)
    nu = (np.arange(r_b) - (r_b - 1) / 2.0) * s + jit + off
    band = float(np.max(np.abs(nu)))
    return nu, band


@dataclasses.dataclass
class Frame:
    wl: Workload
    Y: np.ndarray                 # (p, H_in, W_in) complex64
    bank_a: np.ndarray            # (V, p) complex64
    bank_b: np.ndarray            # (V, q) complex64
    targets: List[Tuple[int, int, int, complex]]   # (r, c, v, beta), cell coordinates
    A: np.ndarray                 # true spatial covariance (p x p)
    tones: np.ndarray             # clutter tones nu_k (cycles/sample)
    mus: np.ndarray               # clutter powers mu_k
    ring_targets: List[Tuple[int, int, int, complex]] = dataclasses.field(default_factory=list)


def _cn(rng: np.random.Generator, shape, dtype=np.float64) -> np.ndarray:
    re = rng.standard_normal(shape, dtype=dtype)
    im = rng.standard_normal(shape, dtype=dtype)
    return (re + 1j * im) * np.sqrt(0.5)


def make_frame(wl: Workload, seed: Optional[int] = None, clutter: bool = True,
               noise: bool = True, targets: bool = True, texture_nu: Optional[float] = None,
               training_targets: int = 0, tone_band: Optional[float] = None) -> Frame:
    """Draw one seeded frame for workload `wl` (see the module docstring)."""
    seed = wl.seed if seed is None else seed
    p, q, H_in, W_in = wl.p, wl.q, wl.H_in, wl.W_in
    Y = np.zeros((p, H_in, W_in), dtype=np.complex64)

    rng_c = np.random.default_rng([seed, STREAM_CLUTTER])
    phi = rng_c.uniform(-np.pi, np.pi)
    A = spatial_cov(p, phi)
    L_A = np.linalg.cholesky(A)
    tones, band = clutter_tones(q, wl.r_b, rng_c, tone_band)
    w = 2.0 ** -np.arange(wl.r_b)
    mus = wl.sigma2 * 10 ** (wl.cnr_db / 10.0) * w / w.sum()
    g = _cn(rng_c, (wl.r_b, H_in, p))                              # g_k(row)
    if clutter:
        lg = np.einsum("ij,krj->kri", L_A, g) * np.sqrt(mus)[:, None, None]
        if texture_nu is not None:
            rng_x = np.random.default_rng([seed, STREAM_TEXTURE])
            tau = np.sqrt(rng_x.gamma(texture_nu, 1.0 / texture_nu, size=H_in))
            lg = lg * tau[None, :, None]
        ph = np.exp(2j * np.pi * tones[:, None] * np.arange(W_in)[None, :])   # (r_b, W_in)
        for i in range(p):
            Y[i] += (lg[:, :, i].T @ ph).astype(np.complex64)     # (H_in, W_in)

    if noise:
        rng_n = np.random.default_rng([seed, STREAM_NOISE])
        for i in range(p):
            Y[i] += (np.sqrt(wl.sigma2) * _cn(rng_n, (H_in, W_in), np.float32)).astype(np.complex64)

    bank_a, bank_b = steering_bank(p, q, wl.V)
    tl: List[Tuple[int, int, int, complex]] = []
    rng_t = np.random.default_rng([seed, STREAM_TARGETS])
    nu = (np.arange(wl.V) - wl.V / 2.0) / wl.V
    allowed = np.nonzero(np.abs(nu) >= max(0.15, band + 1.0 / q))[0]
    if targets and wl.n_targets > 0 and len(allowed) > 0:
        for _ in range(wl.n_targets):
            r0 = int(rng_t.integers(0, wl.H))
            c0 = int(rng_t.integers(0, wl.W))
            v = int(allowed[rng_t.integers(0, len(allowed))])
            snr = rng_t.uniform(wl.snr_db[0], wl.snr_db[1])
            amp = np.sqrt(wl.sigma2 * 10 ** (snr / 10.0))
            beta = amp * np.exp(1j * rng_t.uniform(-np.pi, np.pi))
            blk = beta * np.outer(bank_a[v].astype(np.complex128), bank_b[v].astype(np.complex128))
            Y[:, r0 + wl.ring_r, c0 + wl.ring_a:c0 + wl.ring_a + q] += blk.astype(np.complex64)
            tl.append((r0, c0, v, complex(beta)))
    ring: List[Tuple[int, int, int, complex]] = []
    if training_targets > 0 and tl:
        rng_k = np.random.default_rng([seed, STREAM_CONTAM])
        for (r0, c0, v, beta) in list(tl):
            blk = beta * np.outer(bank_a[v].astype(np.complex128), bank_b[v].astype(np.complex128))
            placed = 0
            while placed < training_targets:
                dr = int(rng_k.integers(-wl.ring_r, wl.ring_r + 1))
                dc = int(rng_k.integers(-wl.ring_a, wl.ring_a + 1))
                if abs(dr) <= wl.guard_r and abs(dc) <= wl.guard_a:
                    continue                        # in the guard box: not training
                r1, c1 = r0 + dr, c0 + dc
                if not (0 <= r1 + wl.ring_r < H_in and 0 <= c1 + wl.ring_a and
                        c1 + wl.ring_a + q <= W_in):
                    continue
                Y[:, r1 + wl.ring_r, c1 + wl.ring_a:c1 + wl.ring_a + q] += blk.astype(np.complex64)
                ring.append((r1, c1, v, beta))
                placed += 1
    return Frame(wl=wl, Y=np.ascontiguousarray(Y), bank_a=bank_a, bank_b=bank_b, targets=tl,
                 A=A, tones=tones, mus=mus, ring_targets=ring)


def random_cells(wl: Workload, count: int, seed: int) -> np.ndarray:
    """Seeded sample of distinct flattened cell indices r * W + c, sorted."""
    rng = np.random.default_rng([seed, STREAM_SIZES])
    total = wl.H * wl.W
    count = min(count, total)
    return np.sort(rng.choice(total, size=count, replace=False)).astype(np.int64)


def tile_batch(n_tiles: int = 256, seed: int = SEED_BASE + 2, V: int = 64,
               cnr_db: float = 40.0) -> List[Workload]:
    """Uneven frame tiles: H ~ logU[32, 512], W ~ logU[32, 384] cells, q uniform
    in {8, 16, 32}, r_b uniform in {2, 3, 4}, n = 2pq training cells (p = 3),
    V velocities, targets at the density of the 1024^2 frame (200 per 1M cells)."""
    rng = np.random.default_rng([seed, STREAM_SIZES])
    out = []
    for k in range(n_tiles):
        H = int(round(math.exp(rng.uniform(math.log(32), math.log(512)))))
        W = int(round(math.exp(rng.uniform(math.log(32), math.log(384)))))
        q = int(rng.choice([8, 16, 32]))
        r_b = int(rng.choice([2, 3, 4]))
        nt = max(1, int(round(200 * H * W / 1048576.0)))
        out.append(make_workload(f"tile{k:03d}", H, W, q, r_b, 2 * 3 * q, V, cnr_db, nt,
                                 (0.0, 15.0), 1000 + k))
    return out


def serving_pool(n_per_q: int = 4, seed: int = SEED_BASE + 4, V: int = 64,
                 qs=(16, 32), r_b: int = 3, lo: int = 256, hi: int = 4096) -> List[Workload]:
    """Frames for the serving stream: sides uniform in [lo, hi] cells, q in qs,
    r_b = 3, n = 2pq, V velocities, 40 dB CNR, targets at the 1024^2 density."""
    rng = np.random.default_rng([seed, STREAM_SIZES])
    out = []
    for q in qs:
        for k in range(n_per_q):
            H = int(rng.integers(lo, hi + 1))
            W = int(rng.integers(lo, hi + 1))
            nt = max(1, int(round(200 * H * W / 1048576.0)))
            out.append(make_workload(f"serve_q{q}_{k}", H, W, q, r_b, 2 * 3 * q, V, 40.0, nt,
                                     (0.0, 15.0), 2000 + 10 * q + k))
    return out


def poisson_arrivals(n: int, rate_hz: float, n_frames: int, seed: int = SEED_BASE + 5):
    """Arrival times (s) of a Poisson stream and the pool index of each request."""
    rng = np.random.default_rng([seed, STREAM_SIZES])
    t = np.cumsum(rng.exponential(1.0 / rate_hz, size=n))
    idx = rng.integers(0, n_frames, size=n)
    return t, idx


def lrkron_timing_case(p: int, q: int, n: int = 5, sigma2: float = 0.1,
                       seed: int = SEED_BASE + 6) -> np.ndarray:
    """Snapshots of the single large-covariance LR-Kron timing workload (Sec. 7.1):
    x_m = vec(X_m^T) ~ CN(0, A (x) I_q + sigma2 I_pq), m < n, with A = u u^H a
    random complex rank-one p x p matrix (|u| = 1) and B = I_q.  Returns
    X (n, p, q) complex64.  sigma2 = 0 gives the noiseless model, whose sample
    covariance is exactly separable."""
    rng = np.random.default_rng([seed, STREAM_CLUTTER])
    u = _cn(rng, p)
    u = u / np.linalg.norm(u)
    w = _cn(rng, (n, q))                                  # B = I: white temporal factor
    X = u[None, :, None] * w[:, None, :]                  # X_m = u w_m^T
    if sigma2 > 0:
        rng_n = np.random.default_rng([seed, STREAM_NOISE])
        X = X + np.sqrt(sigma2) * _cn(rng_n, (n, p, q))
    return np.ascontiguousarray(X.astype(np.complex64))


@dataclasses.dataclass
class MultipassFrame:
    wl: Workload                  # per-pass model (p channels); the frame has K p channels
    K: int
    Y: np.ndarray                 # (K p, H_in, W_in) complex64: pass k on channels [k p, (k+1) p)
    bank_a: np.ndarray            # (K V, K p): velocity v of pass k = row k V + v, a_v on block k
    bank_b: np.ndarray            # (K V, q)
    targets: List[Tuple[int, int, int, int, complex]]   # (pass, r, c, v, beta)


def make_multipass_frame(wl: Workload, K: int = 2, coherence: float = 0.9,
                         seed: Optional[int] = None,
                         tone_band: Optional[float] = None) -> MultipassFrame:
    """K registered passes over the same scene (Sec. 3), stacked as K p channels.

    The clutter of pass k is A_k^{1/2} g_k(row) exp(j 2 pi nu col) per tone,
    with its own spatial covariance A_k (a per-pass phase phi_k: calibration
    differs between passes) and temporal tones shared by all passes (same
    ground); the range-row amplitudes g_k are correlated across passes with
    coefficient `coherence` (g_k = c g_0 + sqrt(1 - c^2) e_k).  The stacked
    clutter spans [U_A1; ...; U_AK] (x) U_B: spatial rank K, temporal rank r_b.
    Noise is white per channel.  Each target moves between passes, so it is
    injected in one pass only (pass chosen at random).  The bank holds every
    velocity once per pass: row k V + v has a_v on the channels of pass k."""
    seed = wl.seed + 17 if seed is None else seed
    p, q, H_in, W_in = wl.p, wl.q, wl.H_in, wl.W_in
    Y = np.zeros((K * p, H_in, W_in), dtype=np.complex64)
    rng_c = np.random.default_rng([seed, STREAM_CLUTTER])
    tones, band = clutter_tones(q, wl.r_b, rng_c, tone_band)
    w = 2.0 ** -np.arange(wl.r_b)
    mus = wl.sigma2 * 10 ** (wl.cnr_db / 10.0) * w / w.sum()
    g0 = _cn(rng_c, (wl.r_b, H_in))
    ph = np.exp(2j * np.pi * tones[:, None] * np.arange(W_in)[None, :])   # (r_b, W_in)
    for k in range(K):
        phi = rng_c.uniform(-np.pi, np.pi)
        L_A = np.linalg.cholesky(spatial_cov(p, phi))
        gk = coherence * g0 + np.sqrt(1 - coherence ** 2) * _cn(rng_c, (wl.r_b, H_in))
        h = _cn(rng_c, (wl.r_b, H_in, p))                 # spatial draw per tone and row
        lg = np.einsum("ij,krj->kri", L_A, h) * (np.sqrt(mus)[:, None] * np.abs(gk))[:, :, None]
        lg = lg * np.exp(1j * np.angle(gk))[:, :, None]
        for i in range(p):
            Y[k * p + i] += (lg[:, :, i].T @ ph).astype(np.complex64)
    rng_n = np.random.default_rng([seed, STREAM_NOISE])
    for ch in range(K * p):
        Y[ch] += (np.sqrt(wl.sigma2) * _cn(rng_n, (H_in, W_in), np.float32)).astype(np.complex64)
    ba, bb = steering_bank(p, q, wl.V)
    bank_a = np.zeros((K * wl.V, K * p), np.complex64)
    bank_b = np.zeros((K * wl.V, q), np.complex64)
    for k in range(K):
        bank_a[k * wl.V:(k + 1) * wl.V, k * p:(k + 1) * p] = ba
        bank_b[k * wl.V:(k + 1) * wl.V] = bb
    rng_t = np.random.default_rng([seed, STREAM_TARGETS])
    nu = (np.arange(wl.V) - wl.V / 2.0) / wl.V
    allowed = np.nonzero(np.abs(nu) >= max(0.15, band + 1.0 / q))[0]
    tl = []
    for _ in range(wl.n_targets):
        kk = int(rng_t.integers(0, K))
        r0, c0 = int(rng_t.integers(0, wl.H)), int(rng_t.integers(0, wl.W))
        v = int(allowed[rng_t.integers(0, len(allowed))])
        amp = np.sqrt(wl.sigma2 * 10 ** (rng_t.uniform(*wl.snr_db) / 10.0))
        beta = amp * np.exp(1j * rng_t.uniform(-np.pi, np.pi))
        blk = beta * np.outer(ba[v].astype(np.complex128), bb[v].astype(np.complex128))
        Y[kk * p:(kk + 1) * p, r0 + wl.ring_r, c0 + wl.ring_a:c0 + wl.ring_a + q] += blk.astype(np.complex64)
        tl.append((kk, r0, c0, v, complex(beta)))
    return MultipassFrame(wl=wl, K=K, Y=np.ascontiguousarray(Y), bank_a=bank_a, bank_b=bank_b,
                          targets=tl)
