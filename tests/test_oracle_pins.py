"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these re-types the oracle's own formulas: each compares it with a
closed form, a library routine used as an independent method, a hand-derived
fixture, an invariant the paper states, or brute force on a tiny input.
"""
import os

import numpy as np
import pytest

import gen
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def crandn(rng, *shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2)


def rand_psd(rng, n, rank):
    G = crandn(rng, n, rank)
    return G @ G.conj().T


def vecF(M):
    return M.flatten(order="F")


# ---------------------------------------------------------------- Alg. 1 ---

def test_alg1_matches_hand_derived_fixture():
    """Sec. 4 Eq. SVD / Alg. 1: p = q = 2 index map derived by hand."""
    rows = []
    with open(os.path.join(GOLDEN, "alg1_p2_q2.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            parts = line.split()
            rows.append([tuple(int(t) for t in e.split(",")) for e in parts[1:]])
    S = np.arange(16, dtype=float).reshape(4, 4) + 1j * np.arange(16).reshape(4, 4) * 0.5
    R = oracle.rearrange(S, 2, 2)
    for J, row in enumerate(rows):
        for P, (i, j) in enumerate(row):
            assert R[J, P] == S[i - 1, j - 1]


@pytest.mark.parametrize("p,q", [(3, 4), (2, 5), (4, 3)])
def test_alg1_rows_are_vectorised_blocks(p, q):
    """Sec. 4 (Eq. SVD): each row of R is vec(M(i, j)) of a q x q block."""
    rng = np.random.default_rng(1)
    S = crandn(rng, p * q, p * q)
    R = oracle.rearrange(S, p, q)
    got = set()
    for J in range(p * p):
        match = [(i, j) for i in range(p) for j in range(p)
                 if np.array_equal(R[J], vecF(S[i * q:(i + 1) * q, j * q:(j + 1) * q]))]
        assert len(match) == 1
        got.add(match[0])
    assert len(got) == p * p


@pytest.mark.parametrize("p,q", [(3, 4), (3, 8), (2, 6)])
def test_alg1_kron_is_rank_one(p, q):
    """R(A (x) B) = vec(A) vec(B)^T (Pitsianis-Van Loan, Sec. 4)."""
    rng = np.random.default_rng(2)
    A = crandn(rng, p, p)
    B = crandn(rng, q, q)
    R = oracle.rearrange(np.kron(A, B), p, q)
    np.testing.assert_allclose(R, np.outer(vecF(A), vecF(B)), atol=1e-12)


# ------------------------------------------------------------ Jacobi -------

@pytest.mark.parametrize("n", [2, 3, 8, 16, 32])
def test_jacobi_matches_lapack(n):
    rng = np.random.default_rng(3 + n)
    M = rand_psd(rng, n, n) - 0.3 * n * np.eye(n)      # indefinite Hermitian
    w, U = oracle.eigh(M)
    w_ref = np.linalg.eigvalsh(M)[::-1]
    np.testing.assert_allclose(w, w_ref, atol=1e-12 * abs(w_ref).max())
    np.testing.assert_allclose(U.conj().T @ U, np.eye(n), atol=1e-12)
    np.testing.assert_allclose(U.conj().T @ M @ U, np.diag(w), atol=1e-11 * abs(w_ref).max())


# ------------------------------------------------------------ SCM ----------

def test_scm_of_separable_snapshots_is_kronecker():
    """Eq. SCM with x = vec(X^T): X = u v^T gives x = u (x) v, so the SCM of
    separable snapshots is (1/n) sum (u u^H) (x) (v v^H)."""
    rng = np.random.default_rng(4)
    p, q, n = 3, 5, 7
    us = crandn(rng, n, p)
    vs = crandn(rng, n, q)
    X = np.stack([np.outer(us[m], vs[m]) for m in range(n)])
    S = oracle.scm(X)
    ref = sum(np.kron(np.outer(us[m], us[m].conj()), np.outer(vs[m], vs[m].conj()))
              for m in range(n)) / n
    np.testing.assert_allclose(S, ref, atol=1e-12)


def test_scm_is_hermitian_psd_with_trace_of_mean_energy():
    rng = np.random.default_rng(5)
    X = crandn(rng, 9, 3, 4)
    S = oracle.scm(X)
    np.testing.assert_allclose(S, S.conj().T, atol=1e-14)
    assert np.linalg.eigvalsh(S).min() > -1e-12
    assert abs(np.trace(S).real - np.mean(np.sum(np.abs(X) ** 2, axis=(1, 2)))) < 1e-12


# ------------------------------------------------------------ Alg. 2 -------

def test_lrkron_exact_recovery_from_kronecker_data():
    """Sec. 4: S = A (x) B exactly with rank(A) <= r_a, rank(B) <= r_b is
    recovered exactly (eta = 0).  The data are all pairs u_s (x) v_t."""
    rng = np.random.default_rng(6)
    p, q, r_b = 3, 6, 2
    h = crandn(rng, p)
    vs = crandn(rng, r_b, q)
    X = np.stack([np.outer(s * h, v) for s in (1.0, 0.5j, -0.7) for v in vs])
    S = oracle.scm(X)
    out = oracle.lrkron(S, p, q, 1, r_b)
    np.testing.assert_allclose(np.kron(out["A"], out["B"]), S, atol=1e-12 * abs(S).max())
    assert out["eta"] < 1e-12
    assert out["iters"] <= 3
    PA = out["UA"] @ out["UA"].conj().T
    np.testing.assert_allclose(PA, np.outer(h, h.conj()) / np.vdot(h, h).real, atol=1e-12)


def test_lrkron_stacked_passes_exact_recovery():
    """Sec. 3 multipass: two passes stacked as p = 6 channels.  Snapshots
    a_s v_t^T over all pairs, with spatial vectors [h1; 0], [0; h2] and a mix
    (rank-2 A), give S = A (x) B exactly; r_a = 2 recovers it (eta = 0) and
    P_A is the projector onto span{[h1; 0], [0; h2]}."""
    rng = np.random.default_rng(16)
    p1, q, r_b = 3, 6, 2
    h1, h2 = crandn(rng, p1), crandn(rng, p1)
    z = np.zeros(p1, complex)
    avs = [np.concatenate([h1, z]), np.concatenate([z, h2]), 0.5j * np.concatenate([h1, h2])]
    vs = crandn(rng, r_b, q)
    X = np.stack([np.outer(a, v) for a in avs for v in vs])
    S = oracle.scm(X)
    out = oracle.lrkron(S, 2 * p1, q, 2, r_b)
    np.testing.assert_allclose(np.kron(out["A"], out["B"]), S, atol=1e-11 * abs(S).max())
    assert out["eta"] < 1e-11
    PA = out["UA"] @ out["UA"].conj().T
    E = np.stack([avs[0], avs[1]], axis=1)
    Q_, _ = np.linalg.qr(E)
    np.testing.assert_allclose(PA, Q_ @ Q_.conj().T, atol=1e-11)
    # with r_a = 1 the rank-2 spatial factor cannot be represented: eta > 0
    assert oracle.lrkron(S, 2 * p1, q, 1, r_b)["eta"] > 1e-3


def test_stacked_bank_measures_each_pass():
    """Sec. 8: with the stacked bank (entry k V + v = a_v on pass k's channels),
    a target present only in pass 1 and orthogonal to both clutter factors
    gives T = |beta|^2 |d|^2 on its pass-1 entry (Sec. 6, projector = I on d)
    and 0 on its pass-0 entry (the two steering vectors are orthogonal)."""
    p1, q, V = 3, 8, 8
    ba, bb = gen.steering_bank(p1, q, V)
    bank_a = np.zeros((2 * V, 2 * p1), complex)
    bank_b = np.zeros((2 * V, q), complex)
    for k in range(2):
        bank_a[k * V:(k + 1) * V, k * p1:(k + 1) * p1] = ba
        bank_b[k * V:(k + 1) * V] = bb
    v, beta = 5, 0.8 - 0.3j
    d1 = np.kron(bank_a[V + v], bank_b[V + v])                  # pass-1 steering, vec(X^T)
    X = beta * np.outer(bank_a[V + v], bank_b[V + v])
    # clutter factors orthogonal to the target: U_A on pass 0 only, U_B
    # orthogonal to b_v
    UA = np.concatenate([ba[1], np.zeros(p1)])[:, None] / np.sqrt(p1)
    w = bb[2] - bb[v] * np.vdot(bb[v], bb[2]) / np.vdot(bb[v], bb[v])
    UB = (w / np.linalg.norm(w))[:, None]
    T, _ = oracle.stat(X, UA, UB, bank_a, bank_b)
    np.testing.assert_allclose(T[V + v], abs(beta) ** 2 * np.vdot(d1, d1).real, rtol=1e-12)
    assert abs(T[v]) < 1e-20
    assert T.argmax() == V + v


def test_lrkron_exact_recovery_given_S():
    rng = np.random.default_rng(7)
    p, q = 3, 5
    A = rand_psd(rng, p, 1)
    B = rand_psd(rng, q, 2)
    out = oracle.lrkron(np.kron(A, B), p, q, 1, 2)
    np.testing.assert_allclose(np.kron(out["A"], out["B"]), np.kron(A, B), atol=1e-11)
    assert abs(np.trace(out["A"]).real - p) < 1e-12        # tr A^ = p normalisation


def test_lrkron_untruncated_is_top_singular_pair():
    """r_a = p, r_b = q: the fixed point of Alg. 2 is the best rank-one fit
    of R(S), i.e. its top singular pair (Van Loan-Pitsianis; library SVD)."""
    rng = np.random.default_rng(8)
    p, q = 3, 4
    X = crandn(rng, 40, p, q)
    S = oracle.scm(X)
    out = oracle.lrkron(S, p, q, p, q)
    R = oracle.rearrange(S, p, q)
    U, s, Vh = np.linalg.svd(R)
    best = s[0] * np.outer(U[:, 0], Vh[0])
    got = np.outer(vecF(out["A"]), vecF(out["B"]))
    np.testing.assert_allclose(got, best, atol=1e-9 * abs(best).max())


def test_lrkron_factors_psd_with_stated_ranks():
    """Sec. 4: A_0 PSD implies A^ (x) B^ PSD Hermitian of rank r_a r_b."""
    rng = np.random.default_rng(9)
    p, q, r_a, r_b = 3, 6, 1, 3
    X = crandn(rng, 30, p, q)
    out = oracle.lrkron(oracle.scm(X), p, q, r_a, r_b)
    for M, r in ((out["A"], r_a), (out["B"], r_b)):
        np.testing.assert_allclose(M, M.conj().T, atol=1e-12 * abs(M).max())
        w = np.linalg.eigvalsh(M)[::-1]
        assert w.min() > -1e-10 * w[0]
        assert np.sum(w > 1e-9 * w[0]) == r
    K = np.kron(out["A"], out["B"])
    assert np.linalg.matrix_rank(K, tol=1e-9 * abs(K).max()) == r_a * r_b


def test_lrkron_fixed_point_is_local_minimum():
    """Tiny brute force (p = 2, q = 3, r_a = 1, r_b = q): no rank-feasible
    perturbation of the fixed point lowers |S - A (x) B|_F (Eq. SparseOpt)."""
    rng = np.random.default_rng(10)
    p, q = 2, 3
    S = oracle.scm(crandn(rng, 12, p, q))
    out = oracle.lrkron(S, p, q, 1, q)
    A, B = out["A"], out["B"]
    f0 = np.linalg.norm(S - np.kron(A, B)) ** 2
    w, U = np.linalg.eigh(A)
    u, lam = U[:, -1], w[-1]
    for _ in range(3000):
        e = 10 ** rng.uniform(-6, -1)
        u2 = u + e * crandn(rng, p)
        A2 = (lam * (1 + e * rng.standard_normal())) * np.outer(u2, u2.conj()) / np.vdot(u2, u2).real
        D = crandn(rng, q, q) * e
        B2 = B + (D + D.conj().T) / 2 * abs(B).max()
        assert np.linalg.norm(S - np.kron(A2, B2)) ** 2 >= f0 * (1 - 1e-12)


def test_lrkron_eta_is_residual_and_decreases():
    rng = np.random.default_rng(11)
    p, q = 3, 6
    S = oracle.scm(crandn(rng, 36, p, q) + np.kron(np.ones((1, p, 1)), crandn(rng, 36, 1, q)) * 3)
    out = oracle.lrkron(S, p, q, 1, 2, eps=0.0, max_iter=30)
    hist = out["eta_hist"]
    assert np.all(np.diff(hist) <= 1e-13)
    assert 0 < hist[-1] < 1


def test_classical_subspace_of_exact_kronecker():
    """Eq. KronUS: for S = A (x) B exact, the leading r_a r_b eigenvectors of
    the dense S span U_A (x) U_B (library eigh as the brute force)."""
    rng = np.random.default_rng(12)
    p, q = 3, 5
    A = rand_psd(rng, p, 1)
    B = rand_psd(rng, q, 2)
    S = np.kron(A, B)
    out = oracle.lrkron(S, p, q, 1, 2)
    w, U = np.linalg.eigh(S)
    top = U[:, -2:]
    P1 = top @ top.conj().T
    K = np.kron(out["UA"], out["UB"])
    np.testing.assert_allclose(P1, K @ K.conj().T, atol=1e-10)


# ----------------------------------------------------------- statistic -----

def _orth_complement_basis(rng, vecs, n, r):
    """r orthonormal columns orthogonal to the given vectors (QR)."""
    M = np.concatenate([np.atleast_2d(vecs).T, crandn(rng, n, r)], axis=1)
    Q, _ = np.linalg.qr(M)
    k = np.atleast_2d(vecs).shape[0]
    return Q[:, k:k + r]


def test_stat_target_orthogonal_to_clutter_gives_alpha_squared():
    """Eq. KronSTAP with P d = d and x = alpha d: T = |alpha|^2 exactly."""
    rng = np.random.default_rng(13)
    p, q, V = 3, 8, 16
    ba, bb = gen.steering_bank(p, q, V)
    v = 3
    UA = _orth_complement_basis(rng, ba[v], p, 1)
    UB = _orth_complement_basis(rng, bb[v], q, 2)
    d = np.kron(ba[v].astype(np.complex128), bb[v].astype(np.complex128)) / np.sqrt(p * q)
    alpha = 2.5 - 1.25j
    T, cond = oracle.stat((alpha * d).reshape(p, q), UA, UB, ba, bb)
    # T = |alpha|^2 |d|^2; the bank entries are complex64, so |d| = 1 to ~1e-7
    assert abs(T[v] - abs(alpha) ** 2 * np.vdot(d, d).real) < 1e-12
    assert abs(cond[v] - 1.0) < 1e-12


def test_classical_stat_equals_projector_from_eigh_of_S():
    """Sec. 5 classical projector: for S = A (x) B exact (rank r_a r_b), I - W W^H
    with W = U_A (x) U_B is I minus the projector onto the leading r_a r_b
    eigenvectors of the dense S (library eigh), so T matches that form."""
    rng = np.random.default_rng(21)
    p, q, V = 3, 6, 12
    A = rand_psd(rng, p, 1)
    B = rand_psd(rng, q, 2)
    S = np.kron(A, B)
    out = oracle.lrkron(S, p, q, 1, 2)
    w, E = np.linalg.eigh(S)
    E = E[:, -2:]
    P = np.eye(p * q) - E @ E.conj().T
    ba, bb = gen.steering_bank(p, q, V)
    X = crandn(rng, p, q) * 2
    T, cond = oracle.stat(X, out["UA"], out["UB"], ba, bb, filter="classical")
    x = X.reshape(-1)
    for v in range(V):
        d = np.kron(ba[v].astype(np.complex128), bb[v].astype(np.complex128)) / np.sqrt(p * q)
        num = abs(np.vdot(d, P @ x)) ** 2
        den = np.vdot(d, P @ d).real
        assert abs(T[v] - num / den) <= 1e-9 * max(1.0, num / den)
        assert abs(cond[v] - den / np.vdot(d, d).real) <= 1e-10


def test_classical_keeps_what_kron_removes():
    """x = alpha d with U_B^H b = 0 but U_A^H a != 0: the classical projector
    leaves d whole (T = |alpha|^2 |d|^2) while Kron-STAP still removes the
    U_A direction (T = |alpha|^2 |F_A a|^2 |b|^2 / pq); and the classical
    projector annihilates U_A (x) U_B itself."""
    rng = np.random.default_rng(22)
    p, q, V = 3, 8, 16
    ba, bb = gen.steering_bank(p, q, V)
    v = 5
    a = ba[v].astype(np.complex128)
    b = bb[v].astype(np.complex128)
    UA = np.linalg.qr(crandn(rng, p, 1))[0]
    UB = _orth_complement_basis(rng, bb[v], q, 2)
    d = np.kron(a, b) / np.sqrt(p * q)
    alpha = -1.5 + 2.0j
    X = (alpha * d).reshape(p, q)
    Tc, _ = oracle.stat(X, UA, UB, ba, bb, filter="classical")
    Tk, _ = oracle.stat(X, UA, UB, ba, bb)
    assert abs(Tc[v] - abs(alpha) ** 2 * np.vdot(d, d).real) < 1e-11
    FAa = a - UA[:, 0] * np.vdot(UA[:, 0], a)
    want = abs(alpha) ** 2 * np.vdot(FAa, FAa).real * np.vdot(b, b).real / (p * q)
    assert abs(Tk[v] - want) < 1e-11
    assert abs(Tc[v] - Tk[v]) > 1e-3
    Xw = 3.0 * np.outer(UA[:, 0], UB[:, 1])          # in span(U_A (x) U_B)
    Tw, _ = oracle.stat(Xw, UA, UB, ba, bb, filter="classical")
    assert np.abs(Tw).max() < 1e-20


def test_stat_matches_factored_form():
    """P = F_A (x) F_B acts on X as F_A X F_B^T, and d^H P d factorises."""
    rng = np.random.default_rng(14)
    p, q, V = 3, 6, 12
    ba, bb = gen.steering_bank(p, q, V)
    UA = np.linalg.qr(crandn(rng, p, 1))[0]
    UB = np.linalg.qr(crandn(rng, q, 2))[0]
    X = crandn(rng, p, q) * 3
    T, cond = oracle.stat(X, UA, UB, ba, bb)
    FA = np.eye(p) - UA @ UA.conj().T
    FB = np.eye(q) - UB @ UB.conj().T
    Z = FA @ X @ FB.T
    for v in range(V):
        num = abs(ba[v].conj() @ Z @ bb[v].conj()) ** 2
        den = np.linalg.norm(FA @ ba[v]) ** 2 * np.linalg.norm(FB @ bb[v]) ** 2
        assert abs(T[v] - num / den) <= 1e-10 * max(1.0, num / den)


def test_stat_white_noise_mean_is_sigma2():
    """x ~ CN(0, sigma^2 I) and fixed P: T_v ~ sigma^2 Exp(1) (Eq. SINRdef)."""
    rng = np.random.default_rng(15)
    p, q, V = 3, 8, 8
    ba, bb = gen.steering_bank(p, q, V)
    UA = np.linalg.qr(crandn(rng, p, 1))[0]
    UB = np.linalg.qr(crandn(rng, q, 2))[0]
    sig2 = 2.0
    Ts = np.array([oracle.stat(np.sqrt(sig2) * crandn(rng, p, q), UA, UB, ba, bb)[0]
                   for _ in range(2500)])
    m = Ts.mean(axis=0)
    assert np.all(np.abs(m / sig2 - 1) < 0.1)
    assert abs(Ts.mean() / sig2 - 1) < 0.03


def test_projector_idempotent_and_annihilates_clutter():
    wl = gen.WORKLOADS["small64"].with_size(6, 7)
    f = gen.make_frame(wl)
    o = oracle.run_workload(f)
    for PA, PB in zip(o["PA"], o["PB"]):
        for Pm, r in ((PA, wl.r_a), (PB, wl.r_b)):
            np.testing.assert_allclose(Pm @ Pm, Pm, atol=1e-12)
            np.testing.assert_allclose(Pm, Pm.conj().T, atol=1e-12)
            assert abs(np.trace(Pm).real - r) < 1e-12
        P = np.kron(np.eye(wl.p) - PA, np.eye(wl.q) - PB)
        UA = np.linalg.eigh(PA)[1][:, -wl.r_a:]
        UB = np.linalg.eigh(PB)[1][:, -wl.r_b:]
        w = crandn(np.random.default_rng(0), wl.q)
        assert np.abs(P @ np.kron(UA, UB)).max() < 1e-12
        assert np.abs(P @ np.kron(UA[:, 0], w)).max() < 1e-12
        assert np.abs(P @ np.kron(w[:wl.p], UB[:, 0])).max() < 1e-12


# ------------------------------------------------------- whole pipeline ----

def _gather(Y, wl, r, c):
    """Brute-force O1 for a tiny test: the ring by its definition."""
    q = wl.q
    X = Y[:, r + wl.ring_r, c + wl.ring_a:c + wl.ring_a + q]
    T = [Y[:, r + dr + wl.ring_r, c + dc + wl.ring_a:c + dc + wl.ring_a + q]
         for dr in range(-wl.ring_r, wl.ring_r + 1) for dc in range(-wl.ring_a, wl.ring_a + 1)
         if not (abs(dr) <= wl.guard_r and abs(dc) <= wl.guard_a)]
    return X, np.stack(T)


def test_cells_pipeline_equals_composed_steps():
    """Per-cell pipeline == ring gather by definition + SCM + Alg. 2 + stat."""
    wl = gen.WORKLOADS["small64"].with_size(5, 6)
    f = gen.make_frame(wl)
    o = oracle.run_workload(f)
    assert wl.n == 48
    for k in [0, 7, 29]:
        r, c = divmod(k, wl.W)
        X, Tr = _gather(f.Y, wl, r, c)
        assert Tr.shape[0] == wl.n
        lr = oracle.lrkron(oracle.scm(Tr), wl.p, wl.q, wl.r_a, wl.r_b)
        T, _ = oracle.stat(X, lr["UA"], lr["UB"], f.bank_a, f.bank_b)
        np.testing.assert_allclose(o["T_all"][k], T, rtol=1e-12, atol=1e-12)
        assert o["vidx"][k] == int(np.argmax(T))


def test_pipeline_cancels_clutter_and_detects_targets():
    """Sanity of generator + oracle: clutter-free T has mean sigma^2 after
    Kron-STAP at 30 dB CNR, and injected targets exceed tau at their velocity."""
    wl = gen.WORKLOADS["small64"]
    f0 = gen.make_frame(wl, targets=False)
    o0 = oracle.run_workload(f0)
    assert abs(o0["T_all"].mean() - wl.sigma2) < 0.05
    assert o0["map"].mean() < 5e-3
    f = gen.make_frame(wl)
    o = oracle.run_workload(f)
    for r, c, v, beta in f.targets:
        k = r * wl.W + c
        assert o["map"][k] == 1
        assert o["T_all"][k, v] > wl.tau


def test_oracle_rejects_bad_arguments():
    wl = gen.WORKLOADS["small64"].with_size(4, 4)
    f = gen.make_frame(wl)
    with pytest.raises(ValueError):
        oracle.kstap_cells(f.Y, wl.q, 1, wl.q, wl.ring_r, wl.ring_a, wl.guard_r, wl.guard_a,
                           f.bank_a, f.bank_b, wl.tau)      # r_b = q is rejected (Sec. 5)
    with pytest.raises(ValueError):
        oracle.run_workload(f, cells=np.array([wl.H * wl.W]))
