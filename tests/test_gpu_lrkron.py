"""One large-covariance LR-Kron fit (kstap_lrkron_fit) against the FP64 oracle's
literal Alg. 1 + Alg. 2 on the dense sample covariance (needs a GPU).

Workload of Sec. 7.1: rank-one A, B = I (r_b = q, untruncated), n = 5.  Bars:
the same iteration count and eta to 1e-9 (the GPU iterates in FP64 on the
Grams); A^ to 1e-6 and B^ to 1e-5 of its largest entry (complex64 outputs).
"""
import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu


def _dense_S(X):
    n, p, q = X.shape
    x = np.stack([X[m].reshape(-1) for m in range(n)]).astype(np.complex128)   # vec(X_m^T)
    return (x.T @ x.conj()) / n


def _fit(X, r_a, eps, max_iter=100):
    import torch
    import paper_1604_03622_b300 as K
    Xd = torch.from_numpy(X).cuda()
    A, B, it, eta = K.kstap_lrkron_fit(Xd, r_a=r_a, eps=eps, max_iter=max_iter)
    torch.cuda.synchronize()
    return A.cpu().numpy(), B.cpu().numpy(), it, eta


@pytest.mark.parametrize("p,q,n,sigma2,r_a,eps", [
    (3, 12, 5, 0.1, 1, 1e-6), (3, 120, 5, 0.1, 1, 1e-6), (3, 120, 5, 0.1, 1, 1e-4),
    (6, 25, 5, 0.1, 1, 1e-6), (3, 40, 5, 0.1, 2, 1e-6), (3, 50, 1, 0.1, 1, 1e-6),
    (4, 33, 7, 0.3, 1, 1e-6)])
def test_lrkron_fit_matches_oracle(p, q, n, sigma2, r_a, eps):
    X = gen.lrkron_timing_case(p, q, n=n, sigma2=sigma2)
    ref = oracle.lrkron(_dense_S(X), p, q, r_a, q, eps=eps, max_iter=100)
    A, B, it, eta = _fit(X, r_a, eps)
    assert it == ref["iters"]
    assert abs(eta - ref["eta"]) <= 1e-9
    assert np.abs(A - ref["A"]).max() <= 1e-6 * np.abs(ref["A"]).max()
    assert np.abs(B - ref["B"]).max() <= 1e-5 * np.abs(ref["B"]).max()


def test_lrkron_fit_noiseless_is_exact():
    """sigma2 = 0: S is exactly A (x) B-hat (separable snapshots), so Alg. 2
    stops after two iterations with eta ~ 0 and A^ (x) B^ reproduces S."""
    p, q = 3, 64
    X = gen.lrkron_timing_case(p, q, sigma2=0.0)
    A, B, it, eta = _fit(X, 1, 1e-6)
    assert it == 2 and eta < 1e-6
    S = _dense_S(X)
    K = np.kron(A.astype(np.complex128), B.astype(np.complex128))
    assert np.abs(K - S).max() <= 1e-5 * np.abs(S).max()


def test_lrkron_fit_large_q_matches_oracle():
    """q = 300 (the oracle's dense S is 900 x 900): same bars."""
    X = gen.lrkron_timing_case(3, 300)
    ref = oracle.lrkron(_dense_S(X), 3, 300, 1, 300, eps=1e-6, max_iter=100)
    A, B, it, eta = _fit(X, 1, 1e-6)
    assert it == ref["iters"] and abs(eta - ref["eta"]) <= 1e-9
    assert np.abs(B - ref["B"]).max() <= 1e-5 * np.abs(ref["B"]).max()


def test_lrkron_fit_q2500_properties():
    """The paper's largest case (p = 3, q = 2500): B^ is Hermitian, tr A^ = p,
    A^ is rank one, and eta lies in (0, 1)."""
    X = gen.lrkron_timing_case(3, 2500)
    A, B, it, eta = _fit(X, 1, 1e-6)
    assert abs(np.trace(A).real - 3) < 1e-5 and abs(np.trace(A).imag) < 1e-5
    w = np.linalg.eigvalsh(A.astype(np.complex128))
    assert w[-2] < 1e-5 * w[-1]
    assert np.abs(B - B.conj().T).max() <= 1e-5 * np.abs(B).max()
    assert 0 < eta < 1 and 2 <= it <= 100
