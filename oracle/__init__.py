"""FP64 CPU oracle for Kron-STAP -- test infrastructure only.

Only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
use this package.  The product path (``paper_1604_03622_b300``) never imports
it, and the two share no code: this file binds ``kstap_oracle.cpp`` (plain
FP64 C++ written from the paper's Alg. 1, Alg. 2, Eq. SCM and Eq. KronSTAP)
through ctypes.  Each function is a marshalling wrapper; the arithmetic and
the paper step it follows are in the C++ file.

Defaults: eps = 1e-15 on |eta_k - eta_{k-1}| (Alg. 2's test).  eta is
stationary at the fixed point, so |delta eta| ~ |delta a|^2: eps = 1e-15
resolves the factors to ~1e-8, below single-precision resolution.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Dict, Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kstap_oracle.cpp")
_LIB = os.path.join(_HERE, "libkstap_oracle.so")
_lib = None

DEFAULT_EPS = 1e-15
DEFAULT_MAX_ITER = 500


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (OpenMP) next to its source."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P, I, D, L = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64
        lib.oracle_scm.argtypes = [P, I, I, I, P]
        lib.oracle_rearrange.argtypes = [P, I, I, P]
        lib.oracle_eigh.argtypes = [P, I, P, P]
        lib.oracle_lrkron.argtypes = [P, I, I, I, I, D, I, P, P, P, P, P, P, P, P, P]
        lib.oracle_lrkron.restype = I
        lib.oracle_stat.argtypes = [P, P, P, I, I, I, I, P, P, I, P, P, I]
        lib.oracle_kstap_cells.argtypes = [P, I, I, I, I, I, I, I, I, I, I, D, I, P, P, I, D,
                                           P, L, P, P, P, P, P, P, P, P, P, P, P, P, I, I]
        lib.oracle_kstap_cells.restype = I
        lib.oracle_num_threads.restype = I
        _lib = lib
    return _lib


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.complex128))


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def scm(Xtr: np.ndarray) -> np.ndarray:
    """S = (1/n) sum x x^H with x = vec(X^T), from training snapshots (n, p, q)."""
    X = _c128(Xtr)
    n, p, q = X.shape
    S = np.zeros((p * q, p * q), np.complex128)
    _load().oracle_scm(_ptr(X), n, p, q, _ptr(S))
    return S


def rearrange(S: np.ndarray, p: int, q: int) -> np.ndarray:
    """R = Rearrange(S) by Alg. 1 (p^2 x q^2)."""
    S = _c128(S)
    R = np.zeros((p * p, q * q), np.complex128)
    _load().oracle_rearrange(_ptr(S), p, q, _ptr(R))
    return R


def eigh(M: np.ndarray):
    """Cyclic-Jacobi eigendecomposition: (w decreasing, U with eigenvector columns)."""
    M = _c128(M)
    n = M.shape[0]
    w = np.zeros(n)
    U = np.zeros((n, n), np.complex128)
    _load().oracle_eigh(_ptr(M), n, _ptr(w), _ptr(U))
    return w, U


def lrkron(S: np.ndarray, p: int, q: int, r_a: int, r_b: int, eps: float = DEFAULT_EPS,
           max_iter: int = DEFAULT_MAX_ITER) -> Dict[str, np.ndarray]:
    """Alg. 2 (LR-Kron) on a given S: A, B (tr A = p), UA, UB, lamA, lamB, wB, eta, iters."""
    S = _c128(S)
    out = dict(A=np.zeros((p, p), np.complex128), B=np.zeros((q, q), np.complex128),
               UA=np.zeros((p, r_a), np.complex128), UB=np.zeros((q, r_b), np.complex128),
               lamA=np.zeros(r_a), lamB=np.zeros(r_b), wB=np.zeros(q), eta=np.zeros(1),
               eta_hist=np.zeros(max_iter))
    it = _load().oracle_lrkron(_ptr(S), p, q, r_a, r_b, float(eps), int(max_iter),
                               _ptr(out["A"]), _ptr(out["B"]), _ptr(out["UA"]), _ptr(out["UB"]),
                               _ptr(out["lamA"]), _ptr(out["lamB"]), _ptr(out["wB"]),
                               _ptr(out["eta"]), _ptr(out["eta_hist"]))
    out["iters"] = int(it)
    out["eta"] = float(out["eta"][0])
    out["eta_hist"] = out["eta_hist"][:it]
    return out


FILTERS = {"kron": 0, "classical": 1}


def stat(X: np.ndarray, UA: np.ndarray, UB: np.ndarray, bank_a: np.ndarray,
         bank_b: np.ndarray, filter: str = "kron"):
    """Statistic T_v for one snapshot X (p x q) with the Kron-STAP projector
    (Eq. KronSTAP) or the classical one (Sec. 5); returns (T, cond)."""
    X, UA, UB, ba, bb = map(_c128, (X, UA, UB, bank_a, bank_b))
    p, q = X.shape
    V = ba.shape[0]
    T = np.zeros(V)
    cond = np.zeros(V)
    _load().oracle_stat(_ptr(X), _ptr(UA), _ptr(UB), p, q, UA.shape[1], UB.shape[1], _ptr(ba),
                        _ptr(bb), V, _ptr(T), _ptr(cond), FILTERS[filter])
    return T, cond


def kstap_cells(Y: np.ndarray, q: int, r_a: int, r_b: int, ring_r: int, ring_a: int,
                guard_r: int, guard_a: int, bank_a: np.ndarray, bank_b: np.ndarray, tau: float,
                cells: Optional[np.ndarray] = None, eps: float = DEFAULT_EPS,
                max_iter: int = DEFAULT_MAX_ITER, want_T_all: bool = True,
                want_proj: bool = True, nthreads: int = 0,
                filter: str = "kron") -> Dict[str, np.ndarray]:
    """Whole per-cell Kron-STAP (O1-O7) on the listed cells of one frame.

    Y is (p, H_in, W_in) complex64; cells are flattened r * W + c indices of
    the H x W cell grid (all cells if None).
    """
    Y = np.ascontiguousarray(Y, dtype=np.complex64)
    p, H_in, W_in = Y.shape
    H = H_in - 2 * ring_r
    W = W_in - 2 * ring_a - q + 1
    if cells is None:
        cells = np.arange(H * W, dtype=np.int64)
    cells = np.ascontiguousarray(cells, dtype=np.int64)
    k = len(cells)
    ba = np.ascontiguousarray(bank_a, dtype=np.complex64)
    bb = np.ascontiguousarray(bank_b, dtype=np.complex64)
    V = ba.shape[0]
    out = dict(Tmax=np.zeros(k), vidx=np.zeros(k, np.int32), map=np.zeros(k, np.uint8),
               lamA=np.zeros((k, r_a)), lamB=np.zeros((k, r_b)), gapB=np.zeros(k),
               iters=np.zeros(k, np.int32), eta=np.zeros(k))
    out["T_all"] = np.zeros((k, V)) if want_T_all else None
    out["cond"] = np.zeros((k, V)) if want_T_all else None
    out["PA"] = np.zeros((k, p, p), np.complex128) if want_proj else None
    out["PB"] = np.zeros((k, q, q), np.complex128) if want_proj else None
    rc = _load().oracle_kstap_cells(
        _ptr(Y), p, H_in, W_in, q, r_a, r_b, ring_r, ring_a, guard_r, guard_a, float(eps),
        int(max_iter), _ptr(ba), _ptr(bb), V, float(tau), _ptr(cells), k, _ptr(out["T_all"]),
        _ptr(out["Tmax"]), _ptr(out["vidx"]), _ptr(out["map"]), _ptr(out["cond"]),
        _ptr(out["PA"]), _ptr(out["PB"]), _ptr(out["lamA"]), _ptr(out["lamB"]),
        _ptr(out["gapB"]), _ptr(out["iters"]), _ptr(out["eta"]), int(nthreads), FILTERS[filter])
    if rc != 0:
        raise ValueError("oracle_kstap_cells: bad arguments")
    out["cells"] = cells
    return out


def run_workload(frame, cells=None, **kw) -> Dict[str, np.ndarray]:
    """kstap_cells on a gen.Frame with its workload's parameters."""
    wl = frame.wl
    return kstap_cells(frame.Y, wl.q, wl.r_a, wl.r_b, wl.ring_r, wl.ring_a, wl.guard_r,
                       wl.guard_a, frame.bank_a, frame.bank_b, wl.tau, cells=cells, **kw)
