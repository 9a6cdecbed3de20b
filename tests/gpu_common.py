"""Shared helpers of the GPU parity tests (test infrastructure)."""
import numpy as np

SIGMA2 = 1.0
TOL_T = 1e-4          # |T_gpu - T_ref| / max(T_ref, sigma^2), single-precision path


def run_gpu(frame, T_all=True, **kw):
    import torch
    from paper_1604_03622_b300.runner import KStap
    wl = frame.wl
    ks = KStap.from_workload(wl, frame.bank_a, frame.bank_b, **kw)
    Y = torch.from_numpy(frame.Y).cuda()
    out = ks.run(Y, T_all=T_all)
    torch.cuda.synchronize()
    res = {k: v.cpu().numpy() for k, v in out.items() if k != "factors"}
    ks.close()
    return res


def t_err(T_gpu, T_ref):
    return np.abs(T_gpu.astype(np.float64) - T_ref) / np.maximum(T_ref, SIGMA2)


def projector(U):
    return np.einsum("...im,...jm->...ij", U, U.conj())


def compare(gpu, ref, cells, tau, tol=TOL_T, check_all_T=True):
    """Element-wise parity of one run against the oracle on the listed cells."""
    k = np.asarray(cells)
    rep = {}
    if check_all_T:
        e = t_err(gpu["T_all"][k], ref["T_all"])
        rep["T_all_max_err"] = float(e.max())
        assert e.max() <= tol, f"T_all error {e.max():.3e} > {tol}"
    e = t_err(gpu["Tmax"][k], ref["Tmax"])
    rep["Tmax_max_err"] = float(e.max())
    assert e.max() <= tol, f"Tmax error {e.max():.3e}"
    # maps identical outside the band |Tmax_ref - tau| <= 2 tol max(tau, 1)
    band = np.abs(ref["Tmax"] - tau) <= 2 * tol * max(tau, 1.0)
    mism = (gpu["map"][k] != ref["map"]) & ~band
    assert not mism.any(), f"{mism.sum()} map mismatches outside the band"
    # argmax where the oracle's top-2 gap is resolvable
    if ref.get("T_all") is not None:
        srt = np.sort(ref["T_all"], axis=1)
        gap = srt[:, -1] - srt[:, -2]
        ok = gap > 2 * tol * np.maximum(srt[:, -1], 1.0)
        bad = (gpu["vidx"][k] != ref["vidx"]) & ok
        assert not bad.any(), f"{bad.sum()} argmax mismatches"
    return rep


def run_sampled(ks, Y, cells):
    """One fit + detect of device frame Y through context `ks` (a KStap); the
    statistic and the maps of the listed cells only, copied to the host (a
    full-size frame's T_all and factors are gigabytes)."""
    import torch
    out = ks.run(Y, T_all=True)
    idx = torch.from_numpy(np.asarray(cells, np.int64)).to(Y.device)
    res = {k: out[k][idx].cpu().numpy() for k in ("T_all", "Tmax", "vidx", "map")}
    torch.cuda.synchronize()
    return res
