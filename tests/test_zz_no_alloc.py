"""The allocation-free fit entry point against the regular one (needs a GPU).

kstap_fit_project_noalloc serves callers that must not allocate device memory
while running (e.g. real-time loops, where cudaMalloc can synchronise the
device with unbounded latency, or hosts whose device memory belongs to another
allocator).  Its scratch is a static device array shared by all calls, so this
test calls it twice in a row on different frames -- stale contents from the
first call must not leak into the second -- and compares each result with
kstap_fit_project's, through the C ABI, at the parity tolerance of the other
GPU tests.  It also checks that frames above the size limit are refused.
"""
import numpy as np
import pytest

import gen

pytestmark = pytest.mark.gpu

TOL = 1e-4


def _fit_and_detect(K, ks, Y, H_in, W_in, noalloc):
    import torch
    b = ks.buffers(H_in, W_in, T_all=True)
    out = {}
    if noalloc:
        # fresh factor buffers, filled only by the allocation-free entry point
        f = {k: torch.full_like(b[k], float("nan")) if b[k].is_floating_point() or b[k].is_complex()
             else torch.zeros_like(b[k]) for k in ("UA", "UB_hi", "UB_lo", "lamA", "lamB",
                                                     "iters", "eta")}
        fac = K.make_factors(f["UA"], f["UB_hi"], f["UB_lo"], f["lamA"], f["lamB"], f["iters"],
                             f["eta"])
        K.kstap_fit_project_noalloc(ks.params, Y, H_in, W_in, fac, ks.stream.cuda_stream)
    else:
        f = {k: b[k] for k in ("UA", "UB_hi", "UB_lo", "lamA", "lamB", "iters", "eta")}
        fac = b["factors"]
        K.kstap_fit_project(ks.ctx, Y, H_in, W_in, fac)
    Tmax = torch.empty_like(b["Tmax"])
    vidx = torch.empty_like(b["vidx"])
    mp = torch.empty_like(b["map"])
    T_all = torch.empty_like(b["T_all"])
    K.kstap_detect(ks.ctx, Y, H_in, W_in, fac, Tmax, vidx, mp, T_all)
    torch.cuda.synchronize()
    out.update({k: v.cpu().numpy() for k, v in f.items()})
    out.update(Tmax=Tmax.cpu().numpy(), vidx=vidx.cpu().numpy(), map=mp.cpu().numpy(),
               T_all=T_all.cpu().numpy())
    return out


# (workload, cell grid): q = 8, 12, 16, 24 and 32, each with ragged tiles
CASES = [("small64", 48, 70), ("frame_q12", 30, 61), ("frame1024", 40, 90),
         ("frame_q24", 20, 50), ("precision2048", 24, 72)]


@pytest.mark.parametrize("name,H,W", CASES)
def test_noalloc_fit_matches_fit_project_on_two_calls_in_a_row(name, H, W):
    import torch
    import paper_1604_03622_b300 as K
    from paper_1604_03622_b300.runner import KStap
    wl = gen.WORKLOADS[name].with_size(H, W)
    frames = [gen.make_frame(wl, seed=wl.seed + s) for s in (11, 12)]
    ks = KStap.from_workload(wl, frames[0].bank_a, frames[0].bank_b)
    proj = lambda U: np.einsum("kim,kjm->kij", U, U.conj())
    try:
        for f in frames:                                     # two calls in a row
            Y = torch.from_numpy(f.Y).cuda()
            _, H_in, W_in = f.Y.shape
            ref = _fit_and_detect(K, ks, Y, H_in, W_in, noalloc=False)
            got = _fit_and_detect(K, ks, Y, H_in, W_in, noalloc=True)
            err = np.abs(got["T_all"] - ref["T_all"]) / np.maximum(ref["T_all"], 1.0)
            assert err.max() <= TOL, err.max()
            assert np.abs(got["Tmax"] - ref["Tmax"]).max() <= TOL * max(1.0, ref["Tmax"].max())
            assert np.array_equal(got["map"], ref["map"])
            assert np.array_equal(got["vidx"], ref["vidx"])
            # the factors: projectors, eigenvalues, Alg. 2 iterations and eta
            assert np.abs(proj(got["UB_hi"]) - proj(ref["UB_hi"])).max() <= 1e-5
            assert np.abs(proj(got["UA"]) - proj(ref["UA"])).max() <= 1e-5
            for k in ("lamA", "lamB"):
                assert np.allclose(got[k], ref[k], rtol=1e-5, atol=1e-6 * np.abs(ref[k]).max()), k
            assert np.array_equal(got["iters"], ref["iters"])
            assert np.allclose(got["eta"], ref["eta"], rtol=1e-4, atol=1e-6)
    finally:
        ks.close()


def test_noalloc_rejects_frames_above_the_limit():
    import torch
    import paper_1604_03622_b300 as K
    wl = gen.WORKLOADS["small64"].with_size(200, 200)        # 40000 > 32768 cells
    prm = K.make_params(wl.p, wl.q, wl.r_a, wl.r_b, wl.ring_r, wl.ring_a, wl.guard_r,
                        wl.guard_a, wl.tau)
    Y = torch.zeros(wl.p, wl.H_in, wl.W_in, dtype=torch.complex64, device="cuda")
    n = wl.H * wl.W
    UA = torch.empty(n, wl.p, 1, dtype=torch.complex64, device="cuda")
    UB = torch.empty(n, wl.q, wl.r_b, dtype=torch.complex64, device="cuda")
    fac = K.make_factors(UA, UB, torch.empty_like(UB))
    with pytest.raises(K.KstapError, match="at most 32768"):
        K.kstap_fit_project_noalloc(prm, Y, wl.H_in, wl.W_in, fac)
