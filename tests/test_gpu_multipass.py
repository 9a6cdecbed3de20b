"""Stacked passes on the GPU (needs a GPU): K = 2 registered passes of a
3-channel array stacked as p = 6 channels, fitted with spatial rank r_a <= 2
(the stacked clutter spans one spatial direction per pass, Sec. 3), and the
noncoherent change map of Sec. 8.  Parity is element by element against the
FP64 oracle on the same seeded frames."""
import dataclasses

import numpy as np
import pytest

import gen
import oracle
from gpu_common import compare, projector

pytestmark = pytest.mark.gpu

K_PASSES = 2


def _frame(name, H, W, seed_shift=0, **kw):
    wl = dataclasses.replace(gen.WORKLOADS[name].with_size(H, W), **kw)
    if seed_shift:
        wl = dataclasses.replace(wl, seed=wl.seed + seed_shift)
    return gen.make_multipass_frame(wl, K=K_PASSES)


def _run(f, r_a, r_b=None, T_all=True):
    import torch
    from paper_1604_03622_b300.runner import KStap
    wl = f.wl
    ks = KStap(K_PASSES * wl.p, wl.q, r_a, r_b or wl.r_b, wl.ring_r, wl.ring_a, wl.guard_r,
               wl.guard_a, wl.tau, f.bank_a, f.bank_b)
    out = ks.run(torch.from_numpy(f.Y).cuda(), T_all=T_all)
    torch.cuda.synchronize()
    res = {k: v.cpu().numpy() for k, v in out.items() if k != "factors"}
    ks.close()
    return res


def _oracle(f, r_a, r_b=None, cells=None):
    wl = f.wl
    return oracle.kstap_cells(f.Y, wl.q, r_a, r_b or wl.r_b, wl.ring_r, wl.ring_a, wl.guard_r,
                              wl.guard_a, f.bank_a, f.bank_b, wl.tau, cells=cells)


# (workload, H, W, r_a, r_b): ragged rows (W not a multiple of the 32-cell
# moments tile or the 8-cell warp tile), both window lengths, both spatial ranks
CASES = [
    ("small64", 20, 43, 2, 2),
    ("frame1024", 12, 37, 2, 3),
    ("small64", 9, 27, 1, 2),
    ("frame1024", 7, 21, 2, 1),
    ("frame1024", 6, 19, 2, 4),
]


@pytest.mark.parametrize("name,H,W,r_a,r_b", CASES)
def test_stacked_pass_parity(name, H, W, r_a, r_b):
    f = _frame(name, H, W, r_b=r_b)        # clutter of temporal rank r_b
    ref = _oracle(f, r_a, r_b)
    gpu = _run(f, r_a, r_b)
    cells = np.arange(H * W)
    rep = compare(gpu, ref, cells, f.wl.tau)
    # projectors of the two factors (Eq. KronSTAP) and the trace-normalised
    # eigenvalues
    # U_A has orthonormal columns (a Jacobi rotation that lost |e^{i phi}| = 1
    # on a subnormal |b|^2 once broke this on cells near a strong target)
    UA = gpu["UA"].astype(np.complex128)
    gram = np.einsum("kim,kin->kmn", UA.conj(), UA)
    assert np.abs(gram - np.eye(r_a)).max() < 1e-5
    PA = projector(gpu["UA"])
    PB = projector(gpu["UB_hi"].astype(np.complex128) + gpu["UB_lo"])
    assert np.abs(PA - ref["PA"]).max() < 1e-4
    assert np.abs(PB - ref["PB"]).max() < 1e-7
    np.testing.assert_allclose(gpu["lamA"], ref["lamA"], rtol=1e-4)
    np.testing.assert_allclose(gpu["lamB"], ref["lamB"], rtol=1e-4)
    # eta of Alg. 2 from the closed form eta^2 = 1 - a^H M a / (|a|^2 tr M) with M
    # accumulated in single precision: the relative error of the ratio
    # (~1e-6) over eta^2 (>= 2.5e-3 here) bounds eta's relative error by ~2e-4
    np.testing.assert_allclose(gpu["eta"], ref["eta"], rtol=2e-4, atol=1e-6)
    print(name, H, W, r_a, r_b, rep)


def test_spatial_projector_rank_two():
    """With r_a = 2 the fitted U_A spans both passes: its projector agrees with
    the oracle's P_A (Eq. KronSTAP) and is idempotent of trace 2."""
    import torch
    from paper_1604_03622_b300.runner import KStap
    f = _frame("small64", 8, 24)
    wl = f.wl
    ks = KStap(6, wl.q, 2, wl.r_b, wl.ring_r, wl.ring_a, wl.guard_r, wl.guard_a, wl.tau,
               f.bank_a, f.bank_b)
    out = ks.run(torch.from_numpy(f.Y).cuda())
    UA = out["UA"].cpu().numpy().astype(np.complex128)      # (cells, 6, 2)
    ks.close()
    ref = _oracle(f, 2)
    PA = np.einsum("kim,kjm->kij", UA, UA.conj())
    assert np.abs(np.einsum("kii->k", PA).real - 2).max() < 1e-4
    assert np.abs(PA - ref["PA"]).max() < 1e-3


def test_change_map():
    """Per-pass maxima and the change map from the stacked T_all: bit-exact
    against numpy on the same T_all, within the statistic's tolerance of the
    oracle, and of the sign that the pass holding each clear target implies."""
    import torch
    import paper_1604_03622_b300 as K
    f = _frame("frame1024", 16, 40, n_targets=6, snr_db=(25.0, 25.0))
    wl = f.wl
    gpu = _run(f, 2)
    T_all = torch.from_numpy(gpu["T_all"]).cuda()
    Tk, ch = K.kstap_change_map(T_all, wl.V, K_PASSES)
    torch.cuda.synchronize()
    Tk, ch = Tk.cpu().numpy(), ch.cpu().numpy()
    per = gpu["T_all"].reshape(-1, K_PASSES, wl.V).max(axis=2).T
    assert np.array_equal(Tk, per)
    assert np.array_equal(ch, per[-1] - per[0])
    ref = _oracle(f, 2)
    rper = ref["T_all"].reshape(-1, K_PASSES, wl.V).max(axis=2).T
    assert (np.abs(Tk - rper) / np.maximum(rper, 1.0)).max() < 1e-4
    clear = 0
    for kk, r, c, v, beta in f.targets:
        cell = r * wl.W + c
        if rper[kk, cell] > 4 * wl.tau and rper[1 - kk, cell] < wl.tau:
            clear += 1
            assert np.sign(ch[cell]) == (1 if kk == K_PASSES - 1 else -1)
    assert clear >= 1
    # the per-pass maxima alone (change = NULL), on the default stream
    ncell = T_all.shape[0]
    Tk2 = torch.empty(K_PASSES, ncell, device=T_all.device)
    torch.cuda.synchronize()
    st = K.lib().kstap_change_map(T_all.data_ptr(), ncell, wl.V, K_PASSES, Tk2.data_ptr(), None,
                                  None)
    assert st == K.KSTAP_OK
    torch.cuda.synchronize()
    assert np.array_equal(Tk2.cpu().numpy(), per)


def test_stacked_pass_all_zero_frame():
    """Y = 0 on both passes: every statistic is 0, every cell finite."""
    f = _frame("small64", 6, 20)
    f = dataclasses.replace(f, Y=np.zeros_like(f.Y))
    gpu = _run(f, 2)
    assert (gpu["T_all"] == 0).all() and (gpu["Tmax"] == 0).all()
    assert (gpu["vidx"] == 0).all()
    assert np.isfinite(gpu["eta"]).all()


def test_stacked_pass_nonfinite_sample():
    """A NaN in one pass flags exactly the cells whose box holds it."""
    f = _frame("small64", 12, 30)
    Y = f.Y.copy()
    Y[4, 6, 20] = complex(np.nan, 0.0)          # pass 1, channel 1
    f = dataclasses.replace(f, Y=Y)
    gpu = _run(f, 2)
    wl = f.wl
    flag = np.zeros((wl.H, wl.W), bool)
    r0, r1 = max(0, 6 - 2 * wl.ring_r), min(wl.H - 1, 6)
    c0, c1 = max(0, 20 - (2 * wl.ring_a + wl.q - 1)), min(wl.W - 1, 20)
    flag[r0:r1 + 1, c0:c1 + 1] = True
    flag = flag.ravel()
    assert np.isnan(gpu["Tmax"][flag]).all() and (gpu["vidx"][flag] == -1).all()
    ok = np.nonzero(~flag)[0]
    assert len(ok) > 0
    ref = _oracle(f, 2, cells=ok)
    compare(gpu, ref, ok, wl.tau)


def test_stacked_pass_batch_strips_and_serving():
    """The stacked-pass context on the batch, strip and serving paths: a batch
    of uneven frames is bit-identical to the frames run one by one; a budget
    a third of the whole workspace runs the frame as row strips (their own
    fixed-point scale: equal to the unsplit frame to 1e-4); a served frame
    equals the frame run alone."""
    import torch
    import paper_1604_03622_b300 as K
    from paper_1604_03622_b300.runner import KStap
    from gpu_common import t_err
    from test_gpu_serving import _served
    sizes = [(9, 30), (1, 1), (14, 17)]
    frames = [_frame("frame1024", H, W, seed_shift=k) for k, (H, W) in enumerate(sizes)]
    f0 = frames[0]
    wl = f0.wl
    mk = lambda **kw: KStap(6, wl.q, 2, wl.r_b, wl.ring_r, wl.ring_a, wl.guard_r, wl.guard_a,
                            wl.tau, f0.bank_a, f0.bank_b, **kw)
    keys = ("Tmax", "vidx", "map", "UA", "UB_hi", "UB_lo", "T_all", "lamA", "eta", "iters")
    ks = mk()
    Ys = [torch.from_numpy(f.Y).cuda() for f in frames]
    alone = [{k: v.cpu().numpy() for k, v in ks.run(Y, T_all=True).items() if k in keys}
             for Y in Ys]
    bufs = [ks.alloc_outputs(Y.shape[1], Y.shape[2], T_all=True) for Y in Ys]
    K.kstap_run_batch(ks.ctx, [ks.frame_desc(Y, b) for Y, b in zip(Ys, bufs)])
    torch.cuda.synchronize()
    for r, b in zip(alone, bufs):
        for k in keys:
            assert np.array_equal(b[k].cpu().numpy(), r[k]), k
    tk = K.kstap_submit(ks.ctx, Ys[2], Ys[2].shape[1], Ys[2].shape[2])
    res = K.kstap_poll(ks.ctx, tk, timeout_us=-1)
    served = _served(K, ks, Ys[2], res)
    for k in ("Tmax", "vidx", "map"):
        assert np.array_equal(served[k], alone[2][k]), k
    K.kstap_release(ks.ctx, tk)
    ks.close()
    # row strips under a small budget
    big = _frame("frame1024", 41, 33, seed_shift=5)
    prm = K.make_params(6, wl.q, 2, wl.r_b, wl.ring_r, wl.ring_a, wl.guard_r, wl.guard_a, wl.tau)
    whole = K.kstap_workspace_bytes(prm, big.wl.H_in, big.wl.W_in)
    Y = torch.from_numpy(big.Y).cuda()
    ks0 = mk()
    ref = ks0.run(Y, T_all=True)["T_all"].cpu().numpy()
    ks0.close()
    ks = mk(hbm_budget_bytes=whole // 3)
    got = ks.run(Y, T_all=True)["T_all"].cpu().numpy()
    ks.close()
    assert t_err(got, ref.astype(np.float64)).max() <= 1e-4


def test_change_map_three_passes_and_flagged_cells():
    """kstap_change_map for K = 3 passes on a synthetic T_all: per-pass maxima
    bit-exact against numpy, change = last minus first pass, and a flagged
    cell (T_all NaN) stays NaN."""
    import torch
    import paper_1604_03622_b300 as K
    rng = np.random.default_rng(31)
    ncell, V, KP = 1000, 7, 3
    T = rng.exponential(size=(ncell, KP * V)).astype(np.float32)
    T[17] = np.nan
    Tk, ch = K.kstap_change_map(torch.from_numpy(T).cuda(), V, KP)
    torch.cuda.synchronize()
    Tk, ch = Tk.cpu().numpy(), ch.cpu().numpy()
    ok = np.ones(ncell, bool)
    ok[17] = False
    per = T.reshape(ncell, KP, V).max(axis=2).T
    assert np.array_equal(Tk[:, ok], per[:, ok])
    assert np.array_equal(ch[ok], per[-1, ok] - per[0, ok])
    assert np.isnan(Tk[:, 17]).all() and np.isnan(ch[17])
    with pytest.raises(ValueError):
        K.kstap_change_map(torch.from_numpy(T).cuda(), V + 1, KP)


def test_stacked_pass_full_size_frame_sampled():
    """The two-pass 1024 x 1024 frame of the bench's stacked-pass leg, run
    whole; all 2V velocities compared on every target cell and 512 random
    cells."""
    import torch
    from gpu_common import run_sampled
    from paper_1604_03622_b300.runner import KStap
    f = _frame("frame1024", 1024, 1024)
    wl = f.wl
    tcells = [r * wl.W + c for _, r, c, _, _ in f.targets]
    cells = np.unique(np.concatenate([tcells, gen.random_cells(wl, 512, seed=10)]).astype(np.int64))
    ks = KStap(K_PASSES * wl.p, wl.q, 2, wl.r_b, wl.ring_r, wl.ring_a, wl.guard_r, wl.guard_a,
               wl.tau, f.bank_a, f.bank_b)
    gpu = run_sampled(ks, torch.from_numpy(f.Y).cuda(), cells)
    ks.close()
    ref = _oracle(f, 2, cells=cells)
    rep = compare(gpu, ref, np.arange(len(cells)), wl.tau)
    print(rep)
