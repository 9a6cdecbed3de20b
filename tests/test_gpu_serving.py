"""Serving loop (kstap_submit / kstap_poll / kstap_release) on a GPU.

Every served result must be bit-identical to the same frame run alone through
kstap_fit_project + kstap_detect, whatever it was batched with; the HBM
budget must bound admission and refuse frames that can never fit.
"""
import numpy as np
import pytest

import gen

pytestmark = pytest.mark.gpu


def _served(K, ks, Y, res):
    """Copy the library-owned device results of one request to numpy."""
    import torch
    n = res.H * res.W
    torch.cuda.synchronize()
    return {name: _wrap(ptr, n, dt).clone().cpu().numpy()
            for name, ptr, dt in (("Tmax", res.Tmax, torch.float32),
                                  ("vidx", res.vidx, torch.int32),
                                  ("map", res.map, torch.uint8))}


def _wrap(ptr, n, dt):
    """A torch view of library-owned device memory (read once, then copied)."""
    import torch
    return torch.as_tensor(_DevArray(ptr, n, dt), device="cuda")


class _DevArray:
    def __init__(self, ptr, n, dt):
        import torch
        typestr = {torch.float32: "<f4", torch.int32: "<i4", torch.uint8: "|u1"}[dt]
        self.__cuda_array_interface__ = dict(shape=(n,), typestr=typestr, data=(ptr, False),
                                             version=3)


@pytest.mark.parametrize("precision", ["fp32", "fp16x3"])
def test_served_results_equal_alone_and_in_the_mix(precision):
    import torch
    import paper_1604_03622_b300 as K
    from paper_1604_03622_b300.runner import KStap
    base = gen.WORKLOADS["frame1024"]
    sizes = [(40, 70), (13, 29), (64, 33), (7, 7), (50, 90), (21, 61)]
    frames = [gen.make_frame(base.with_size(H, W), seed=base.seed + 500 + k)
              for k, (H, W) in enumerate(sizes)]
    ks = KStap.from_workload(frames[0].wl, frames[0].bank_a, frames[0].bank_b,
                             precision=precision)
    Ys = [torch.from_numpy(f.Y).cuda() for f in frames]
    alone = []
    for Y in Ys:
        b = ks.run(Y)
        alone.append({k: b[k].cpu().numpy() for k in ("Tmax", "vidx", "map")})
    K.kstap_serve_config(ks.ctx, 4, 2)
    host = [torch.from_numpy(f.Y).pin_memory() for f in frames]
    tickets = []
    for k, (Y, Yh) in enumerate(zip(Ys, host)):          # alternate device / host frames
        if k % 2:
            tickets.append(K.kstap_submit(ks.ctx, Yh, Yh.shape[1], Yh.shape[2], on_host=True))
        else:
            tickets.append(K.kstap_submit(ks.ctx, Y, Y.shape[1], Y.shape[2]))
    for k, tk in enumerate(tickets):
        r = K.kstap_poll(ks.ctx, tk, timeout_us=-1)
        assert r.H * r.W == frames[k].wl.cells
        assert r.t_submit_us <= r.t_admit_us <= r.t_done_us
        got = _served(K, ks, Ys[k], r)
        for key in ("Tmax", "vidx", "map"):
            assert np.array_equal(got[key], alone[k][key]), (k, key)
        K.kstap_release(ks.ctx, tk)
    with pytest.raises(K.KstapError, match="ENOTFOUND"):
        K.kstap_release(ks.ctx, tickets[0])
    ks.close()


def test_budget_bounds_admission_and_refuses_oversized_frames():
    import torch
    import paper_1604_03622_b300 as K
    from paper_1604_03622_b300.runner import KStap
    base = gen.WORKLOADS["small64"]
    f_small = gen.make_frame(base.with_size(30, 30))
    one = K.kstap_workspace_bytes(
        K.make_params(3, 8, 1, 2, base.ring_r, base.ring_a, base.guard_r, base.guard_a, 1.0),
        f_small.wl.H_in, f_small.wl.W_in)
    budget = int(2.5 * (one + 200_000))          # room for about two frames at a time
    ks = KStap.from_workload(f_small.wl, f_small.bank_a, f_small.bank_b,
                             hbm_budget_bytes=budget)
    Y = torch.from_numpy(f_small.Y).cuda()
    ref = ks.run(Y)["Tmax"].cpu().numpy()
    tks = [K.kstap_submit(ks.ctx, Y, Y.shape[1], Y.shape[2]) for _ in range(6)]
    res = [K.kstap_poll(ks.ctx, t, timeout_us=-1) for t in tks]
    for t, r in zip(tks, res):
        assert np.array_equal(_served(K, ks, Y, r)["Tmax"], ref)
        K.kstap_release(ks.ctx, t)
    # a tall frame is served as row strips within the budget ...
    tall = gen.make_frame(base.with_size(160, 30))
    Yt = torch.from_numpy(tall.Y).cuda()
    tk = K.kstap_submit(ks.ctx, Yt, Yt.shape[1], Yt.shape[2])
    r = K.kstap_poll(ks.ctx, tk, timeout_us=-1)
    assert r.H == 160 and np.isfinite(_served(K, ks, Yt, r)["Tmax"]).all()
    K.kstap_release(ks.ctx, tk)
    # ... but a frame so wide that even a 4-row strip exceeds it is refused
    wide = gen.make_frame(base.with_size(4, 20000))
    Yw = torch.from_numpy(wide.Y).cuda()
    with pytest.raises(K.KstapError, match="ENOMEM"):
        K.kstap_submit(ks.ctx, Yw, Yw.shape[1], Yw.shape[2])
    ks.close()


def test_strips_under_a_small_budget_match_oracle():
    """A budget too small for the whole workspace: kstap_fit_project runs the
    frame as row strips, and the server admits strips one by one.  Strips take
    their own fixed-point scale, so results agree with the unsplit frame to
    rounding: checked against the oracle at the parity tolerance."""
    import torch
    import oracle
    import paper_1604_03622_b300 as K
    from paper_1604_03622_b300.runner import KStap
    from gpu_common import compare, t_err
    base = gen.WORKLOADS["frame1024"]
    f = gen.make_frame(base.with_size(61, 45), seed=base.seed + 900)
    wl = f.wl
    whole = K.kstap_workspace_bytes(K.make_params(3, 16, 1, 3, wl.ring_r, wl.ring_a, wl.guard_r,
                                                  wl.guard_a, wl.tau), wl.H_in, wl.W_in)
    Y = torch.from_numpy(f.Y).cuda()
    ks0 = KStap.from_workload(wl, f.bank_a, f.bank_b)
    ref = {k: v.cpu().numpy() for k, v in ks0.run(Y, T_all=True).items() if k != "factors"}
    ks0.close()
    ks = KStap.from_workload(wl, f.bank_a, f.bank_b, hbm_budget_bytes=whole // 3)
    got = {k: v.cpu().numpy() for k, v in ks.run(Y, T_all=True).items() if k != "factors"}
    assert t_err(got["T_all"], ref["T_all"].astype(np.float64)).max() <= 1e-4
    o = oracle.run_workload(f, want_proj=False)
    compare(got, o, np.arange(wl.H * wl.W), wl.tau)
    tk = K.kstap_submit(ks.ctx, Y, Y.shape[1], Y.shape[2])
    r = K.kstap_poll(ks.ctx, tk, timeout_us=-1)
    served = _served(K, ks, Y, r)
    assert t_err(served["Tmax"], o["Tmax"]).max() <= 1e-4
    K.kstap_release(ks.ctx, tk)
    ks.close()
