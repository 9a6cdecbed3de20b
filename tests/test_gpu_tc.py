"""Tensor-core route of the statistic (KSTAP_FP16X3 / KSTAP_BF16X3) against the
FP64 oracle (needs a GPU).

The fit is the single-precision path's; only the velocity-bank contraction
runs on the tensor cores (tcgen05, hi + lo 16-bit splits, FP32 accumulation).
Bars: |T - T_ref| / max(T_ref, sigma^2) <= 2e-4 for FP16X3 (11 + 11 mantissa
bits per factor) and <= 1e-3 for BF16X3 (8 + 8 bits), the bound stated for
the 16-bit routes; maps outside the band, argmax where resolvable."""
import dataclasses

import numpy as np
import pytest

import gen
import oracle
from gpu_common import compare, run_gpu, t_err

pytestmark = pytest.mark.gpu

TOL = {"fp16x3": 2e-4, "bf16x3": 1e-3}


def _wl(name, H, W, **over):
    wl = gen.WORKLOADS[name].with_size(H, W)
    return dataclasses.replace(wl, **over) if over else wl


@pytest.mark.parametrize("precision", ["fp16x3", "bf16x3"])
@pytest.mark.parametrize("name,H,W,r_b", [("small64", 37, 45, 2), ("frame1024", 29, 70, 3),
                                          ("precision2048", 13, 40, 4),
                                          ("frame1024", 9, 37, 1), ("small64", 9, 37, 4)])
def test_tc_parity(precision, name, H, W, r_b):
    wl = _wl(name, H, W, r_b=r_b)
    f = gen.make_frame(wl)
    ref = oracle.run_workload(f)
    gpu = run_gpu(f, precision=precision)
    cells = np.arange(wl.H * wl.W)
    rep = compare(gpu, ref, cells, wl.tau, tol=TOL[precision])
    print(precision, name, H, W, r_b, rep)


def test_tc_factors_equal_fp32_route():
    """The precision switch changes only the statistic: the fitted factors are
    bit-identical, and T agrees with the FP32 route to the 16-bit bar."""
    wl = _wl("frame1024", 21, 50)
    f = gen.make_frame(wl)
    a = run_gpu(f)
    b = run_gpu(f, precision="fp16x3")
    for k in ("UA", "UB_hi", "UB_lo", "lamA", "lamB", "iters", "eta"):
        assert np.array_equal(a[k], b[k]), k
    assert t_err(b["T_all"], a["T_all"].astype(np.float64)).max() <= 2e-4


def test_tc_deterministic_and_status_clean():
    import torch
    import paper_1604_03622_b300 as K
    from paper_1604_03622_b300.runner import KStap
    wl = _wl("precision2048", 11, 50)
    f = gen.make_frame(wl)
    ks = KStap.from_workload(wl, f.bank_a, f.bank_b, precision="fp16x3")
    Y = torch.from_numpy(f.Y).cuda()
    o1 = {k: v.clone() for k, v in ks.run(Y, T_all=True).items() if k != "factors"}
    o2 = ks.run(Y, T_all=True)
    K.kstap_device_status(ks.ctx)
    for k, v in o1.items():
        assert torch.equal(v, o2[k]), k
    ks.close()


def test_tc_rejects_large_bank():
    import torch
    import paper_1604_03622_b300 as K
    from paper_1604_03622_b300.runner import KStap
    wl = _wl("frame1024", 9, 37)
    a, b = gen.steering_bank(wl.p, wl.q, 160)
    with pytest.raises(K.KstapError, match="EINVAL"):
        KStap.from_workload(wl, a, b, precision="fp16x3")
