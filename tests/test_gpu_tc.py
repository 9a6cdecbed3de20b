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


def test_tc_batch_and_graph_bit_identical_to_per_frame():
    """Batches and CUDA graphs of the tensor-core route reproduce the per-frame
    calls bit for bit, whatever the launch tuning (no atomics in value paths;
    the near-blind queue order does not change any value)."""
    import torch
    import paper_1604_03622_b300 as K
    from paper_1604_03622_b300.runner import KStap
    keys = ("Tmax", "vidx", "map", "T_all", "UB_hi")
    groups = []
    for name, sizes, seed0 in (("frame1024", [(7, 40), (33, 29), (1, 1), (20, 70)], 0),
                               ("precision2048", [(6, 40), (11, 17)], 7)):
        base = gen.WORKLOADS[name]
        fr = [gen.make_frame(base.with_size(H, W), seed=base.seed + 300 + seed0 + k)
              for k, (H, W) in enumerate(sizes)]
        ks = KStap.from_workload(fr[0].wl, fr[0].bank_a, fr[0].bank_b, precision="fp16x3")
        Ys = [torch.from_numpy(f.Y).cuda() for f in fr]
        ref = [{k: v.cpu().numpy() for k, v in ks.run(Y, T_all=True).items() if k in keys}
               for Y in Ys]
        groups.append((ks, Ys, ref))
    for ks, Ys, ref in groups:
        for waves, tc in ((1, 16), (16, 0)):
            K.kstap_set_tuning(ks.ctx, waves, tc)
            bufs = [ks.alloc_outputs(Y.shape[1], Y.shape[2], T_all=True) for Y in Ys]
            K.kstap_run_batch(ks.ctx, [ks.frame_desc(Y, b) for Y, b in zip(Ys, bufs)])
            torch.cuda.synchronize()
            for r, b in zip(ref, bufs):
                for k in keys:
                    assert np.array_equal(b[k].cpu().numpy(), r[k]), (waves, tc, k)
    bufs = [[ks.alloc_outputs(Y.shape[1], Y.shape[2], T_all=True) for Y in Ys]
            for ks, Ys, _ in groups]
    descs = [[ks.frame_desc(Y, b) for Y, b in zip(Ys, bg)]
             for (ks, Ys, _), bg in zip(groups, bufs)]
    graph = K.kstap_graph_create([g[0].ctx for g in groups], descs)
    K.kstap_graph_launch(graph, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    for (ks, Ys, ref), bg in zip(groups, bufs):
        for r, b in zip(ref, bg):
            for k in keys:
                assert np.array_equal(b[k].cpu().numpy(), r[k]), k
    K.kstap_graph_destroy(graph)
    for ks, _, _ in groups:
        K.kstap_device_status(ks.ctx)
        ks.close()
