"""The boundary's full (q, r_b) domain against the FP64 oracle (needs a GPU).

Beyond the configurations' q in {8, 16, 32} and r_b in {2, 3, 4}, the
library takes q in {12, 24} (a cell's q rows on a group of 16 or 32 lanes,
the lanes past q idle; the tensor-core bank pads its contraction to whole
K steps of 16) and any 1 <= r_b <= min(q - 1, 8) (Sec. 4's EIG_{r_b}; ranks
above 4 on the single-precision bank).  Every case is checked element by
element: T of
every cell and velocity within the route's bar, maps outside the band
around tau, argmax where resolvable, projectors and eigenvalues.
"""
import dataclasses

import numpy as np
import pytest

import gen
import oracle
from gpu_common import TOL_T, compare, projector, run_gpu, t_err

pytestmark = pytest.mark.gpu

TOL_TC = {"fp16x3": 2e-4, "bf16x3": 1e-3}


def _wl(name, H, W, **over):
    wl = gen.WORKLOADS[name].with_size(H, W)
    return dataclasses.replace(wl, **over) if over else wl


def _check_factors(gpu, ref, gap_floor=1e-6):
    PA = projector(gpu["UA"])
    PB = projector(gpu["UB_hi"].astype(np.complex128) + gpu["UB_lo"])
    assert np.abs(PA - ref["PA"]).max() < 1e-5
    ok = ref["gapB"] >= gap_floor     # the projector of an ill-gapped B is not pinned
    assert np.abs(PB - ref["PB"])[ok].max() < 1e-8
    np.testing.assert_allclose(gpu["lamA"], ref["lamA"], rtol=1e-5)
    np.testing.assert_allclose(gpu["lamB"][ok], ref["lamB"][ok], rtol=1e-4)


@pytest.mark.parametrize("name,H,W,r_b", [
    ("frame_q12", 37, 45, 3),    # q = 12: 16-lane groups, 4 idle lanes; ragged tiles
    ("frame_q12", 9, 70, 1),
    ("frame_q12", 11, 33, 4),
    ("frame_q24", 21, 40, 4),    # q = 24: 32-lane groups, 16-cell B tiles
    ("frame_q24", 9, 37, 2),
])
def test_parity_q12_q24(name, H, W, r_b):
    wl = _wl(name, H, W, r_b=r_b)
    f = gen.make_frame(wl)
    ref = oracle.run_workload(f)
    gpu = run_gpu(f)
    rep = compare(gpu, ref, np.arange(wl.H * wl.W), wl.tau)
    _check_factors(gpu, ref)
    print(name, H, W, r_b, rep)


@pytest.mark.parametrize("precision", ["fp16x3", "bf16x3"])
@pytest.mark.parametrize("name,H,W,r_b", [("frame_q12", 19, 41, 3), ("frame_q24", 13, 40, 4)])
def test_tensor_core_bank_q12_q24(precision, name, H, W, r_b):
    """q = 12 pads the bank GEMM's contraction from 24 to 32 (zero columns)."""
    wl = _wl(name, H, W, r_b=r_b)
    f = gen.make_frame(wl)
    ref = oracle.run_workload(f)
    gpu = run_gpu(f, precision=precision)
    rep = compare(gpu, ref, np.arange(wl.H * wl.W), wl.tau, tol=TOL_TC[precision])
    print(precision, name, r_b, rep)


@pytest.mark.parametrize("name,r_b", [
    ("small64", 5),       # q = 8
    ("frame_q12", 6),
    ("frame1024", 8),     # q = 16
    ("frame_q24", 7),
    ("precision2048", 5),
    ("precision2048", 8),
])
def test_parity_high_rank_b(name, r_b):
    """r_b > 4: the subspace iteration on r_b vectors (its r_b x r_b Gram,
    Cholesky and Ritz matrices spill from registers), with the block
    Rayleigh-Ritz path on min(q, r_b + 4) vectors for ill-gapped cells."""
    wl = _wl(name, 9, 37, r_b=r_b)
    f = gen.make_frame(wl)
    ref = oracle.run_workload(f)
    gpu = run_gpu(f)
    ok = ref["gapB"] >= 1e-6
    e = t_err(gpu["T_all"], ref["T_all"])
    assert e[ok].max() <= TOL_T, f"max T error {e[ok].max():.3e}"
    assert ok.mean() > 0.5, "the generator should give most cells a resolvable rank-r_b B"
    cells = np.nonzero(ok)[0]
    compare(gpu, {k: ref[k][ok] for k in ("T_all", "Tmax", "vidx", "map")}, cells, wl.tau)
    _check_factors(gpu, ref)
    print(name, r_b, "cells", len(ok), "gap >= 1e-6:", int(ok.sum()), "max err", e[ok].max())


def test_classical_filter_and_spatial_rank_two_at_q12():
    wl = _wl("frame_q12", 13, 29)
    f = gen.make_frame(wl)
    ref = oracle.run_workload(f, filter="classical")
    gpu = run_gpu(f, filter="classical")
    compare(gpu, ref, np.arange(wl.H * wl.W), wl.tau)
    wl2 = dataclasses.replace(wl, r_a=2)
    f2 = gen.make_frame(wl2)
    ref2 = oracle.run_workload(f2)
    gpu2 = run_gpu(f2)
    compare(gpu2, ref2, np.arange(wl2.H * wl2.W), wl2.tau)


@pytest.mark.parametrize("name,r_b", [("frame_q12", 3), ("frame_q24", 4), ("frame1024", 6)])
def test_recomputed_lags_and_batches_bit_identical(name, r_b):
    """The B pass that recomputes the lag sums (no lag store) and a batch of
    uneven frames give the per-frame results bit for bit."""
    import torch
    import paper_1604_03622_b300 as K
    from paper_1604_03622_b300.runner import KStap
    base = dataclasses.replace(gen.WORKLOADS[name], r_b=r_b)
    frames = [gen.make_frame(base.with_size(H, W), seed=base.seed + 300 + k)
              for k, (H, W) in enumerate([(7, 40), (19, 23), (1, 1)])]
    ks = KStap.from_workload(frames[0].wl, frames[0].bank_a, frames[0].bank_b)
    Ys = [torch.from_numpy(f.Y).cuda() for f in frames]
    keys = ("Tmax", "vidx", "map", "UA", "UB_hi", "UB_lo", "T_all", "lamB", "eta", "iters")
    ref = [{k: v.cpu().numpy() for k, v in ks.run(Y, T_all=True).items() if k in keys}
           for Y in Ys]
    K.kstap_set_tuning(ks.ctx, 4, 0, lag_store=0)
    for Y, r in zip(Ys, ref):
        got = ks.run(Y, T_all=True)
        for k in keys:
            assert np.array_equal(got[k].cpu().numpy(), r[k]), ("recompute", k)
    K.kstap_set_tuning(ks.ctx, 2, 0, lag_store=1)
    bufs = [ks.alloc_outputs(Y.shape[1], Y.shape[2], T_all=True) for Y in Ys]
    K.kstap_run_batch(ks.ctx, [ks.frame_desc(Y, b) for Y, b in zip(Ys, bufs)])
    torch.cuda.synchronize()
    for b, r in zip(bufs, ref):
        for k in keys:
            assert np.array_equal(b[k].cpu().numpy(), r[k]), ("batch", k)
    ks.close()
