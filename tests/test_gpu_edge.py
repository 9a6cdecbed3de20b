"""Edge cases of the CUDA path (needs a GPU): non-finite input samples, an
all-zero frame, the Alg. 2 iteration cap and the largest training box this
build accepts.  Every case checks either the oracle (FP64) or a property that
is fixed without one."""
import dataclasses

import numpy as np
import pytest

import gen
import oracle
from gpu_common import compare

pytestmark = pytest.mark.gpu


def _run(frame, T_all=True, **kw):
    """One fit + detect through the C ABI; returns host arrays and the fit report."""
    import torch
    import paper_1604_03622_b300 as K
    from paper_1604_03622_b300.runner import KStap
    ks = KStap.from_workload(frame.wl, frame.bank_a, frame.bank_b, **kw)
    out = ks.run(torch.from_numpy(frame.Y).cuda(), T_all=T_all)
    report = K.kstap_fit_report(ks.ctx)
    torch.cuda.synchronize()
    res = {k: v.cpu().numpy() for k, v in out.items() if k != "factors"}
    ks.close()
    return res, report


def _box_flags(wl, bad):
    """Cells whose box (rows r .. r + 2 ring_r, columns c .. c + 2 ring_a + q - 1
    of the input, any channel) contains one of the (channel, row, col) samples."""
    flag = np.zeros((wl.H, wl.W), bool)
    span_r, span_c = 2 * wl.ring_r, 2 * wl.ring_a + wl.q - 1
    for _, row, col in bad:
        r0, r1 = max(0, row - span_r), min(wl.H - 1, row)
        c0, c1 = max(0, col - span_c), min(wl.W - 1, col)
        if r0 <= r1 and c0 <= c1:
            flag[r0:r1 + 1, c0:c1 + 1] = True
    return flag.ravel()


def test_nonfinite_samples_flag_their_cells_only():
    wl = gen.WORKLOADS["small64"].with_size(40, 56)
    f = gen.make_frame(wl)
    Y = f.Y.copy()
    bad = [(1, 20, 30), (0, 5, 70), (2, 45, 10)]
    Y[1, 20, 30] = complex(np.nan, 0.5)
    Y[0, 5, 70] = complex(1.0, np.inf)
    Y[2, 45, 10] = complex(-np.inf, 0.0)
    f = dataclasses.replace(f, Y=Y)
    gpu, (nonconv, nonfinite, _) = _run(f)
    flag = _box_flags(wl, bad)
    assert 0 < flag.sum() < flag.size
    assert nonfinite == int(flag.sum())
    # flagged cells: Tmax NaN, vidx -1, map 0, T_all NaN, iters -1, eta NaN
    assert np.isnan(gpu["Tmax"][flag]).all()
    assert (gpu["vidx"][flag] == -1).all()
    assert (gpu["map"][flag] == 0).all()
    assert np.isnan(gpu["T_all"][flag]).all()
    assert (gpu["iters"][flag] == -1).all()
    assert np.isnan(gpu["eta"][flag]).all()
    # every other cell is finite and matches the oracle on the same frame
    ok = np.nonzero(~flag)[0]
    assert np.isfinite(gpu["T_all"][ok]).all() and (gpu["vidx"][ok] >= 0).all()
    assert (gpu["iters"][ok] >= 1).all()
    ref = oracle.run_workload(f, cells=ok)
    compare({k: v for k, v in gpu.items()}, ref, ok, wl.tau)


def test_all_zero_frame():
    """Y = 0: no clutter, no signal.  Every statistic is 0 (|d^H P x|^2 = 0 with
    d^H P d > 0), so Tmax = 0, vidx = 0 (lowest index of the tie), map = 0."""
    wl = gen.WORKLOADS["frame1024"].with_size(9, 40)
    f = gen.make_frame(wl)
    f = dataclasses.replace(f, Y=np.zeros_like(f.Y))
    gpu, (nonconv, nonfinite, _) = _run(f)
    assert nonfinite == 0
    assert (gpu["Tmax"] == 0).all() and (gpu["T_all"] == 0).all()
    assert (gpu["vidx"] == 0).all() and (gpu["map"] == 0).all()
    assert np.isfinite(gpu["lamA"]).all() and np.isfinite(gpu["eta"]).all()


def test_iteration_cap_reported():
    """max_iter = 1 stops Alg. 2 after one update: the report counts the cells
    that had not met eps, and iters never exceeds the cap."""
    wl = gen.WORKLOADS["small64"].with_size(16, 24)
    f = gen.make_frame(wl)
    gpu, (nonconv, nonfinite, _) = _run(f, max_iter=1)
    assert gpu["iters"].max() == 1
    assert 0 < nonconv <= wl.H * wl.W
    assert nonfinite == 0
    # with the default cap every cell converges and the report is clean
    gpu, (nonconv, _, _) = _run(f, T_all=False)
    assert nonconv == 0 and gpu["iters"].max() < 64


def test_largest_training_box_q32():
    """ring_r = 12, ring_a = 19 (25 x 39 box, the largest with <= 1024 samples
    at this height) at q = 32: the largest shared-memory footprint of the
    moments and B passes.  Full parity against the oracle."""
    wl = dataclasses.replace(gen.WORKLOADS["precision2048"].with_size(5, 21), ring_r=12,
                             ring_a=19, guard_r=1, guard_a=2, n_targets=2)
    f = gen.make_frame(wl)
    ref = oracle.run_workload(f)
    gpu, (nonconv, nonfinite, _) = _run(f)
    assert nonconv == 0 and nonfinite == 0
    compare(gpu, ref, np.arange(wl.H * wl.W), wl.tau)
