"""Batched path (kstap_run_batch, CUDA graph, autotuner) against the per-frame
path and the oracle (needs a GPU).

A batch runs the same kernels with the same tiling of each frame, so every
output must be bit-identical to the per-frame calls, whatever the batch
composition and the launch tuning.
"""
import numpy as np
import pytest

import gen
import oracle
from gpu_common import compare

pytestmark = pytest.mark.gpu

KEYS = ("Tmax", "vidx", "map", "UA", "UB_hi", "UB_lo", "T_all", "lamB", "eta", "iters")


def _frames(name, sizes, seed0=0):
    base = gen.WORKLOADS[name]
    return [gen.make_frame(base.with_size(H, W), seed=base.seed + 100 + seed0 + k)
            for k, (H, W) in enumerate(sizes)]


def _np(b):
    return {k: b[k].cpu().numpy() for k in KEYS if k in b}


def test_batch_bit_identical_to_per_frame_and_tuning_invariant():
    import torch
    import paper_1604_03622_b300 as K
    from paper_1604_03622_b300.runner import KStap
    frames = _frames("frame1024", [(7, 40), (33, 29), (1, 1), (64, 70), (12, 5)])
    ks = KStap.from_workload(frames[0].wl, frames[0].bank_a, frames[0].bank_b)
    Ys = [torch.from_numpy(f.Y).cuda() for f in frames]
    ref = []
    for Y in Ys:
        ref.append(_np(ks.run(Y, T_all=True)))
    for waves, tc in ((4, 0), (1, 16), (16, 32), (64, 0)):
        K.kstap_set_tuning(ks.ctx, waves, tc)
        bufs = [ks.alloc_outputs(Y.shape[1], Y.shape[2], T_all=True) for Y in Ys]
        K.kstap_run_batch(ks.ctx, [ks.frame_desc(Y, b) for Y, b in zip(Ys, bufs)])
        torch.cuda.synchronize()
        for r, b in zip(ref, bufs):
            got = _np(b)
            for k in KEYS:
                assert np.array_equal(got[k], r[k]), (waves, tc, k)
    ks.close()


def test_graph_of_two_classes_matches_per_frame_and_oracle():
    import torch
    import paper_1604_03622_b300 as K
    from paper_1604_03622_b300.runner import KStap
    fa = _frames("small64", [(20, 31), (9, 64)])
    fb = _frames("precision2048", [(6, 40), (11, 17)], seed0=7)
    ka = KStap.from_workload(fa[0].wl, fa[0].bank_a, fa[0].bank_b)
    kb = KStap.from_workload(fb[0].wl, fb[0].bank_a, fb[0].bank_b)
    groups = [(ka, fa), (kb, fb)]
    ref, Ys, bufs, descs = [], [], [], []
    for ks, fr in groups:
        Yg = [torch.from_numpy(f.Y).cuda() for f in fr]
        ref.append([_np(ks.run(Y, T_all=True)) for Y in Yg])
        bg = [ks.alloc_outputs(Y.shape[1], Y.shape[2], T_all=True) for Y in Yg]
        Ys.append(Yg)
        bufs.append(bg)
        descs.append([ks.frame_desc(Y, b) for Y, b in zip(Yg, bg)])
    graph = K.kstap_graph_create([ka.ctx, kb.ctx], descs)
    for _ in range(2):                       # replay twice
        K.kstap_graph_launch(graph, torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        for g in range(2):
            for r, b in zip(ref[g], bufs[g]):
                got = _np(b)
                for k in KEYS:
                    assert np.array_equal(got[k], r[k]), (g, k)
    K.kstap_graph_destroy(graph)
    # and the graph's results against the oracle
    for (ks, fr), bg in zip(groups, bufs):
        for f, b in zip(fr, bg):
            o = oracle.run_workload(f, want_proj=False)
            compare(_np(b), o, np.arange(f.wl.H * f.wl.W), f.wl.tau)
    ka.close()
    kb.close()


def test_autotune_picks_a_candidate_and_keeps_results():
    import torch
    import paper_1604_03622_b300 as K
    from paper_1604_03622_b300.runner import KStap
    frames = _frames("small64", [(40, 50), (17, 80), (64, 64)])
    ks = KStap.from_workload(frames[0].wl, frames[0].bank_a, frames[0].bank_b)
    Ys = [torch.from_numpy(f.Y).cuda() for f in frames]
    ref = [_np(ks.run(Y, T_all=True)) for Y in Ys]
    bufs = [ks.alloc_outputs(Y.shape[1], Y.shape[2], T_all=True) for Y in Ys]
    descs = [ks.frame_desc(Y, b) for Y, b in zip(Ys, bufs)]
    t = K.kstap_autotune(ks.ctx, descs, reps=2)
    assert t.waves in (1, 2, 4, 8, 16, 32, 64) and t.tc in (16, 32) and t.ms_per_batch > 0
    K.kstap_run_batch(ks.ctx, descs)
    torch.cuda.synchronize()
    for r, b in zip(ref, bufs):
        got = _np(b)
        for k in KEYS:
            assert np.array_equal(got[k], r[k]), k
    ks.close()


@pytest.mark.parametrize("name,sizes", [("small64", [(20, 45), (9, 70)]),
                                        ("frame1024", [(7, 40), (33, 29), (1, 1)]),
                                        ("precision2048", [(6, 40), (11, 17)])])
def test_recomputed_lags_bit_identical_to_lag_store(name, sizes):
    """lag_store = 0 (the B pass recomputes the exact lag sums from its frame
    tile, no store in the workspace) gives the same bits as the store, per
    frame and in a batch: the sums are exact integers either way."""
    import torch
    import paper_1604_03622_b300 as K
    from paper_1604_03622_b300.runner import KStap
    frames = _frames(name, sizes)
    ks = KStap.from_workload(frames[0].wl, frames[0].bank_a, frames[0].bank_b)
    Ys = [torch.from_numpy(f.Y).cuda() for f in frames]
    ref = [_np(ks.run(Y, T_all=True)) for Y in Ys]
    K.kstap_set_tuning(ks.ctx, 4, 0, lag_store=0)
    for r, Y in zip(ref, Ys):
        got = _np(ks.run(Y, T_all=True))
        for k in KEYS:
            assert np.array_equal(got[k], r[k]), ("per frame", k)
    bufs = [ks.alloc_outputs(Y.shape[1], Y.shape[2], T_all=True) for Y in Ys]
    K.kstap_run_batch(ks.ctx, [ks.frame_desc(Y, b) for Y, b in zip(Ys, bufs)])
    torch.cuda.synchronize()
    for r, b in zip(ref, bufs):
        got = _np(b)
        for k in KEYS:
            assert np.array_equal(got[k], r[k]), ("batch", k)
    ks.close()
