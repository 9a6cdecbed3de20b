"""Convenience wrapper: torch-owned device buffers around one libkstap context.

Holds the per-frame output tensors and calls the C ABI; no arithmetic of the
method happens here.
"""
from __future__ import annotations

from typing import Dict, Optional

import torch

from . import (kstap_create, kstap_destroy, kstap_detect, kstap_fit_project, make_factors,
               make_params)


class KStap:
    """One context (bank, stream, workspace) plus factor/output buffers."""

    def __init__(self, p, q, r_a, r_b, ring_r, ring_a, guard_r, guard_a, tau, bank_a, bank_b,
                 eps=0.0, max_iter=0, hbm_budget_bytes=0, device="cuda:0", stream=None,
                 precision="fp32", filter="kron"):
        self.dev = torch.device(device)
        self.p, self.q, self.r_a, self.r_b = p, q, r_a, r_b
        self.ring_r, self.ring_a = ring_r, ring_a
        self.params = make_params(p, q, r_a, r_b, ring_r, ring_a, guard_r, guard_a, tau, eps,
                                  max_iter, precision, filter)
        self.bank_a = torch.as_tensor(bank_a).to(self.dev, torch.complex64).contiguous()
        self.bank_b = torch.as_tensor(bank_b).to(self.dev, torch.complex64).contiguous()
        self.V = self.bank_a.shape[0]
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.dev)
        self.ctx = kstap_create(self.params, self.bank_a, self.bank_b, self.V, hbm_budget_bytes,
                                self.stream.cuda_stream)
        self._bufs: Dict[tuple, Dict[str, torch.Tensor]] = {}

    @classmethod
    def from_workload(cls, wl, bank_a, bank_b, **kw):
        return cls(wl.p, wl.q, wl.r_a, wl.r_b, wl.ring_r, wl.ring_a, wl.guard_r, wl.guard_a,
                   wl.tau, bank_a, bank_b, **kw)

    def cells(self, H_in, W_in):
        return H_in - 2 * self.ring_r, W_in - 2 * self.ring_a - self.q + 1

    def buffers(self, H_in, W_in, T_all=False) -> Dict[str, torch.Tensor]:
        key = (H_in, W_in, T_all)
        if key not in self._bufs:
            H, W = self.cells(H_in, W_in)
            n = H * W
            d = self.dev
            b = dict(
                UA=torch.empty(n, self.p, self.r_a, dtype=torch.complex64, device=d),
                UB_hi=torch.empty(n, self.q, self.r_b, dtype=torch.complex64, device=d),
                UB_lo=torch.empty(n, self.q, self.r_b, dtype=torch.complex64, device=d),
                lamA=torch.empty(n, self.r_a, dtype=torch.float32, device=d),
                lamB=torch.empty(n, self.r_b, dtype=torch.float32, device=d),
                iters=torch.empty(n, dtype=torch.int32, device=d),
                eta=torch.empty(n, dtype=torch.float32, device=d),
                Tmax=torch.empty(n, dtype=torch.float32, device=d),
                vidx=torch.empty(n, dtype=torch.int32, device=d),
                map=torch.empty(n, dtype=torch.uint8, device=d))
            if T_all:
                b["T_all"] = torch.empty(n, self.V, dtype=torch.float32, device=d)
            b["factors"] = make_factors(b["UA"], b["UB_hi"], b["UB_lo"], b["lamA"], b["lamB"],
                                        b["iters"], b["eta"])
            self._bufs[key] = b
        return self._bufs[key]

    def alloc_outputs(self, H_in, W_in, T_all=False) -> Dict[str, torch.Tensor]:
        """Fresh (not cached) factor and output buffers for one frame."""
        key_bufs = self._bufs.pop((H_in, W_in, T_all), None)
        b = self.buffers(H_in, W_in, T_all)
        self._bufs.pop((H_in, W_in, T_all), None)
        if key_bufs is not None:
            self._bufs[(H_in, W_in, T_all)] = key_bufs
        return b

    def frame_desc(self, Y: torch.Tensor, b: Dict[str, torch.Tensor]):
        """Batch descriptor of frame Y with output buffers b.  It holds raw
        device pointers: the caller keeps Y and b alive while it is used."""
        from . import make_frame
        _, H_in, W_in = Y.shape
        return make_frame(Y, H_in, W_in, b["factors"], b["Tmax"], b["vidx"], b["map"],
                          b.get("T_all"))

    def run(self, Y: torch.Tensor, T_all: bool = False) -> Dict[str, torch.Tensor]:
        """fit_project + detect on a device frame Y (p, H_in, W_in) complex64."""
        assert Y.is_cuda and Y.dtype == torch.complex64 and Y.is_contiguous()
        _, H_in, W_in = Y.shape
        b = self.buffers(H_in, W_in, T_all)
        kstap_fit_project(self.ctx, Y, H_in, W_in, b["factors"])
        kstap_detect(self.ctx, Y, H_in, W_in, b["factors"], b["Tmax"], b["vidx"], b["map"],
                     b.get("T_all"))
        return b

    def close(self):
        if self.ctx:
            kstap_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
