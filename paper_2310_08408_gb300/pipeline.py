"""Host-staged pipeline: a batch that lives in pinned host memory streams through a device
computation chunk by chunk. The upload of chunk i+1 and the download of chunk i-1 run on their own
CUDA streams while chunk i computes, so the host<->device copies overlap the kernels instead of
adding to them (the copy engines of each direction and the SMs work at the same time).

Only scheduling lives here: device staging buffers (`depth` slots per input and output), three
streams and the events that order them. The computation is whatever `fn` launches on the current
stream, which is where the library's entry points launch.
"""
from __future__ import annotations

import math

import torch


class HostPipeline:
    """in_specs / out_specs: lists of (per-item shape, dtype); chunk: items per device pass;
    depth: staging slots (2 = double buffering)."""

    def __init__(self, in_specs, out_specs, chunk: int, depth: int = 2, device="cuda"):
        if chunk < 1 or depth < 1:
            raise ValueError("chunk and depth must be >= 1")
        self.chunk, self.depth = int(chunk), int(depth)
        mk = lambda specs: [[torch.empty((self.chunk, *shape), dtype=dt, device=device)
                             for shape, dt in specs] for _ in range(self.depth)]
        self.dev_in, self.dev_out = mk(in_specs), mk(out_specs)
        self.s_up, self.s_comp, self.s_down = (torch.cuda.Stream(device) for _ in range(3))
        ev = lambda: [torch.cuda.Event() for _ in range(self.depth)]
        self.ev_up, self.ev_comp, self.ev_down = ev(), ev(), ev()

    @property
    def compute_stream(self) -> torch.cuda.Stream:
        return self.s_comp

    def run(self, host_in, host_out, fn) -> None:
        """host_in / host_out: lists of pinned host tensors [B][...] matching the specs.
        fn(dev_in, dev_out, lo, n) computes items lo..lo+n-1 on the current stream, reading the
        views dev_in (n items each) and writing the views dev_out. The work is ordered after
        everything already queued on the caller's stream, and the caller's stream waits for the
        last download (no host synchronisation)."""
        B = int(host_in[0].shape[0])
        for t in list(host_in) + list(host_out):
            if t.shape[0] != B:
                raise ValueError("host tensors must share the batch dimension")
        caller = torch.cuda.current_stream()
        start = torch.cuda.Event()
        start.record(caller)
        for s in (self.s_up, self.s_comp, self.s_down):
            s.wait_event(start)
        for i in range(math.ceil(B / self.chunk)):
            k = i % self.depth
            lo = i * self.chunk
            n = min(B, lo + self.chunk) - lo
            with torch.cuda.stream(self.s_up):
                if i >= self.depth:  # slot k's inputs are free once chunk i - depth computed
                    self.s_up.wait_event(self.ev_comp[k])
                for h, d in zip(host_in, self.dev_in[k]):
                    d[:n].copy_(h[lo:lo + n], non_blocking=True)
                self.ev_up[k].record(self.s_up)
            with torch.cuda.stream(self.s_comp):
                self.s_comp.wait_event(self.ev_up[k])
                if i >= self.depth:  # slot k's outputs are free once chunk i - depth downloaded
                    self.s_comp.wait_event(self.ev_down[k])
                fn([d[:n] for d in self.dev_in[k]], [d[:n] for d in self.dev_out[k]], lo, n)
                self.ev_comp[k].record(self.s_comp)
            with torch.cuda.stream(self.s_down):
                self.s_down.wait_event(self.ev_comp[k])
                for h, d in zip(host_out, self.dev_out[k]):
                    h[lo:lo + n].copy_(d[:n], non_blocking=True)
                self.ev_down[k].record(self.s_down)
        end = torch.cuda.Event()
        end.record(self.s_down)
        caller.wait_event(end)
