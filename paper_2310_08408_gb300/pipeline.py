"""Host-staged pipeline: a batch that lives in pinned host memory streams through a device
computation chunk by chunk. The upload of chunk i+1 and the download of chunk i-1 run on their own
CUDA streams while chunk i computes, so the host<->device copies overlap the kernels instead of
adding to them (the copy engines of each direction and the SMs work at the same time).

Only scheduling lives here: device staging buffers (`depth` slots per input and output), three
streams and the events that order them. The computation is whatever `fn` launches on the current
stream, which is where the library's entry points launch.

`run` is one self-contained pass: its first upload and last download have no computation to hide
behind. For a loop of passes over the same batch (the steps of an optimisation), the overlapped
mode (`prime`, `run_overlapped`, `finish`) hides them too: every pass uploads the first chunk of the
next pass after its own first chunk has computed, and downloads the last chunk of the previous pass
while its own first chunk computes, so that only the loop's first upload and last download are left
outside the computation. The alternating mode (`prime_alternating`, `run_alternating`, `finish`)
keeps the whole batch in one chunk and two slots: a pass computes from one slot while the next
pass's input goes up into the other and the previous pass's results come down from it.
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
        self._pending = None  # overlapped passes: the last chunk whose download is still due

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

    # ------------------------------------------------------------------ overlapped passes
    def _chunks(self, B):
        n_c = math.ceil(B / self.chunk)
        if n_c > self.depth:
            raise ValueError("overlapped passes need a staging slot per chunk (depth >= chunks)")
        return [(i, i * self.chunk, min(B, (i + 1) * self.chunk) - i * self.chunk) for i in range(n_c)]

    def _join_start(self):
        caller = torch.cuda.current_stream()
        start = torch.cuda.Event()
        start.record(caller)
        for s in (self.s_up, self.s_comp, self.s_down):
            s.wait_event(start)
        return caller

    def _join_end(self, caller):
        for s in (self.s_up, self.s_comp, self.s_down):
            ev = torch.cuda.Event()
            ev.record(s)
            caller.wait_event(ev)

    def prime(self, host_in) -> None:
        """Uploads the first chunk of the first overlapped pass (ordered after the caller's
        stream; the caller's stream waits for it)."""
        B = int(host_in[0].shape[0])
        _, lo, n = self._chunks(B)[0]
        caller = self._join_start()
        with torch.cuda.stream(self.s_up):
            for h, d in zip(host_in, self.dev_in[0]):
                d[:n].copy_(h[lo:lo + n], non_blocking=True)
        self._join_end(caller)
        self._pending = None

    def run_overlapped(self, host_in, host_out, fn) -> None:
        """One pass as `run`, with the first chunk already uploaded (by `prime` or the previous
        pass) and the last chunk's download left to the next pass (or `finish`). Every chunk has
        its own staging slot. Work is ordered after the caller's stream, which waits for the pass
        (so each pass is one unit that a CUDA graph can capture and replay)."""
        B = int(host_in[0].shape[0])
        chunks = self._chunks(B)
        last = len(chunks) - 1
        caller = self._join_start()
        pend = None
        with torch.cuda.stream(self.s_down):  # the previous pass's last chunk
            if self._pending is not None:
                k, lo, n, outs = self._pending
                for h, d in zip(outs, self.dev_out[k]):
                    h[lo:lo + n].copy_(d[:n], non_blocking=True)
                pend = torch.cuda.Event()
                pend.record(self.s_down)
        with torch.cuda.stream(self.s_up):  # chunks 1..last: their slots are free
            for i, lo, n in chunks[1:]:
                for h, d in zip(host_in, self.dev_in[i]):
                    d[:n].copy_(h[lo:lo + n], non_blocking=True)
                self.ev_up[i].record(self.s_up)
        for i, lo, n in chunks:
            with torch.cuda.stream(self.s_comp):
                if i > 0:
                    self.s_comp.wait_event(self.ev_up[i])
                if i == last and pend is not None:
                    self.s_comp.wait_event(pend)  # slot `last` is downloaded before it is rewritten
                fn([d[:n] for d in self.dev_in[i]], [d[:n] for d in self.dev_out[i]], lo, n)
                self.ev_comp[i].record(self.s_comp)
            if i == 0:  # the next pass's first chunk, once this pass's first chunk has read slot 0
                with torch.cuda.stream(self.s_up):
                    self.s_up.wait_event(self.ev_comp[0])
                    for h, d in zip(host_in, self.dev_in[0]):
                        d[:n].copy_(h[lo:lo + n], non_blocking=True)
            if i < last:
                with torch.cuda.stream(self.s_down):
                    self.s_down.wait_event(self.ev_comp[i])
                    for h, d in zip(host_out, self.dev_out[i]):
                        h[lo:lo + n].copy_(d[:n], non_blocking=True)
        _, lo, n = chunks[last]
        self._pending = (last, lo, n, list(host_out))
        self._join_end(caller)

    def run_alternating(self, host_in, host_out, fn, parity: int) -> None:
        """One pass over the whole batch as one chunk, the passes of a loop alternating between two
        staging slots: pass k (parity k % 2) computes from slot `parity`, whose input the previous
        pass (or `prime_alternating`) uploaded, while the next pass's input is uploaded into the
        other slot and the previous pass's results are downloaded from it, so that nothing inside a
        pass waits on a copy. Needs chunk >= batch and depth >= 2; `finish` downloads the last
        pass's results. Each parity is one unit that a CUDA graph can capture."""
        B = int(host_in[0].shape[0])
        if self.chunk < B or self.depth < 2:
            raise ValueError("alternating passes need the whole batch in one chunk and two slots")
        p, o = parity & 1, 1 - (parity & 1)
        caller = self._join_start()
        with torch.cuda.stream(self.s_down):  # the previous pass's results, from the other slot
            if self._pending is not None:
                k, lo, n, outs = self._pending
                for h, d in zip(outs, self.dev_out[k]):
                    h[lo:lo + n].copy_(d[:n], non_blocking=True)
        with torch.cuda.stream(self.s_up):  # the next pass's input, into the other slot
            for h, d in zip(host_in, self.dev_in[o]):
                d[:B].copy_(h[:B], non_blocking=True)
        with torch.cuda.stream(self.s_comp):
            fn([d[:B] for d in self.dev_in[p]], [d[:B] for d in self.dev_out[p]], 0, B)
        self._pending = (p, 0, B, list(host_out))
        self._join_end(caller)

    def prime_alternating(self, host_in, parity: int = 0) -> None:
        """Uploads the input of the first alternating pass into slot `parity`."""
        B = int(host_in[0].shape[0])
        caller = self._join_start()
        with torch.cuda.stream(self.s_up):
            for h, d in zip(host_in, self.dev_in[parity & 1]):
                d[:B].copy_(h[:B], non_blocking=True)
        self._join_end(caller)
        self._pending = None

    def tail_due(self, host_out, batch: int, parity=None) -> None:
        """Marks the last pass's results as still to be downloaded, for a loop of passes replayed
        from CUDA graphs (a replay does not update this object): overlapped passes (parity None)
        leave their last chunk, alternating passes their whole batch in slot `parity`."""
        if parity is None:
            i, lo, n = self._chunks(batch)[-1]
            self._pending = (i, lo, n, list(host_out))
        else:
            self._pending = (parity & 1, 0, batch, list(host_out))

    def finish(self) -> None:
        """Downloads the last chunk of the last overlapped pass (the caller's stream waits)."""
        if getattr(self, "_pending", None) is None:
            return
        caller = self._join_start()
        k, lo, n, outs = self._pending
        with torch.cuda.stream(self.s_down):
            for h, d in zip(outs, self.dev_out[k]):
                h[lo:lo + n].copy_(d[:n], non_blocking=True)
        self._join_end(caller)
        self._pending = None
