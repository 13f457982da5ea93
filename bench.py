#!/usr/bin/env python3
"""Throughput benchmark of the GB300 RS / CZT hot path (XLuminA, arXiv 2310.08408).

Workload (rs2048): a batch of 16 complex64 source fields on a 2048 x 2048 grid (pitch 0.5 um,
lambda 0.633 um), each a Gaussian (w0 = 200 um) times a seeded uniform [0, 2 pi) phase, shaped by
an SLM phase mask per field (the trained parameters, starting flat); the distances cycle through
z = 0.5, 2 and 10 mm; CZT maps onto a 512 x 512 window over the central 64 um. Inputs are
synthetic (the paper's benchmarks use a Gaussian beam through a phase mask at 2048^2,
Introduction and Methods, "Features and performance"); all 16 inputs (537 MB) and the step's
intermediates exceed the 126 MB L2, so no flush is needed between steps.

One step is one gradient evaluation of every field through both propagators and an Adam step
on the masks, every stage a library call:
    U = SLM(src, phi)                              xl_apply_elements
    A = RS(U, z)  (input spectrum saved)           xl_rs_propagate_save
    C = CZT(U, z) (distance-gradient sums saved)   xl_czt_propagate_save (second stream, with
                                                   C's loss, beside the RS forward)
    L = S(|A|^2) + S(|C|^2), gA, gC = dL/dA, dL/dC xl_intensity_loss_and_grad (second-moment
                                                   spot sizes and their field gradients)
    gU, dL/dz = RS^H gA                            xl_rs_propagate_backward_saved
    gU, dL/dz += CZT^H gC                          xl_czt_propagate_backward_saved (accumulate)
    dL/dphi = SLM^H gU                             xl_apply_elements_backward
    phi <- Adam(phi, dL/dphi)                      xl_step_advance, xl_adam_step
(the distances are differentiated but not stepped: the propagation tables stay cached).
`value` = RS/CZT propagations per second (four a field: RS, CZT and their adjoints; whole job),
`grads_per_s` = gradient evaluations (fields) per second.

`--impl reference` times the FP64 CPU oracle (the only reference this build has) on the host
cores: each step is the same composition for ONE field of the batch.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import re
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

LAM = 0.633
ZS = (500.0, 2000.0, 10_000.0)
N, PITCH, W0 = 2048, 0.5, 200.0
M, WIN_W = 512, 64.0
LR = 0.01
E2E_CHUNK = 8  # fields per device pass of the end-to-end (host-staged) measurement
MB = 1e6


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=60)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="xl", choices=["xl", "reference"])
    p.add_argument("--batch", type=int, default=16)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--e2e-chunk", type=int, default=E2E_CHUNK,
                   help="fields per device pass of the end-to-end measurement")
    p.add_argument("--autotune", action="store_true", help="time the launch variants here "
                   "instead of loading --plan")
    p.add_argument("--plan", default=os.path.join(ROOT, "paper_2310_08408_gb300", "plans",
                                                  "gb300_c64.txt"),
                   help="launch plan file (xl_tune_load); empty: the built-in plan")
    p.add_argument("--no-next", action="store_true", help="skip the angular-spectrum CZT, "
                   "beam-splitter and cuFFT-comparison measurements")
    p.add_argument("--no-configs", action="store_true", help="skip the other workloads "
                   "(complex128 RS 256^2, VRS / VCZT 2048^2)")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--e2e-depth", type=int, default=3,
                   help="staging slots of the end-to-end pipeline (at least one per chunk of a step: "
                        "consecutive steps overlap)")
    p.add_argument("--e2e-mode", default="alternate", choices=["overlap", "alternate"],
                   help="end-to-end pipeline: chunks with consecutive steps overlapped, or the whole "
                        "batch alternating between two staging slots")
    p.add_argument("--e2e-eager", action="store_true",
                   help="end-to-end steps as eager launches instead of one CUDA graph replay")
    p.add_argument("--no-table", action="store_true", help="skip the batched optical-table section")
    p.add_argument("--table-setups", type=int, default=256)
    p.add_argument("--table-steps", type=int, default=4)
    return p.parse_args()


# ----------------------------------------------------------------------------- clocks
class Clocks:
    """nvidia-smi sampling (every 50 ms) of SM clock and throttle reasons during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")
    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, index: int):
        self.proc = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons = [], [], set()
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                smax.append(float(f[1]))
            except ValueError:
                continue
            for name, v in zip(self.NAMES, f[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- roofline
def fft_flops(L: int) -> float:
    """Algorithmic flops of one complex FFT of length L (5 L log2 L convention)."""
    return 5.0 * L * math.log2(L)


def czt_plan(n: int, m: int):
    """(L, S) of one CZT axis, the rule the library applies (xl_czt.cu czt_axis_plan): the grid
    side in S segments, each a cyclic convolution of length L = 2^ceil(log2(ceil(n/S) + m - 1)),
    the least (S + 1) L log2 L + 4 S L."""
    best, cost, S = None, math.inf, 1
    while S <= 64 and S <= n:
        seg = -(-n // S)
        if (S - 1) * seg < n:
            L = 64
            while L < seg + m - 1:
                L *= 2
            if L <= 8192:
                c = (S + 1) * L * math.log2(L) + 4 * S * L
                if c < cost * (1 - 1e-9):
                    best, cost = (L, S), c
        S *= 2
    return best


# Algorithmic bytes of one 2048^2 field (per-unit figures: what the method must
# read and write, complex64 = 8 B, float32 masks = 4 B): the four propagations and the rest of the
# gradient step.
UNIT_BYTES = {
    "rs": 3 * N * N * 8 + (N + 1) ** 2 * 8,             # in + out + transfer-spectrum quadrant
    "rs_adj_dz": 4 * N * N * 8 + 2 * (N + 1) ** 2 * 8,  # + the input and the dh/dz quadrant
    "czt": N * N * 8 + M * M * 8,                       # in + window out (chirps ~0)
    "czt_adj_dz": 2 * N * N * 8 + M * M * 8,            # + the input for dL/dz
    "slm": N * N * (8 + 4 + 8),                         # src, phi in; U out
    "loss": N * N * 8 + M * M * 8,                      # |A|^2, |C|^2 sums
    "loss_bwd": 2 * (N * N + M * M) * 8,                # fields in, gradients out
    "slm_bwd": N * N * (8 + 8 + 4 + 4),                 # gU, src, phi in; dL/dphi out
    "adam": N * N * 4 * 7,                              # p, m, v, g in; p, m, v out
}
UNIT_FLOPS_RS = 2 * N * fft_flops(2 * N) + 2 * (2 * N) * (2 * fft_flops(2 * N) + 6 * 2 * N)


def kernel_model(name: str, fields: float):
    """(algorithmic flops, algorithmic bytes) of ONE launch of kernel family `name` on the
    benchmark workload (complex64) processing `fields` 2048^2 fields. Bytes are the compulsory
    reads + writes of that pass; flops count every FFT at its padded length (5 L log2 L) plus 6
    flops per complex multiply."""
    n, m, cs = N, M, 8
    L = int(re.search(r"<(\d+)>", name).group(1)) if "<" in name else 0
    nb = fields
    if name.startswith("rs_pass1"):
        return nb * n * fft_flops(L), nb * (n * n + 2 * n * n) * cs
    if name.startswith("rs_pass3"):
        return nb * n * fft_flops(L), nb * (2 * n * n + n * n) * cs
    if name.startswith("rs_pass2_m0_save"):  # also stores the input's 2D spectrum (4 n^2)
        return nb * 2 * n * (2 * fft_flops(L) + 6 * L), nb * (8 * n * n + (n + 1) ** 2) * cs
    if name.startswith("rs_pass2_m0"):
        return nb * 2 * n * (2 * fft_flops(L) + 6 * L), nb * (4 * n * n + (n + 1) ** 2) * cs
    if name.startswith("rs_pass2_m4"):  # adjoint with the saved spectrum: T in/out, spectrum in
        return nb * 2 * n * (2 * fft_flops(L) + 14 * L), nb * (8 * n * n + 2 * (n + 1) ** 2) * cs
    if name.startswith("rs_pass2_m2"):
        return nb * 2 * n * (3 * fft_flops(L) + 14 * L), nb * (6 * n * n + 2 * (n + 1) ** 2) * cs
    if name.startswith("czt_") and L:
        _, S = czt_plan(n, m)
        dz = "_dz" in name
        rows = n if "_x" in name else m  # rows the pass transforms (x: grid rows; y: window columns)
        fl = rows * ((S + 1) * fft_flops(L) + (S * (12 if dz else 6) + 12) * L)
        if name.startswith("czt_fwd_x"):
            by = n * n + n * m + (n * L if dz else 0)
        elif name.startswith("czt_fwd_y"):
            by = n * m + m * m + (m * L + m * m if dz else 0)
        elif name.startswith("czt_adj_y"):
            by = m * m + n * m + (m * m + n * m + m * L if dz else 0)
        else:  # dz (as the step runs it): the forward input, the saved sums a2 and g_in read
            # back (the pass adds into the RS adjoint's gradient); the T-plane term is the y pass's
            by = n * m + n * n + (2 * n * n + n * L if dz else 0)
        return nb * fl, nb * by * cs
    if name == "elements_fwd":
        return None, nb * UNIT_BYTES["slm"]
    if name in ("elements_bwd", "elements_bwd_mask"):
        return None, nb * UNIT_BYTES["slm_bwd"]
    if name == "adam":
        return None, nb * UNIT_BYTES["adam"]
    if name == "loss_grad":  # the step runs it on A (2048^2) and on C (512^2)
        return None, nb * (n * n + m * m) * 2 * cs / 2
    if name.startswith("loss_sweep"):
        return None, nb * (n * n + m * m) * cs / 2
    return None, None


def load_traffic():
    """Per-field DRAM traffic of kernel families from the committed ncu summary (a launch moves
    that many bytes for each field it processes), valid only while the kernel sources are
    unchanged (hash recorded with the counters)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return {}
    try:
        data = json.load(open(path))
        from paper_2310_08408_gb300 import build
        if data.get("csrc_hash") != build.source_hash():
            return {}
        return data.get("bytes_per_field", {})
    except Exception:
        return {}


# ----------------------------------------------------------------------------- workload
def make_inputs(rank: int, batch: int):
    from paper_2310_08408_gb300 import inputs
    g = inputs.Grid.centred(N, PITCH)
    w = inputs.Window.centred(M, WIN_W)
    from paper_2310_08408_gb300.replicas import rank_seed
    seed = rank_seed(inputs.SEED0 + 2, rank)
    U = np.stack([inputs.gaussian_random_phase(g, W0, seed + b) for b in range(batch)]
                 ).astype(np.complex64)
    zs = [ZS[b % 3] for b in range(batch)]
    return g, w, U, zs


def inputs_seed(rank: int) -> int:
    from paper_2310_08408_gb300 import inputs
    from paper_2310_08408_gb300.replicas import rank_seed
    return rank_seed(inputs.SEED0 + 5, rank)


# Library entry points one step calls, in order (the bench line's `step_parts`).
STEP_PARTS = ["xl_step_advance", "xl_apply_elements (SLM)", "xl_rs_propagate_save",
              "xl_czt_propagate_save", "xl_intensity_loss_and_grad (A, C)",
              "xl_rs_propagate_backward_saved (+ dL/dz)",
              "xl_czt_propagate_backward_saved (+ dL/dz, accumulate)",
              "xl_apply_elements_backward (dL/dphi)", "xl_adam_step (phi)"]


class GpuStep:
    """The benchmark step (module docstring) on device-resident buffers, all through the C ABI.
    run(lo, n) steps fields lo..lo+n-1 (their masks and moments); src / zs override the sources
    and distances of those fields (the end-to-end pipeline passes its staged chunk)."""

    def __init__(self, xl, torch, g, w, src_dev, zs, chunk=None):
        self.xl, self.torch, self.g, self.w, self.zs = xl, torch, g, w, list(zs)
        self.src = src_dev
        B = src_dev.shape[0]
        cap = chunk or B  # fields per run()
        dev = src_dev.device
        self.wg = (M, M, w.dxo, w.dyo, w.xo0, w.yo0)  # the camera grid of the window field
        self.phi = torch.zeros((B, N, N), dtype=torch.float32, device=dev)
        self.m, self.v = torch.zeros_like(self.phi), torch.zeros_like(self.phi)
        self.t = torch.zeros(1, dtype=torch.int32, device=dev)
        e = lambda *s: torch.empty(*s, dtype=torch.complex64, device=dev)
        self.U, self.A, self.gA = (e((cap, N, N)) for _ in range(3))
        self.C, self.gC = e((cap, M, M)), e((cap, M, M))
        self.S_rs = xl.save_buffer(self.U)
        self.S_czt = xl.czt_save_buffer(self.U, g, w)
        self.props = 4 * B
        self.last = None
        # the CZT forward and its loss depend only on U, like the RS forward: they run on a second
        # stream so that their blocks fill the SMs the RS passes leave idle (False: one stream, as
        # the per-kernel profile wants its launches apart)
        self.side = torch.cuda.Stream(device=dev)
        self.concurrent = True

    def run(self, lo=0, n=None, src=None, zs=None, advance=True):
        xl, g, w = self.xl, self.g, self.w
        n = self.src.shape[0] - lo if n is None else n
        s = slice(lo, lo + n)
        src = self.src[s] if src is None else src
        zs = self.zs[s] if zs is None else zs
        U, A, C, gA, gC = (b[:n] for b in (self.U, self.A, self.C, self.gA, self.gC))
        q4 = lambda t: t.view(t.shape[0], 1, t.shape[-2], t.shape[-1])
        slm = [dict(kind=xl.SLM, phi_x=self.phi[s])]
        if advance:
            xl.step_advance(self.t)
        xl.apply_elements(q4(src), g, LAM, slm, out=q4(U))
        main = self.torch.cuda.current_stream()
        if self.concurrent:
            self.side.wait_stream(main)
        with self.torch.cuda.stream(self.side if self.concurrent else main):
            xl.czt_propagate(U, g, w, LAM, zs, out=C, saved=self.S_czt[:n])
            lC, _ = xl.intensity_loss_and_grad(q4(C), self.wg, 1, out=q4(gC))
        xl.rs_propagate(U, g, LAM, zs, out=A, saved=self.S_rs[:n])
        lA, _ = xl.intensity_loss_and_grad(q4(A), g, 1, out=q4(gA))
        if self.concurrent:
            main.wait_stream(self.side)
        # the spot-size losses are blind to a constant phase on A and C: phase-invariant dL/dz
        gU_rs, gz_rs = xl.rs_propagate_backward(gA, None, g, LAM, zs, want_field=True, want_dz=True,
                                                phase_invariant=True, saved=self.S_rs[:n])
        xl.czt_propagate_backward(gC, g, w, LAM, zs, u_in=U, want_dz=True, phase_invariant=True,
                                  saved=self.S_czt[:n], g_in=gU_rs, g_z=gz_rs, accumulate=True)
        _, gpx, _, _ = xl.apply_elements_backward(q4(gU_rs), q4(src), g, LAM, slm, want_field=False,
                                                  want_phi=True, want_params=False)
        xl.adam_step(self.phi[s], self.m[s], self.v[s], gpx[0], LR, self.t)
        self.last = (lA, lC, gz_rs, gpx[0])
        return self.last

    def __call__(self):
        return self.run()

# ----------------------------------------------------------------------------- optical tables
TABLE_CFG = dict(wavelength=0.6328, extent=1024.0, w0=200.0, f=5000.0, cam_m=256, cam_width=64.0,
                 lr=0.01, lr_z=1.0)
TABLE_WINDOW = (256, 256, 0.25, 0.25, -32.0, -32.0)  # the tables' camera window
TABLE_BYTES_1024 = 1.2e9  # algorithmic bytes of one 1024^2 table gradient evaluation


def inputs_grid(n: int):
    """The centred grid of side n: pitch 0.5 um at the headline size, 1024 um / n for the tables."""
    from paper_2310_08408_gb300 import inputs
    return inputs.Grid.centred(n, PITCH if n == N else 1024.0 / n)


def table_section(xl, torch, setups: int, steps: int, seed: int, hbm: float):
    """Batched optical tables: `setups` setups with N drawn from {512, 1024, 2048} (seeded,
    pitch = 1024 um / N), fwd + bwd + Adam per step replayed from one CUDA graph; compared with
    the same library in complex128, one setup per call, eager launches (the plain FP64
    single-instance GPU path), timed per grid size and weighted by the same mix."""
    from paper_2310_08408_gb300 import inputs
    u = inputs.uniform(seed, setups)
    grid_n = [512 * (2 ** int(3 * x)) for x in u]
    init = [[0.3, 20_000.0, 20_000.0] for _ in range(setups)]
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    b = xl.Batch(TABLE_CFG, grid_n, init, seed)
    b.step(use_graph=True)   # eager warm-up (sizes every workspace)
    b.step(use_graph=True)   # capture + first replay
    torch.cuda.synchronize()
    n0 = xl.launch_count()
    e0.record(stream)
    for _ in range(steps):
        b.step(use_graph=True)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    # launch gaps: the graph replay against the sum of its kernels' own durations (one eager step
    # with every launch bracketed by CUDA events on its stream)
    xl.profile_enable(True)
    b.step(use_graph=False)
    torch.cuda.synchronize()
    prof = xl.profile_report()
    xl.profile_enable(False)
    k_ms = sum(v[1] for v in prof.values())
    k_n = sum(v[0] for v in prof.values())
    b.close()
    # one table of 1024^2 (complex64, graph replay): the single-setup rate
    one = xl.Batch(TABLE_CFG, [1024], [[0.3, 20_000.0, 20_000.0]], seed)
    one.step(use_graph=True)
    one.step(use_graph=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(20):
        one.step(use_graph=True)
    e1.record(stream)
    torch.cuda.synchronize()
    ms1024 = e0.elapsed_time(e1) / 20
    one.close()
    # the complex128 single-instance path, one setup per size
    f64 = {}
    for n in (512, 1024, 2048):
        one = xl.Batch(dict(TABLE_CFG, dtype="c128"), [n], [[0.3, 20_000.0, 20_000.0]], seed)
        one.step(use_graph=False)
        torch.cuda.synchronize()
        e0.record(stream)
        one.step(use_graph=False)
        e1.record(stream)
        torch.cuda.synchronize()
        f64[n] = e0.elapsed_time(e1)
        one.close()
    t64 = sum(f64[n] for n in grid_n)
    # per-plane checkpointing at 2048^2: step time and bytes a setup in both modes (4 setups)
    ckpt = {}
    for mode in (0, 1):
        cb = xl.Batch(dict(TABLE_CFG, checkpoint=mode), [2048] * 4, [[0.3, 20_000.0, 20_000.0]] * 4, seed)
        cb.step(use_graph=True)
        cb.step(use_graph=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(5):
            cb.step(use_graph=True)
        e1.record(stream)
        torch.cuda.synchronize()
        ckpt[f"checkpoint{mode}"] = {"ms_per_step": e0.elapsed_time(e1) / 5,
                                     "bytes_per_setup": cb.memory() / 4}
        cb.close()
    counts = {n: grid_n.count(n) for n in (512, 1024, 2048)}
    # HBM bound of a gradient evaluation: TABLE_BYTES_1024 per 1024^2 setup, in proportion to the
    # pixel count for the other sizes
    bound_ms = sum(TABLE_BYTES_1024 * (n / 1024) ** 2 for n in grid_n) / (hbm * 1e9) * 1e3
    bound1024 = TABLE_BYTES_1024 / (hbm * 1e9) * 1e3
    return {"workload": f"{setups} optical tables (N mix {counts}), fwd+bwd+Adam, CUDA graph",
            "grads_per_s": setups / (ms / 1000.0), "ms_per_step": ms,
            "fp64_single_instance_grads_per_s": setups / (t64 / 1000.0),
            "fp64_ms_per_setup": f64,
            "table1024_grads_per_s": 1000.0 / ms1024,
            "frac_of_hbm_bound": bound_ms / ms, "table1024_frac_of_hbm_bound": bound1024 / ms1024,
            "hbm_bound_note": f"{TABLE_BYTES_1024 / 1e9:.1f} GB per 1024^2 gradient evaluation (fwd 0.4 + "
                              "bwd 0.8, with the trained distances' spectrum regeneration), scaled by "
                              "pixels, at measured HBM",
            "launches_per_step": k_n, "kernel_ms_per_step": k_ms,
            "top_kernels_ms": {k: round(v[1], 3) for k, v in
                               sorted(prof.items(), key=lambda kv: -kv[1][1])[:10]},
            "launch_gap_frac": max(0.0, 1.0 - k_ms / ms),
            "launch_gap_note": "1 - (sum of the step's kernel durations, CUDA events per launch) / "
                               "(graph replay time per step)",
            "speedup_vs_fp64_single_instance": t64 / ms,
            "checkpointing_2048": dict(ckpt, workload="4 tables of 2048^2, graph replay; "
                                       "0: RS / VRS input spectra kept, 1: plane fields only")}


# ----------------------------------------------------------------------------- further rows
def cufft_comparison(xl, torch, g, U_dev, zs, steps: int = 10):
    """Timing comparison only (not the product path): the RS forward of the same batch through
    torch.fft (cuFFT, complex64): zero-pad to 2N, 2D FFT, multiply by a 2N x 2N spectrum per
    distance, inverse 2D FFT, crop. The spectra are placeholders (unit-modulus values), so only
    the time is compared, against the library's xl.rs_propagate of the same fields, both after
    warm-up, CUDA events on the current stream."""
    B, n = U_dev.shape[0], U_dev.shape[-1]
    L = 2 * n
    dev = U_dev.device
    dists = sorted(set(zs))
    gen = torch.Generator(device="cpu").manual_seed(11)
    H = torch.polar(torch.ones(len(dists), L, L), 6.283185307179586 * torch.rand(len(dists), L, L, generator=gen)
                    ).to(torch.complex64).to(dev)
    idx = [dists.index(z) for z in zs]
    X = torch.zeros((B, L, L), dtype=torch.complex64, device=dev)
    out = torch.empty_like(U_dev)

    def cufft_step():
        X.zero_()
        X[:, :n, :n] = U_dev
        F = torch.fft.fft2(X)
        for i in range(B):
            F[i].mul_(H[idx[i]])
        out.copy_(torch.fft.ifft2(F)[:, :n, :n])

    A = torch.empty_like(U_dev)
    ours = lambda: xl.rs_propagate(U_dev, g, LAM, zs, out=A)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    res = {}
    for name, f in (("cufft_ms", cufft_step), ("xl_ms", ours)):
        for _ in range(3):
            f()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):
            f()
        e1.record(stream)
        torch.cuda.synchronize()
        res[name] = e0.elapsed_time(e1) / steps
    del X, H
    torch.cuda.empty_cache()
    return {"workload": f"RS forward, {B} x {n}^2 complex64 padded to {L}^2, z cycling {dists}",
            "cufft_ms": res["cufft_ms"], "xl_ms": res["xl_ms"],
            "xl_speedup": res["cufft_ms"] / res["xl_ms"],
            "note": "torch.fft (cuFFT) pipeline with placeholder spectra: timing comparison only"}


def next_rows_section(xl, torch, g, w, U_dev, zs, hbm_gbs: float, steps: int = 10):
    """Device throughput of the rows beyond the headline step, on the same 2048^2 inputs:
    the angular-spectrum CZT onto the 512^2 window (forward + adjoint with distance gradient)
    and the beam splitter (forward and adjoint with the ratio gradient) on [B][2][2048^2]
    fields, the latter against the measured HBM bandwidth (it moves each pixel once)."""
    from paper_2310_08408_gb300 import inputs
    B = U_dev.shape[0]
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    G = torch.from_numpy(inputs.random_unit(9, (1, M, M)).astype(np.complex64)).cuda().expand(B, M, M).contiguous()

    def timed(fn, k):
        fn()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(k):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / k

    def as_step():
        xl.asczt_propagate(U_dev, g, w, LAM, zs)
        xl.asczt_propagate_backward(G, U_dev, g, w, LAM, zs, want_field=True, want_dz=True)

    ms_as = timed(as_step, steps)
    xl.profile_enable(True)
    as_step()
    torch.cuda.synchronize()
    prof = xl.profile_report()
    xl.profile_enable(False)
    kern = {k: {"launches": v[0], "ms": v[1]} for k, v in prof.items()}
    # beam splitter on two-component fields
    a = U_dev.unsqueeze(1).expand(B, 2, N, N).contiguous()
    b = torch.flip(a, dims=[3]).contiguous()
    ot, orr = torch.empty_like(a), torch.empty_like(a)
    R = torch.linspace(0.2, 0.8, B, dtype=torch.float64, device="cuda")
    nbytes = a.numel() * a.element_size()
    ms_f = timed(lambda: xl.beam_splitter(a, b, R, out_t=ot, out_r=orr), steps)
    ms_b = timed(lambda: xl.beam_splitter_backward(ot, orr, a, b, R), steps)
    del a, b, ot, orr
    fwd_gbs = 4 * nbytes / (ms_f / 1000.0) / 1e9
    bwd_gbs = 6 * nbytes / (ms_b / 1000.0) / 1e9
    return {"asczt": {"workload": f"{B} x 2048^2 -> 512^2 over 64 um, z cycling {{0.5, 2, 10}} mm, "
                                  "forward + adjoint + dz", "propagations_per_s": 2 * B / (ms_as / 1000.0),
                      "ms_per_step": ms_as, "kernels": kern},
            "beam_splitter": {"workload": f"{B} x 2 x 2048^2 complex64 per port",
                              "fwd_ms": ms_f, "fwd_gbs": fwd_gbs, "bwd_ms": ms_b, "bwd_gbs": bwd_gbs,
                              "fwd_frac_of_measured_hbm": fwd_gbs / hbm_gbs,
                              "bwd_frac_of_measured_hbm": bwd_gbs / hbm_gbs,
                              "bytes": "fwd 2 fields read + 2 written; bwd 4 read + 2 written"}}


# ----------------------------------------------------------------------------- other workloads
def configs_section(xl, torch, steps: int = 10):
    """The other workloads of the benchmark set, device-timed (CUDA events, after warm-up):
    complex128 RS at 256^2 (z = 10 mm, one field) and the vectorial workload at 2048^2 (VRS and
    VCZT onto 512^2, z = 5 mm, a radially polarised Gaussian and a random Jones field; forward with
    saved sums, adjoint with dL/dz)."""
    from paper_2310_08408_gb300 import inputs
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, k):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(k):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / k

    out = {}
    w1 = inputs.WORKLOADS["rs256_c128"]
    g1 = inputs.Grid.centred(w1["n"], w1["pitch"])
    x, y = g1.coords()
    lens = np.exp(-1j * (2 * np.pi / w1["wavelength"]) * (x[None, :] ** 2 + y[:, None] ** 2) / (2 * w1["f"]))
    u1 = (inputs.gaussian(g1, w1["w0"]) * lens * np.exp(1j * inputs.random_phase(g1, w1["seed"])))
    U1 = torch.from_numpy(u1[None].astype(np.complex128)).cuda()
    ms1 = timed(lambda: xl.rs_propagate(U1, g1, w1["wavelength"], [w1["z"]]), 4 * steps)
    out["rs256_c128"] = {"workload": "RS 256^2 complex128, pitch 1 um, z = 10 mm, one field "
                                     "(padded 512^2)", "propagations_per_s": 1000.0 / ms1,
                         "ms_per_propagation": ms1}
    w3 = inputs.WORKLOADS["vrs2048"]
    g3 = inputs.Grid.centred(w3["n"], w3["pitch"])
    win3 = inputs.Window.centred(w3["window_m"], w3["window_w"])
    exy = np.stack([inputs.radial_gaussian(g3, w3["w0"]),
                    inputs.random_jones(g3, w3["w0"], w3["seed"])]).astype(np.complex64)
    E = torch.from_numpy(exy).cuda()
    z3 = [w3["z"]] * 2
    Sv = xl.save_buffer(E, 2)
    Sc = xl.czt_save_buffer(E, g3, win3, vectorial=1)
    Gv = torch.from_numpy(inputs.random_unit(31, (2, 3, N, N)).astype(np.complex64)).cuda()
    Gc = torch.from_numpy(inputs.random_unit(32, (2, 3, M, M)).astype(np.complex64)).cuda()
    lam3 = w3["wavelength"]

    def vstep():
        xl.vrs_propagate(E, g3, lam3, z3, saved=Sv)
        xl.vrs_propagate_backward(Gv, None, g3, lam3, z3, want_field=True, want_dz=True, saved=Sv)
        xl.czt_propagate(E, g3, win3, lam3, z3, vectorial=1, saved=Sc)
        xl.czt_propagate_backward(Gc, g3, win3, lam3, z3, vectorial=1, u_in=E, want_dz=True, saved=Sc)

    ms3 = timed(vstep, steps)
    xl.profile_enable(True)
    vstep()
    torch.cuda.synchronize()
    prof = xl.profile_report()
    xl.profile_enable(False)
    out["vrs2048"] = {"workload": "VRS and VCZT (512^2 over 64 um) at 2048^2 complex64, z = 5 mm, "
                                  "2 fields (radial Gaussian, random Jones), forward with saved "
                                  "sums + adjoint with dL/dz",
                      "propagations_per_s": 4 * 2 / (ms3 / 1000.0), "ms_per_step": ms3,
                      "kernels": {k: {"launches": v[0], "ms": v[1]} for k, v in prof.items()}}
    del E, Sv, Sc, Gv, Gc
    torch.cuda.empty_cache()
    return out


# ----------------------------------------------------------------------------- CPU oracle
def oracle_step(src, phi, g, w, z, adam_state):
    """The step's composition for one field with the FP64 oracle (module docstring). Returns the
    stepped mask, the Adam state and the step's losses, dL/dz and dL/dphi."""
    import oracle
    wg = (M, M, w.dxo, w.dyo, w.xo0, w.yo0)
    slm = [dict(kind=oracle.SLM, phi_x=phi)]
    src = src.astype(np.complex128)[None]
    U = oracle.apply_elements(src, g.astuple(), LAM, slm)[0]
    A = oracle.rs_conv(U, g.dx, g.dy, LAM, z)
    C = oracle.czt_conv(U, g.astuple(), w.astuple(), LAM, z)
    lA, _ = oracle.intensity_loss(A[None], g.astuple(), 1)
    lC, _ = oracle.intensity_loss(C[None], wg, 1)
    gA = oracle.intensity_loss_backward(A[None], g.astuple(), 1)[0]
    gC = oracle.intensity_loss_backward(C[None], wg, 1)[0]
    gU = (oracle.rs_conv(gA, g.dx, g.dy, LAM, z, oracle.K_H, adjoint=True)
          + oracle.czt_conv(gC, g.astuple(), w.astuple(), LAM, z, adjoint=True))
    k = 2 * np.pi / LAM
    # phase-invariant distance gradients (the losses ignore a constant phase on A and C)
    dz = (np.real(np.vdot(gA, oracle.rs_conv(U, g.dx, g.dy, LAM, z, oracle.K_DH))) - np.real(1j * k * np.vdot(gA, A))
          + np.real(np.vdot(gC, oracle.czt_conv(U, g.astuple(), w.astuple(), LAM, z, 3)))
          - np.real(1j * k * np.vdot(gC, C)))
    _, gpx, _, _ = oracle.apply_elements_backward(gU[None], src, g.astuple(), LAM, slm)
    m, v, t = adam_state
    t += 1
    oracle.adam(phi, m, v, gpx[0], LR, t)  # in place
    return phi, (m, v, t), {"loss_a": lA, "loss_c": lC, "dz": float(dz), "gphi": gpx[0]}


def cpu_sample(U, g, w, zs, steps=1):
    import oracle
    oracle.build()
    phi = np.zeros((N, N))
    st = (np.zeros((N, N)), np.zeros((N, N)), 0)
    t0 = time.perf_counter()
    for i in range(steps):
        phi, st, _ = oracle_step(U[i % len(U)], phi, g, w, zs[i % len(zs)], st)
    dt = time.perf_counter() - t0
    return {"value": 4 * steps / dt, "unit": "propagations/s", "cores": oracle.get_threads(),
            "kind": "oracle",
            "sample": f"{steps} of the {len(U)} fields of one step (SLM, RS, CZT, losses, their "
                      f"adjoints with dL/dz, SLM adjoint, Adam at 2048^2 -> 512^2, FP64 C++ "
                      f"oracle), {dt:.1f} s"}


# ----------------------------------------------------------------------------- main
METRIC = "RS/CZT propagations/s at 2048^2 (fwd + adjoint) and grads/s"


def bench_config(batch: int, world: int) -> dict:
    """The workload both arms report (the reference arm times a bounded sample of it)."""
    return {"workload": "rs2048 gradient step: batch 16 x 2048^2 complex64 sources, pitch 0.5 um, "
                        "lambda 0.633 um, z cycling {0.5, 2, 10} mm; SLM mask -> RS (4096^2 padded) "
                        "and CZT to 512^2 over 64 um -> second-moment spot sizes -> adjoints with "
                        "dL/dz -> mask gradient -> Adam on the masks",
            "global_batch": batch * world, "grid": N, "window": M,
            "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
            "l2": "inputs (537 MB per GPU) exceed L2; no flush"}


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    g, w, U, zs = make_inputs(0, 3)
    import oracle
    oracle.build()
    phi = np.zeros((N, N))
    st = (np.zeros((N, N)), np.zeros((N, N)), 0)
    for i in range(a.warmup):
        phi, st, _ = oracle_step(U[i % 3], phi, g, w, zs[i % 3], st)
    t0 = time.perf_counter()
    for i in range(a.steps):
        phi, st, _ = oracle_step(U[i % 3], phi, g, w, zs[i % 3], st)
    dt = time.perf_counter() - t0
    v = 4 * a.steps / dt
    line = {
        "impl": "reference", "metric": METRIC,
        "value": v, "unit": "propagations/s", "n_gpus": a.gpus, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": 1000 * dt / max(a.steps, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": bench_config(a.batch, 1),
        "cpu_baseline": {"value": v, "unit": "propagations/s", "cores": oracle.get_threads(),
                         "kind": "oracle",
                         "sample": "one field of the batch per step (SLM, RS, CZT, losses, their "
                                   "adjoints with dL/dz, SLM adjoint, Adam in FP64 on the host "
                                   "cores), the fields and distances cycling"},
        "e2e": {"value": v, "unit": "propagations/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    a = parse()
    if a.impl == "reference":
        return run_reference(a)
    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2310_08408_gb300 import build, xl
    build.build()
    xl.load()
    B = a.batch
    g, w, U_host, zs = make_inputs(rank, B)
    U_pin = torch.from_numpy(U_host).pin_memory()
    U_dev = U_pin.to("cuda", non_blocking=True)
    torch.cuda.synchronize()
    step = GpuStep(xl, torch, g, w, U_dev, zs)

    from paper_2310_08408_gb300 import replicas

    def barrier():
        replicas.barrier("cuda")

    # launch plan: the autotuner's rows-per-block choice for every pass of this grid and window,
    # from the packaged GB300 plan or (--autotune) timed here; untimed set-up, results identical
    # for every choice
    tune = None
    if a.autotune:
        for grid_n in ((N,) if a.no_table else (N, 512, 1024)):
            gt = inputs_grid(grid_n)
            xl.autotune(gt, w if grid_n == N else TABLE_WINDOW, xl.C64, reps=5)
    elif a.plan:
        xl.tune_load(a.plan)
    if a.autotune or a.plan:
        import tempfile
        fd, tpath = tempfile.mkstemp(suffix=".txt")
        os.close(fd)
        xl.tune_save(tpath)
        tune = [ln for ln in open(tpath).read().splitlines() if not ln.startswith("#")]
        os.unlink(tpath)

    clocks = Clocks(local)
    for _ in range(a.warmup):
        step()
    barrier()
    n0 = xl.launch_count()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(a.steps):
        step()
    e1.record(stream)
    barrier()
    ms = e0.elapsed_time(e1)
    launches = (xl.launch_count() - n0) // max(a.steps, 1)
    ck = clocks.stop()
    ms = replicas.max_over_ranks(ms, "cuda")
    value = replicas.whole_job_rate(step.props, world, a.steps, ms)
    grads = replicas.whole_job_rate(B, world, a.steps, ms)
    ms_step = ms / a.steps

    # batch 1 (one field per step) at each distance: the latency-bound end of the same step
    batch1 = None
    if B > 1:
        batch1 = {}
        for z in ZS:
            i = zs.index(z)
            s1 = GpuStep(xl, torch, g, w, U_dev[i:i + 1].contiguous(), [z])
            for _ in range(3):
                s1()
            barrier()
            k1 = max(10, a.steps // 2)
            e0.record(stream)
            for _ in range(k1):
                s1()
            e1.record(stream)
            barrier()
            ms1 = e0.elapsed_time(e1) / k1
            batch1[f"z{z / 1000:g}mm"] = {"value": s1.props / (ms1 / 1000.0), "unit": "propagations/s",
                                          "ms_per_step": ms1, "steps": k1}
            del s1
        torch.cuda.empty_cache()

    # per-kernel durations (CUDA events recorded by the library on its launch stream), one stream
    step.concurrent = False
    xl.profile_enable(True)
    for _ in range(3):
        step()
    torch.cuda.synchronize()
    prof = xl.profile_report()
    xl.profile_enable(False)
    step.concurrent = True
    total = sum(v[1] for v in prof.values())
    peaks = {}
    pk_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk_path):
        peaks = json.load(open(pk_path))
    hbm = peaks.get("hbm_gbs", 6800.0)
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    clk = ck.get("sm_mhz") or 1900.0
    fp32_peak = sms * 128 * 2 * clk * 1e6 / 1e12  # TFLOP/s, CUDA-core FMA rate at the sampled clock
    traffic_pf = load_traffic()

    def fields_per_launch(name, cnt):
        """Fields one launch of kernel family `name` processed: the step makes two passes of
        the RS row kernels (forward and adjoint) and of the loss kernels (A and C), one of every
        other kernel per field; the library batches the fields of a call into fewer launches."""
        twice = name.startswith(("rs_pass1", "rs_pass3", "loss_"))
        return (2 if twice else 1) * B / (cnt / 3)

    kernels = {}
    for k_, (cnt_k, tot_k) in prof.items():
        fpl = fields_per_launch(k_, cnt_k)
        ent = {"launches": cnt_k // 3, "ms_per_step": tot_k / 3, "share": tot_k / total if total else None}
        fl, nb = kernel_model(k_, fpl)
        avg = tot_k / cnt_k / 1000.0
        if nb is not None:
            ent["fields_per_launch"] = fpl
            ent["hbm_gbs"] = nb / avg / 1e9
            ent["hbm_frac"] = nb / avg / 1e9 / hbm
        if fl is not None:
            ent["tflops"] = fl / avg / 1e12
            ent["alu_frac"] = fl / avg / 1e12 / fp32_peak
            ent["bound"] = "alu" if fl / (fp32_peak * 1e12) >= nb / (hbm * 1e9) else "hbm"
        elif nb is not None:
            ent["bound"] = "hbm"
        if k_ in traffic_pf and nb:
            ent["traffic_ratio"] = traffic_pf[k_] * fpl / nb
        kernels[k_] = ent

    # roofline of the dominant kernel: its algorithmic flops against the FP32 CUDA-core peak (the
    # RS / CZT units are ALU-bound at their algorithmic bytes), with the HBM fraction of the
    # per-unit algorithmic bytes beside it
    roof = None
    modelled = {k: v for k, v in prof.items() if kernel_model(k, 1.0)[1] is not None}
    if modelled:
        name, (cnt, tot) = max(modelled.items(), key=lambda kv: kv[1][1])
        avg_s = tot / cnt / 1000.0
        fpl = fields_per_launch(name, cnt)
        fl, nb = kernel_model(name, fpl)
        unit = "rs" if name.startswith("rs_") else "czt"
        unit_bytes = fpl * (UNIT_BYTES["rs_adj_dz"] if "m4" in name else UNIT_BYTES[unit])
        traffic = traffic_pf[name] * fpl if name in traffic_pf else None
        if fl is None:  # a bandwidth kernel (elements, loss, Adam): its bytes against HBM
            ach = nb / avg_s / 1e9
            roof = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                    "traffic": traffic, "kernel": name, "share": tot / total if total else None,
                    "peak_note": "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                    "traffic_ratio": (traffic / nb) if traffic else None}
        else:
            ach = fl / avg_s / 1e12
            roof = {"bound": "alu", "achieved": ach, "peak": fp32_peak, "unit": "TFLOP/s",
                    "frac": ach / fp32_peak, "traffic": traffic, "kernel": name,
                    "share": tot / total if total else None,
                    "peak_note": f"FP32 CUDA-core FMA rate derived from unit counts and clock: {sms} SMs "
                                 f"x 128 lanes x 2 x {clk:.0f} MHz (median sampled clock)",
                    "alg_flops_per_launch": fl, "alg_bytes_per_launch": nb,
                    "unit_bytes_per_launch": unit_bytes,
                    "unit_hbm_frac": unit_bytes / avg_s / 1e9 / hbm,
                    "unit_hbm_note": "the per-unit algorithmic bytes of the fields this launch "
                                     "processes (whole propagation) / its duration / measured HBM",
                    "traffic_ratio": (traffic / nb) if traffic else None}
    step_bytes = B * sum(UNIT_BYTES.values())
    e2e_alg = {"bytes_per_step": step_bytes, "frac_of_measured_hbm": step_bytes / (ms_step / 1000.0) / 1e9 / hbm,
               "note": "the step's algorithmic bytes (every stage's compulsory reads and writes) / "
                       "ms_per_step / measured HBM"}

    # end to end: pinned host sources -> device, the step, the losses, distance gradients and
    # mask gradients back to pinned host buffers, streamed in chunks of E2E_CHUNK fields so that
    # the copies overlap the kernels
    e2e = None
    if not a.no_e2e:
        from paper_2310_08408_gb300.pipeline import HostPipeline
        alt = a.e2e_mode == "alternate"
        ch = B if alt else min(a.e2e_chunk, B)
        loss_h = torch.empty((B, 2), dtype=torch.float64).pin_memory()
        gz_h = torch.empty((B,), dtype=torch.float64).pin_memory()
        gphi_h = torch.empty((B, N, N), dtype=torch.float32).pin_memory()
        outs_h = [loss_h, gz_h, gphi_h]
        ke = max(10, a.steps // 2)  # timed end-to-end steps (after a.warmup untimed ones)
        nchunk = -(-B // ch)
        pipe = HostPipeline([((N, N), U_pin.dtype)],
                            [((2,), torch.float64), ((), torch.float64), ((N, N), torch.float32)],
                            chunk=ch, depth=2 if alt else max(a.e2e_depth, nchunk))
        with torch.cuda.stream(pipe.compute_stream):
            sc = GpuStep(xl, torch, g, w, U_dev, zs, chunk=ch)

        def chunk_step(ins, outs, lo, n):
            (src,), (lo_, gz, gphi) = ins, outs
            lA, lC, gzc, gpc = sc.run(lo, n, src=src, zs=zs[lo:lo + n], advance=(lo == 0))
            lo_[:, 0].copy_(lA)
            lo_[:, 1].copy_(lC)
            gz.copy_(gzc)
            gphi.copy_(gpc)

        # consecutive steps overlap (the timed region starts with the first step's first upload and
        # ends with the last step's last download). overlap: chunks of the batch, each step
        # uploading the next step's first chunk and downloading the previous step's last chunk
        # while it computes; alternate: the whole batch in one chunk, steps alternating between two
        # staging slots (a step computes from one while the next step's input goes up into the
        # other and the previous step's results come down from it)
        def e2e_step(par):
            if alt:
                pipe.run_alternating([U_pin], outs_h, chunk_step, par)
            else:
                pipe.run_overlapped([U_pin], outs_h, chunk_step)

        def prime():
            if alt:
                pipe.prime_alternating([U_pin], 0)
            else:
                pipe.prime([U_pin])

        prime()
        e2e_step(0)
        e2e_step(1)
        # each step (uploads, the chunks' calls, downloads) as one CUDA graph (one per slot parity
        # when alternating), so that each timed step is one launch and host-side enqueue jitter
        # cannot stall the pipeline; eager launches if the capture fails
        launchers, mode = [lambda: e2e_step(0), lambda: e2e_step(1)], "eager"
        if not a.e2e_eager:
            torch.cuda.synchronize()
            try:
                graphs = []
                for par in ((0, 1) if alt else (0,)):
                    gr = torch.cuda.CUDAGraph()
                    with torch.cuda.graph(gr, capture_error_mode="thread_local"):
                        e2e_step(par)
                    graphs.append(gr)
                for gr in graphs:
                    gr.replay()
                torch.cuda.synchronize()
                launchers = [gr.replay for gr in graphs] * (1 if alt else 2)
                mode = "cuda_graph"
            except Exception as ex:  # noqa: BLE001 - reported in the JSON line
                torch.cuda.synchronize()
                mode = f"eager (graph capture failed: {type(ex).__name__})"
        ck_e2e = Clocks(local)  # clocks of the end-to-end region, reported with it
        for i in range(a.warmup):
            launchers[i % 2]()
        pipe.tail_due(outs_h, B, ((a.warmup - 1) % 2) if alt else None)
        pipe.finish()
        torch.cuda.synchronize()
        barrier()
        e0.record(stream)
        prime()
        for i in range(ke):
            launchers[i % 2]()
        pipe.tail_due(outs_h, B, ((ke - 1) % 2) if alt else None)
        pipe.finish()
        e1.record(stream)
        barrier()
        e2e_clocks = ck_e2e.stop()
        ems = e0.elapsed_time(e1)
        ems = replicas.max_over_ranks(ems, "cuda")
        # the host link alone on this machine: one whole-batch pinned upload and download
        link = {}
        for name, dst, src in (("h2d_gbs", U_dev, U_pin), ("d2h_gbs", gphi_h, step.phi)):
            dst.copy_(src, non_blocking=True)
            torch.cuda.synchronize()
            e0.record(stream)
            dst.copy_(src, non_blocking=True)
            e1.record(stream)
            e1.synchronize()
            link[name] = src.numel() * src.element_size() / (e0.elapsed_time(e1) / 1000.0) / 1e9
        e2e = {"value": replicas.whole_job_rate(step.props, world, ke, ems), "unit": "propagations/s",
               "h2d_bytes_per_step": int(U_pin.numel() * 8),
               "d2h_bytes_per_step": int(loss_h.numel() * 8 + gz_h.numel() * 8 + gphi_h.numel() * 4),
               "d2h": "losses, dL/dz and dL/dphi of every field",
               "ms_per_step": ems / ke, "host_link": link, "launch": mode, "chunk": ch,
               "depth": 2 if alt else max(a.e2e_depth, nchunk), "steps": ke, "clocks": e2e_clocks,
               "overlap": ("whole batch, steps alternating between two staging slots" if alt else
                           "each step uploads the next step's first chunk and downloads the "
                           "previous step's last chunk while it computes")}
        del sc, pipe
        torch.cuda.empty_cache()

    cfgs = None
    if not a.no_configs:
        cfgs = configs_section(xl, torch)

    nxt = None
    if not a.no_next:
        nxt = next_rows_section(xl, torch, g, w, U_dev, zs, hbm)
        nxt["cufft_comparison"] = cufft_comparison(xl, torch, g, U_dev, zs)

    table = None
    if not a.no_table:
        table = table_section(xl, torch, a.table_setups, a.table_steps, inputs_seed(rank), hbm)

    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        cpu = cpu_sample(U_host, g, w, zs, steps=1)

    if rank == 0:
        line = {
            "metric": METRIC,
            "value": value, "unit": "propagations/s", "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c64 (f32, f64 phases)",
            "data": "synthetic",
            "config": bench_config(B, world),
            "grads_per_s": grads,
            "tables_grads_per_s": table["grads_per_s"] if table else None,
            "tables_frac_of_hbm_bound": table["frac_of_hbm_bound"] if table else None,
            "gpu_launches": int(launches),
            "clocks": ck,
            "roofline": roof,
            "e2e_alg": e2e_alg,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "step_parts": STEP_PARTS,
            "batch1": batch1,
            "configs": cfgs,
            "tables": table,
            "next_rows": nxt,
            "autotune": tune,
            "kernels": kernels,
            "kernels_note": "per-kernel times from 3 profiled steps on one stream; the timed steps run "
                            "the CZT forward and its loss on a second stream beside the RS forward",
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
