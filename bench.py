#!/usr/bin/env python3
"""Throughput benchmark of the GB300 RS / CZT hot path (XLuminA, arXiv 2310.08408).

Workload (rs2048): a batch of 16 complex64 fields on a 2048 x 2048 grid (pitch 0.5 um,
lambda 0.633 um), each a Gaussian (w0 = 200 um) times a seeded uniform [0, 2 pi) phase; the
distances cycle through z = 0.5, 2 and 10 mm; CZT maps onto a 512 x 512 window over the central
64 um. Inputs are synthetic (the paper's propagation benchmark uses a Gaussian beam at 2048^2,
Fig. 1b); all 16 inputs (537 MB) exceed the 126 MB L2, so no flush is needed between steps.

One step is one gradient evaluation of every field through both propagators:
    A = RS(U, z),  C = CZT(U, z)                              (forward propagations)
    L = S(|A|^2) + S(|C|^2)  (second-moment spot size of each plane)
    dL/dU = RS^H(dL/dA) + CZT^H(dL/dC),  dL/dz from the dh/dz spectrum
with U = SLM(phi) applied to the source, dL/dphi from the element adjoint and an Adam step on phi.
Parts not yet present in the library are skipped and listed in the JSON ("step_parts").
`value` = RS/CZT propagations per second (forward and adjoint, whole job), `grads_per_s` = field
gradient evaluations per second.

`--impl reference` times the FP64 CPU oracle (the only reference this build has) on the host
cores: each step is the same composition for ONE field of the batch.
"""
from __future__ import annotations

import argparse
import json
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
E2E_CHUNK = 2  # fields per device pass of the end-to-end (host-staged) measurement


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
    p.add_argument("--no-next", action="store_true", help="skip the angular-spectrum CZT and "
                   "beam-splitter measurements")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--e2e-depth", type=int, default=3,
                   help="staging slots of the end-to-end pipeline (3: a late download of chunk i does not stall chunk i + 2)")
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
    return 5.0 * L * np.log2(L)


def kernel_model(name: str, dims: dict):
    """(algorithmic flops, algorithmic bytes) of ONE launch of kernel family `name` on the
    benchmark workload (complex64). Bytes are the compulsory reads + writes of that pass;
    flops count every FFT at its padded length plus 6 flops per complex multiply."""
    n, m, cs = dims["n"], dims["m"], 8
    L = int(re.search(r"<(\d+)>", name).group(1)) if "<" in name else 0
    nb = dims.get("per_launch", 1)
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
    if name.startswith("czt_fwd_x") or name.startswith("czt_adj_x"):
        return nb * n * (2 * fft_flops(L) + 18 * L), nb * (n * n + n * m) * cs
    if name.startswith("czt_fwd_y") or name.startswith("czt_adj_y"):
        return nb * m * (2 * fft_flops(L) + 18 * L), nb * (n * m + m * m) * cs
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


def step_parts(xl):
    have = {"rs": True, "czt": True}
    for fn in ("apply_elements", "intensity_loss", "adam_step"):
        have[fn] = hasattr(xl, fn)
    return have


class GpuStep:
    """The benchmark step on device-resident buffers (all through the C ABI)."""

    def __init__(self, xl, torch, g, w, U_dev, zs):
        self.xl, self.torch, self.g, self.w, self.zs = xl, torch, g, w, zs
        self.U = U_dev
        B = U_dev.shape[0]
        dev = U_dev.device
        from paper_2310_08408_gb300 import inputs
        # fixed seeded cotangents (the loss gradients until the loss kernels are present)
        self.GA = torch.from_numpy(inputs.random_unit(7, (1, N, N)).astype(np.complex64)).to(dev).expand(B, N, N).contiguous()
        self.GC = torch.from_numpy(inputs.random_unit(8, (1, M, M)).astype(np.complex64)).to(dev).expand(B, M, M).contiguous()
        self.A = torch.empty_like(U_dev)
        self.C = torch.empty((B, M, M), dtype=U_dev.dtype, device=dev)
        # the forward RS keeps the row transforms of U for the adjoint's distance gradient
        self.S = xl.save_buffer(U_dev)
        self.props = 4 * B

    def __call__(self):
        xl = self.xl
        xl.rs_propagate(self.U, self.g, LAM, self.zs, out=self.A, saved=self.S)
        xl.czt_propagate(self.U, self.g, self.w, LAM, self.zs, out=self.C)
        gc = xl.czt_propagate_backward(self.GC, self.g, self.w, LAM, self.zs)
        ga, gz = xl.rs_propagate_backward(self.GA, None, self.g, LAM, self.zs, want_field=True,
                                          want_dz=True, saved=self.S)
        self.gA, self.gC = ga, gc
        self.gz = gz
        return self.A, self.C, self.gz


# ----------------------------------------------------------------------------- optical tables
TABLE_CFG = dict(wavelength=0.6328, extent=1024.0, w0=200.0, f=5000.0, cam_m=256, cam_width=64.0,
                 lr=0.01, lr_z=1.0)
TABLE_WINDOW = (256, 256, 0.25, 0.25, -32.0, -32.0)  # the tables' camera window


def inputs_grid(n: int):
    """The centred grid of side n: pitch 0.5 um at the headline size, 1024 um / n for the tables."""
    from paper_2310_08408_gb300 import inputs
    return inputs.Grid.centred(n, PITCH if n == N else 1024.0 / n)


def table_section(xl, torch, setups: int, steps: int, seed: int):
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
    counts = {n: grid_n.count(n) for n in (512, 1024, 2048)}
    return {"workload": f"{setups} optical tables (N mix {counts}), fwd+bwd+Adam, CUDA graph",
            "grads_per_s": setups / (ms / 1000.0), "ms_per_step": ms,
            "fp64_single_instance_grads_per_s": setups / (t64 / 1000.0),
            "fp64_ms_per_setup": f64,
            "table1024_grads_per_s": 1000.0 / ms1024,
            "speedup_vs_fp64_single_instance": t64 / ms}


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


# ----------------------------------------------------------------------------- CPU oracle
def oracle_step(U1, g, w, z, GA, GC):
    """The step's composition for one field with the FP64 oracle."""
    import oracle
    u = U1.astype(np.complex128)
    A = oracle.rs_conv(u, g.dx, g.dy, LAM, z)
    C = oracle.czt_conv(u, g.astuple(), w.astuple(), LAM, z)
    gc = oracle.czt_conv(GC, g.astuple(), w.astuple(), LAM, z, adjoint=True)
    ga = oracle.rs_conv(GA, g.dx, g.dy, LAM, z, oracle.K_H, adjoint=True)
    dz = np.real(np.vdot(GA, oracle.rs_conv(u, g.dx, g.dy, LAM, z, oracle.K_DH)))
    return A, C, ga + gc, dz


def cpu_sample(U, g, w, zs, steps=1):
    import oracle
    from paper_2310_08408_gb300 import inputs
    GA = inputs.random_unit(7, (N, N)).astype(np.complex64).astype(np.complex128)
    GC = inputs.random_unit(8, (M, M)).astype(np.complex64).astype(np.complex128)
    oracle.build()
    t0 = time.perf_counter()
    for i in range(steps):
        oracle_step(U[i % len(U)], g, w, zs[i % len(zs)], GA, GC)
    dt = time.perf_counter() - t0
    # the oracle step holds 5 propagation-sized sums per field (4 propagations + the dz one);
    # count the 4 propagations as in the GPU step
    return {"value": 4 * steps / dt, "unit": "propagations/s", "cores": oracle.get_threads(),
            "kind": "oracle",
            "sample": f"{steps} of the {len(U)} fields of one step (RS, CZT, CZT^H, RS^H + dz at "
                      f"2048^2 -> 512^2, FP64 C++ oracle), {dt:.1f} s"}


# ----------------------------------------------------------------------------- main
METRIC = "RS/CZT propagations/s at 2048^2 (fwd + adjoint) and grads/s"


def bench_config(batch: int, world: int) -> dict:
    """The workload both arms report (the reference arm times a bounded sample of it)."""
    return {"workload": "rs2048: batch 16 x 2048^2 complex64, pitch 0.5 um, "
                        "lambda 0.633 um, z cycling {0.5, 2, 10} mm; RS (4096^2 padded) "
                        "and CZT to 512^2 over 64 um; forward + adjoint + dz",
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
    from paper_2310_08408_gb300 import inputs
    GA = inputs.random_unit(7, (N, N)).astype(np.complex64).astype(np.complex128)
    GC = inputs.random_unit(8, (M, M)).astype(np.complex64).astype(np.complex128)
    for i in range(a.warmup):
        oracle_step(U[i % 3], g, w, zs[i % 3], GA, GC)
    t0 = time.perf_counter()
    for i in range(a.steps):
        oracle_step(U[i % 3], g, w, zs[i % 3], GA, GC)
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
                         "sample": "one field of the batch per step (RS, CZT, CZT^H, RS^H + dz in "
                                   "FP64 on the host cores), the fields and distances cycling"},
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

    # batch 1 (one field per step, z = 0.5 mm): the latency-bound end of the same step
    batch1 = None
    if B > 1:
        s1 = GpuStep(xl, torch, g, w, U_dev[:1].contiguous(), zs[:1])
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
        batch1 = {"value": s1.props / (ms1 / 1000.0), "unit": "propagations/s", "ms_per_step": ms1,
                  "steps": k1, "note": "one 2048^2 field, z = 0.5 mm, same four propagations"}
        del s1

    # per-kernel durations (CUDA events recorded by the library on its launch stream)
    xl.profile_enable(True)
    for _ in range(3):
        step()
    torch.cuda.synchronize()
    prof = xl.profile_report()
    xl.profile_enable(False)
    total = sum(v[1] for v in prof.values())
    top = max(prof.items(), key=lambda kv: kv[1][1]) if prof else None
    roof = None
    peaks = {}
    pk_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk_path):
        peaks = json.load(open(pk_path))
    hbm = peaks.get("hbm_gbs", 6800.0)
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    def fields_per_launch(name, cnt):
        """Fields one launch of kernel family `name` processed: the step makes two passes of
        the row kernels (forward and adjoint RS) and one of every other kernel per field; the
        library batches the fields of a call into fewer launches."""
        per_step = (2 if name.startswith(("rs_pass1", "rs_pass3")) else 1) * B
        return per_step / (cnt / 3)

    if top is not None:
        name, (cnt, tot) = top
        avg_s = tot / cnt / 1000.0
        flops, nbytes = kernel_model(name, {"n": N, "m": M,
                                            "per_launch": fields_per_launch(name, cnt)})
        clk = ck.get("sm_mhz") or 1900.0
        fp32_peak = sms * 128 * 2 * clk * 1e6 / 1e12  # TFLOP/s, CUDA-core FMA rate at the sampled clock
        per_field = load_traffic().get(name)
        traffic = per_field * fields_per_launch(name, cnt) if per_field is not None else None
        if flops is not None:
            t_alu = flops / (fp32_peak * 1e12)
            t_mem = nbytes / (hbm * 1e9)
            if t_alu >= t_mem:
                ach = flops / avg_s / 1e12
                roof = {"bound": "alu", "achieved": ach, "peak": fp32_peak, "unit": "TFLOP/s",
                        "frac": ach / fp32_peak, "traffic": traffic, "kernel": name,
                        "share": tot / total if total else None,
                        "peak_note": f"FP32 CUDA-core FMA rate: {sms} SMs x 128 lanes x 2 x "
                                     f"{clk:.0f} MHz (median sampled clock)",
                        "hbm_frac_of_measured": nbytes / avg_s / 1e9 / hbm}
            else:
                ach = nbytes / avg_s / 1e9
                roof = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                        "frac": ach / hbm, "traffic": traffic, "kernel": name,
                        "share": tot / total if total else None,
                        "peak_note": "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"}
    kernels = {}
    clk_k = ck.get("sm_mhz") or 1900.0
    fp32_k = sms * 128 * 2 * clk_k * 1e6 / 1e12
    for k, (cnt_k, tot_k) in prof.items():
        fpl = fields_per_launch(k, cnt_k)
        ent = {"launches": cnt_k // 3, "ms_per_step": tot_k / 3, "fields_per_launch": fpl}
        fl, nb = kernel_model(k, {"n": N, "m": M, "per_launch": fpl})
        if fl is not None:  # each kernel against the roof its model says bounds it
            avg = tot_k / cnt_k / 1000.0
            alu = fl / (fp32_k * 1e12) >= nb / (hbm * 1e9)
            ent["bound"] = "alu" if alu else "hbm"
            ent["frac"] = (fl / avg / 1e12 / fp32_k) if alu else (nb / avg / 1e9 / hbm)
            ent["hbm_gbs"] = nb / avg / 1e9
            ent["tflops"] = fl / avg / 1e12
        kernels[k] = ent

    # end to end: pinned host input -> device, the step, results back to pinned host buffers,
    # streamed in chunks of E2E_CHUNK fields so that the copies overlap the kernels
    e2e = None
    if not a.no_e2e:
        from paper_2310_08408_gb300.pipeline import HostPipeline
        A_h = torch.empty(step.A.shape, dtype=step.A.dtype).pin_memory()
        C_h = torch.empty(step.C.shape, dtype=step.C.dtype).pin_memory()
        gz_h = torch.empty((B,), dtype=torch.float64).pin_memory()
        ke = max(10, a.steps // 2)  # timed end-to-end steps (after a.warmup untimed ones)
        ch = min(a.e2e_chunk, B)
        pipe = HostPipeline([((N, N), U_pin.dtype)],
                            [((N, N), step.A.dtype), ((M, M), step.C.dtype), ((), torch.float64)],
                            chunk=ch, depth=a.e2e_depth)
        with torch.cuda.stream(pipe.compute_stream):
            S_c = xl.save_buffer(step.U[:ch])
        GA_c, GC_c = step.GA[:ch], step.GC[:ch]

        def chunk_step(ins, outs, lo, n):
            (U,), (A, C, gz) = ins, outs
            zc = zs[lo:lo + n]
            xl.rs_propagate(U, g, LAM, zc, out=A, saved=S_c[:n])
            xl.czt_propagate(U, g, w, LAM, zc, out=C)
            xl.czt_propagate_backward(GC_c[:n], g, w, LAM, zc)
            _, gzc = xl.rs_propagate_backward(GA_c[:n], None, g, LAM, zc, want_field=True,
                                              want_dz=True, saved=S_c[:n])
            gz.copy_(gzc)

        def e2e_step():
            pipe.run([U_pin], [A_h, C_h, gz_h], chunk_step)

        e2e_step()
        # the whole step (uploads, the chunks' propagations, downloads) as one CUDA graph, so that
        # each timed step is one launch and host-side enqueue jitter cannot stall the pipeline;
        # eager launches if the capture fails
        launch, mode = e2e_step, "eager"
        if not a.e2e_eager:
            torch.cuda.synchronize()
            try:
                graph = torch.cuda.CUDAGraph()
                with torch.cuda.graph(graph, capture_error_mode="thread_local"):
                    e2e_step()
                graph.replay()
                torch.cuda.synchronize()
                launch, mode = graph.replay, "cuda_graph"
            except Exception as ex:  # noqa: BLE001 - reported in the JSON line
                torch.cuda.synchronize()
                mode = f"eager (graph capture failed: {type(ex).__name__})"
        ck_e2e = Clocks(local)  # clocks of the end-to-end region, reported with it
        for _ in range(a.warmup):
            launch()
        torch.cuda.synchronize()
        barrier()
        e0.record(stream)
        for _ in range(ke):
            launch()
        e1.record(stream)
        barrier()
        e2e_clocks = ck_e2e.stop()
        ems = e0.elapsed_time(e1)
        ems = replicas.max_over_ranks(ems, "cuda")
        # the host link alone on this machine: one whole-batch pinned upload and download
        link = {}
        for name, dst, src in (("h2d_gbs", step.U, U_pin), ("d2h_gbs", A_h, step.A)):
            dst.copy_(src, non_blocking=True)
            torch.cuda.synchronize()
            e0.record(stream)
            dst.copy_(src, non_blocking=True)
            e1.record(stream)
            e1.synchronize()
            link[name] = src.numel() * src.element_size() / (e0.elapsed_time(e1) / 1000.0) / 1e9
        e2e = {"value": replicas.whole_job_rate(step.props, world, ke, ems), "unit": "propagations/s",
               "h2d_bytes_per_step": int(U_pin.numel() * 8),
               "d2h_bytes_per_step": int(A_h.numel() * 8 + C_h.numel() * 8 + gz_h.numel() * 8),
               "ms_per_step": ems / ke, "host_link": link, "launch": mode, "chunk": ch, "depth": a.e2e_depth, "steps": ke,
               "clocks": e2e_clocks}

    nxt = None
    if not a.no_next:
        nxt = next_rows_section(xl, torch, g, w, U_dev, zs, hbm)
        nxt["cufft_comparison"] = cufft_comparison(xl, torch, g, U_dev, zs)

    table = None
    if not a.no_table:
        table = table_section(xl, torch, a.table_setups, a.table_steps, inputs_seed(rank))

    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        cpu = cpu_sample(U_host, g, w, zs, steps=1)

    if rank == 0:
        line = {
            "metric": METRIC,
            "value": value, "unit": "propagations/s", "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms / a.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c64 (f32, f64 phases)",
            "data": "synthetic",
            "config": bench_config(B, world),
            "grads_per_s": grads,
            "batch1": batch1,
            "tables": table,
            "next_rows": nxt,
            "autotune": tune,
            "step_parts": step_parts(xl),
            "gpu_launches": int(launches),
            "clocks": ck,
            "roofline": roof,
            "kernels": kernels,
            "e2e": e2e,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
