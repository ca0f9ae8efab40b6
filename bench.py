#!/usr/bin/env python
"""Benchmark of the SDMM-SARA hot path on GB300.

Workload (default ``sdmm1024``, the largest single-GPU problem): 1024 x 1024
image of 5000 Gaussian sources plus a k^-2 diffuse field, M = 2^21
visibilities (half Gaussian variable density, half on 200 radial arcs),
Kaiser-Bessel 6 x 6, 2048 x 2048 grid, FP32 with FP64 reductions, SARA
(Dirac + db1..db8, 4 levels), 10 CG steps per x-update.  ``sdmm256`` (256 x
256, M = 65536, KB 6 x 6, reweighting every 60 iterations) is the
L2-resident secondary line.  One step = one SDMM iteration (Algorithm 1
steps 5-9).  Inputs are seeded and synthetic.

Printed: one JSON line with SDMM iterations/s (device-timed, inputs resident,
L2 flushed between steps), the Phi + Phi^H visibility rate, the end-to-end
rate through the C ABI with host buffers, the roofline of the dominant kernel,
the FP64 CPU oracle as a reported baseline, SM clocks and kernel launches.

``--impl reference`` times the FP64 CPU oracle on the host cores on the same
workload and metric.  Under torchrun each rank solves its own independent
problem (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1307_4370_gb300 import inputs  # noqa: E402

REWEIGHT_EVERY = 60
ROUNDS = 5
L2_FLUSH_BYTES = 512 << 20
QUALITY_ITERS = 60
METRIC = "SDMM-SARA iterations/sec"
UNIT = "iterations/s"


def nvtx_range(name):
    """Open (name) or close (None) an NVTX range, for kernel profilers' filters."""
    import torch
    try:
        if name is None:
            torch.cuda.nvtx.range_pop()
        else:
            torch.cuda.nvtx.range_push(name)
    except (RuntimeError, AttributeError):
        pass


def parse_args():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="sdmm1024", choices=sorted(inputs.WORKLOADS) + ["batch32"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-quality", action="store_true", help="skip the equal-iteration SNR of c64 and bf16 y")
    ap.add_argument("--no-batch", action="store_true", help="skip the 32-problem batched measurement")
    ap.add_argument("--cpu-seconds", type=float, default=20.0, help="budget of the oracle sample")
    ap.add_argument("--kernel", choices=["kb", "gauss"], default="kb",
                    help="interpolation kernel of G: Kaiser-Bessel or the paper's Gaussian")
    ap.add_argument("--prior", choices=["sara", "tv"], default="sara",
                    help="SARA (eq. delta) or the TV prior with positivity (FGP prox, 20 inner iterations)")
    ap.add_argument("--blocks", type=int, default=0,
                    help="distributed-block form (one l2 ball per block of equal size); 0 = one ball")
    ap.add_argument("--precision", choices=["c64", "bf16"], default="c64",
                    help="storage of the measured visibilities y (bf16 pairs with per-4096 scales)")
    return ap.parse_args()


def workload_config(w: inputs.Workload) -> dict:
    return {"workload": f"{w.name}: {w.n}x{w.n} image, M={w.M} visibilities, KB {w.J}x{w.J}, "
                        f"{2 * w.n}x{2 * w.n} grid, SARA 9 bases x 4 levels, CG {w.cg_iters} steps",
            "n": w.n, "M": w.M, "J": w.J, "cg_iters": w.cg_iters,
            "reweight_every": REWEIGHT_EVERY, "rounds": ROUNDS}


# ---------------------------------------------------------------------------
# FP64 CPU oracle: the reported baseline (and the reference arm)
# ---------------------------------------------------------------------------
def block_table(M: int, R: int, eps: float, l2_bound):
    """R equal consecutive blocks and their chi^2 bounds (sigma_n recovered from
    eps); ``l2_bound`` is the oracle's (CPU leg) or the library's (GPU arm)."""
    offsets = [M * i // R for i in range(R + 1)]
    sig = eps / math.sqrt(M + 2 * math.sqrt(M))
    return offsets, [l2_bound(offsets[i + 1] - offsets[i], sig) for i in range(R)]


def oracle_rate(w: inputs.Workload, budget_s: float, max_iters: int | None = None, kernel: str = "kb",
                blocks: int = 0, prior: str = "sara"):
    """SDMM iterations/s of the FP64 oracle on a bounded sample of the workload."""
    from oracle import sdmm as osdmm, simulate

    p = inputs.make_problem(w)
    y, eps = simulate.visibilities(p.x_true, p.uv, w.J, p.noise_unit, w.isnr_db, kernel=kernel)
    ops = simulate.operators(p.uv, w.n, w.J, kernel=kernel)
    wts = np.ones((9, w.n, w.n))
    if prior == "tv":
        st = osdmm.init_state_tv(ops, y, (w.n, w.n))
        wtv = np.ones((w.n, w.n))

        def iteration():
            osdmm.sdmm_iteration_tv(ops, st, y, eps, wtv, w.cg_iters)
    elif blocks > 0:
        offsets, eps_b = block_table(w.M, blocks, eps, simulate.l2_bound)
        st = osdmm.init_state_blocks(ops, y, offsets, (w.n, w.n))

        def iteration():
            osdmm.sdmm_iteration_blocks(ops, st, y, eps_b, offsets, wts, w.cg_iters)
    else:
        st = osdmm.init_state(ops, y, (w.n, w.n))

        def iteration():
            osdmm.sdmm_iteration(ops, st, y, eps, wts, w.cg_iters)
    iteration()  # the first iteration is trivial (x_hat = 0)
    done, t0 = 0, time.perf_counter()
    while True:
        iteration()
        done += 1
        el = time.perf_counter() - t0
        if el >= budget_s or (max_iters is not None and done >= max_iters):
            break
    return done / el, done, el


def oracle_rate_by_parts(w: inputs.Workload, budget_s: float, kernel: str = "kb"):
    """SDMM iterations/s of the FP64 oracle on a workload whose single
    iteration outlasts the budget: the oracle's own Phi, Phi^H, Psi^H and Psi
    calls are timed on the workload's data, and one iteration is counted as
    (k + 1) (Phi + Phi^H) + Psi^H + Psi (the operator applications of
    Algorithm 1 with k CG steps; the entrywise updates are left out, which
    favours the oracle)."""
    from oracle import measurement as me, sara as osara

    p = inputs.make_problem(w)
    x = p.x_true.astype(np.complex128)
    t0 = time.perf_counter()
    y = me.phi(x, p.uv, w.J, kernel=kernel)
    t_phi = time.perf_counter() - t0
    t0 = time.perf_counter()
    xa = me.phi_adj(y, p.uv, w.n, w.J, kernel=kernel)
    t_adj = time.perf_counter() - t0
    t0 = time.perf_counter()
    a = osara.sara_analysis(xa, 4)
    t_psiadj = time.perf_counter() - t0
    t0 = time.perf_counter()
    osara.sara_synthesis(a, 4)
    t_psi = time.perf_counter() - t0
    per_iter = (w.cg_iters + 1) * (t_phi + t_adj) + t_psiadj + t_psi
    el = t_phi + t_adj + t_psiadj + t_psi
    return 1.0 / per_iter, el, (t_phi, t_adj, t_psiadj, t_psi)


def cpu_baseline_entry(w, budget_s, max_iters=None, kernel: str = "kb", blocks: int = 0,
                       prior: str = "sara") -> dict:
    if w.n >= 1024 and prior == "sara" and blocks == 0:
        rate, el, t = oracle_rate_by_parts(w, budget_s, kernel)
        return {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle", "steps_timed": 1,
                "sample": f"one call each of the FP64 numpy oracle's Phi ({t[0]:.1f} s), Phi^H ({t[1]:.1f} s), "
                          f"Psi^H ({t[2]:.1f} s) and Psi ({t[3]:.1f} s) on the {w.name} workload "
                          f"({el:.1f} s in all), scaled to one SDMM iteration as "
                          f"{w.cg_iters + 1} (Phi + Phi^H) + Psi^H + Psi; single thread; "
                          f"host has {os.cpu_count()} cores"}
    rate, done, el = oracle_rate(w, budget_s, max_iters, kernel, blocks, prior)
    return {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle", "steps_timed": done,
            "sample": f"{done} SDMM iterations (after one untimed) of the {w.name} workload, FP64 numpy "
                      f"oracle, single thread, {el:.1f} s; host has {os.cpu_count()} cores"}


def run_reference(args, w):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    # bounded: about a minute of oracle work whatever --steps is
    budget = min(60.0, max(10.0, 0.2 * (args.steps + args.warmup)))
    entry = cpu_baseline_entry(w, budget, kernel=args.kernel, blocks=args.blocks, prior=args.prior)
    # "steps" is what was actually timed (the oracle's own sample, bounded in time)
    out = {"impl": "reference", "metric": METRIC, "value": entry["value"], "unit": UNIT,
           "n_gpus": args.gpus, "steps": entry["steps_timed"], "warmup": args.warmup,
           "steps_requested": args.steps,
           "ms_per_step": 1e3 / entry["value"], "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {**workload_config(w), "prior": args.prior, "kernel": args.kernel, "blocks": args.blocks},
           "cpu_baseline": entry,
           "e2e": {"value": entry["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines: list[str] = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.gpu), "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except OSError:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if parts[5 + k].lower() in ("active", "1", "yes"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def algorithmic_bytes(w: inputs.Workload, q: int = 9) -> dict:
    """Unique bytes each kernel family must move per launch (averaged over the
    launches of one SDMM step); complex64 = 8 B, uv = 8 B per visibility."""
    N, M, k = w.n * w.n, w.M, w.cg_iters
    c = 8
    D = q * N
    return {
        # first CG step: read r; later steps and the x_hat pass: read r, w, p, s, x,
        # write p, s, x, r (single-reduction CG update); always write n x 2n rows
        "row_fwd": ((3 + (k - 1) * 11 + 11) * N * c) / (k + 1),
        "col_fwd": 6 * N * c,                          # read n x 2n, write 2n x 2n
        "degrid": 4 * N * c + 4 * M * c,               # SDMM: read grid, uv, z2, y; write s2
        "grid": 4 * N * c + 2 * M * c,                 # read uv + vis, write the grid
        # CG steps, G^T G in one pass: read the grid and the frequencies
        # (8 B per visibility), write the second grid
        "gram": 8 * N * c + 8 * M,
        "col_inv": 6 * N * c,
        # CG: read n x 2n rows and r, write w; SDMM: also x_hat, z3, x1 in, z3 out
        "row_inv": (k * 4 * N * c + 7 * N * c) / (k + 1),
        "sdmm_l2": 5 * M * c,                          # s2, z2, y in; z2, v out
        # all levels of all planes: x in, z1 / w in, z1 / u1 out (w float32)
        "dwt_level": (N * c + D * (c + 4 + 2 * c)) / 4,
        "idwt_level": (D * c + N * c) / 4,
        "dirac": 4 * N * c,
        # TV prior: one FGP iteration reads b, r, s, p, q, w and writes p, q, r', s';
        # the finishing pass reads b, p, q, x_hat, w and writes z1, x1
        "tv_fgp": 9 * N * c + 4 * N,
        "tv_finish": 6 * N * c + 4 * N,
        "tv_init": 7 * N * c,
    }


KERNEL_SOURCE = {"row_fwd": "nufft.cu", "col_fwd": "nufft.cu", "degrid": "gridding.cu", "grid": "gridding.cu",
                 "gram": "gridding.cu", "tv_fgp": "tv.cu", "tv_finish": "tv.cu", "tv_init": "tv.cu",
                 "col_inv": "nufft.cu", "row_inv": "nufft.cu", "dwt_level": "sara.cu", "idwt_level": "sara.cu",
                 "dirac": "sara.cu", "sdmm_l2": "vecops.cu"}


def dram_traffic(workload: str, kernel: str):
    """DRAM bytes per launch of `kernel` from the committed ncu capture of this
    workload, or None when there is none or the kernel's source file changed
    after the capture (the record carries the file's SHA-256)."""
    import hashlib

    src = KERNEL_SOURCE.get(kernel)
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    if src is None or not os.path.exists(path):
        return None
    src_path = os.path.join(ROOT, "paper_1307_4370_gb300", "csrc", src)
    if not os.path.exists(src_path):
        return None
    with open(src_path, "rb") as f:
        sha = hashlib.sha256(f.read()).hexdigest()
    with open(path) as f:
        for ln in f:
            parts = ln.split()
            if len(parts) == 4 and not ln.startswith("#") and parts[0] == workload and parts[1] == kernel:
                return int(parts[2]) if parts[3] == sha else None
    return None


def peaks() -> tuple[float, str]:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def rank_workload(w: inputs.Workload, rank: int) -> inputs.Workload:
    """The independent problem a rank solves: same shape, its own seed."""
    return inputs.Workload(**{**w.__dict__, "seed": w.seed + 1000 * rank})


def max_over_ranks(value: float, device) -> float:
    """Largest value over all ranks (the timing rule: the slowest rank counts)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_gpu(args, w):
    import torch
    import torch.distributed as dist

    from paper_1307_4370_gb300 import binding

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    cpu_entry = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu_entry = cpu_baseline_entry(w, args.cpu_seconds, kernel=args.kernel, blocks=args.blocks,
                                       prior=args.prior)

    # each rank: its own independent problem of the same shape
    p = inputs.make_problem(rank_workload(w, rank))
    from paper_1307_4370_gb300 import autotune
    tune = autotune.autotune_tile(w.n, p.uv, w.J, reps=10)  # grid-tile schedule, measured and cached
    ctx = binding.Context(w.n, p.uv.astype(np.float32), J=w.J, tile=tune["tile"], kernel=args.kernel)
    x_true = torch.tensor(p.x_true.astype(np.complex64), device=dev)
    y0 = ctx.phi(x_true)
    sig = float(torch.linalg.vector_norm(y0).item()) / math.sqrt(w.M) * 10 ** (-w.isnr_db / 20)
    noise = torch.tensor(p.noise_unit.astype(np.complex64), device=dev)
    y = y0 + sig * noise
    eps = binding.l2_bound(w.M, sig)
    st = ctx.sdmm_state()
    if args.prior == "tv":
        st.set_prior("tv")
    st.init(y, eps, cg_iters=w.cg_iters)
    if args.blocks > 0:
        st.set_blocks(*block_table(w.M, args.blocks, eps, binding.l2_bound))
    if args.precision == "bf16":
        st.set_data_bf16(y)
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    state = {"iters": 0, "round": 0}

    def one_step():
        if state["iters"] > 0 and state["iters"] % REWEIGHT_EVERY == 0 and state["round"] < ROUNDS - 1:
            state["round"] += 1
            st.reweight(state["round"])
        st.step()
        state["iters"] += 1

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # --- device-timed steps (value) -------------------------------------
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    l0 = binding.launch_count()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier()
    nvtx_range("timed_steps")  # the range a launch-list capture of the timed steps filters on
    for k in range(args.steps):
        flush.fill_(float(k))                # evict L2 between steps (not timed)
        evs[k][0].record(stream)
        one_step()
        evs[k][1].record(stream)
    nvtx_range(None)
    barrier()
    gpu_launches = binding.launch_count() - l0
    step_ms = [a.elapsed_time(b) for a, b in evs]
    total_ms = max_over_ranks(float(np.sum(step_ms)), dev)
    value = world * args.steps / (total_ms / 1e3)

    # --- Phi + Phi^H visibility rate (public calls, L2 flushed) ----------
    xr = torch.randn(w.n, w.n, dtype=torch.complex64, device=dev)
    yv = torch.empty(w.M, dtype=torch.complex64, device=dev)
    xa = torch.empty(w.n, w.n, dtype=torch.complex64, device=dev)
    reps = 50
    pe = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for k in range(reps):
        flush.fill_(float(k))
        pe[k][0].record(stream)
        ctx.phi(xr, out=yv)
        ctx.phi_adj(yv, out=xa)
        pe[k][1].record(stream)
    torch.cuda.synchronize()
    phi_ms = float(np.mean([a.elapsed_time(b) for a, b in pe]))
    gvis = world * w.M / (phi_ms / 1e3) / 1e9

    # --- end to end through the C ABI with host buffers -----------------
    y_host = y.cpu().pin_memory()
    x_host = torch.empty((w.n, w.n), dtype=torch.complex64).pin_memory()
    e2e_steps = max(1, min(args.steps, 100))
    barrier()
    t0 = time.perf_counter()
    for k in range(e2e_steps):
        flush.fill_(float(k))
        if args.precision == "bf16":
            st.set_data_bf16(y_host)  # H2D of this step's data, stored as bf16 on the device
        else:
            st.set_data(y_host)       # H2D of this step's data
        one_step()
        st.get_image(x_host)     # D2H of the step's result (synchronises)
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t0, dev)
    # the flush is inside this wall-clock region: take it out with its own timing
    fl = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(10)]
    for a, b in fl:
        a.record(stream)
        flush.fill_(1.0)
        b.record(stream)
    torch.cuda.synchronize()
    flush_s = float(np.mean([a.elapsed_time(b) for a, b in fl])) / 1e3
    e2e_value = world * e2e_steps / max(e2e_s - e2e_steps * flush_s, 1e-9)
    clocks = sampler.stop()

    # --- final-image SNR of the two storage forms of y at equal iteration count
    quality = None
    if rank == 0 and not args.no_quality:
        x_true_r = torch.tensor(p.x_true.astype(np.float32), device=dev)
        quality = {"iterations": QUALITY_ITERS}
        for form in ("c64", "bf16"):
            sq = ctx.sdmm_state()
            if args.prior == "tv":
                sq.set_prior("tv")
            sq.init(y, eps, cg_iters=w.cg_iters)
            if args.blocks > 0:
                sq.set_blocks(*block_table(w.M, args.blocks, eps, binding.l2_bound))
            if form == "bf16":
                sq.set_data_bf16(y)
            for _ in range(QUALITY_ITERS):
                sq.step()
            quality[f"snr_db_{form}"] = snr_db(x_true_r, sq.get_image().reshape(w.n, w.n))
            sq.close()
        quality["note"] = ("SNR = 20 log10(||x|| / ||x - Re x_hat||) (§6) after the same number of SDMM iterations "
                           "from x_hat = 0, complex64 y and bf16-stored y with FP32 scales per 4096")

    # --- 32 uneven problems batched (the batching workload), on rank 0 ------
    batch = None
    if rank == 0 and world == 1 and not args.no_batch:
        batch = measure_batch(min(args.steps, 20), 3)

    # --- per-kernel times (profiled steps) and the roofline ---------------
    ctx.profile_enable(True)
    prof_steps = min(args.steps, 30)
    for k in range(prof_steps):
        flush.fill_(float(k))
        one_step()
    prof = ctx.profile_collect()
    ctx.profile_enable(False)
    dom = max(prof, key=lambda r: r[2])
    abytes = algorithmic_bytes(w)
    peak, peak_kind = peaks()
    per_launch_s = dom[2] / dom[1] / 1e3
    achieved = abytes.get(dom[0], float("nan")) / per_launch_s / 1e9
    total_prof = sum(r[2] for r in prof)
    kernels = {nm: {"launches": n_, "ms": round(ms, 4), "share": round(ms / total_prof, 4),
                    "us_per_launch": round(ms / n_ * 1e3, 2),
                    "alg_GBps": (round(abytes[nm] / (ms / n_ / 1e3) / 1e9, 1) if nm in abytes else None)}
               for nm, n_, ms in prof}

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {**workload_config(w), "prior": args.prior, "kernel": args.kernel, "blocks": args.blocks,
                       "y_storage": args.precision,
                       "l2": f"flushed between timed steps ({L2_FLUSH_BYTES >> 20} MiB write)",
                       "cuda_graph": True, "tile": tune["tile"], "tile_ms": tune["timings"],
                       "parallelism": f"{world} independent problems (one per GPU)"},
            "phi_phiadj": {"value": gvis, "unit": "Gvis/s", "ms": phi_ms},
            "roofline": {"bound": "hbm", "kernel": dom[0], "achieved": achieved, "peak": peak,
                         "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": dram_traffic(w.name, dom[0]), "alg_bytes_per_launch": abytes.get(dom[0]),
                         "us_per_launch": per_launch_s * 1e6},
            "kernels": kernels,
            "cpu_baseline": cpu_entry,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 8 * w.M,
                    "d2h_bytes_per_step": 8 * w.n * w.n},
            "gpu_launches": gpu_launches,
            "quality": quality,
            "batch32": batch,
            "clocks": clocks,
        }
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


def snr_db(x_true, x_hat) -> float:
    """Reconstruction SNR of §6, 20 log10(||x|| / ||x - x_hat||), of the real image."""
    import torch

    xr = x_hat.real.double() if torch.is_complex(x_hat) else x_hat.double()
    xt = x_true.double()
    return float(20.0 * torch.log10(torch.linalg.vector_norm(xt) / torch.linalg.vector_norm(xt - xr)).item())


def measure_batch(steps: int, warmup: int) -> dict:
    """32 uneven problems advanced together (one CUDA graph per batch iteration)
    against the same problems stepped one after another; final-image SNRs of
    both (the batch only changes the schedule, so the iterates are equal)."""
    import torch

    from paper_1307_4370_gb300 import binding

    ws = inputs.batch_workloads(32)

    def make_states():
        out = []
        for w in ws:
            p = inputs.make_problem(w)
            ctx = binding.Context(w.n, p.uv.astype(np.float32), J=w.J)
            xt = torch.tensor(p.x_true.astype(np.complex64), device="cuda")
            y0 = ctx.phi(xt)
            sig = float(torch.linalg.vector_norm(y0).item()) / math.sqrt(w.M) * 10 ** (-w.isnr_db / 20)
            y = y0 + sig * torch.tensor(p.noise_unit.astype(np.complex64), device="cuda")
            st = ctx.sdmm_state()
            st.init(y, binding.l2_bound(w.M, sig), cg_iters=w.cg_iters)
            out.append((ctx, st, torch.tensor(p.x_true.astype(np.float32), device="cuda")))
        return out

    K = max(1, min(steps, 50))
    W = max(3, warmup)
    made = make_states()
    states = [st for _, st, _ in made]
    batch = binding.Batch(states)
    batch.step(W)
    stream = torch.cuda.current_stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    l0 = binding.launch_count()
    a.record(stream)
    batch.step(K)
    b.record(stream)
    torch.cuda.synchronize()
    launches = binding.launch_count() - l0
    batched_ms = a.elapsed_time(b)
    snr_b = [snr_db(xt, st.get_image().reshape(xt.shape)) for _, st, xt in made]
    batch.close()
    # the same problems, fresh, stepped one after another with their own graphs
    made2 = make_states()
    for _ in range(W):
        for _, st, _ in made2:
            st.step()
    torch.cuda.synchronize()
    a.record(stream)
    for _ in range(K):
        for _, st, _ in made2:
            st.step()
    b.record(stream)
    torch.cuda.synchronize()
    seq_ms = a.elapsed_time(b)
    snr_s = [snr_db(xt, st.get_image().reshape(xt.shape)) for _, st, xt in made2]
    total_iters = K * len(ws)
    return {"value": total_iters / (batched_ms / 1e3), "unit": "instance-iterations/s", "steps": K, "warmup": W,
            "ms_per_step": batched_ms / K, "gpu_launches": launches,
            "sizes": [[w.n, w.M, w.J] for w in ws],
            "snr_db_mean": float(np.mean(snr_b)),
            "sequential": {"value": total_iters / (seq_ms / 1e3), "unit": "instance-iterations/s",
                           "snr_db_mean": float(np.mean(snr_s)),
                           "note": "same problems, one CUDA-graph step per problem in turn"},
            "l2": "not flushed (one graph per batch iteration)"}


def run_batch(args):
    import torch

    torch.cuda.set_device(0)
    r = measure_batch(args.steps, args.warmup)
    out = {"metric": "SDMM-SARA instance-iterations/sec (32 uneven problems)", "value": r["value"],
           "unit": r["unit"], "n_gpus": 1, "steps": r["steps"], "warmup": r["warmup"],
           "ms_per_step": r["ms_per_step"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32", "data": "synthetic",
           "config": {"workload": "batch32: 32 problems, n in {128,192,256,384,512}, M in [0.2N, 2N], J in {4,6}",
                      "sizes": r["sizes"], "l2": r["l2"]},
           "quality": {"snr_db_mean_batched": r["snr_db_mean"],
                       "snr_db_mean_sequential": r["sequential"]["snr_db_mean"],
                       "iterations": r["steps"] + r["warmup"]},
           "sequential": r["sequential"], "gpu_launches": r["gpu_launches"]}
    print(json.dumps(out), flush=True)


def main():
    args = parse_args()
    if args.workload == "batch32":
        run_batch(args)
        return
    w = inputs.WORKLOADS[args.workload]
    if args.impl == "reference":
        run_reference(args, w)
    else:
        run_gpu(args, w)


if __name__ == "__main__":
    main()
