"""Autotuner of the grid-tile schedule of G and G^T.

The tile side (8..64 cells) decides how the visibilities are grouped for the
degridding gather and the gridding adjoint: larger tiles duplicate fewer
footprints across tile edges, smaller tiles give more, lighter work units.
The best choice depends on the image side n, the number of visibilities M,
the kernel support J and the GPU, so it is measured: each candidate context
times the operator mix of one SDMM iteration (Phi + Phi^H and a 10-step CG
solve, whose G^T G runs in the one-pass Gram form) with CUDA events, and the
fastest is kept, cached per (device, n, M, J) in a JSON file.  The schedule never changes the operator;
all candidates compute the same Phi up to floating-point summation order.
"""
from __future__ import annotations

import json
import os

import numpy as np
import torch

from . import binding

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "purify_gb300", "autotune.json")
CANDIDATES = (16, 32, 64)


def valid_tiles(n: int, J: int, candidates=CANDIDATES) -> list[int]:
    L = 2 * n
    return [t for t in candidates if t >= J and L % t == 0 and L // t >= 2]


def _key(n: int, M: int, J: int) -> str:
    dev = torch.cuda.get_device_name(torch.cuda.current_device()) if torch.cuda.is_available() else "cpu"
    return f"{dev}|n={n}|M={M}|J={J}"


def _load(path: str) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _save(path: str, table: dict) -> None:
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def time_phi_pair(ctx: binding.Context, reps: int = 20) -> float:
    """Mean milliseconds of one Phi followed by one Phi^H."""
    x = torch.randn(ctx.n, ctx.n, dtype=torch.complex64, device=ctx.device)
    y = torch.empty(ctx.M, dtype=torch.complex64, device=ctx.device)
    xa = torch.empty(ctx.n, ctx.n, dtype=torch.complex64, device=ctx.device)
    for _ in range(3):
        ctx.phi(x, out=y)
        ctx.phi_adj(y, out=xa)
    s = torch.cuda.current_stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(s)
    for _ in range(reps):
        ctx.phi(x, out=y)
        ctx.phi_adj(y, out=xa)
    b.record(s)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def time_cg(ctx: binding.Context, iters: int = 10, reps: int = 5) -> float:
    """Mean milliseconds of a CG solve of ``iters`` steps on Q = Phi^H Phi + 2I
    (the x-update of every SDMM iteration; G^T G runs in its one-pass form)."""
    b = torch.randn(ctx.n, ctx.n, dtype=torch.complex64, device=ctx.device)
    x0 = torch.zeros_like(b)
    ctx.cg_solve(b, x0, iters)
    s = torch.cuda.current_stream()
    a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(s)
    for _ in range(reps):
        ctx.cg_solve(b, x0, iters)
    e.record(s)
    torch.cuda.synchronize()
    return a.elapsed_time(e) / reps


def autotune_tile(n: int, uv, J: int, levels: int = 4, bases_mask: int = binding.SARA_MASK,
                  cache_path: str | None = DEFAULT_CACHE, reps: int = 20, refresh: bool = False) -> dict:
    """Pick the tile side for (n, M, J); returns {"tile", "ms", "timings"}."""
    uv = np.asarray(uv, dtype=np.float32)
    M = int(uv.shape[0])
    key = _key(n, M, J)
    table = _load(cache_path) if cache_path else {}
    if not refresh and key in table:
        return table[key]
    timings = {}
    for t in valid_tiles(n, J):
        ctx = binding.Context(n, uv, J=J, levels=levels, bases_mask=bases_mask, tile=t)
        # the operator mix of one SDMM iteration: a CG solve (Gram form) plus Phi and Phi^H
        timings[str(t)] = time_phi_pair(ctx, reps) + time_cg(ctx, 10, max(1, reps // 4))
        ctx.close()
    best = min(timings, key=timings.get)
    entry = {"tile": int(best), "ms": timings[best], "timings": timings}
    if cache_path:
        table[key] = entry
        _save(cache_path, table)
    return entry
