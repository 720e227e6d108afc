"""Autotuner for the inverse-update scheme of a crowd and its CTA width: Sherman-Morrison
or a delayed (Woodbury) window of rank k, with 128, 160 or 256 threads per walker, chosen by
timing a few generations of each candidate on the current GPU; then (`tune_plan`) the move
kernel's plan for the winner: how the orbital stencil reaches shared memory (TMA copies
or per-thread loads) and the shared-memory layout (shared or compact).  Results are cached
in a JSON file keyed by system size, crowd size, precision and GPU name.

The timing uses CUDA events on a dedicated stream around qmc_sweep(1) calls; the crowd
under test is built from the same workload the caller will run.
"""
from __future__ import annotations

import json
import os

import numpy as np

DEFAULT_CANDIDATES = (("sm", 1), ("delayed", 2), ("delayed", 4), ("delayed", 8),
                      ("delayed", 16), ("delayed", 32), ("delayed", 64))
WIDTHS = (128, 160, 256)


def cache_path() -> str:
    return os.environ.get("QMCGB_TUNE_CACHE",
                          os.path.join(os.path.dirname(os.path.abspath(__file__)),
                                       ".autotune_cache.json"))


def _key(wl, precision: str, gpu: str) -> str:
    return (f"{gpu}|N={wl.n_el}|n={wl.n_up}|G={wl.grid}|W={wl.n_walkers}|NI={wl.n_ions}|"
            f"{precision}|v3")


def time_candidate(wl, precision: str, update: str, k: int, gens: int = 4,
                   warmup: int = 2, cta_threads: int = 0, staging: str = "auto",
                   layout: str = "auto", want=None) -> float:
    """Median milliseconds of one generation of the crowd with this update scheme (inf
    when the configuration does not fit the GPU, or when `want` (a dict of
    kernel_config entries) is given and the library's plan differs from it)."""
    import torch

    from . import qmcgb
    prev = torch.cuda.current_stream()
    s = torch.cuda.Stream()
    torch.cuda.set_stream(s)
    try:
        try:
            c = qmcgb.Crowd.from_workload(wl, precision=precision, update=update, delay_rank=k,
                                          stream=s.cuda_stream, cta_threads=cta_threads,
                                          staging=staging, layout=layout)
        except qmcgb.QmcError as e:
            if e.status == qmcgb.QMC_ERR_UNSUPPORTED:
                return float("inf")
            raise
        if want and any(c.kernel_config[key] != v for key, v in want.items()):
            c.close()
            return float("inf")
        c.qmc_load_positions(np.ascontiguousarray(wl.positions()))
        c.qmc_recompute()
        for _ in range(warmup):
            c.qmc_sweep(1, stats=False)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(gens)]
        for a, b in ev:
            a.record(s)
            c.qmc_sweep(1, stats=False)
            b.record(s)
        torch.cuda.synchronize()
        ms = sorted(a.elapsed_time(b) for a, b in ev)
        c.close()
        return ms[len(ms) // 2]
    finally:
        torch.cuda.set_stream(prev)


def tune(wl, precision: str = "mixed", candidates=DEFAULT_CANDIDATES, gens: int = 4,
         use_cache: bool = True, widths=WIDTHS):
    """(update, k, cta_threads, {candidate: ms}) for the fastest candidate; cached per GPU
    and shape."""
    import torch
    gpu = torch.cuda.get_device_name()
    key = _key(wl, precision, gpu)
    path = cache_path()
    cache = {}
    if use_cache and os.path.exists(path):
        try:
            cache = json.load(open(path))
        except (OSError, ValueError):
            cache = {}
        if key in cache:
            e = cache[key]
            return e["update"], e["k"], e["nt"], e["table"]
    table = {}
    for nt in widths:
        for update, k in candidates:
            table[f"{update}:{k}:{nt}"] = time_candidate(wl, precision, update, k, gens=gens,
                                                         cta_threads=nt)
    best = min(table, key=table.get)
    update, k, nt = best.split(":")[0], int(best.split(":")[1]), int(best.split(":")[2])
    cache[key] = {"update": update, "k": k, "nt": nt, "table": table}
    try:
        with open(path + ".tmp", "w") as fh:
            json.dump(cache, fh, indent=1)
        os.replace(path + ".tmp", path)
    except OSError:
        pass
    return update, k, nt, table


def tune_plan(wl, precision: str, update: str, k: int, cta_threads: int, gens: int = 4,
              use_cache: bool = True):
    """(staging, layout, {plan: ms}) for the fastest move-kernel plan of a tuned scheme:
    stencil staging 'auto' (TMA where the library can: one copy per move, or the ring of
    boxes beyond 256 orbitals) or 'ldg' (per-thread loads), layout 'shared' or 'compact'.
    Plans the library cannot build (or builds identically to another) are skipped."""
    import torch
    gpu = torch.cuda.get_device_name()
    key = _key(wl, precision, gpu) + f"|plan|{update}:{k}:{cta_threads}"
    path = cache_path()
    cache = {}
    if use_cache and os.path.exists(path):
        try:
            cache = json.load(open(path))
        except (OSError, ValueError):
            cache = {}
        if key in cache:
            e = cache[key]
            return e["staging"], e["layout"], e["table"]
    table = {}
    seen = set()
    from . import qmcgb
    for staging in ("auto", "ldg"):
        for layout in ("shared", "compact"):
            try:
                c = qmcgb.Crowd.from_workload(wl, precision=precision, update=update,
                                              delay_rank=k, cta_threads=cta_threads,
                                              staging=staging, layout=layout, n_walkers=1)
            except qmcgb.QmcError:
                continue
            cfg = c.kernel_config
            c.close()
            sig = (cfg["stencil_tma"], cfg["layout"], cfg["b_in_smem"], cfg["tc_flush"])
            if sig in seen:
                continue
            seen.add(sig)
            table[f"{staging}:{layout}"] = time_candidate(
                wl, precision, update, k, gens=gens, cta_threads=cta_threads, staging=staging,
                layout=layout, want={"stencil_tma": cfg["stencil_tma"], "layout": cfg["layout"]})
    best = min(table, key=table.get)
    staging, layout = best.split(":")
    cache[key] = {"staging": staging, "layout": layout, "table": table}
    try:
        with open(path + ".tmp", "w") as fh:
            json.dump(cache, fh, indent=1)
        os.replace(path + ".tmp", path)
    except OSError:
        pass
    return staging, layout, table
