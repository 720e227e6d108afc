"""Electron-move throughput of the PbyP crowd move on one GB300 (or N replicas).

Metric: electron moves per second over the crowd (walkers x electrons x generations /
time), FP32-mixed path (headline `value`) next to the FP64 path, with the energy each
reaches.  A step is one generation: every electron of every walker proposed once
(Alg. 1 lines 4-9), pending delayed updates applied, the FP64 recompute at its cadence,
and the local energy (line 11).  Inputs are device resident when the timed region starts;
L2 is flushed (a 256 MiB write) between timed steps, outside the per-step CUDA events.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (test infrastructure) on the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "electron moves/sec over crowd, FP32-mixed vs FP64 GPU, at stated energy error"
UNIT = "electron-moves/s"
CSRC = os.path.join(ROOT, "paper_2209_14487_gb300", "csrc")


def bytes_per_move(n, N, s, p_acc, update, k):
    """Algorithmic bytes of one electron move (stencil, inverse column, positions and
    distance rows, accepted rows, and the inverse update)."""
    b = 64 * n * s + n * s + 8 * N * s + p_acc * 5 * n * s
    if update == "sm":
        b += p_acc * 2 * n * n * s
    else:
        b += 2 * n * k * s + p_acc * (2 * n * s + 3 * n * n * s / k)
    return b


def source_sha() -> str:
    h = hashlib.sha256()
    for f in sorted(os.listdir(CSRC)):
        if f.endswith((".cu", ".cuh", ".h")):
            h.update(open(os.path.join(CSRC, f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, or None when the
    kernel sources changed since the capture."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        d = json.load(open(path))
        e = d.get(kernel)
        if e and e.get("source_sha") == source_sha():
            return e.get("bytes_per_launch")
    except Exception:
        return None
    return None


def l2_copy_peak():
    """GB/s of an L2-resident elementwise copy (read + write bytes): 40 launches of
    b = a * 1 over buffers of 16, 24 or 32 MiB each (both buffers together stay within the
    129 MB L2), captured once in a CUDA graph so that the launches run back to back; the
    best of 5 replays of each size after warm-up, the best size reported.  (Single
    device-to-device copies of such buffers, timed launch by launch, measured lower: their
    launch gaps are comparable to a copy.)"""
    import torch
    best_gbs = 0.0
    for mib in (16, 24, 32):
        n = mib * 1024 * 1024 // 4
        a = torch.ones(n, dtype=torch.float32, device="cuda")
        b = torch.empty_like(a)
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(s):
            for _ in range(3):
                torch.mul(a, 1.0, out=b)
            with torch.cuda.graph(g, stream=s):
                for _ in range(40):
                    torch.mul(a, 1.0, out=b)
        torch.cuda.synchronize()
        for _ in range(2):
            g.replay()
        best = float("inf")
        for _ in range(5):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            g.replay()
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1) / 1000.0)
        best_gbs = max(best_gbs, 40 * 2 * 4 * n / best / 1e9)
        del g, a, b
    return best_gbs


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms in the background."""

    Q = ("uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.uuid = uuid
        self.proc = None
        # the raw samples go to $QMCGB_CLOCKS_DIR (default: the temporary directory)
        d = os.environ.get("QMCGB_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(d, f"clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 8:
                continue
            rows.append(parts)
        if self.uuid:
            mine = [r for r in rows if self.uuid in r[0]]
            rows = mine or rows
        try:
            sm = [float(r[1]) for r in rows]
            smax = max(float(r[2]) for r in rows)
        except (ValueError, IndexError):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unparsed"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4)
                          if r[4 + k].lower() in ("active", "1", "yes")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": reasons, "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_max(x: float, ws: int) -> float:
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64,
                     device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(x: float, ws: int) -> float:
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64,
                     device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t)
    return float(t.item())


def aggregate_value(units_per_rank: float, seconds_local: float, ws: int) -> float:
    """Whole-job throughput: every rank processes `units_per_rank`; the job takes as long
    as the slowest rank."""
    return ws * units_per_rank / reduce_max(seconds_local, ws)


def barrier(ws: int):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


# synthetic nonlocal channels for --nlpp: amplitudes, widths (l = 0, 1, 2) and the cutoff
NLPP = ((1.2, -0.8, 0.5), (0.7, 0.9, 0.8), 1.5)
# Ewald Coulomb for --coulomb: alpha L and mmax; the ion charge makes the cell neutral


def coulomb_args(wl):
    return (wl.n_el / max(1, wl.n_ions), 8.0 / wl.L, 10)


LAYOUT = "auto"  # the move kernel's shared-memory layout (--layout)
STAGING = "auto"  # how each move's orbital stencil reaches shared memory (--staging)


def make_crowd(wl, precision, update, k, stream, crowd_id, nt=0, nlpp=None, coulomb=None):
    from paper_2209_14487_gb300 import qmcgb
    c = qmcgb.Crowd.from_workload(wl, precision=precision, update=update, delay_rank=k,
                                  stream=stream, cta_threads=nt,
                                  layout=LAYOUT if precision == "mixed" else "auto",
                                  staging=STAGING if precision == "mixed" else "auto")
    if nlpp is not None:
        c.qmc_load_nlpp(*nlpp)
    if coulomb is not None:
        c.qmc_load_coulomb(*coulomb)
    c.qmc_load_positions(np.ascontiguousarray(wl.positions(crowd_id=crowd_id)))
    c.qmc_recompute()
    return c


def time_path(wl, precision, update, k, steps, warmup, crowd_id, flush_buf, nt=0, nlpp=None,
              coulomb=None, energy=None):
    """Per-step CUDA-event timing of qmc_sweep(1) on torch's current stream.  Then, outside
    the timed region: the cost of a generation that carries the FP64 recompute (timed
    alone, so that its share 1/n_recompute can be added to every step), and with `energy`
    = (equilibration, generations) the E_L of an equilibrated chain of the same crowd."""
    import torch
    stream = torch.cuda.Stream()  # a real stream: torch's default is the legacy NULL stream
    torch.cuda.set_stream(stream)
    c = make_crowd(wl, precision, update, k, stream.cuda_stream, crowd_id, nt, nlpp, coulomb)
    eloc = torch.zeros((warmup + steps, wl.n_walkers), dtype=torch.float64, device="cuda")
    for g in range(warmup):
        c.qmc_sweep(1, eloc[g], stats=False)
    torch.cuda.synchronize()
    n_rc = wl.n_recompute
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    gens = []
    guard = precision == "mixed"
    rep0 = c.qmc_get_guard()[1] if guard else 0
    launches0 = c.launch_count
    for s in range(steps):
        flush_buf.add_(1.0)  # write 256 MiB on this stream: evicts the previous step from L2
        gens.append(c.generation)
        ev[s][0].record(stream)
        c.qmc_sweep(1, eloc[warmup + s], stats=False)
        ev[s][1].record(stream)
    torch.cuda.synchronize()
    launches = c.launch_count - launches0
    repairs = (c.qmc_get_guard()[1] - rep0) if guard else None
    ms = [a.elapsed_time(b) for a, b in ev]
    # steps without the FP64 recompute run exactly one launch of the fused move kernel
    due = [n_rc > 0 and (g + 1) % n_rc == 0 for g in gens]
    plain = [m for m, d in zip(ms, due) if not d]
    e = eloc[warmup:].double().cpu().numpy()
    # acceptance ratio of the chain (one more generation, after the timed region)
    c2 = c.qmc_sweep(2, None, stats=True)
    p_acc = c2.n_accept / max(1, c2.n_moves)
    # a generation with the recompute (sweep without E_L, FP64 LU of every walker, E_L),
    # timed alone under the same L2 flush, three times
    rc_ms = []
    if n_rc > 0:
        g_next = c.generation
        for _ in range(3):
            c.generation = (c.generation // n_rc + 1) * n_rc - 1
            flush_buf.add_(1.0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            c.qmc_sweep(1, None, stats=False)
            b.record(stream)
            torch.cuda.synchronize()
            rc_ms.append(a.elapsed_time(b))
        c.generation = g_next
    chain = None
    if energy is not None:
        n_eq, n_e, snap = energy
        c.qmc_sweep(n_eq, None, stats=False)
        ech = torch.zeros((n_e, wl.n_walkers), dtype=torch.float64, device="cuda")
        snaps, repairs_chain = [], 0
        step = snap if snap else n_e
        for g0 in range(0, n_e, step):
            g1 = min(n_e, g0 + step)
            st = c.qmc_sweep(g1 - g0, ech[g0:g1], stats=True)
            repairs_chain += getattr(st, "n_repair", 0)
            if snap:  # the chain's configuration and its E_L after generation g1 - 1
                snaps.append((c.qmc_get_positions(), ech[g1 - 1].cpu().numpy()))
        chain = {"eloc": ech.cpu().numpy(), "repairs": repairs_chain, "snaps": snaps}
    c.close()
    torch.cuda.set_stream(torch.cuda.default_stream())
    return {"ms": ms, "plain_ms": plain, "eloc": e, "p_acc": p_acc, "launches": launches,
            "due": due, "recompute_step_ms": rc_ms, "chain": chain, "repairs": repairs}


def amortised(r, n_rc):
    """Per-step times with the FP64 recompute's share: a timed step that carried no
    recompute gets (recompute generation - plain generation) / n_recompute added; a timed
    step that carried one keeps its own time (so no recompute is counted twice)."""
    if n_rc <= 0 or not r["recompute_step_ms"]:
        return list(r["ms"]), 0.0
    plain = r["plain_ms"] or r["ms"]
    extra = max(0.0, statistics.mean(r["recompute_step_ms"]) - statistics.mean(plain))
    return [m if d else m + extra / n_rc for m, d in zip(r["ms"], r["due"])], extra


def crowds_path(wl, n_crowds, update, k, steps, warmup, flush_buf, nt=0):
    """The workload's walkers split over `n_crowds` crowds, each on its own CUDA stream
    (the batched driver's crowds, Alg. 4): every step enqueues one qmc_sweep(1) per crowd
    (asynchronous: E_L stays on the device) between a start event the crowds' streams wait
    on and an end event that waits on all of them."""
    import dataclasses

    import torch
    main = torch.cuda.Stream()
    torch.cuda.set_stream(main)
    Wc = wl.n_walkers // n_crowds
    wlc = dataclasses.replace(wl, n_walkers=Wc)
    streams = [torch.cuda.Stream() for _ in range(n_crowds)]
    crowds = [make_crowd(wlc, "mixed", update, k, s.cuda_stream, i, nt)
              for i, s in enumerate(streams)]
    eloc = [torch.zeros(Wc, dtype=torch.float64, device="cuda") for _ in range(n_crowds)]
    torch.cuda.synchronize()
    ms = []
    for g in range(warmup + steps):
        flush_buf.add_(1.0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(main)
        for s in streams:
            s.wait_event(a)
        for c, e in zip(crowds, eloc):
            c.qmc_sweep(1, e, stats=False)
        for s in streams:
            d = torch.cuda.Event()
            d.record(s)
            main.wait_event(d)
        b.record(main)
        if g >= warmup:
            ms.append((a, b))
    torch.cuda.synchronize()
    out = [x.elapsed_time(y) for x, y in ms]
    for c in crowds:
        c.close()
    torch.cuda.set_stream(torch.cuda.default_stream())
    return out, Wc * n_crowds


def scan_main(args, wl, ws, rank, cfg):
    """Throughput against walkers per GPU (the shape of the paper's Fig. 5 scan) and against
    the number of crowds the walkers are split into, mixed path."""
    import dataclasses

    import torch
    try:
        uuid = str(torch.cuda.get_device_properties(torch.cuda.current_device()).uuid)
    except Exception:
        uuid = None
    flush = torch.zeros(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    update = "sm" if args.update == "auto" else args.update
    k = 1 if update == "sm" else (args.delay_rank or 8)
    nt = args.cta_threads
    walkers = [int(x) for x in args.walker_scan.split(",")] if args.walker_scan else []
    crowds = [int(x) for x in args.crowds.split(",")] if args.crowds else []
    scan, cscan = [], []
    barrier(ws)
    with ClockSampler(uuid) as clk:
        for W in walkers:
            r = time_path(dataclasses.replace(wl, n_walkers=W), "mixed", update, k, args.steps,
                          args.warmup, rank, flush, nt)
            plain = r["plain_ms"] or r["ms"]
            scan.append({"walkers": W, "value": W * wl.n_el / (statistics.mean(r["ms"]) / 1e3),
                         "ms_per_step": statistics.mean(r["ms"]),
                         "ms_per_plain_step": statistics.mean(plain)})
        for C in crowds:
            ms, Wt = crowds_path(wl, C, update, k, args.steps, args.warmup, flush, nt)
            cscan.append({"crowds": C, "walkers": Wt,
                          "value": Wt * wl.n_el / (statistics.mean(ms) / 1e3),
                          "ms_per_step": statistics.mean(ms)})
    torch.cuda.synchronize()
    barrier(ws)
    head = (scan or cscan)[-1]
    out = {"metric": METRIC, "value": head["value"] * ws, "unit": UNIT, "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms_per_step"],
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
           "data": "synthetic",
           "config": dict(cfg, mode="scan", precision="mixed", update=f"{update} k={k}",
                          cta_threads=nt or "library", parallelism=f"replicas x{ws}"),
           "walker_scan": scan, "crowd_scan": cscan, "clocks": clk.summary()}
    if rank == 0:
        print(json.dumps(out))


def batch_main(args, ws, rank, cfg):
    """The mixed-size batch (64/192/384 electrons with 512/256/128 walkers): one launch per
    generation for every walker of the three crowds (qmc_batch_sweep, CUDA graph replay),
    against the same crowds swept one after the other."""
    import torch

    from paper_2209_14487_gb300 import qmcgb, workloads
    try:
        uuid = str(torch.cuda.get_device_properties(torch.cuda.current_device()).uuid)
    except Exception:
        uuid = None
    flush = torch.zeros(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    nt = args.cta_threads or 128  # one width for the whole batch
    wls = [make() for make in workloads.MIXED_BATCH]
    crowds = []
    for wl in wls:
        c = qmcgb.Crowd.from_workload(wl, precision="mixed", stream=stream.cuda_stream,
                                      cta_threads=nt)
        c.qmc_load_positions(np.ascontiguousarray(wl.positions(crowd_id=rank)))
        c.qmc_recompute()
        crowds.append(c)
    b = qmcgb.Batch(crowds)
    moves = sum(wl.n_walkers * wl.n_el for wl in wls)

    def timed(step):
        ms = []
        for g in range(args.warmup + args.steps):
            flush.add_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            if g >= args.warmup:
                ms.append((e0, e1))
        torch.cuda.synchronize()
        return [a.elapsed_time(z) for a, z in ms]

    barrier(ws)
    with ClockSampler(uuid) as clk:
        l0 = b.launch_count
        ms_b = timed(lambda: b.qmc_batch_sweep(1, eloc=False, stats=False))
        launches = b.launch_count - l0
        ms_s = timed(lambda: [c.qmc_sweep(1, stats=False) for c in crowds])
    _, st = b.qmc_batch_sweep(1, eloc=False, stats=True)
    barrier(ws)
    value = aggregate_value(moves * args.steps, sum(ms_b) / 1000.0, ws)
    t_b = statistics.mean(ms_b) / 1000.0
    bpg = sum(wl.n_walkers * wl.n_el *
              bytes_per_move(wl.n_orb, wl.n_el, 4, s_.n_accept / max(1, s_.n_moves), "sm", 1)
              for wl, s_ in zip(wls, st))
    hbm, src = peaks()
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": statistics.mean(ms_b), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": "mixed-size batch: " + " + ".join(
               f"{wl.name} ({wl.n_el} e, {wl.n_walkers} walkers)" for wl in wls),
               "step": "one generation of every walker of the three crowds",
               "l2": cfg["l2"], "precision": "mixed", "update": "sm", "cta_threads": nt,
               "parallelism": f"replicas x{ws}"},
           "sequential": {"value": aggregate_value(moves * args.steps, sum(ms_s) / 1000.0, ws),
                          "ms_per_step": statistics.mean(ms_s), "unit": UNIT},
           "roofline": {"bound": "hbm", "achieved": bpg / t_b / 1e9, "peak": hbm, "unit": "GB/s",
                        "frac": bpg / t_b / 1e9 / hbm, "traffic": None,
                        "kernel": "move_kernel_batch<float> (fused generation, three crowds)",
                        "bytes_per_generation": bpg, "peak_source": src},
           "gpu_launches": launches, "clocks": clk.summary()}
    b.close()
    for c in crowds:
        c.close()
    torch.cuda.set_stream(torch.cuda.default_stream())
    if rank == 0:
        print(json.dumps(out))


def dmc_path(wl, update, k, steps, warmup, flush_buf, nt=0, target_frac=0.8, feedback=0.1,
             ws=1, crowd_id=0):
    """Fixed-node DMC generations of the mixed path: qmc_sweep(1) with E_L read back to the
    host, then qmc_dmc_branch (reweighting, branching and the device gather of the new
    population) and the trial-energy feedback E_T = E_est - feedback ln(W / W_target) / tau.
    The crowd starts full (W = capacity) and W_target = target_frac x capacity.  With
    several ranks E_est and W are the whole population's and the ranks even out their
    walkers after each branching (population.exchange).  Each generation is bracketed by
    CUDA events on the crowd's stream; moves = W x N of that generation."""
    import torch

    from paper_2209_14487_gb300 import population, qmcgb
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    cap = wl.n_walkers
    target = max(1, int(round(target_frac * cap)))
    c = qmcgb.Crowd.from_workload(wl, precision="mixed", update=update, delay_rank=k,
                                  stream=stream.cuda_stream, cta_threads=nt, dmc=True,
                                  layout=LAYOUT, staging=STAGING)
    layout = c.kernel_config["layout"]
    staging = {0: "per-thread loads", 1: "one TMA copy per move",
               2: "TMA ring"}[c.kernel_config["stencil_tma"]]
    c.qmc_load_positions(np.ascontiguousarray(wl.positions(crowd_id=crowd_id)))
    c.qmc_recompute()
    e_prev = np.zeros(cap)
    c.qmc_local_energy_batch(e_prev)
    e_trial = float(e_prev.mean())
    if ws > 1:
        e_trial, _ = population.global_estimate(float(cap), float(e_prev.sum()), cap)
    ev_s, ev_b, moves, sizes, e_est_hist = [], [], [], [], []
    launches0 = rep0 = None
    for g in range(warmup + steps):
        timed = g >= warmup
        if timed and launches0 is None:
            torch.cuda.synchronize()
            launches0 = c.launch_count
            rep0 = c.qmc_get_guard()[1]
        e_new = np.zeros((1, c.W))
        if timed:
            flush_buf.add_(1.0)  # evicts the previous generation from L2
            a, m, b = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            a.record(stream)
            moves.append(c.W * wl.n_el)
        c.qmc_sweep(1, e_new, stats=False)
        if timed:
            m.record(stream)
        st, e_prev = c.qmc_dmc_branch(e_prev, e_new[0], e_trial)
        if ws > 1:
            e_est, n_all = population.global_estimate(st.w_sum, st.we_sum, st.n_after)
            e_trial = population.trial_energy(e_est, n_all, ws * target, wl.tau, feedback)
            e_prev = population.exchange(c, e_prev)
        else:
            e_est = st.we_sum / st.w_sum
            e_trial = population.trial_energy(e_est, st.n_after, target, wl.tau, feedback)
        if timed:
            b.record(stream)
            ev_s.append((a, m))
            ev_b.append((a, b))
            sizes.append(st.n_after)
            e_est_hist.append(e_est)
    torch.cuda.synchronize()
    launches = c.launch_count - launches0
    repairs = c.qmc_get_guard()[1] - rep0
    # a generation carrying the FP64 recompute (every wl.n_recompute generations), timed
    # alone, against plain sweeps of the same population
    rc_ms, plain_ms = [], []
    if wl.n_recompute > 0:
        g_next = c.generation
        for due in (False, True, False, True):
            c.generation = ((c.generation // wl.n_recompute + 1) * wl.n_recompute - 1 if due
                            else (c.generation // wl.n_recompute + 1) * wl.n_recompute)
            flush_buf.add_(1.0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            c.qmc_sweep(1, None, stats=False)
            b.record(stream)
            torch.cuda.synchronize()
            (rc_ms if due else plain_ms).append(a.elapsed_time(b))
        c.generation = g_next
    st2 = c.qmc_sweep(1, None, stats=True)
    p_acc = st2.n_accept / max(1, st2.n_moves)
    c.close()
    torch.cuda.set_stream(torch.cuda.default_stream())
    return {"ms": [a.elapsed_time(b) for a, b in ev_b],
            "sweep_ms": [a.elapsed_time(b) for a, b in ev_s], "moves": moves,
            "sizes": sizes, "e_est": e_est_hist, "p_acc": p_acc, "launches": launches,
            "capacity": cap, "target": target, "repairs": repairs, "layout": layout,
            "staging": staging,
            "recompute_step_ms": rc_ms, "plain_probe_ms": plain_ms}


def dmc_main(args, wl, ws, rank, cfg):
    """The --dmc line: fixed-node DMC generations (sweep + branching) of the mixed path."""
    import torch
    from paper_2209_14487_gb300 import qmcgb  # noqa: F401
    try:
        uuid = str(torch.cuda.get_device_properties(torch.cuda.current_device()).uuid)
    except Exception:
        uuid = None
    flush = torch.zeros(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    update, k, nt = args.update, args.delay_rank or 8, args.cta_threads
    tune_table = None
    if update == "auto":
        from paper_2209_14487_gb300 import autotune
        update, k, tuned_nt, tune_table = autotune.tune(
            wl, "mixed", candidates=(("sm", 1), ("delayed", 8), ("delayed", 16), ("delayed", 32)),
            gens=2, widths=(128, 256))
        nt = nt or tuned_nt
    elif update == "sm":
        k = 1
    barrier(ws)
    torch.cuda.synchronize()
    with ClockSampler(uuid) as clk:
        r = dmc_path(wl, update, k, args.steps, args.warmup, flush, nt, ws=ws, crowd_id=rank)
    torch.cuda.synchronize()
    barrier(ws)
    # the FP64 recompute's share: (recompute generation - plain generation) / n_recompute
    # added to every timed generation
    extra = 0.0
    if r["recompute_step_ms"]:
        extra = max(0.0, statistics.mean(r["recompute_step_ms"]) -
                    statistics.mean(r["plain_probe_ms"]))
    ms_all = [m + extra / wl.n_recompute for m in r["ms"]] if extra else list(r["ms"])
    # DMC populations differ between ranks: all ranks' moves over the slowest rank's time
    value = reduce_sum(float(sum(r["moves"])), ws) / reduce_max(sum(ms_all) / 1000.0, ws)
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": statistics.mean(ms_all),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
           "data": "synthetic",
           "recompute": {"every": wl.n_recompute, "recompute_ms": extra,
                         "recompute_step_ms": statistics.mean(r["recompute_step_ms"])
                         if r["recompute_step_ms"] else None,
                         "note": "a generation with the FP64 recompute minus a plain one, "
                                 "timed alone; its 1/every share is in value"},
           "config": dict(cfg, mode="fixed-node DMC: sweep + E_L to host + reweighting, "
                                    "branching and device gather + E_T feedback",
                          capacity=r["capacity"], target_walkers=r["target"],
                          precision="mixed", update=f"{update} k={k}",
                          cta_threads=nt or "library", layout=r["layout"],
                          stencil=r["staging"],
                          parallelism=f"replicas x{ws}")}
    if tune_table is not None:
        out["autotune"] = {"ms_per_generation": tune_table, "chosen": f"{update}:{k}:{nt}"}
    sweep_rate = sum(r["moves"]) / (sum(r["sweep_ms"]) / 1000.0)
    out["dmc"] = {"sweep_only_value": sweep_rate, "unit": UNIT,
                  "branch_ms_mean": statistics.mean(b - a for a, b in
                                                    zip(r["sweep_ms"], r["ms"])),
                  "walkers_min": min(r["sizes"]), "walkers_max": max(r["sizes"]),
                  "walkers_mean": statistics.mean(r["sizes"]),
                  "e_est_mean": statistics.mean(r["e_est"]), "acceptance": r["p_acc"],
                  "guard_repairs": r["repairs"],
                  "walker_generations": int(sum(r["moves"]) / wl.n_el)}
    hbm, src = peaks()
    W_mean = statistics.mean(r["moves"]) / wl.n_el
    bpm = bytes_per_move(wl.n_orb, wl.n_el, 4, r["p_acc"], update, k)
    achieved = sweep_rate * bpm / 1e9
    out["roofline"] = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                       "frac": achieved / hbm, "traffic": None,
                       "kernel": "move_kernel<float> (fused generation)",
                       "bytes_per_move": bpm, "walkers_mean": W_mean, "peak_source": src}
    out["gpu_launches"] = r["launches"]
    out["clocks"] = clk.summary()
    if not args.no_fp64:
        # the FP64 path on the same system: Sherman-Morrison sweeps (its delayed window
        # does not fit in shared memory at this size; the library takes the compact
        # layout) of the DMC population's target walker count, timed like the mixed VMC
        # path (L2 flushed between generations, the recompute amortised); outside the
        # clock record of the DMC generations above
        import dataclasses
        wl64 = dataclasses.replace(wl, n_walkers=r["target"])
        f = time_path(wl64, "fp64", "sm", 1, args.fp64_steps, 3, rank, flush, 128)
        ms64, _ = amortised(f, wl64.n_recompute)
        v64 = aggregate_value(wl64.n_walkers * wl.n_el * len(ms64), sum(ms64) / 1000.0, ws)
        out["fp64"] = {"value": v64, "unit": UNIT, "ms_per_step": statistics.mean(ms64),
                       "update": "sm", "layout": "compact", "walkers": wl64.n_walkers,
                       "steps": len(ms64), "mode": "VMC sweeps (no fixed node, no branching)",
                       "compare_with": "dmc.sweep_only_value"}
        out["mixed_over_fp64"] = sweep_rate / v64
    if rank == 0 and not args.no_cpu:
        rate, cores, sample = cpu_oracle_rate(wl, target_s=10.0, max_gens=1,
                                              walkers=args.cpu_walkers)
        out["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                               "sample": sample + " (VMC sweep of the oracle)",
                               "cpu": cpu_model()}
    if rank == 0:
        print(json.dumps(out))


def eloc_error(wl, snaps):
    """The mixed path's E_L error where the sampling plays no part: at configurations of
    its own chain (one per energy block), E_L(mixed) - E_L(FP64 path: FP64 recompute of
    the same positions, then E_L)."""
    from paper_2209_14487_gb300 import qmcgb
    c = qmcgb.Crowd.from_workload(wl, precision="fp64")
    d = []
    for R, el in snaps:
        c.qmc_load_positions(np.ascontiguousarray(R))
        c.qmc_recompute()
        e64 = np.zeros(wl.n_walkers)
        c.qmc_local_energy_batch(e64)
        d.append(el - e64)
    c.close()
    d = np.concatenate(d)
    return {"samples": int(d.size), "mean": float(d.mean()),
            "sem": float(d.std(ddof=1) / math.sqrt(d.size)) if d.size > 1 else None,
            "rms": float(np.sqrt((d * d).mean())), "max_abs": float(np.abs(d).max()),
            "note": "E_L(mixed) - E_L(fp64) at the mixed chain's own configurations, one "
                    "per block: the mixed path's energy error without the sampling noise"}


def energy_stats(e: np.ndarray, block: int = 10):
    """Mean of E_L [generations][walkers] and its error from blocks of `block` generations
    (crowd averages per generation, then block means)."""
    g = e.mean(axis=1)
    nb = len(g) // block
    if nb < 2:
        return float(g.mean()), float("nan")
    b = g[: nb * block].reshape(nb, block).mean(axis=1)
    return float(b.mean()), float(b.std(ddof=1) / math.sqrt(nb))


def e2e_run(wl, precision, update, k, steps, crowd_id, nt=0):
    """Through the public API from pinned host buffers: create, load table, ions, Jastrow
    and positions, recompute, then `steps` sweeps each returning E_L to the host."""
    import torch

    from paper_2209_14487_gb300 import qmcgb
    table = torch.from_numpy(np.ascontiguousarray(wl.table())).pin_memory()
    R = torch.from_numpy(np.ascontiguousarray(wl.positions(crowd_id=crowd_id))).pin_memory()
    e_host = torch.zeros(wl.n_walkers, dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    c = qmcgb.Crowd(wl.n_up, wl.n_dn, wl.n_orb, wl.n_ions, wl.grid, wl.L, wl.n_walkers, wl.tau,
                    precision=precision, update=update, delay_rank=k,
                    n_recompute=wl.n_recompute, drift=wl.drift, potential=wl.potential,
                    seed=wl.seed, cta_threads=nt)
    if wl.n_ions:
        c.qmc_load_ions(wl.ions)
    if wl.j2_uu is not None:
        c.qmc_load_jastrow(qmcgb.QMC_J2_UU, wl.j2_uu.coefs, wl.j2_uu.rc)
        c.qmc_load_jastrow(qmcgb.QMC_J2_UD, wl.j2_ud.coefs, wl.j2_ud.rc)
    if wl.j1 is not None:
        c.qmc_load_jastrow(qmcgb.QMC_J1, wl.j1.coefs, wl.j1.rc)
    c.qmc_load_orbitals(table)
    c.qmc_load_positions(R)
    c.qmc_recompute()
    for _ in range(steps):
        c.qmc_sweep(1, e_host, stats=False)
    t1 = time.perf_counter()
    c.close()
    h2d = table.numel() * 8 + R.numel() * 8 + wl.ions.size * 8
    moves = wl.n_walkers * wl.n_el * steps
    return moves / (t1 - t0), h2d / steps, wl.n_walkers * 8


def cpu_oracle_rate(wl, target_s=12.0, max_gens=None, walkers=None, threads=None):
    """Moves/s of the CPU oracle (as it stands) on a bounded sample of the workload: all
    walkers, or the first `walkers` of them; all host threads, or `threads` of them."""
    import oracle
    oracle.build()
    all_threads = oracle.num_threads()
    if threads:
        oracle.set_num_threads(threads)
    try:
        return _cpu_oracle_rate(oracle, wl, target_s, max_gens, walkers)
    finally:
        oracle.set_num_threads(all_threads)


def _cpu_oracle_rate(oracle, wl, target_s, max_gens, walkers):
    osys = oracle.OracleSystem(wl)
    R = wl.positions()
    if walkers:
        R = np.ascontiguousarray(R[:walkers])
    W = R.shape[0]
    crowd = oracle.OracleCrowd(osys, R)
    t0 = time.perf_counter()
    crowd.sweep(1)
    t1 = time.perf_counter()
    per_gen = t1 - t0
    gens = max(1, int(target_s / max(per_gen, 1e-6)))
    if max_gens:
        gens = min(gens, max_gens)
    t0 = time.perf_counter()
    e, na = crowd.sweep(gens)
    t1 = time.perf_counter()
    rate = W * wl.n_el * gens / (t1 - t0)
    return rate, oracle.num_threads(), f"{gens} generation(s) x {W} walkers x {wl.n_el} electrons"


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return os.uname().machine


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="pw128")
    ap.add_argument("--walkers", type=int, default=None,
                    help="walkers per GPU (default: the workload's)")
    ap.add_argument("--delay-rank", type=int, default=None)
    ap.add_argument("--update", default="auto", choices=["auto", "sm", "delayed"])
    ap.add_argument("--cta-threads", type=int, default=0, choices=[0, 128, 160, 256],
                    help="threads per walker CTA (0: tuned with --update auto, else the "
                         "library's choice)")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--fp64-steps", type=int, default=2,
                    help="--dmc: timed generations of the FP64 arm")
    ap.add_argument("--staging", default="auto", choices=["auto", "ldg"],
                    help="stencil staging (auto: TMA where the library can; ldg: per-thread "
                         "loads)")
    ap.add_argument("--layout", default="auto", choices=["auto", "shared", "compact"],
                    help="the move kernel's shared-memory layout (auto: the library's pick)")
    ap.add_argument("--equilibrate", type=int, default=200,
                    help="untimed generations before the energy chain of each path")
    ap.add_argument("--energy-gens", type=int, default=800,
                    help="generations of the energy chain (0: no energy comparison)")
    ap.add_argument("--energy-block", type=int, default=40,
                    help="generations per block of the energy error (longer than the "
                         "chain's autocorrelation)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--dmc", action="store_true",
                    help="fixed-node DMC generations (sweep + branching) instead of VMC")
    ap.add_argument("--tau", type=float, default=None,
                    help="time step (default: the workload's; DMC wants about 0.01)")
    ap.add_argument("--cpu-walkers", type=int, default=None,
                    help="walkers of the CPU oracle sample (default: all)")
    ap.add_argument("--nlpp", action="store_true",
                    help="also time the mixed path with the synthetic nonlocal term in E_L")
    ap.add_argument("--coulomb", action="store_true",
                    help="also time the mixed path with the Ewald Coulomb energy in E_L")
    ap.add_argument("--batch", action="store_true",
                    help="the mixed-size batch (64/192/384 electrons) in one launch per generation")
    ap.add_argument("--walker-scan", default=None,
                    help="comma-separated walkers per GPU: throughput against crowd size")
    ap.add_argument("--crowds", default=None,
                    help="comma-separated crowd counts: the walkers split over crowds on "
                         "their own streams")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    global LAYOUT, STAGING
    LAYOUT = args.layout
    STAGING = args.staging

    from paper_2209_14487_gb300 import workloads
    wl = workloads.WORKLOADS[args.workload]()
    if args.walkers:
        wl.n_walkers = args.walkers
    if args.tau:
        wl.tau = args.tau
    ws, rank, local = dist_env()
    update = args.update
    k = args.delay_rank or (1 if update == "sm" else 8)
    cfg = {
        "workload": f"{wl.name}: {wl.n_el} electrons ({wl.n_up}/{wl.n_dn}), {wl.n_orb} orbitals "
                    f"on {wl.grid}^3, {wl.n_ions} ions, L={wl.L:g}, J1({wl.j1.K if wl.j1 else 0})"
                    f"+J2({wl.j2_uu.K if wl.j2_uu else 0}), {wl.n_walkers} walkers/GPU, "
                    f"tau={wl.tau}, FP64 recompute every {wl.n_recompute} generations",
        "walkers_per_gpu": wl.n_walkers, "electrons": wl.n_el,
        "step": "one generation (all electrons of all walkers proposed once + E_L)",
        "l2": "flushed between timed steps (256 MiB write outside the per-step events)",
    }

    if args.impl == "reference":
        if ws > 1 and rank != 0:
            return
        n_gen = args.steps + args.warmup
        import oracle
        oracle.build()
        osys = oracle.OracleSystem(wl)
        W = wl.n_walkers
        crowd = oracle.OracleCrowd(osys, wl.positions())
        t0 = time.perf_counter()
        crowd.sweep(1)
        per_gen = time.perf_counter() - t0
        # bounded sample: whole run within ~3 minutes; fewer walkers when one generation
        # of the full crowd is too slow
        budget = 150.0 / max(1, n_gen)
        Ws = W if per_gen <= budget else max(1, int(W * budget / per_gen))
        if Ws < W:
            crowd = oracle.OracleCrowd(osys, wl.positions()[:Ws])
        for _ in range(args.warmup):
            crowd.sweep(1)
        t0 = time.perf_counter()
        crowd.sweep(args.steps)
        dt = time.perf_counter() - t0
        rate = Ws * wl.n_el * args.steps / dt
        cores = oracle.num_threads()
        sample = f"{args.steps} generations x {Ws} of {W} walkers x {wl.n_el} electrons"
        print(json.dumps({
            "impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * dt / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": cfg,
            "cpu_baseline": {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample, "cpu": cpu_model()},
            "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
        }))
        return

    import torch
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    from paper_2209_14487_gb300 import qmcgb  # noqa: F401
    try:
        uuid = str(torch.cuda.get_device_properties(torch.cuda.current_device()).uuid)
    except Exception:
        uuid = None
    if args.batch:
        batch_main(args, ws, rank, cfg)
        if ws > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return
    if args.walker_scan or args.crowds:
        scan_main(args, wl, ws, rank, cfg)
        if ws > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return
    if args.dmc:
        dmc_main(args, wl, ws, rank, cfg)
        if ws > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return
    flush = torch.zeros(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MiB

    tune_table = None
    plan_table = None
    if update == "auto":
        from paper_2209_14487_gb300 import autotune
        update, k, tuned_nt, tune_table = autotune.tune(wl, "mixed")
        if not args.cta_threads:
            args.cta_threads = tuned_nt
        if args.staging == "auto" and args.layout == "auto":
            STAGING, LAYOUT, plan_table = autotune.tune_plan(wl, "mixed", update, k,
                                                             args.cta_threads)
    barrier(ws)
    torch.cuda.synchronize()
    energy = ((args.equilibrate, args.energy_gens, args.energy_block)
              if args.energy_gens > 0 else None)
    with ClockSampler(uuid) as clk:
        mixed = time_path(wl, "mixed", update, k, args.steps, args.warmup, rank, flush,
                          args.cta_threads, energy=energy)
        fp64 = None
        if not args.no_fp64:
            fp64 = time_path(wl, "fp64", "sm", 1, args.steps, args.warmup, rank, flush,
                             args.cta_threads,
                             energy=None if energy is None else energy[:2] + (0,))
    torch.cuda.synchronize()
    barrier(ws)

    moves_step = wl.n_walkers * wl.n_el
    ms_mixed, extra_mixed = amortised(mixed, wl.n_recompute)
    value = aggregate_value(moves_step * args.steps, sum(ms_mixed) / 1000.0, ws)
    t_mixed = ws * moves_step * args.steps / value
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1000.0 * t_mixed / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
           "data": "synthetic", "config": dict(cfg, precision="mixed: fp32 orbitals, Jastrow, "
                                               "ratios and inverse; fp64 recompute and energy",
                                               update=f"{update} k={k}",
                                               cta_threads=args.cta_threads or "library",
                                               parallelism=f"replicas x{ws}")}
    if tune_table is not None:
        out["autotune"] = {"ms_per_generation": tune_table,
                           "chosen": f"{update}:{k}:{args.cta_threads}"}
        if plan_table is not None:
            out["autotune"]["plan_ms_per_generation"] = plan_table
            out["autotune"]["plan"] = f"staging={STAGING} layout={LAYOUT}"
    out["recompute"] = {
        "every": wl.n_recompute,
        "recompute_ms": extra_mixed,
        "recompute_step_ms": statistics.mean(mixed["recompute_step_ms"])
        if mixed["recompute_step_ms"] else None,
        "plain_step_ms": statistics.mean(mixed["plain_ms"] or mixed["ms"]),
        "note": "recompute_ms = a generation carrying the FP64 recompute (sweep, LU of every "
                "walker, E_L) minus a plain generation, timed alone; ms_per_step and value "
                "include recompute_ms / every on each step that carried none"}
    out["guard"] = {"tol": qmcgb.GUARD_TOL_DEFAULT, "repairs_in_timed_steps": mixed["repairs"],
                    "walker_generations": wl.n_walkers * args.steps}
    if energy is not None:
        blk = args.energy_block
        e_m, s_m = energy_stats(mixed["chain"]["eloc"], block=blk)
        out["energy"] = {"equilibration_generations": args.equilibrate,
                         "generations": args.energy_gens, "block_generations": blk,
                         "mixed": {"mean": e_m, "sigma": s_m,
                                   "guard_repairs": mixed["chain"]["repairs"]}}
        if not args.no_fp64 and mixed["chain"]["snaps"]:
            out["energy"]["eloc_error_same_configs"] = eloc_error(wl, mixed["chain"]["snaps"])
    if fp64 is not None:
        ms64, _ = amortised(fp64, wl.n_recompute)
        v64 = aggregate_value(moves_step * args.steps, sum(ms64) / 1000.0, ws)
        t64 = ws * moves_step * args.steps / v64
        out["fp64"] = {"value": v64, "unit": UNIT,
                       "ms_per_step": 1000.0 * t64 / args.steps, "update": "sm"}
        if energy is not None:
            e_d, s_d = energy_stats(fp64["chain"]["eloc"], block=args.energy_block)
            out["energy"]["fp64"] = {"mean": e_d, "sigma": s_d}
            out["energy"]["diff_sigma"] = abs(e_m - e_d) / math.hypot(s_m, s_d)
        out["mixed_over_fp64"] = out["value"] / out["fp64"]["value"]
    # roofline of the dominant kernel (the fused move kernel, one launch per plain step)
    hbm, src = peaks()
    plain = mixed["plain_ms"] or mixed["ms"]
    t_launch = statistics.mean(plain) / 1000.0
    bpm = bytes_per_move(wl.n_orb, wl.n_el, 4, mixed["p_acc"], update, k)
    achieved = moves_step * bpm / t_launch / 1e9
    out["roofline"] = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                       "frac": achieved / hbm, "traffic": ncu_traffic("move_kernel<float>"),
                       "kernel": "move_kernel<float> (fused generation)",
                       "bytes_per_move": bpm, "acceptance": mixed["p_acc"],
                       "peak_source": src}
    # the table, rows and inverses of a 256-walker pw128 crowd stay in L2 during a
    # generation: the same algorithmic bytes against the measured L2 copy bandwidth
    l2 = l2_copy_peak()
    out["roofline_l2"] = {"bound": "l2", "achieved": achieved, "peak": l2, "unit": "GB/s",
                          "frac": achieved / l2,
                          "peak_source": "measured here: L2-resident elementwise copy "
                                         "(16-32 MiB buffers, 40 launches in a CUDA graph)"}
    out["gpu_launches"] = mixed["launches"]
    extras = []
    if args.nlpp:
        extras.append(("nlpp", dict(nlpp=NLPP),
                       {"amplitudes": NLPP[0], "widths": NLPP[1], "rc": NLPP[2]}))
    if args.coulomb:
        ca = coulomb_args(wl)
        extras.append(("coulomb", dict(coulomb=ca), {"Z": ca[0], "alpha": ca[1], "mmax": ca[2]}))
    for name, kw, desc in extras:
        with ClockSampler(uuid) as clk_x:
            xr = time_path(wl, "mixed", update, k, args.steps, args.warmup, rank, flush,
                           args.cta_threads, **kw)
        v_x = aggregate_value(moves_step * args.steps, sum(xr["ms"]) / 1000.0, ws)
        e_x, s_x = energy_stats(xr["eloc"])
        out[name] = {"value": v_x, "unit": UNIT, "ms_per_step": 1000.0 * ws * moves_step / v_x,
                     "parameters": desc, "energy": {"mean": e_x, "sigma": s_x},
                     "launches_per_step": xr["launches"] / args.steps,
                     "clocks": clk_x.summary()}
    out["clocks"] = clk.summary()
    if not args.no_e2e:
        rate, h2d, d2h = e2e_run(wl, "mixed", update, k, args.steps, rank, args.cta_threads)
        rate = aggregate_value(moves_step * args.steps, moves_step * args.steps / rate, ws)
        out["e2e"] = {"value": rate, "unit": UNIT, "h2d_bytes_per_step": h2d,
                      "d2h_bytes_per_step": d2h,
                      "note": "create + host loads (table, ions, Jastrow, positions) + recompute "
                              "+ K sweeps returning E_L to pinned host memory, wall clock"}
    if rank == 0 and not args.no_cpu:
        rate, cores, sample = cpu_oracle_rate(wl, walkers=args.cpu_walkers)
        r1, _, s1 = cpu_oracle_rate(wl, target_s=5.0, walkers=args.cpu_walkers, threads=1)
        out["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                               "sample": sample, "cpu": cpu_model(),
                               "one_core": {"value": r1, "sample": s1}}
    if rank == 0:
        print(json.dumps(out))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
