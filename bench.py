"""Benchmark: Static and Dynamic Frontier Leiden on the largest single-GPU
workload, a Chung-Lu web-graph stand-in with 2.0e9 CSR entries.

Workload (one GPU, default): Chung-Lu with degree exponent 2.1 (endpoint
probabilities proportional to (i + 10)^(-1/1.1), expected degrees capped at
sqrt(2m)), 5e7 vertices, 1.0e9 undirected edges (2.0e9 CSR entries, int64
offsets), integer weights uniform in 1..4, generated on the device; random
batches of 1e-7 .. 1e-1 |E| undirected updates (decades; 80% insertions
between uniform vertex pairs, 20% deletions of uniform existing edges, unit
weight), each applied to the base graph separately (Sec. 5.1.4).  The CSR
(16 GB) is far larger than the 129 MB L2, so no flush is needed between
steps.  ``--workload rmat`` runs the R-MAT scale-22 workload instead (4.19M
vertices, 1.3e8 entries, batches of 1e-5 .. 1e-3 |E|); its figures also
appear in the default line under "rmat_s22".

One step, all on the device: apply the step's batch to the base graph (a1),
DF update from the base graph's membership (a2..a10), then Static Leiden on
the same updated graph (a4..a10).  The headline value is Static Leiden's CSR
entries processed per second per pass, sum_p nnz(G'_p) / t_static; the DF
update time is reported beside it (p50 / p99 per batch size, and the speedup
over Static on the same G^t).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun each rank runs an independent replica (its own seed): the
method has no data-path exchange, so scaling is weak and there is no
collective beyond the timing barrier.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "edges/s per Leiden pass; DF batch update time & p50/p99 vs GPU Static, same GPU"
SCALE, EDGE_FACTOR = 22, 16
RMAT_FRACS = (1e-5, 1e-4, 1e-3)
RMAT_SEED = 0x1EDE0 + 1
CL_N, CL_M = 50_000_000, 1_000_000_000
CL_FRACS = (1e-7, 1e-6, 1e-5, 1e-4, 1e-3, 1e-2, 1e-1)
CL_SEED = 0x1EDE0 + 2
# the oracle's bounded sample of the Chung-Lu workload: the same recipe at
# 1/CL_SAMPLE_DIV of the vertices and edges
CL_SAMPLE_DIV = 32


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=14)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--scale", type=int, default=SCALE)
    ap.add_argument("--sched", default="det", choices=["det", "async"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--workload", default="cl",
                    choices=["cl", "rmat", "serving", "lowdeg", "temporal", "ablation", "smscale"])
    ap.add_argument("--no-serving-extra", action="store_true",
                    help="skip the compact serving figures of the default Chung-Lu line")
    ap.add_argument("--no-temporal-extra", action="store_true",
                    help="skip the temporal-stream figures of the default Chung-Lu line")
    ap.add_argument("--no-rmat-extra", action="store_true",
                    help="skip the compact R-MAT scale-22 figures of the default Chung-Lu line")
    ap.add_argument("--cl-div", type=int, default=1,
                    help="--profile-static on the Chung-Lu recipe at 1/k of its vertices and edges")
    ap.add_argument("--record-traffic", default=None,
                    help="ncu CSV of the first-pass decide kernels' DRAM bytes: write the traffic figure of the "
                         "workload to profiles/ (with --profile-json, the JSON line of the profiled run)")
    ap.add_argument("--profile-json", default=None)
    ap.add_argument("--profile-static", action="store_true",
                    help="run one Static Leiden on the workload graph and print its statistics (for profilers)")
    ap.add_argument("--lowdeg-samples", type=int, default=3, help="batches per size on the low-degree graphs")
    ap.add_argument("--serving-graphs", type=int, default=64)
    ap.add_argument("--serving-max-n", type=float, default=1e7)
    ap.add_argument("--serving-per-graph", type=int, default=10)
    ap.add_argument("--serving-load", type=float, default=0.7)
    ap.add_argument("--serving-slots", type=int, default=3)
    ap.add_argument("--serving-budget-gb", type=float, default=120.0)
    ap.add_argument("--serving-autotune", type=int, default=0)
    ap.add_argument("--serving-seed", type=int, default=5)
    ap.add_argument("--serving-small-n", type=int, default=1 << 16)
    ap.add_argument("--serving-small-nnz", type=int, default=1 << 18)
    ap.add_argument("--serving-small-workers", type=int, default=2)
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:  # noqa: BLE001 -- the file is written by the driver
        return 6800.0, "fallback"


# The decide kernels' sources: a DRAM-traffic figure measured by ncu (stored
# under profiles/) stays valid only while these files are unchanged.
DECIDE_SOURCES = ("paper_2405_11658_gb300/csrc/move.cu", "paper_2405_11658_gb300/csrc/hub.cu",
                  "paper_2405_11658_gb300/csrc/internal.h", "paper_2405_11658_gb300/csrc/common.cuh",
                  "paper_2405_11658_gb300/csrc/api.cu")
TRAFFIC_FILES = {"cl": os.path.join(ROOT, "profiles", "decide_traffic_cl.json"),
                 "rmat": os.path.join(ROOT, "profiles", "decide_traffic_rmat22.json")}


def decide_sources_sha():
    import hashlib
    h = hashlib.sha256()
    for f in DECIDE_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def measured_traffic(workload, entries_per_launch):
    """DRAM bytes per first-pass local-moving launch (one colour class) of the
    decide kernels, from the ncu capture recorded in profiles/, scaled to this
    run's entries per launch when the capture was taken on a smaller case --
    or None when there is none for this workload or the kernels changed since
    it was taken."""
    try:
        with open(TRAFFIC_FILES[workload]) as f:
            d = json.load(f)
    except (OSError, ValueError, KeyError):
        return None
    if d.get("source_sha256") != decide_sources_sha():
        return None
    per_entry = d.get("dram_bytes_per_scanned_entry")
    if per_entry is not None and entries_per_launch:
        return float(per_entry) * entries_per_launch
    return float(d["dram_bytes_per_launch"])


class Clocks:
    """Samples nvidia-smi SM clocks and throttle reasons during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:  # noqa: BLE001
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:  # noqa: BLE001
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx = max(mx, float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


def host_info():
    """The host's core count and CPU model (the oracle's baseline runs on it)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                model = ln.split(":", 1)[1].strip()
                break
    except Exception:  # noqa: BLE001
        pass
    return {"nproc": os.cpu_count(), "cpu_model": model}


# ---------------------------------------------------------------------------
# Workloads.  Each provides the device graph, one batch per step, the host
# copy for the end-to-end leg and the oracle's bounded sample.
# ---------------------------------------------------------------------------
class RmatWorkload:
    key = "rmat"

    def __init__(self, scale=SCALE):
        self.scale = scale
        self.fracs = RMAT_FRACS

    def config(self, n, nnz, sched, world):
        return {"workload": f"rmat-s{self.scale}-ef{EDGE_FACTOR}: batch apply + DF update + Static Leiden",
                "graph": f"R-MAT scale {self.scale}, edge factor {EDGE_FACTOR}, a/b/c/d=0.57/0.19/0.19/0.05",
                "vertices": n, "csr_entries": nnz, "batch_fracs": list(self.fracs),
                "schedule": sched, "l2": l2_note(8 * (n + 1) + 8 * nnz), "parallelism": f"replicas x{world}"}

    def host_graph(self, seed):
        from paper_2405_11658_gb300 import synth as S
        return S.rmat(self.scale, EDGE_FACTOR, 0.57, 0.19, 0.19, seed=seed)

    def build(self, L, dev, seed, nsteps):
        """(G0, host (off, idx, w), [(frac, dE, iE)] per step, max_nnz)."""
        from paper_2405_11658_gb300 import synth as S
        g = self.host_graph(seed)
        off, idx, w = g
        pairs = S.undirected_pairs(*g)
        nedges = len(pairs[0])
        batches = []
        for k in range(nsteps):
            frac = self.fracs[k % len(self.fracs)]
            d, i = S.random_batch(*g, max(2, int(round(frac * nedges))), seed=1000 + k, pairs=pairs)
            batches.append((frac, L.Edges.from_numpy(d, device=dev), L.Edges.from_numpy(i, device=dev)))
        max_nnz = len(idx) + 2 * max(b[2].count for b in batches) + 16
        return L.Graph.from_numpy(off, idx, w, device=dev), g, batches, max_nnz

    def cpu_sample(self):
        g = self.host_graph(RMAT_SEED)
        return g, (f"first pass of Static Leiden (DET) on the same R-MAT graph, {len(g[1])} CSR entries")


class ChungLuWorkload:
    key = "cl"

    def __init__(self, n=CL_N, m=CL_M):
        self.n, self.m = n, m
        self.fracs = CL_FRACS

    def config(self, n, nnz, sched, world):
        return {"workload": f"chung-lu-{self.n:.0e}v-{2 * self.m:.1e}e: batch apply + DF update + Static Leiden",
                "graph": "Chung-Lu, degree exponent 2.1, expected degrees capped at sqrt(2m), "
                         "integer weights uniform in 1..4, generated on the device",
                "vertices": n, "csr_entries": nnz, "batch_fracs": list(self.fracs),
                "schedule": sched, "l2": l2_note(8 * (n + 1) + 8 * nnz), "parallelism": f"replicas x{world}"}

    def build(self, L, dev, seed, nsteps):
        import torch
        from paper_2405_11658_gb300 import synth_device as D
        (off, idx, w), (keys, wk) = D.chung_lu(self.n, self.m, 2.1, 1, 4, seed=seed, device=dev)
        batches = []
        for k in range(nsteps):
            frac = self.fracs[k % len(self.fracs)]
            d, i = D.random_batch(self.n, keys, wk, max(2, int(round(frac * self.m))), seed=1000 + k)
            batches.append((frac, L.Edges(*d), L.Edges(*i)))
        del keys, wk
        torch.cuda.empty_cache()
        max_nnz = idx.numel() + 2 * max(b[2].count for b in batches) + 16
        return L.Graph(off, idx, w), None, batches, max_nnz

    def cpu_sample(self):
        from paper_2405_11658_gb300 import synth as S
        n, m = self.n // CL_SAMPLE_DIV, self.m // CL_SAMPLE_DIV
        g = S.chung_lu(n, m, 2.1, 1, 4, seed=CL_SEED)
        return g, (f"first pass of Static Leiden (DET) on a Chung-Lu graph of the same recipe at "
                   f"1/{CL_SAMPLE_DIV} of the vertices and edges ({n} vertices, {len(g[1])} CSR entries)")


WORKLOADS = {"cl": ChungLuWorkload, "rmat": RmatWorkload}


def cpu_baseline(g, sample, max_passes=1):
    """The oracle as it stands, single-threaded, on the first pass of Static
    Leiden over a bounded sample of the workload: CSR entries per second of
    that pass."""
    import oracle as O
    t0 = time.perf_counter()
    r = O.static(*g, O.LeidenOpts(max_passes=max_passes))
    wall = time.perf_counter() - t0
    st = r.stats
    edges = sum(st["nnz"][:st["passes"]])
    secs = sum(st["t_pass"][:st["passes"]])
    return {"value": edges / secs, "unit": "edges/s", "cores": 1, "kind": "oracle",
            "sample": f"{sample}; {wall:.1f} s of CPU work", "seconds": round(wall, 3), "host": host_info()}


def l2_note(csr_bytes):
    """How the timed steps stand with the 129 MB L2 (no flush between steps)."""
    if csr_bytes > 129e6:
        return f"inputs larger than L2 (CSR {csr_bytes / 1e9:.1f} GB), no flush"
    return f"inputs smaller than L2 (CSR {csr_bytes / 1e6:.0f} MB): L2-warm steps, no flush"


def workload_of(args):
    return RmatWorkload(args.scale) if args.workload == "rmat" else ChungLuWorkload()


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    wl = workload_of(args)
    g, sample = wl.cpu_sample()
    vals = []
    for _ in range(args.warmup):
        pass  # the oracle has no warm-up state
    t0 = time.perf_counter()
    for _ in range(args.steps):
        vals.append(cpu_baseline(g, sample))
    total = time.perf_counter() - t0
    v = statistics.mean(x["value"] for x in vals)
    n, nnz = (wl.n, 2 * wl.m) if wl.key == "cl" else (len(g[0]) - 1, len(g[1]))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "edges/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic",
            "config": wl.config(n, nnz, args.sched, world),
            "cpu_baseline": {"kind": "oracle", "cores": 1, "sample": vals[0]["sample"], "value": v,
                             "unit": "edges/s", "host": vals[0]["host"]},
            "e2e": {"value": v, "unit": "edges/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def combine_ranks(total_ms, static_ms, edges, launches, world, device):
    """Whole-job figures of independent replicas: the slowest rank's times
    (max over ranks) and the work of all ranks (sums).  One process per GPU;
    the reduction runs on the process group's backend (NCCL on the GPUs)."""
    if world <= 1:
        return total_ms, static_ms, edges, launches
    import torch
    import torch.distributed as dist
    t = torch.tensor([total_ms, static_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    e = torch.tensor([edges, launches], dtype=torch.float64, device=device)
    dist.all_reduce(e)
    return float(t[0]), float(t[1]), float(e[0]), int(e[1])


def run_graph(args, wl, L, dev, stream, rank, world, steps, warmup, e2e_steps, with_clocks=True):
    """The timed steps of one graph workload on this rank; returns the
    figures (device times are this rank's, not yet combined)."""
    import torch
    nsteps = warmup + steps
    seed = (CL_SEED if wl.key == "cl" else RMAT_SEED) + 7919 * rank
    G0, host, batches, max_nnz = wl.build(L, dev, seed, nsteps)
    n, nnz = G0.n, G0.nnz
    opts = L.Opts(sched=L.DET if args.sched == "det" else L.ASYNC)
    ctx = L.Context(max_n=n, max_nnz=max_nnz, stream=stream)
    Cs, _ = ctx.static(G0, opts, want_q=False)
    # base membership with consistent auxiliary information (K, Sigma): one
    # ND pass over the unchanged graph returns C0 together with K0 and S0
    C0, K0, S0, _ = ctx.update(G0, Cs, None, None, "ND", opts, want_q=False)
    del Cs
    rec = []

    def step(k, timed):
        frac, dE, iE = batches[k]
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ev[0].record(stream)
        Gt = ctx.apply_batch(G0, dE, iE, cap_nnz=max_nnz)
        ev[1].record(stream)
        ctx.update(Gt, C0, dE, iE, "DF", opts, prior_K=K0, prior_Sigma=S0, want_q=False)
        ev[2].record(stream)
        st_df = ctx.stats()
        if timed:
            ctx.set_timing(True)
        ctx.static(Gt, opts, want_q=False)
        ev[3].record(stream)
        if timed:
            ctx.set_timing(False)
        st = ctx.stats()
        torch.cuda.synchronize()
        t = [ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2]), ev[2].elapsed_time(ev[3])]
        rec.append({"frac": frac, "apply_ms": t[0], "df_ms": t[1], "static_ms": t[2],
                    "static_edges": sum(st["nnz"][:st["passes"]]), "stats": st,
                    "df_affected0": st_df["affected0"]})

    for k in range(warmup):
        step(k, False)
    rec.clear()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clk = Clocks(torch.cuda.current_device()) if with_clocks else None
    if clk:
        clk.__enter__()
    launches0 = L.kernel_launches()
    t0 = time.perf_counter()
    e_start = torch.cuda.Event(enable_timing=True)
    e_end = torch.cuda.Event(enable_timing=True)
    e_start.record(stream)
    for k in range(warmup, nsteps):
        step(k, True)
    e_end.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    launches = L.kernel_launches() - launches0
    if clk:
        clk.__exit__(None, None, None)
    out = {"n": n, "nnz": nnz, "rec": rec, "total_ms": e_start.elapsed_time(e_end), "wall": wall,
           "launches": launches, "clocks": clk.summary() if clk else None}

    # end to end through the public API from pinned host buffers: the graph
    # copied in, Static Leiden, the labels copied out, every step
    if e2e_steps > 0:
        if host is None:
            host = (G0.off.cpu().numpy(), G0.idx.cpu().numpy(), G0.w.cpu().numpy())
        off_h = torch.from_numpy(host[0]).pin_memory()
        idx_h = torch.from_numpy(host[1]).pin_memory()
        w_h = torch.from_numpy(host[2]).pin_memory()
        m_h = torch.empty(n, dtype=torch.int32).pin_memory()
        # pinned host copies of a few batches for the DF end-to-end leg
        host_batches = []
        for frac in sorted({b[0] for b in batches})[:2]:
            _, dE, iE = next(b for b in batches if b[0] == frac)
            host_batches.append((frac, tuple(x.cpu().pin_memory() for x in (dE.src, dE.dst, dE.w)),
                                 tuple(x.cpu().pin_memory() for x in (iE.src, iE.dst, iE.w))))
        del G0, batches
        torch.cuda.empty_cache()
        Gd = L.Graph(torch.empty_like(off_h, device=dev), torch.empty_like(idx_h, device=dev),
                     torch.empty_like(w_h, device=dev))
        mdev = torch.empty(n, dtype=torch.int32, device=dev)
        e_edges, e_ms = 0, 0.0
        for k in range(e2e_steps + 1):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record(stream)
            Gd.off.copy_(off_h, non_blocking=True)
            Gd.idx.copy_(idx_h, non_blocking=True)
            Gd.w.copy_(w_h, non_blocking=True)
            ctx.static(Gd, opts, out=mdev, want_q=False)
            m_h.copy_(mdev, non_blocking=True)
            b.record(stream)
            torch.cuda.synchronize()
            st = ctx.stats()
            if k > 0:  # the first round is a warm-up
                e_edges += sum(st["nnz"][:st["passes"]])
                e_ms += a.elapsed_time(b)
        out["e2e"] = {"value": e_edges / (e_ms / 1000.0), "unit": "edges/s",
                      "h2d_bytes_per_step": int(off_h.nbytes + idx_h.nbytes + w_h.nbytes),
                      "d2h_bytes_per_step": int(n * 4)}
        # DF end to end: the batch copied in from pinned host memory, G^t built,
        # the DF update from the base membership, the membership copied out
        Gd.off.copy_(off_h)
        Gd.idx.copy_(idx_h)
        Gd.w.copy_(w_h)
        torch.cuda.synchronize()
        df_e2e = {}
        for k in range(e2e_steps + 1):
            frac, dE, iE = host_batches[k % len(host_batches)]
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record(stream)
            dD = L.Edges(*(x.to(dev, non_blocking=True) for x in dE))
            iD = L.Edges(*(x.to(dev, non_blocking=True) for x in iE))
            Gt = ctx.apply_batch(Gd, dD, iD, cap_nnz=max_nnz)
            ctx.update(Gt, C0, dD, iD, "DF", opts, prior_K=K0, prior_Sigma=S0, out=mdev, want_q=False)
            m_h.copy_(mdev, non_blocking=True)
            b.record(stream)
            torch.cuda.synchronize()
            del Gt
            if k > 0:
                r = df_e2e.setdefault(f"{frac:g}", {"ms": [], "h2d": 0})
                r["ms"].append(a.elapsed_time(b))
                r["h2d"] = int(sum(x.nbytes for x in dE) + sum(x.nbytes for x in iE))
        out["e2e_df"] = {key: {"ms_p50": float(np.median(v["ms"])), "samples": len(v["ms"]),
                               "h2d_bytes_per_update": v["h2d"], "d2h_bytes_per_update": int(n * 4)}
                         for key, v in df_e2e.items()}
        del Gd, off_h, idx_h, w_h
    ctx.close()
    torch.cuda.empty_cache()
    return out


def summarise(wl, out, static_ms, static_edges):
    """Per-batch-size DF / Static figures and the first-pass decide roofline."""
    rec = out["rec"]
    df = {}
    for frac in wl.fracs:
        rs = [r for r in rec if r["frac"] == frac]
        if not rs:
            continue
        d = sorted(r["df_ms"] for r in rs)
        s = sorted(r["static_ms"] for r in rs)
        df[f"{frac:g}"] = {"df_ms_p50": float(np.percentile(d, 50)), "df_ms_p99": float(np.percentile(d, 99)),
                           "static_ms_p50": float(np.percentile(s, 50)),
                           "speedup_vs_static": float(np.median(s) / np.median(d)),
                           "apply_ms_p50": float(np.median([r["apply_ms"] for r in rs])),
                           "df_affected0_p50": int(np.median([r["df_affected0"] for r in rs])),
                           "samples": len(rs)}
    # roofline of the dominant kernel family: the local-moving decide kernels
    # of the first pass (every vertex of the input graph, the same work in
    # every step), one launch = the decide kernels of one colour class
    mv_bytes = sum(r["stats"]["move0_bytes"] for r in rec)
    mv_ms = sum(r["stats"]["move0_kernel_ms"] for r in rec)
    mv_launches = sum(r["stats"]["move0_kernel_launches"] for r in rec)
    mv_entries = sum(r["stats"]["move0_scanned_entries"] for r in rec)
    all_bytes = sum(r["stats"]["move_bytes"] for r in rec)
    all_ms = sum(r["stats"]["move_kernel_ms"] for r in rec)
    peak, peak_kind = peaks()
    achieved = (mv_bytes / mv_launches) / ((mv_ms / mv_launches) / 1000.0) / 1e9 if mv_ms > 0 else None
    last = rec[-1]["stats"] if rec else {}
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": (achieved / peak) if achieved else None,
            "traffic": measured_traffic(wl.key, mv_entries / max(1, mv_launches)),
            "kernel": "first-pass local-move decide kernels (all degree tiers), per colour class",
            "peak_kind": peak_kind,
            "bytes_per_launch": mv_bytes / max(1, mv_launches),
            "ms_per_launch": mv_ms / max(1, mv_launches), "launches": mv_launches,
            "entries_per_launch": mv_entries / max(1, mv_launches),
            "all_passes_achieved": (all_bytes / (all_ms / 1000.0) / 1e9) if all_ms else None}
    return {"static_ms_mean": static_ms / max(1, len(rec)), "static_edges_per_s": static_edges / (static_ms / 1000.0),
            "static_passes": last.get("passes"), "static_iters": last.get("iters"),
            "static_nnz_per_pass": last.get("nnz"), "df": df, "roofline": roof}


def run_ours(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    import paper_2405_11658_gb300 as L
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    wl = workload_of(args)
    out = run_graph(args, wl, L, dev, stream, rank, world, args.steps, args.warmup, args.e2e_steps)
    rec = out["rec"]
    static_ms = sum(r["static_ms"] for r in rec)
    static_edges = sum(r["static_edges"] for r in rec)
    # max over ranks of the device time
    total_ms, static_ms_all, static_edges_all, launches = combine_ranks(out["total_ms"], static_ms, static_edges,
                                                                         out["launches"], world, dev)
    value = static_edges_all / (static_ms_all / 1000.0)
    summ = summarise(wl, out, static_ms, static_edges)

    # the R-MAT scale-22 figures beside the Chung-Lu line (not timed into it)
    rmat = None
    if wl.key == "cl" and not args.no_rmat_extra:
        rw = RmatWorkload(SCALE)
        ro = run_graph(args, rw, L, dev, stream, rank, world, 6, 3, 0, with_clocks=False)
        r_ms = sum(r["static_ms"] for r in ro["rec"])
        r_edges = sum(r["static_edges"] for r in ro["rec"])
        rs = summarise(rw, ro, r_ms, r_edges)
        rmat = {"config": rw.config(ro["n"], ro["nnz"], args.sched, world), "value": r_edges / (r_ms / 1000.0),
                "unit": "edges/s", **{k: rs[k] for k in ("static_ms_mean", "static_passes", "df")},
                "roofline_frac": rs["roofline"]["frac"], "roofline_achieved": rs["roofline"]["achieved"]}

    temporal = None
    if wl.key == "cl" and not args.no_temporal_extra:
        temporal = run_temporal_graph(args, L, dev, stream)
    serving = None
    if wl.key == "cl" and not args.no_serving_extra:
        serving = run_serving_compact(L)

    base = None
    if rank == 0 and not args.no_cpu_baseline:
        g, sample = wl.cpu_sample()
        base = cpu_baseline(g, sample)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "edges/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / max(1, args.steps), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": wl.config(out["n"], out["nnz"], args.sched, world),
            **{k: summ[k] for k in ("static_ms_mean", "static_passes", "static_iters", "static_nnz_per_pass", "df")},
            "roofline": summ["roofline"],
            "cpu_baseline": base,
            "e2e": out.get("e2e"),
            "e2e_df": out.get("e2e_df"),
            "gpu_launches": launches,
            "clocks": out["clocks"],
            "wall_s": out["wall"],
        }
        if rmat is not None:
            line["rmat_s22"] = rmat
        if temporal is not None:
            line["temporal"] = temporal
        if serving is not None:
            line["serving"] = serving
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


TEMPORAL_N, TEMPORAL_EVENTS = 1_140_000, 7_830_000
TEMPORAL_FRACS = (1e-5, 1e-4, 1e-3)
TEMPORAL_SEED = 0x1EDE0 + 5


def run_temporal_graph(args, L, dev, stream, batches_per_size=100, every=10):
    """The temporal workload (Sec. 5.3) on a synthetic interaction stream the
    size of wiki-talk-temporal (1.14M vertices, 7.83M events): 90% preloaded,
    then, for each batch size of 1e-5, 1e-4 and 1e-3 |E_T| events, 100
    consecutive insertion batches applied in turn, each followed by a DF
    update from the previous update's membership, K and Sigma.  Every
    ``every``-th batch also times Static, ND and DS on the same G^t.  Returns
    the per-size figures."""
    import torch
    from paper_2405_11658_gb300 import synth as S
    src, dst = S.temporal_stream(TEMPORAL_N, TEMPORAL_EVENTS, seed=TEMPORAL_SEED)
    g0, rest = S.temporal_split(TEMPORAL_N, src, dst, 0.9)
    opts = L.Opts(sched=L.DET if args.sched == "det" else L.ASYNC)

    def timed(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        r = fn()
        b.record(stream)
        b.synchronize()
        return r, a.elapsed_time(b)

    out = {}
    cap_all = len(g0[1]) + 2 * int(round(max(TEMPORAL_FRACS) * TEMPORAL_EVENTS)) * batches_per_size + 16
    with L.Context(max_n=TEMPORAL_N, max_nnz=cap_all, stream=stream) as ctx:
        G0 = L.Graph.from_numpy(*g0, device=dev)
        Cs, _ = ctx.static(G0, opts, want_q=False)
        C0, K0, S0, _ = ctx.update(G0, Cs, None, None, "ND", opts, want_q=False)
        for frac in TEMPORAL_FRACS:
            size = max(1, int(round(frac * TEMPORAL_EVENTS)))
            batches = S.temporal_batches(rest, size, batches_per_size)
            G, C, K, Sg = G0, C0, K0, S0
            rec = {"df": [], "static": [], "nd": [], "ds": [], "apply": [], "affected": []}
            for k, ins in enumerate(batches):
                iE = L.Edges.from_numpy(ins, device=dev)
                G, t_apply = timed(lambda: ctx.apply_batch(G, None, iE, cap_nnz=cap_all))
                (C, K, Sg, _), t_df = timed(lambda: ctx.update(G, C, None, iE, "DF", opts, prior_K=K,
                                                               prior_Sigma=Sg, want_q=False))
                rec["apply"].append(t_apply)
                rec["df"].append(t_df)
                rec["affected"].append(ctx.stats()["affected0"])
                if k % every == every - 1:
                    _, t = timed(lambda: ctx.static(G, opts, want_q=False))
                    rec["static"].append(t)
                    for mode in ("ND", "DS"):
                        _, t = timed(lambda: ctx.update(G, C, None, iE, mode, opts, prior_K=K, prior_Sigma=Sg,
                                                        want_q=False))
                        rec[mode.lower()].append(t)
            q_df = ctx.modularity(G, C)
            _, q_static = ctx.static(G, opts)
            s50 = float(np.median(rec["static"]))
            out[f"{frac:g}"] = {
                "batch_events": size, "batches": len(batches),
                "df_ms_p50": float(np.percentile(rec["df"], 50)), "df_ms_p99": float(np.percentile(rec["df"], 99)),
                "static_ms_p50": s50, "nd_ms_p50": float(np.median(rec["nd"])),
                "ds_ms_p50": float(np.median(rec["ds"])), "apply_ms_p50": float(np.median(rec["apply"])),
                "df_speedup_vs_static": s50 / float(np.median(rec["df"])),
                "nd_speedup_vs_static": s50 / float(np.median(rec["nd"])),
                "ds_speedup_vs_static": s50 / float(np.median(rec["ds"])),
                "df_affected0_p50": int(np.median(rec["affected"])),
                "q_df_after_chain": q_df, "q_static_same_graph": q_static}
    return {"graph": f"synthetic interaction stream, {TEMPORAL_N} vertices, {TEMPORAL_EVENTS} events "
                     f"({len(g0[1]) // 2} static edges preloaded from the first 90%)",
            "by_batch": out}


def _compact_serving_graph(k):
    """Graph k of the compact serving mix: 16 small planted-partition graphs
    (1e4..3e4 vertices, mean degree ~8: inside the persistent path's limits)
    and 8 larger R-MAT graphs (scale 16..20, edge factor 8..16), each with a
    stream of 12 update batches of 1e-6..1e-3 |E| (80/20, valid in any order)."""
    from paper_2405_11658_gb300 import synth as S
    rng = np.random.default_rng(0x5E7 + k)
    if k < 16:
        n = int(10 ** rng.uniform(4.0, np.log10(3e4)))
        comms = max(4, n // 400)
        g = S.planted_partition(n, comms, 7.0 / (n / comms), 1.0 / n, 0x5E70 + k)
        kind = "pp"
    else:
        scale = 16 + (k - 16) % 5
        g = S.rmat(scale, 8 if k % 2 else 16, 0.57, 0.19, 0.19, seed=0x5E70 + k)
        kind = f"rmat{scale}"
    off, idx, w = g
    n = len(off) - 1
    eu, ev, ew = S.undirected_pairs(off, idx, w)
    keys = np.sort(eu * n + ev)
    perm = rng.permutation(len(eu))
    used, stream = 0, []
    for _ in range(12):
        size = max(2, int(round(10 ** rng.uniform(-6, -3) * len(eu))))
        nd = size // 5
        pick = perm[used:used + nd]
        used += nd
        dels = (eu[pick].astype(np.int32), ev[pick].astype(np.int32), ew[pick].astype(np.int32))
        a = rng.integers(0, n, size=2 * size + 16)
        b = rng.integers(0, n, size=2 * size + 16)
        lo, hi = np.minimum(a, b), np.maximum(a, b)
        cand = lo * n + hi
        pos = np.minimum(np.searchsorted(keys, cand), len(keys) - 1)
        cand = np.unique(cand[(lo != hi) & (keys[pos] != cand)])[:size - nd]
        ins = ((cand // n).astype(np.int32), (cand % n).astype(np.int32), np.ones(len(cand), np.int32))
        stream.append((dels, ins))
    return kind, g, stream


def run_serving_compact(L):
    """A compact serving run for the default line: 24 resident graphs; update
    batches arrive in bursts (exponential gaps) that each bring one batch for
    every small graph and one for two of the large ones, so requests arrive
    while others run, small graphs are batched into persistent launches and
    large ones overlap on the large-graph workers.  Returns updates/s, p50/p99
    latency overall and per path, and graphs per persistent launch."""
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(min(8, os.cpu_count() or 1)) as pool:
        work = pool.map(_compact_serving_graph, range(24), chunksize=1)
    rng = np.random.default_rng(11)
    cfg = dict(hbm_budget=40 << 30, large_slots=2, small_max_graphs=32,
               large_max_n=max(len(g[0]) for _, g, _ in work),
               large_max_nnz=int(max(len(g[1]) for _, g, _ in work) * 1.2) + 4096,
               small_max_n=1 << 16, small_max_nnz=1 << 18, small_batch_n=1 << 21, small_batch_nnz=1 << 24,
               growth=0.05, small_workers=1, min_persistent=4)
    with L.Server(**cfg) as srv:
        ids = []
        for _, g, _ in work:
            gid, rid = srv.admit(*g)
            srv.wait(rid)
            ids.append(gid)
        small = [k for k, (kind, _, _) in enumerate(work) if kind == "pp"]
        large = [k for k in range(len(work)) if k not in small]
        nxt = [0] * len(work)
        submitted = []
        t0 = time.perf_counter()
        for burst in range(12):
            time.sleep(rng.exponential(0.05))
            for k in small + list(rng.choice(large, size=2, replace=False)):
                if nxt[k] < len(work[k][2]):
                    dels, ins = work[k][2][nxt[k]]
                    nxt[k] += 1
                    submitted.append(srv.submit(ids[k], dels, ins))
        infos = [srv.wait(r) for r in submitted]
        t1 = time.perf_counter()
        st = srv.stats()
    ok = [x for x in infos if x["status"] == 0]
    lat = np.array([x["latency_ms"] for x in ok])
    per_path = {}
    for path, name in ((0, "persistent"), (1, "large"), (2, "small_alone")):
        v = np.array([x["latency_ms"] for x in ok if x["path"] == path])
        if len(v):
            per_path[name] = {"requests": int(len(v)), "p50_ms": float(np.percentile(v, 50)),
                              "p99_ms": float(np.percentile(v, 99))}
    sizes = [x["launch_graphs"] for x in ok if x["path"] == 0]
    return {"workload": "24 resident graphs (16 planted partitions of 1e4..3e4 vertices, 8 R-MAT of "
                        "scale 16..20), 12 bursts of DF update batches of 1e-6..1e-3 |E|",
            "updates_per_s": len(ok) / (t1 - t0), "requests": len(infos), "failed": len(infos) - len(ok),
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "paths": per_path, "mean_graphs_per_persistent_launch": float(np.mean(sizes)) if sizes else None,
            "persistent_launches": st.get("small_launches")}


SERVING_METRIC = "serving: DF updates/s with p50/p99 per-batch latency, many resident graphs"


def _serving_graph(job):
    """Graph k of the serving workload and its update stream: log-spaced sizes
    from 1e4 to max_n vertices (most of them small), planted-partition and
    R-MAT alternating below 2e5 vertices and R-MAT above, edge factors 8 to
    32 (8 above 1e6 vertices).  The stream holds batches of 1e-6..1e-3 |E|
    (log-uniform): 80% insertions of pairs that are not edges of the graph,
    20% deletions of distinct edges of the graph, so every batch stays valid
    whatever ran before it."""
    k, count, max_n, seed, per_graph = job
    from paper_2405_11658_gb300 import synth as S
    x = k / max(1, count - 1)
    n = int(round(10 ** (4 + (np.log10(max_n) - 4) * x * x)))
    ef = (8, 16, 32)[k % 3] if n <= 1_000_000 else 8
    if n <= 200_000 and k % 2 == 0:
        comms = max(4, n // 500)
        g = S.planted_partition(n, comms, min(0.5, 2.0 * ef / (n / comms)), 0.1 * ef / n, seed + k)
        kind = "pp"
    else:
        scale = max(10, int(round(np.log2(n))))
        g = S.rmat(scale, ef, 0.57, 0.19, 0.19, seed=seed + k)
        kind = f"rmat{scale}"
    off, idx, w = g
    n = len(off) - 1
    eu, ev, ew = S.undirected_pairs(off, idx, w)
    keys = np.sort(eu * n + ev)
    rng = np.random.default_rng(seed * 1000 + k)
    perm = rng.permutation(len(eu))
    used = 0
    stream = []
    for _ in range(per_graph):
        frac = 10 ** rng.uniform(-6, -3)
        size = max(1, int(round(frac * len(eu))))
        nd = size // 5
        ni = size - nd
        pick = perm[used:used + nd]
        used += nd
        dels = (eu[pick].astype(np.int32), ev[pick].astype(np.int32), ew[pick].astype(np.int32))
        a = rng.integers(0, n, size=2 * ni + 16)
        b = rng.integers(0, n, size=2 * ni + 16)
        lo, hi = np.minimum(a, b), np.maximum(a, b)
        cand = lo * n + hi
        pos = np.minimum(np.searchsorted(keys, cand), len(keys) - 1)
        ok = (lo != hi) & (keys[pos] != cand)
        cand = np.unique(cand[ok])[:ni]
        ins = ((cand // n).astype(np.int32), (cand % n).astype(np.int32), np.ones(len(cand), np.int32))
        stream.append((frac, dels, ins))
    return kind, g, stream


def serving_workload(count, max_n, seed, per_graph, procs):
    """The graphs and streams, built by a pool of `procs` processes (spawned:
    the caller has not touched the GPU yet)."""
    import multiprocessing as mp
    jobs = [(k, count, max_n, seed, per_graph) for k in range(count)]
    if procs <= 1:
        return [_serving_graph(j) for j in jobs]
    with mp.get_context("spawn").Pool(procs) as pool:
        return pool.map(_serving_graph, sorted(jobs, key=lambda j: -j[0]), chunksize=1)[::-1]


def run_serving(args):
    """Poisson arrivals of update batches over many resident graphs; prints
    one JSON line (updates/s, p50 / p99 latency per path)."""
    t0 = time.perf_counter()
    work = serving_workload(args.serving_graphs, args.serving_max_n, 0x1EDE0 + 4, args.serving_per_graph + 1,
                            min(16, os.cpu_count() or 1))
    graphs = [(kind, g) for kind, g, _ in work]
    streams = [st for _, _, st in work]
    del work
    gen_s = time.perf_counter() - t0
    import torch
    torch.cuda.set_device(0)
    import paper_2405_11658_gb300 as L
    rng = np.random.default_rng(args.serving_seed)
    cfg = dict(hbm_budget=int(args.serving_budget_gb * (1 << 30)), large_slots=args.serving_slots,
               small_max_graphs=64, large_max_n=max(len(g[0]) for _, g in graphs),
               large_max_nnz=int(max(len(g[1]) for _, g in graphs) * 1.3) + 4096,
               small_max_n=args.serving_small_n, small_max_nnz=args.serving_small_nnz,
               small_batch_n=1 << 22, small_batch_nnz=1 << 25, growth=0.05,
               autotune_trials=args.serving_autotune, small_workers=args.serving_small_workers)
    with L.Server(**cfg) as srv:
        ids, admit_rids = [], []
        t_adm = time.perf_counter()
        for _, g in graphs:
            gid, rid = srv.admit(*g)
            ids.append(gid)
            admit_rids.append(rid)
        for r in admit_rids:
            info = srv.wait(r)
            assert info["status"] == 0, info
        admit_s = time.perf_counter() - t_adm
        # calibration: one batch per graph, all at once
        t_cal = time.perf_counter()
        rids = [srv.submit(ids[k], *streams[k][0][1:]) for k in range(len(graphs))]
        for r in rids:
            srv.wait(r)
        cal_s = time.perf_counter() - t_cal
        mu = len(graphs) / cal_s
        lam = args.serving_load * mu
        # timed: Poisson arrivals at rate lam over a random graph order
        order = [(k, j) for k in range(len(graphs)) for j in range(1, args.serving_per_graph + 1)]
        rng.shuffle(order)
        nxt = [1] * len(graphs)
        submitted = []
        launches0 = L.kernel_launches()
        with Clocks(0) as clk:
            t_start = time.perf_counter()
            t_next = t_start
            for k, _ in order:
                t_next += rng.exponential(1.0 / lam)
                delay = t_next - time.perf_counter()
                if delay > 0:
                    time.sleep(delay)
                frac, dels, ins = streams[k][nxt[k]]
                nxt[k] += 1
                submitted.append((k, frac, srv.submit(ids[k], dels, ins)))
            infos = [(k, frac, srv.wait(r)) for k, frac, r in submitted]
            t_end = time.perf_counter()
        launches = L.kernel_launches() - launches0
        st = srv.stats()
    ok = [x for x in infos if x[2]["status"] == 0]
    lat = np.array([x[2]["latency_ms"] for x in ok])
    per_path = {}
    for path, name in ((0, "persistent"), (1, "large"), (2, "small_alone")):
        v = np.array([x[2]["latency_ms"] for x in ok if x[2]["path"] == path])
        if len(v):
            per_path[name] = {"requests": int(len(v)), "p50_ms": float(np.percentile(v, 50)),
                              "p99_ms": float(np.percentile(v, 99))}
    launch_sizes = [x[2]["launch_graphs"] for x in ok if x[2]["path"] == 0]
    line = {
        "metric": SERVING_METRIC, "value": len(ok) / (t_end - t_start), "unit": "updates/s", "n_gpus": 1,
        "steps": len(order), "warmup": len(graphs), "ms_per_step": 1000 * (t_end - t_start) / max(1, len(order)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": f"serving: {len(graphs)} resident graphs, 1e4..{args.serving_max_n:.0e} vertices, "
                               f"Poisson DF update batches of 1e-6..1e-3 |E|",
                   "graphs": [f"{kind}:{len(g[0]) - 1}:{len(g[1])}" for kind, g in graphs],
                   "arrival_rate_per_s": lam, "load": args.serving_load, "large_slots": args.serving_slots,
                   "budget_gb": args.serving_budget_gb, "autotune_trials": args.serving_autotune,
                   "small_limits": [args.serving_small_n, args.serving_small_nnz],
                   "small_workers": args.serving_small_workers},
        "p50_ms": float(np.percentile(lat, 50)) if len(lat) else None,
        "p99_ms": float(np.percentile(lat, 99)) if len(lat) else None,
        "paths": per_path, "failed": len(infos) - len(ok),
        "mean_graphs_per_persistent_launch": float(np.mean(launch_sizes)) if launch_sizes else None,
        "server": st, "gpu_launches": launches, "clocks": clk.summary(),
        "gen_s": gen_s, "admit_s": admit_s, "calibration_s": cal_s,
    }
    print(json.dumps(line))
    return 0

LOWDEG_FRACS = (1e-6, 1e-5, 1e-4, 1e-3)


def _lowdeg_graph(job):
    """One low-degree graph at full size and its batches: (name, graph,
    [(frac, dels, ins), ...]), samples batches per size."""
    name, samples = job
    from paper_2405_11658_gb300 import synth as S
    if name == "grid":
        g = S.grid(5000, 0.05, 0.001, seed=0x1EDE0 + 3)
    else:
        g = S.kmer(100_000_000, 64.0, 2.1, seed=0x1EDE0 + 4)
    pairs = S.undirected_pairs(*g)
    nedges = len(pairs[0])
    batches = []
    for i, frac in enumerate(LOWDEG_FRACS):
        for k in range(samples):
            size = max(2, int(round(frac * nedges)))
            batches.append((frac, *S.random_batch(*g, size, seed=2000 + 10 * i + k, pairs=pairs)))
    return name, g, batches


def run_lowdeg(args):
    """Static, DS and DF Leiden on the two low-degree graphs at full size
    (5000 x 5000 grid with 5% of edges removed and 0.1% |V| shortcuts;
    1e8-vertex k-mer-like paths with mean degree 2.1), batches of 1e-6 ..
    1e-3 |E|; prints one JSON line."""
    import multiprocessing as mp
    jobs = [("kmer", args.lowdeg_samples), ("grid", args.lowdeg_samples)]
    with mp.get_context("spawn").Pool(2) as pool:
        work = pool.map(_lowdeg_graph, jobs, chunksize=1)
    import torch
    import paper_2405_11658_gb300 as L
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    opts = L.Opts(sched=L.DET if args.sched == "det" else L.ASYNC)
    out, tot_edges, tot_ms = {}, 0, 0.0
    peak, peak_kind = peaks()

    def timed(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        r = fn()
        b.record(stream)
        b.synchronize()
        return r, a.elapsed_time(b)

    launches0 = L.kernel_launches()
    with Clocks(0) as clk:
        for name, g, batches in sorted(work):
            off, idx, w = g
            n, nnz = len(off) - 1, len(idx)
            max_nnz = nnz + 2 * max(len(b[2][0]) for b in batches) + 16
            G0 = L.Graph.from_numpy(off, idx, w, device=dev)
            with L.Context(max_n=n, max_nnz=max_nnz, stream=stream) as ctx:
                for _ in range(args.warmup):
                    Cs, _ = ctx.static(G0, opts, want_q=False)
                st_ms, st_edges, mv = [], [], []
                for _ in range(args.steps):
                    ctx.set_timing(True)
                    (Cs, _), ms = timed(lambda: ctx.static(G0, opts, want_q=False))
                    ctx.set_timing(False)
                    st = ctx.stats()
                    st_ms.append(ms)
                    st_edges.append(sum(st["nnz"][:st["passes"]]))
                    mv.append((st["move0_bytes"], st["move0_kernel_ms"], st["move0_kernel_launches"]))
                C0, K0, S0, _ = ctx.update(G0, Cs, None, None, "ND", opts, want_q=False)
                per = {}
                for frac, dels, ins in batches:
                    dE, iE = L.Edges.from_numpy(dels, device=dev), L.Edges.from_numpy(ins, device=dev)
                    Gt, t_apply = timed(lambda: ctx.apply_batch(G0, dE, iE, cap_nnz=max_nnz))
                    rec = per.setdefault(f"{frac:g}", {"apply": [], "DS": [], "DF": [], "static": [], "affected": []})
                    rec["apply"].append(t_apply)
                    for mode in ("DS", "DF"):
                        _, t = timed(lambda: ctx.update(Gt, C0, dE, iE, mode, opts, prior_K=K0, prior_Sigma=S0,
                                                        want_q=False))
                        rec[mode].append(t)
                        if mode == "DF":
                            rec["affected"].append(ctx.stats()["affected0"])
                    _, t = timed(lambda: ctx.static(Gt, opts, want_q=False))
                    rec["static"].append(t)
                    del Gt
                res = {}
                for key, rec in per.items():
                    s50 = float(np.median(rec["static"]))
                    res[key] = {"apply_ms_p50": float(np.median(rec["apply"])), "static_ms_p50": s50,
                                "df_affected0_p50": int(np.median(rec["affected"])), "samples": len(rec["DF"])}
                    for mode in ("DS", "DF"):
                        res[key][f"{mode.lower()}_ms_p50"] = float(np.percentile(rec[mode], 50))
                        res[key][f"{mode.lower()}_ms_p99"] = float(np.percentile(rec[mode], 99))
                        res[key][f"{mode.lower()}_speedup_vs_static"] = s50 / float(np.median(rec[mode]))
                b, ms, nl = (sum(x[i] for x in mv) for i in range(3))
                ach = (b / nl) / ((ms / nl) / 1000.0) / 1e9 if ms > 0 else None
                out[name] = {"vertices": n, "csr_entries": nnz, "static_ms_mean": float(np.mean(st_ms)),
                             "static_edges_per_s": sum(st_edges) / (sum(st_ms) / 1000.0),
                             "static_passes": st["passes"], "static_iters": st["iters"],
                             "first_pass_decide": {"achieved_gbs": ach, "frac": (ach / peak) if ach else None,
                                                   "ms_per_launch": ms / max(1, nl), "launches": nl},
                             "batches": res}
                tot_edges += sum(st_edges)
                tot_ms += sum(st_ms)
    launches = L.kernel_launches() - launches0
    line = {"metric": METRIC, "value": tot_edges / (tot_ms / 1000.0), "unit": "edges/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_ms / max(1, 2 * args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic",
            "config": {"workload": "low-degree: 5000x5000 grid (5% edges removed, 0.1%|V| shortcuts) and "
                                   "1e8-vertex k-mer-like paths (mean 64, degree 2.1); Static, DS, DF",
                       "batch_fracs": list(LOWDEG_FRACS), "samples_per_size": args.lowdeg_samples,
                       "schedule": args.sched, "l2": "inputs larger than L2 (CSR 0.8 and 1.7 GB), no flush",
                       "peak_gbs": peak, "peak_kind": peak_kind},
            "graphs": out, "gpu_launches": launches, "clocks": clk.summary()}
    print(json.dumps(line))
    return 0


def run_temporal(args):
    """``--workload temporal``: the temporal figures as their own JSON line."""
    import torch
    torch.cuda.set_device(0)
    import paper_2405_11658_gb300 as L
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    launches0 = L.kernel_launches()
    with Clocks(0) as clk:
        t0 = time.perf_counter()
        res = run_temporal_graph(args, L, dev, stream)
        wall = time.perf_counter() - t0
    by = res["by_batch"]
    tot_ms = sum(v["df_ms_p50"] * v["batches"] for v in by.values())
    tot_b = sum(v["batches"] for v in by.values())
    line = {"metric": "DF update time per temporal batch (p50/p99) vs GPU Static, same GPU",
            "value": tot_ms / max(1, tot_b), "unit": "ms/batch (DF, p50 over sizes)", "n_gpus": 1,
            "steps": tot_b, "warmup": 0, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "int64", "data": "synthetic",
            "config": {"workload": "temporal: 90% preload, 100 consecutive insertion batches per size, "
                                   "DF chained on the returned membership, K and Sigma",
                       "graph": res["graph"], "batch_fracs_of_events": list(TEMPORAL_FRACS),
                       "schedule": args.sched},
            "by_batch": by, "gpu_launches": L.kernel_launches() - launches0, "clocks": clk.summary(),
            "wall_s": wall}
    print(json.dumps(line))
    return 0


ABLATION_FRACS = (1e-7, 1e-6, 1e-5, 1e-4, 1e-3, 1e-2, 1e-1)
ABLATION_VARIANTS = (("full_refine", 1, True), ("subset_refine", 0, True), ("optimized_aggregation", 0, False))


def _ablation_graphs():
    from paper_2405_11658_gb300 import synth as S
    yield "rmat-s22", S.rmat(SCALE, EDGE_FACTOR, 0.57, 0.19, 0.19, seed=RMAT_SEED)
    yield "grid-5000", S.grid(5000, 0.05, 0.001, seed=0x1EDE0 + 3)


def run_ablation(args):
    """The paper's ablation of DF Leiden (Sec. 4.2-4.4 and its figure): Full
    Refine (every community refined in the first pass), Subset Refine (only
    the changed ones) and Optimized Aggregation (Subset Refine with the
    size-tiered aggregation kernels; the other two aggregate every community
    through one bucketed method), on R-MAT scale 22 and the 5000 x 5000 grid,
    batches of 1e-7 .. 1e-1 |E| (samples per size: --lowdeg-samples).
    Reports the DF update time and modularity per variant and batch size."""
    import torch
    from paper_2405_11658_gb300 import synth as S
    torch.cuda.set_device(0)
    import paper_2405_11658_gb300 as L
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    out = {}
    launches0 = L.kernel_launches()
    with Clocks(0) as clk:
        for name, g in _ablation_graphs():
            pairs = S.undirected_pairs(*g)
            nedges = len(pairs[0])
            batches = []
            for i, frac in enumerate(ABLATION_FRACS):
                for k in range(args.lowdeg_samples):
                    d, ins = S.random_batch(*g, max(2, int(round(frac * nedges))), seed=3000 + 10 * i + k,
                                            pairs=pairs)
                    batches.append((frac, L.Edges.from_numpy(d, device=dev), L.Edges.from_numpy(ins, device=dev)))
            max_nnz = len(g[1]) + 2 * max(b[2].count for b in batches) + 16
            G0 = L.Graph.from_numpy(*g, device=dev)
            res = {}
            with L.Context(max_n=G0.n, max_nnz=max_nnz, stream=stream) as ctx:
                Cs, _ = ctx.static(G0, L.Opts(), want_q=False)
                C0, K0, S0, _ = ctx.update(G0, Cs, None, None, "ND", L.Opts(), want_q=False)
                static_ms = []
                for frac, dE, iE in batches:
                    Gt = ctx.apply_batch(G0, dE, iE, cap_nnz=max_nnz)
                    key = f"{frac:g}"
                    for vname, full, uniform in ABLATION_VARIANTS:
                        ctx.set_agg_policy(uniform)
                        opts = L.Opts(refine_all_first_pass=full)
                        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                        a.record(stream)
                        _, _, _, q = ctx.update(Gt, C0, dE, iE, "DF", opts, prior_K=K0, prior_Sigma=S0)
                        b.record(stream)
                        b.synchronize()
                        st = ctx.stats()
                        r = res.setdefault(key, {}).setdefault(vname, {"ms": [], "q": [], "agg_ms": []})
                        r["ms"].append(a.elapsed_time(b))
                        r["q"].append(q)
                        r["agg_ms"].append(sum(st["t_agg_ms"]))
                    ctx.set_agg_policy(False)
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    _, qs = ctx.static(Gt, L.Opts())
                    b.record(stream)
                    b.synchronize()
                    static_ms.append(a.elapsed_time(b))
                    res[key].setdefault("static_q", []).append(qs)
                    del Gt
            summ = {}
            for key, r in res.items():
                summ[key] = {"static_q": float(np.mean(r["static_q"]))}
                for vname, _, _ in ABLATION_VARIANTS:
                    summ[key][vname] = {"df_ms_p50": float(np.median(r[vname]["ms"])),
                                        "agg_ms_p50": float(np.median(r[vname]["agg_ms"])),
                                        "q_mean": float(np.mean(r[vname]["q"]))}
                base = summ[key]["full_refine"]["df_ms_p50"]
                for vname, _, _ in ABLATION_VARIANTS:
                    summ[key][vname]["relative_to_full_refine"] = summ[key][vname]["df_ms_p50"] / base
            out[name] = {"vertices": G0.n, "csr_entries": G0.nnz, "static_ms_p50": float(np.median(static_ms)),
                         "by_batch": summ}
    line = {"metric": "DF update time, Full Refine / Subset Refine / Optimized Aggregation (relative)",
            "value": float(np.mean([v["by_batch"][k]["optimized_aggregation"]["relative_to_full_refine"]
                                    for v in out.values() for k in v["by_batch"]])),
            "unit": "DF time of Optimized Aggregation relative to Full Refine (mean over graphs and sizes)",
            "n_gpus": 1, "higher_is_better": False, "dtype": "int64", "data": "synthetic",
            "config": {"workload": "ablation: DF Leiden with Full Refine, Subset Refine, Optimized Aggregation",
                       "batch_fracs": list(ABLATION_FRACS), "samples_per_size": args.lowdeg_samples},
            "graphs": out, "gpu_launches": L.kernel_launches() - launches0, "clocks": clk.summary()}
    print(json.dumps(line))
    return 0


SMSCALE_COUNTS = (8, 16, 32, 64, 128)


def run_smscale(args):
    """Static and DF Leiden (1e-4 |E| batch) on R-MAT scale 22 with the
    context restricted to 8, 16, 32, 64 and 128 SMs (green contexts) and on
    the whole GPU: the counterpart of the paper's strong-scaling study over
    1..64 threads (Sec. 5.2).  Times are the calls' wall times (the calls
    synchronise), median of --steps runs; every SM count must return the same
    membership."""
    import torch
    from paper_2405_11658_gb300 import synth as S
    torch.cuda.set_device(0)
    import paper_2405_11658_gb300 as L
    g = RmatWorkload(args.scale).host_graph(RMAT_SEED)
    dels, ins = S.random_batch(*g, max(2, int(round(1e-4 * len(g[1]) / 2))), seed=77)
    G = L.Graph.from_numpy(*g)
    dE, iE = L.Edges.from_numpy(dels), L.Edges.from_numpy(ins)
    total = torch.cuda.get_device_properties(0).multi_processor_count
    rows, ref_hash = [], None
    with Clocks(0) as clk:
        for sms in list(SMSCALE_COUNTS) + [None]:
            kw = {"sm_count": sms} if sms else {}
            with L.Context(max_n=G.n, max_nnz=G.nnz + 2 * iE.count + 16, **kw) as ctx:
                Gt = ctx.apply_batch(G, dE, iE)
                Cs, _ = ctx.static(G, L.Opts(), want_q=False)
                C0, K0, S0, _ = ctx.update(G, Cs, None, None, "ND", L.Opts(), want_q=False)
                st_ms, df_ms = [], []
                for _ in range(max(1, args.steps)):
                    m, _ = ctx.static(Gt, L.Opts(), want_q=False)
                    st_ms.append(ctx.stats()["total_ms"])
                    ctx.update(Gt, C0, dE, iE, "DF", L.Opts(), prior_K=K0, prior_Sigma=S0, want_q=False)
                    df_ms.append(ctx.stats()["total_ms"])
                h = int(torch.sum(m.to(torch.int64) * (torch.arange(G.n, device=m.device) % 65521)))
                ref_hash = h if ref_hash is None else ref_hash
                rows.append({"sms": ctx.sms, "static_ms": float(np.median(st_ms)), "df_ms": float(np.median(df_ms)),
                             "same_membership": h == ref_hash})
    base = rows[0]
    for r in rows:
        r["static_speedup_vs_fewest"] = base["static_ms"] / r["static_ms"]
        r["df_speedup_vs_fewest"] = base["df_ms"] / r["df_ms"]
    # speedup per doubling of the SM count, from the fewest to the most SMs
    full = rows[-1]
    dbl = np.log2(full["sms"] / base["sms"])
    line = {"metric": "Static / DF Leiden time vs SM count (green contexts), R-MAT scale 22",
            "value": float((base["static_ms"] / full["static_ms"]) ** (1.0 / dbl)) if dbl > 0 else None,
            "unit": "Static speedup per doubling of the SMs", "n_gpus": 1, "higher_is_better": True,
            "dtype": "int64", "data": "synthetic",
            "config": {"workload": "sm scaling", "graph": f"R-MAT scale {args.scale}, edge factor {EDGE_FACTOR}",
                       "df_batch": "1e-4 |E|", "sm_total": total, "runs_per_point": max(1, args.steps)},
            "points": rows,
            "df_speedup_per_doubling": float((base["df_ms"] / full["df_ms"]) ** (1.0 / dbl)) if dbl > 0 else None,
            "clocks": clk.summary()}
    print(json.dumps(line))
    return 0


DECIDE_KERNEL_PREFIXES = ("decide_", "hub_")


def record_traffic(args):
    """Writes profiles/decide_traffic_<workload>.json from an ncu capture of
    the first pass's local-moving range (--metrics dram__bytes_read.sum,
    dram__bytes_write.sum, gpu__time_duration.sum; --nvtx-include
    "local_move_pass0/") and the JSON line the same --profile-static command
    printed: DRAM bytes of the decide kernels per colour class and per scanned
    CSR entry, next to their algorithmic bytes."""
    import csv
    rows = list(csv.reader(open(args.record_traffic)))
    start = next(k for k, r in enumerate(rows) if r and r[0] == "ID")
    hdr = rows[start]
    ki, mn, mv, mu = (hdr.index(x) for x in ("Kernel Name", "Metric Name", "Metric Value", "Metric Unit"))
    scale = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "nsecond": 1e-9, "usecond": 1e-6,
             "msecond": 1e-3, "second": 1.0}
    rd = wr = 0.0
    kernels = 0
    for r in rows[start + 1:]:
        if len(r) <= mv or not r[ki].split("<")[0].split("(")[0].replace("void ", "").strip().startswith(
                DECIDE_KERNEL_PREFIXES):
            continue
        v = float(r[mv].replace(",", "")) * scale.get(r[mu], 1.0)
        if r[mn] == "dram__bytes_read.sum":
            rd += v
            kernels += 1
        elif r[mn] == "dram__bytes_write.sum":
            wr += v
    prof = None
    for ln in open(args.profile_json):
        ln = ln.strip()
        if ln.startswith("{"):
            prof = json.loads(ln)
    subs = prof["move0_kernel_launches"]
    out = {"workload": prof["workload"], "capture": os.path.basename(args.record_traffic),
           "source_sha256": decide_sources_sha(), "sub_sweeps": subs, "decide_kernel_launches": kernels,
           "dram_read_bytes": rd, "dram_write_bytes": wr,
           "dram_bytes_per_launch": (rd + wr) / subs,
           "algorithmic_bytes_per_launch": prof["move0_bytes"] / subs,
           "scanned_entries_per_launch": prof["move0_scanned_entries"] / subs,
           "dram_bytes_per_scanned_entry": (rd + wr) / prof["move0_scanned_entries"]}
    path = TRAFFIC_FILES[args.workload]
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out))
    return 0


def run_profile_static(args):
    """One Static Leiden (DET) on the workload's graph (``--workload cl`` or
    ``rmat``; ``--cl-div k`` takes the Chung-Lu recipe at 1/k of the vertices
    and edges) with the decide kernels timed; prints the run's statistics as
    one JSON line.  A profiler run over this command sees exactly one run's
    launches (local-moving inside the NVTX range "local_move", its first pass
    in "local_move_pass0", refinement in "refine", aggregation in
    "aggregate")."""
    import torch
    torch.cuda.set_device(0)
    import paper_2405_11658_gb300 as L
    if args.workload == "cl":
        from paper_2405_11658_gb300 import synth_device as D
        n, m = CL_N // args.cl_div, CL_M // args.cl_div
        (off, idx, w), _ = D.chung_lu(n, m, 2.1, 1, 4, seed=CL_SEED, device="cuda")
        torch.cuda.empty_cache()
        G = L.Graph(off, idx, w)
        name = f"chung-lu {n} vertices {2 * m} entries static leiden"
    else:
        g = RmatWorkload(args.scale).host_graph(RMAT_SEED)
        G = L.Graph.from_numpy(*g)
        name = f"rmat-s{args.scale}-ef{EDGE_FACTOR} static leiden"
    with L.Context(max_n=G.n, max_nnz=G.nnz + 16) as ctx:
        ctx.set_timing(True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, q = ctx.static(G, L.Opts(sched=L.DET if args.sched == "det" else L.ASYNC))
        torch.cuda.synchronize()
        ms = 1000 * (time.perf_counter() - t0)
        st = ctx.stats()
    keep = ("passes", "iters", "nv", "nnz", "moves", "refine_moves", "move_kernel_ms", "move_kernel_launches",
            "move_scanned_entries", "move_scanned_vertices", "move_bytes", "move0_kernel_ms",
            "move0_kernel_launches", "move0_bytes", "move0_scanned_entries", "t_move_ms", "t_refine_ms",
            "t_agg_ms", "wide_passes")
    print(json.dumps({"workload": name, "ms": ms, "q": q, **{k: st[k] for k in keep}}))
    return 0


def main():
    args = parse()
    if args.record_traffic:
        return record_traffic(args)
    if args.profile_static:
        return run_profile_static(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "serving":
        return run_serving(args)
    if args.workload == "lowdeg":
        return run_lowdeg(args)
    if args.workload == "temporal":
        return run_temporal(args)
    if args.workload == "ablation":
        return run_ablation(args)
    if args.workload == "smscale":
        return run_smscale(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
