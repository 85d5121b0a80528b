#!/usr/bin/env python
"""Benchmark of the LST hot path on GB300 (one JSON line on rank 0).

Workload: PU200-like synthetic events (4000 helix tracks, pT pdf ~ 1/pT^2 above 0.5 GeV,
|eta| < 2.4, 20 % noise hits, 6 barrel layers + 5 disks per side) with pixel seeds (1 %
pT / 1 mrad smear, 10 % fakes), so that every step of the chain runs: binning, MD, LS, T3,
T5, pLS lookup, pT3, pT5, duplicate removal, track candidates.  A step is one batch of
--batch events through the whole chain.

  value     events/s, batched + CUDA graph, inputs resident in HBM (lst_run_batch_device)
  e2e       events/s through lst_submit_batch / lst_collect_batch with host buffers (copies inside the timed region)
  per_event events/s and p50/p99 latency of the plain per-event launch (lst_run_event)
  served    p50/p99 latency and events/s of the continuous-batching loop (lst_serve_replay)
  roofline  the kernel with the largest device time, algorithmic bytes / CUDA-event time
  cpu_baseline  the CPU oracle on the host cores, on a bounded sample of the same events

--impl reference times the CPU oracle itself on the same workload and metric.
Multi-GPU: one process per GPU (torchrun), each a replica on its own events (weak scaling).
"""
import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "events/s + p99 event latency at PU200-like load, served vs per-event; oracle-exact"
WORKLOAD = "pu200_4000trk_20pct_noise_with_pixel_seeds"
KERNEL_SOURCES = ["paper_2407_18231_gb300/csrc/lst_kernels.cu", "paper_2407_18231_gb300/csrc/lst_cuts.cuh",
                  "paper_2407_18231_gb300/csrc/lst_device.cuh"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="lst", choices=["lst", "reference"])
    ap.add_argument("--batch", type=int, default=32, help="events per step")
    ap.add_argument("--pool", type=int, default=4, help="distinct resident batches rotated over")
    ap.add_argument("--per-event", type=int, default=48, help="events for the per-event leg (0 = skip)")
    ap.add_argument("--served", type=int, default=2048, help="events for the served leg (0 = skip)")
    ap.add_argument("--served-rate", type=float, default=0.0, help="offered Hz (0: 0.8 x batched rate)")
    ap.add_argument("--cpu-sample", type=int, default=8, help="events for the CPU-oracle baseline (0 = skip)")
    ap.add_argument("--tune", type=int, default=1, help="autotune the launch configuration first (1) or not (0)")
    ap.add_argument("--config", default="", help="fixed launch configuration block_size,blocks_per_sm,ls_list_cap "
                                                 "(skips the autotuner)")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def make_events(n, first):
    import lst_synth as S
    return [S.make_event("pu200", first + i, with_pls=True) for i in range(n)]


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "200"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() in ("active", "1"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- CPU oracle
def cpu_oracle_rate(events, geom_modules):
    import oracle
    og = oracle.Geometry(geom_modules)
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    oracle.run_many(og, events, n_threads=cores, convert=False)
    dt = time.perf_counter() - t0
    return len(events) / dt, cores, dt


def reference_arm(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import lst_synth as S
    geom = S.geometry(False)
    per_step = max(1, min(args.batch, 4))
    evs = make_events(per_step * 2, 10_000)
    import oracle
    og = oracle.Geometry(geom.modules)
    cores = os.cpu_count() or 1
    for w in range(args.warmup):
        oracle.run_many(og, evs[:per_step], n_threads=cores, convert=False)
    t0 = time.perf_counter()
    for k in range(args.steps):
        oracle.run_many(og, evs[(k % 2) * per_step:(k % 2 + 1) * per_step], n_threads=cores, convert=False)
    dt = time.perf_counter() - t0
    rate = args.steps * per_step / dt
    line = {"metric": METRIC, "value": rate, "unit": "events/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "events_per_step": per_step, "parallelism": "host threads over events"},
            "cpu_baseline": {"value": rate, "unit": "events/s", "cores": cores, "kind": "oracle",
                             "sample": f"{per_step} PU200-like events per step, all host cores"},
            "e2e": {"value": rate, "unit": "events/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- ranks
def aggregate(elapsed_ms: float, events_per_rank: int):
    """Weak scaling over replicas: every rank processed events_per_rank events, the job
    took as long as the slowest rank.  Returns (events/s of the whole job, max ms)."""
    import torch
    import torch.distributed as dist
    ws = dist.get_world_size() if dist.is_available() and dist.is_initialized() else 1
    if ws > 1:
        dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
        t = torch.tensor([elapsed_ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed_ms = float(t.item())
    return ws * events_per_rank / (elapsed_ms * 1e-3), elapsed_ms


# ---------------------------------------------------------------- roofline
def kernel_hash():
    """Hash of the kernel sources' code: comments and blank lines do not count."""
    h = hashlib.sha1()
    for p in KERNEL_SOURCES:
        src = open(os.path.join(ROOT, p)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        h.update("\n".join(l.rstrip() for l in src.splitlines() if l.strip()).encode())
    return h.hexdigest()[:12]


def recorded_traffic(kernel):
    """dram bytes per launch of `kernel` from the committed ncu summary, if its source hash matches."""
    path = os.path.join(ROOT, "profiles", "traffic.md")
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    m = re.search(rf"^\|\s*{re.escape(kernel)}\s*\|\s*([0-9a-f]+)\s*\|\s*(\d+)\s*\|", txt, re.M)
    if not m or m.group(1) != kernel_hash():
        return None
    return int(m.group(2))


def algorithmic_bytes(kernel, st, n_units):
    """Minimum bytes a kernel must move, from the object counts of one batch.

    Records: hit 16 B (x,y,z,r) + 4 B index; MD 60 B (two float4 points, a float4 of
    tolerances, unit, two hit indices); LS 8 B; T3 12 B; T5 28 B; pLS 80 B in, 36 B params;
    pT3/pT5 12 B; per-unit counts/offsets 4 B each."""
    h, md, ls, t3, t5 = st["n_hits"], st["n_md"], st["n_ls"], st["n_t3"], st["n_t5"]
    p, pt3, pt5 = st["n_pls"], st["n_pt3"], st["n_pt5"]
    md_rec = 52  # what a join reads of an MD: two float4 points, tolerances, unit
    table = {
        "md_count": h * 20 + n_units * 12,
        "md_fill": h * 20 + n_units * 8 + md * 60,
        "ls_count": md * (md_rec + 8) + n_units * 8,
        "ls_fill": md * (md_rec + 8) + n_units * 8 + ls * 8,
        "t3_count": md * (md_rec + 8) + ls * 4,
        "t3_fill": md * (md_rec + 8) + ls * 4 + t3 * 12,
        "t5_count": md * md_rec + t3 * 12 + md * 8,
        "t5_fill": md * md_rec + t3 * 12 + md * 8 + t5 * 28,
        "pt3_count": p * (36 + 4 * 37) + t3 * 12 + md * md_rec,
        "pt3_fill": p * (36 + 4 * 37) + t3 * 12 + md * md_rec + pt3 * 12,
        "pt5_count": p * (36 + 4 * 37) + t5 * 24 + md * md_rec,
        "pt5_fill": p * (36 + 4 * 37) + t5 * 24 + md * md_rec + pt5 * 12,
        "hits_sort": h * (16 + 16 + 4),
        "pls_prep": p * (80 + 36 + 4 * 37),
    }
    return table.get(kernel)


# FP32 operations (add, sub, mul, div, sqrt, compare; abs is free) of the LS cuts, counted
# from their expressions: the r-z pointing test on every connection-map candidate pair, the
# bending test and the chord-direction tests of both MDs on every LS that comes out.  A
# lower bound on the cut arithmetic any implementation of the selection performs.
LS_OPS_RZ = 21
LS_OPS_REST = 20 + 38


def algorithmic_ops(kernel, st):
    if kernel == "ls_count" and st.get("ls_candidates"):
        return LS_OPS_RZ * st["ls_candidates"] + LS_OPS_REST * st["n_ls"]
    return None


def alu_peak(n_sm, sm_mhz):
    """FP32 ops/s: every SM issues 128 FP32 lanes per clock (4 partitions x 32)."""
    return n_sm * 128 * sm_mhz * 1e6


def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
        return
    ws, rank, local = dist_env()
    import torch
    import paper_2407_18231_gb300 as lst
    from paper_2407_18231_gb300 import validation as V
    import lst_synth as S
    if ws > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    lst.build()
    geom = S.geometry(False)
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}

    B, P = args.batch, args.pool
    events = make_events(B * P, 100_000 * rank)
    batches = [events[i * B:(i + 1) * B] for i in range(P)]

    # device-resident inputs, one concatenated set per batch
    def to_device(evs):
        cat = lambda k: torch.from_numpy(np.ascontiguousarray(np.concatenate([getattr(e, k) for e in evs]))).to(dev)  # noqa
        x, y, z = cat("x"), cat("y"), cat("z")
        det = torch.from_numpy(np.concatenate([e.det for e in evs]).view(np.int32)).to(dev)
        pls = torch.from_numpy(np.concatenate([e.pls for e in evs]).view(np.uint8)).to(dev)
        hoff = torch.tensor(np.concatenate([[0], np.cumsum([e.n_hits for e in evs])]).astype(np.int32), device=dev)
        poff = torch.tensor(np.concatenate([[0], np.cumsum([e.n_pls for e in evs])]).astype(np.int32), device=dev)
        desc = lst.lst_batch_dev(len(evs), int(hoff[-1]), int(poff[-1]), max(e.n_hits for e in evs),
                                 x.data_ptr(), y.data_ptr(), z.data_ptr(), det.data_ptr(), hoff.data_ptr(),
                                 pls.data_ptr(), poff.data_ptr())
        return desc, (x, y, z, det, pls, hoff, poff)

    dev_batches = [to_device(b) for b in batches]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2
    tuning = {}
    if args.config:
        bs, bps, cap = (int(v) for v in args.config.split(","))
        tuning = {"block_size": bs, "blocks_per_sm": bps, "ls_list_cap": cap}
    elif args.tune:
        from paper_2407_18231_gb300 import autotune
        space = {"block_size": [128, 256], "blocks_per_sm": [4, 8, 12], "ls_list_cap": [128, 512]}
        tuning = autotune.tune(geom.modules, events[:B], device=local, space=space, reps=5)["best"]
    sess = lst.Session(geom.modules, device=local, **tuning)
    # the library runs on this stream, so events recorded on it bracket its kernels
    stream = torch.cuda.Stream(dev)
    assert stream.cuda_stream != 0

    # every resident batch at least once before timing: buffers sized, graph captured
    n_warm = max(args.warmup, P)
    for k in range(n_warm):
        sess.run_batch_device(dev_batches[k % P][0], stream.cuda_stream)
        sess.batch_finish(B, timeout_ms=120000)
    stats = sess.stats()
    reruns_before = stats["reruns"]
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    with ClockSampler(local) as clk, torch.cuda.stream(stream):
        torch.cuda.synchronize()
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        elapsed_ms = 0.0
        for k in range(args.steps):
            flush.zero_()  # between timed iterations: evict L2 (not timed)
            t_start.record(stream)
            sess.run_batch_device(dev_batches[k % P][0], stream.cuda_stream)
            t_end.record(stream)
            # status check of the step (overflow re-run, bad input) after the timed region
            sess.batch_finish(B, timeout_ms=120000)
            elapsed_ms += t_start.elapsed_time(t_end)
        torch.cuda.synchronize()
    if sess.stats()["reruns"] != reruns_before:
        raise RuntimeError("a timed step re-ran after a list overflow; warm-up did not size the buffers")
    if ws > 1:
        torch.distributed.barrier()
    value, elapsed_ms = aggregate(elapsed_ms, args.steps * B)
    kernels_per_step = stats["kernels"]

    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return

    # ---- end to end: host buffers through the asynchronous batch API (lst_submit_batch /
    # lst_collect_batch): one batch in flight while the next is packed and uploaded; every
    # step's H2D copy and the read-back of its candidates fall inside the timed region
    sess_h = lst.Session(geom.modules, device=local, **tuning)
    for k in range(max(args.warmup, P) + 1):  # both slots: buffers sized, graphs captured
        t_w = sess_h.submit_batch(batches[k % P])
        for i in sess_h.collect_batch(sess_h.submit_batch(batches[(k + 1) % P])) + sess_h.collect_batch(t_w):
            sess_h.release(i)
    torch.cuda.synchronize()
    e2e_steps = max(3, min(args.steps, 10))
    d2h = 0
    t0 = time.perf_counter()
    ticket = sess_h.submit_batch(batches[0])
    for k in range(e2e_steps):
        nxt = sess_h.submit_batch(batches[(k + 1) % P]) if k + 1 < e2e_steps else None
        ids = sess_h.collect_batch(ticket)
        tcs, _ = sess_h.candidates_batch(ids)
        d2h += len(tcs) * 76 + (B + 1) * 4 + 256
        for i in ids:
            sess_h.release(i)
        ticket = nxt
    e2e_s = time.perf_counter() - t0
    e2e = {"value": e2e_steps * B / e2e_s, "unit": "events/s",
           "h2d_bytes_per_step": int(np.mean([sum(e.n_hits * 16 + e.n_pls * 80 for e in b) + 2 * (B + 1) * 4
                                              for b in batches])),
           "d2h_bytes_per_step": int(d2h / e2e_steps), "api": "lst_submit_batch / lst_collect_batch, one batch in flight"}

    # ---- physics: track-level metrics (Sec. 3) of the first batch's candidates, not timed
    phys_ids = sess_h.run_batch(batches[0])
    tcs, counts = sess_h.candidates_batch(phys_ids)
    for i in phys_ids:
        sess_h.release(i)
    offs = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    c_all, c_ot = [], []
    for k, e in enumerate(batches[0]):
        tc = tcs[offs[k]:offs[k + 1]]
        sel = (e.tracks["pt"] >= 0.9) & (np.abs(e.tracks["eta"]) < 2.4)
        c_all.append(V.event_counts(tc, e.sim, e.pls_sim, len(e.tracks), sel))
        c_ot.append(V.event_counts(tc[tc["type"] != lst.TC_PLS], e.sim, e.pls_sim, len(e.tracks), sel))
    r_all, r_ot = V.rates(c_all), V.rates(c_ot)
    physics = {"events": B, "selection": "simulated tracks with pT >= 0.9 GeV and |eta| < 2.4",
               "match": "more than 75 % of a candidate's hits from one simulated track (Sec. 3)",
               "efficiency": r_all["efficiency"], "fake_rate": r_all["fake_rate"],
               "duplicate_rate": r_all["duplicate_rate"],
               "without_pls_only": {"efficiency": r_ot["efficiency"], "fake_rate": r_ot["fake_rate"],
                                    "duplicate_rate": r_ot["duplicate_rate"]}}

    # ---- per-event launch: latency of single events
    per_event = None
    if args.per_event:
        for i in sess_h.run_batch(batches[0]):  # size the main pipeline for any single event
            sess_h.release(i)
        lat = []
        for e in events[: args.per_event]:
            t0 = time.perf_counter()
            rid = sess_h.run_event(e)
            sess_h.candidates(rid)
            lat.append(time.perf_counter() - t0)
            sess_h.release(rid)
        lat = np.array(lat[2:])
        per_event = {"events_per_s": float(1.0 / lat.mean()), "p50_ms": float(np.percentile(lat, 50) * 1e3),
                     "p99_ms": float(np.percentile(lat, 99) * 1e3), "events": int(len(lat))}

    # ---- served: Poisson arrivals into the continuous-batching loop
    served = None
    if args.served:
        rate = args.served_rate or 0.8 * value
        rng = np.random.default_rng(7)
        arrival = np.cumsum(rng.exponential(1.0 / rate, args.served))
        evs = [events[i % len(events)] for i in range(args.served)]
        lat, ntc, _, wall = sess_h.serve_replay(evs, arrival, n_slots=4, max_batch=B)
        served = {"offered_hz": rate, "events_per_s": args.served / wall, "p50_ms": float(np.percentile(lat, 50) * 1e3),
                  "p99_ms": float(np.percentile(lat, 99) * 1e3), "events": args.served, "slots": 4,
                  "max_batch": B}

    # ---- roofline of the dominant kernel (profile mode: CUDA events around every kernel)
    prof_sess = lst.Session(geom.modules, device=local, profile=True, **tuning)
    acc = {}
    reps = 3
    for r in range(reps + 1):
        prof_sess.run_batch_device(dev_batches[r % P][0], stream.cuda_stream)
        prof_sess.batch_finish(B, timeout_ms=120000)
        if r == 0:
            continue
        for name, (n, ms) in prof_sess.profile().items():
            a = acc.setdefault(name, [0, 0.0])
            a[0] += n
            a[1] += ms
    pst = prof_sess.stats()
    top = max(acc.items(), key=lambda kv: kv[1][1])
    kname, (nl, tot_ms) = top
    per_launch_ms = tot_ms / nl
    n_units = B * geom.n_modules
    algo = algorithmic_bytes(kname, pst, n_units)
    ops = algorithmic_ops(kname, pst)
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    roof = None
    share = tot_ms / sum(v[1] for v in acc.values())
    hbm = None
    if algo is not None:
        achieved = algo / (per_launch_ms * 1e-3) / 1e9
        hbm = {"achieved": achieved, "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
               "peak_source": peak_src, "algorithmic_bytes": algo}
    if ops is not None:
        # the cut chain is FP32 arithmetic on an L2-resident working set: the ALU roof binds
        n_sm = torch.cuda.get_device_properties(local).multi_processor_count
        mhz = clk.summary().get("sm_max_mhz") or 2070.0
        peak = alu_peak(n_sm, mhz) / 1e12
        achieved = ops / (per_launch_ms * 1e-3) / 1e12
        roof = {"bound": "alu", "kernel": kname, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": recorded_traffic(kname),
                "peak_source": f"derived: {n_sm} SMs x 128 FP32 lanes x {mhz:.0f} MHz",
                "algorithmic_ops": ops, "ls_candidates": pst["ls_candidates"], "ms_per_launch": per_launch_ms,
                "kernel_share": share, "hbm": hbm}
    elif hbm is not None:
        roof = {"bound": "hbm", "kernel": kname, "traffic": recorded_traffic(kname), "ms_per_launch": per_launch_ms,
                "kernel_share": share, **hbm}
    kernel_times = {k: round(v[1] / reps, 4) for k, v in sorted(acc.items(), key=lambda kv: -kv[1][1])}

    # ---- CPU oracle on a bounded sample of the same events
    cpu = None
    if args.cpu_sample:
        rate_cpu, cores, dt = cpu_oracle_rate(events[: args.cpu_sample], geom.modules)
        cpu = {"value": rate_cpu, "unit": "events/s", "cores": cores, "kind": "oracle",
               "sample": f"{args.cpu_sample} of the benchmark's events, threads over events, {dt:.1f} s"}

    clocks = clk.summary()
    line = {
        "metric": METRIC, "value": value, "unit": "events/s", "n_gpus": ws, "steps": args.steps,
        "warmup": n_warm, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "events_per_step": B, "mean_hits_per_event": float(np.mean([e.n_hits for e in events])),
                   "mean_pls_per_event": float(np.mean([e.n_pls for e in events])),
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                   "mode": "batched persistent kernels, CUDA graph replay",
                   "tuning": tuning or "defaults",
                   "l2": "256 MB buffer written between timed steps; inputs rotate over "
                         f"{P} resident batches"},
        "e2e": e2e, "per_event": per_event, "served": served, "physics": physics,
        "objects_per_step": {k: stats[k] for k in ("n_md", "n_ls", "n_t3", "n_t5", "n_pt3", "n_pt5", "n_tc")},
        "roofline": roof, "kernel_ms_per_step": kernel_times, "cpu_baseline": cpu, "clocks": clocks,
        "gpu_launches": kernels_per_step * args.steps,
    }
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
