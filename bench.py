#!/usr/bin/env python
"""Benchmark of the LST hot path on GB300 (one JSON line on rank 0).

Workload: PU200-like synthetic events (4000 helix tracks, pT pdf ~ 1/pT^2 above 0.5 GeV,
|eta| < 2.4, 20 % noise hits, 6 barrel layers + 5 disks per side) with pixel seeds (1 %
pT / 1 mrad smear, 10 % fakes), so that every step of the chain runs: binning, MD, LS, T3,
T5, pLS lookup, pT3, pT5, duplicate removal, track candidates.  A step is one batch of
--batch events through the whole chain.

  value      events/s, batched + CUDA graph, inputs resident in HBM (lst_run_batch_device)
  parity     after timing, sampled events of a timed batch against the CPU oracle, bit for bit
  sustained  the same step repeated for --sustain seconds (clock evidence under load)
  e2e        events/s through lst_submit_batch / lst_collect_batch with host buffers (copies inside the timed region)
  per_event  events/s and p50/p99 latency of the plain per-event launch (lst_run_event)
  served     p50/p99 latency and events/s of the continuous-batching loop (lst_serve_replay)
  serving_sweep  the serving workload (U{2000..8000} tracks) at 1-20 kHz offered, 1, 8 and
             64 GB budgets, slots' batches one after another or sharing the device
  workloads  the tiny event (us/event), the 64-event barrel batch, the 16-event
             high-occupancy batch with seeds and the headline batch in the geometry with
             tilted inner-barrel modules (events/s, objects/s), each with a parity check
  roofline   the kernel with the largest device time, algorithmic work / CUDA-event time;
             the MD and LS stages' HBM fraction beside it
  seeding    LST as a seeder (Sec. 2, Table 1): unlinked seeds handed on, quads only or
             quads and triplets, and the simulated tracks LST's tracks plus those seeds cover
  cpu_baseline  the CPU oracle on the host cores (1 thread, 2 threads pinned to 2 cores,
             all cores) on the benchmark's own events

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
# serving: two slots of up to 16 events each, sharing the device -- the lowest p99 latency
# measured at 12 and 16.6 kHz of PU200-like events among 2-8 slots of 4-32 events, at the
# same throughput (4.3 ms at 16.6 kHz against 17.6 ms for four slots of 32)
SERVE_SLOTS, SERVE_BATCH = 2, 16
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
    ap.add_argument("--cpu-sample", type=int, default=1, help="CPU-oracle baseline (0 = skip)")
    ap.add_argument("--sustain", type=float, default=2.0, help="seconds of the sustained run (0 = skip)")
    ap.add_argument("--sweep", type=int, default=1, help="serving sweep over rates and budgets (0 = skip)")
    ap.add_argument("--legs", type=int, default=1, help="tiny / barrel-batch / high-occupancy legs (0 = skip)")
    ap.add_argument("--parity", type=int, default=3, help="events of a timed batch checked against the oracle")
    ap.add_argument("--tune", type=int, default=1, help="autotune the launch configuration first (1) or not (0)")
    ap.add_argument("--workload", default="pu200", choices=["pu200", "highocc"],
                    help="events of the timed batches (profiling: highocc = 12000 tracks, 30 %% noise)")
    ap.add_argument("--t5", default="cuts", choices=["cuts", "learned"],
                    help="T5 selection of the timed and end-to-end sessions (learned: the shipped network)")
    ap.add_argument("--config", default="", help="fixed launch configuration block_size,blocks_per_sm,ls_list_cap "
                                                 "(skips the autotuner)")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def make_events(n, first, workload="pu200"):
    import lst_synth as S
    return [S.make_event(workload, first + i, with_pls=True) for i in range(n)]


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
def _oracle_seconds(og, events, threads, cpus=None):
    """Wall seconds of the oracle over `events` on `threads` host threads (optionally
    pinned to the CPU set `cpus`: the calling thread's affinity, which the oracle's threads
    inherit)."""
    import oracle
    old = os.sched_getaffinity(0) if cpus else None
    try:
        if cpus:
            os.sched_setaffinity(0, cpus)
        t0 = time.perf_counter()
        oracle.run_many(og, events, n_threads=threads, convert=False)
        return time.perf_counter() - t0
    finally:
        if old:
            os.sched_setaffinity(0, old)


def check_pending(pending):
    """CPU leg: the oracle on every event whose GPU candidates were kept, field by field."""
    import oracle
    geoms, out = {}, {}
    for label, k, tc, ev, modules, t5_weights in pending:
        key = (id(modules), None if t5_weights is None else id(t5_weights))
        if key not in geoms:
            geoms[key] = oracle.Geometry(modules)
            oracle.set_t5_mlp(geoms[key], t5_weights)
        r = out.setdefault(label, {"events": [], "identical": True,
                                   "compared": "every track-candidate field, pT and score bit for bit"})
        r["events"].append(k)
        r["identical"] = r["identical"] and tc_parity(tc, oracle.run(geoms[key], ev))
    return out


def cpu_oracle_rates(events, geom_modules):
    """The oracle as it stands on the host cores, on the benchmark's own events: one thread,
    two threads pinned to two cores (the paper's CPU setup, Sec. 3), and every core (at
    least two events per core so that no core idles).  A bounded sample: about 10 s."""
    import oracle
    og = oracle.Geometry(geom_modules)
    cpus = sorted(os.sched_getaffinity(0))
    cores = len(cpus)
    n1 = min(len(events), 6)
    n2 = min(len(events), 8)
    na = min(len(events), 2 * cores)
    t1 = _oracle_seconds(og, events[:n1], 1)
    t2 = _oracle_seconds(og, events[:n2], 2, set(cpus[:2]))
    ta = _oracle_seconds(og, events[:na], cores)
    return {"value": na / ta, "unit": "events/s", "cores": cores, "kind": "oracle",
            "rates": {"1_thread": n1 / t1, "2_threads_pinned_2_cores": n2 / t2, f"{cores}_threads": na / ta},
            "sample": f"the benchmark's first PU200-like events with seeds: {n1} on 1 thread ({t1:.1f} s), "
                      f"{n2} on 2 threads pinned to 2 cores ({t2:.1f} s), {na} on {cores} threads ({ta:.1f} s)"}


def reference_arm(args):
    """The CPU oracle as the reference arm: every step runs 2 x cores of the benchmark's
    events on all host cores (threads over events)."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import lst_synth as S
    import oracle
    geom = S.geometry(False)
    cores = len(os.sched_getaffinity(0))
    per_step = 2 * cores
    evs = make_events(per_step, 0)
    og = oracle.Geometry(geom.modules)
    for w in range(args.warmup):
        oracle.run_many(og, evs, n_threads=cores, convert=False)
    t0 = time.perf_counter()
    for k in range(args.steps):
        oracle.run_many(og, evs, n_threads=cores, convert=False)
    dt = time.perf_counter() - t0
    rate = args.steps * per_step / dt
    cpu = cpu_oracle_rates(evs, geom.modules)
    line = {"metric": METRIC, "value": rate, "unit": "events/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "events_per_step": per_step, "parallelism": f"{cores} host threads over events"},
            "cpu_baseline": {"value": rate, "unit": "events/s", "cores": cores, "kind": "oracle",
                             "rates": cpu["rates"],
                             "sample": f"{per_step} PU200-like events per step (the GPU benchmark's first events), "
                                       f"all {cores} host cores; {cpu['sample']}"},
            "e2e": {"value": rate, "unit": "events/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- parity
def tc_parity(tc, ora):
    """Track candidates of one event against the oracle's: every field, floats bit for bit."""
    if len(tc) != len(ora["tc_type"]):
        return False
    checks = [np.array_equal(tc["type"], ora["tc_type"]), np.array_equal(tc["obj"], ora["tc_obj"]),
              np.array_equal(tc["pls"], ora["tc_pls"]), np.array_equal(tc["ot"], ora["tc_ot"]),
              np.array_equal(tc["pix"], ora["tc_pix"]),
              tc["pt"].astype(np.float32).tobytes() == ora["tc_pt"].tobytes(),
              tc["score"].astype(np.float32).tobytes() == ora["tc_score"].tobytes()]
    return bool(all(checks))


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


def to_device(evs, dev):
    """One concatenated, device-resident copy of a batch's inputs (lst_batch_dev + owners)."""
    import torch
    import paper_2407_18231_gb300 as lst
    cat = lambda k: torch.from_numpy(np.ascontiguousarray(np.concatenate([getattr(e, k) for e in evs]))).to(dev)  # noqa
    x, y, z = cat("x"), cat("y"), cat("z")
    det = torch.from_numpy(np.concatenate([e.det for e in evs]).view(np.int32)).to(dev)
    pls_all = np.concatenate([e.pls for e in evs])
    pls = torch.from_numpy(pls_all.view(np.uint8) if len(pls_all) else np.zeros(80, np.uint8)).to(dev)
    hoff = torch.tensor(np.concatenate([[0], np.cumsum([e.n_hits for e in evs])]).astype(np.int32), device=dev)
    poff = torch.tensor(np.concatenate([[0], np.cumsum([e.n_pls for e in evs])]).astype(np.int32), device=dev)
    desc = lst.lst_batch_dev(len(evs), int(hoff[-1]), int(poff[-1]), max(e.n_hits for e in evs),
                             x.data_ptr(), y.data_ptr(), z.data_ptr(), det.data_ptr(), hoff.data_ptr(),
                             pls.data_ptr(), poff.data_ptr())
    return desc, (x, y, z, det, pls, hoff, poff)


OBJ_KEYS = ("n_md", "n_ls", "n_t3", "n_t5", "n_pt3", "n_pt5", "n_tc")


def time_device_batches(sess, dev_batches, n_ev, stream, flush, steps, warmup):
    """Warm-up, then `steps` device-resident batches timed with CUDA events on the
    library's stream, L2 flushed between steps; returns (ms per step, stats of the run)."""
    import torch
    for k in range(max(warmup, len(dev_batches))):
        sess.run_batch_device(dev_batches[k % len(dev_batches)][0], stream.cuda_stream)
        sess.batch_finish(n_ev, timeout_ms=120000)
    t_a = torch.cuda.Event(enable_timing=True)
    t_b = torch.cuda.Event(enable_timing=True)
    ms = 0.0
    with torch.cuda.stream(stream):
        for k in range(steps):
            flush.zero_()
            t_a.record(stream)
            sess.run_batch_device(dev_batches[k % len(dev_batches)][0], stream.cuda_stream)
            t_b.record(stream)
            sess.batch_finish(n_ev, timeout_ms=120000)
            ms += t_a.elapsed_time(t_b)
    return ms / steps, sess.stats()


def sampled_candidates(sess, dev_batch, n_ev, events, picks, stream, label, modules, pending, t5_weights=None):
    """One more run of a resident batch keeping its results: the picked events' candidates
    are queued for the CPU leg, which checks them against the oracle (with the same T5
    network when ``t5_weights`` is set); returns the track-level rates of the whole batch."""
    sess.run_batch_device(dev_batch, stream.cuda_stream)
    _, ids = sess.batch_finish(n_ev, timeout_ms=120000, keep_results=True)
    for k in picks:
        pending.append((label, int(k), sess.candidates(ids[k]), events[k], modules, t5_weights))
    tcs = [sess.candidates(i) for i in ids]
    for i in ids:
        sess.release(i)
    return track_rates(tcs, events)


def track_rates(tcs, events):
    """Efficiency, fake and duplicate rates (Sec. 3 definitions) of the events' candidates,
    with and without the pLS-only candidates."""
    import paper_2407_18231_gb300 as lst
    from paper_2407_18231_gb300 import validation as V
    c_all, c_ot = [], []
    for tc, e in zip(tcs, events):
        sel = (e.tracks["pt"] >= 0.9) & (np.abs(e.tracks["eta"]) < 2.4)
        c_all.append(V.event_counts(tc, e.sim, e.pls_sim, len(e.tracks), sel))
        c_ot.append(V.event_counts(tc[tc["type"] != lst.TC_PLS], e.sim, e.pls_sim, len(e.tracks), sel))
    a, o = V.rates(c_all), V.rates(c_ot)
    return {"efficiency": a["efficiency"], "fake_rate": a["fake_rate"], "duplicate_rate": a["duplicate_rate"],
            "without_pls_only": {"efficiency": o["efficiency"], "fake_rate": o["fake_rate"],
                                 "duplicate_rate": o["duplicate_rate"]}}


def workload_legs(local, dev, flush, stream, pending):
    """The other workloads: the tiny event per launch, the 64-event barrel batch (tuned),
    the 16-event high-occupancy batch with seeds (curvature cuts, then the learned T5
    selection), the headline batch with the learned T5 selection, and the PU200-like batch
    in the geometry with tilted inner-barrel modules; a sampled event of each is queued for
    the CPU leg's oracle check."""
    import lst_synth as S
    import paper_2407_18231_gb300 as lst
    from paper_2407_18231_gb300 import autotune
    out = {}
    # tiny: plain per-event launch, latency-bound
    gb = S.geometry(True)
    ev = S.make_event("tiny")
    sess = lst.Session(gb.modules, device=local)
    for _ in range(20):
        sess.release(sess.run_event(ev))
    lat = []
    for _ in range(300):
        t0 = time.perf_counter()
        rid = sess.run_event(ev)
        tc = sess.candidates(rid)
        lat.append(time.perf_counter() - t0)
        sess.release(rid)
    lat = np.array(lat)
    out["tiny"] = {"us_per_event_p50": float(np.median(lat) * 1e6), "us_per_event_p99": float(np.percentile(lat, 99) * 1e6),
                   "events_per_s": float(1.0 / lat.mean()), "hits": ev.n_hits, "tcs": int(len(tc)),
                   "api": "lst_run_event + lst_get_candidates (host buffers)"}
    pending.append(("tiny", 0, tc, ev, gb.modules, None))
    sess.close()
    # 64-event barrel batch (U{500..6000} tracks like tiny), launch configuration tuned on it
    evs = [S.make_event("batched", i) for i in range(64)]
    best = autotune.tune(gb.modules, evs, device=local, reps=3,
                         space={"block_size": [128, 256, 512], "blocks_per_sm": [4, 8], "ls_list_cap": [512, 1024]})
    sess = lst.Session(gb.modules, device=local, **best["best"])
    db = [to_device(evs, dev)]
    ms, st = time_device_batches(sess, db, 64, stream, flush, 10, 3)
    objs = sum(st[k] for k in OBJ_KEYS)
    sampled_candidates(sess, db[0][0], 64, evs, [7], stream, "barrel_batch64", gb.modules, pending)
    out["barrel_batch64"] = {"events_per_s": 64 / (ms * 1e-3), "objects_per_s": objs / (ms * 1e-3),
                             "ms_per_batch": ms, "objects_per_batch": {k: st[k] for k in OBJ_KEYS},
                             "mean_hits_per_event": float(np.mean([e.n_hits for e in evs])),
                             "tuning": best["best"]}
    sess.close()
    # 16-event high-occupancy batch with seeds, with the curvature cuts and with the learned
    # T5 selection (the shipped network), and the headline batch with the network
    gf = S.geometry(False)
    w = lst.load_t5_mlp()
    evs = [S.make_event("highocc", i) for i in range(16)]
    db = [to_device(evs, dev)]
    for label, weights in (("highocc_batch16", None), ("highocc_batch16_learned_t5", w)):
        sess = lst.Session(gf.modules, device=local)
        sess.set_t5_selection(weights)
        ms, st = time_device_batches(sess, db, 16, stream, flush, 10, 3)
        objs = sum(st[k] for k in OBJ_KEYS)
        phys = sampled_candidates(sess, db[0][0], 16, evs, [3], stream, label, gf.modules, pending, weights)
        out[label] = {"events_per_s": 16 / (ms * 1e-3), "objects_per_s": objs / (ms * 1e-3),
                      "ms_per_batch": ms, "objects_per_batch": {k: st[k] for k in OBJ_KEYS},
                      "mean_hits_per_event": float(np.mean([e.n_hits for e in evs])), "physics": phys,
                      "t5_selection": "curvature cuts" if weights is None else "learned (shipped network)"}
        sess.close()
    evs = make_events(32, 0)
    db = [to_device(evs, dev)]
    sess = lst.Session(gf.modules, device=local)
    sess.set_t5_selection(w)
    ms, st = time_device_batches(sess, db, 32, stream, flush, 10, 3)
    objs = sum(st[k] for k in OBJ_KEYS)
    phys = sampled_candidates(sess, db[0][0], 32, evs, [5], stream, "pu200_batch32_learned_t5", gf.modules, pending, w)
    out["pu200_batch32_learned_t5"] = {"events_per_s": 32 / (ms * 1e-3), "objects_per_s": objs / (ms * 1e-3),
                                       "ms_per_batch": ms, "objects_per_batch": {k: st[k] for k in OBJ_KEYS},
                                       "physics": phys, "t5_selection": "learned (shipped network)"}
    sess.close()
    # the headline workload in the geometry with tilted inner-barrel modules
    gt = S.geometry(False, True)
    evs = [S.make_event("pu200", i, with_pls=True, realistic=True) for i in range(32)]
    sess = lst.Session(gt.modules, device=local)
    db = [to_device(evs, dev)]
    ms, st = time_device_batches(sess, db, 32, stream, flush, 10, 3)
    objs = sum(st[k] for k in OBJ_KEYS)
    sampled_candidates(sess, db[0][0], 32, evs, [9], stream, "pu200_tilted_batch32", gt.modules, pending)
    out["pu200_tilted_batch32"] = {"events_per_s": 32 / (ms * 1e-3), "objects_per_s": objs / (ms * 1e-3),
                                   "ms_per_batch": ms, "objects_per_batch": {k: st[k] for k in OBJ_KEYS},
                                   "mean_hits_per_event": float(np.mean([e.n_hits for e in evs])),
                                   "geometry": "tilted inner-barrel rows (|z| >= 45 cm, layers 1-3)"}
    sess.close()
    # the geometry whose outer endcap rings are 2S modules (r known to half a 5 cm strip there):
    # events of 1000 tracks, since the half-strip tolerance multiplies the T3 and T5 combinatorics
    g2 = S.geometry(False, False, True)
    evs = [S.make_event("pu200", i, n_tracks=1000, with_pls=True, endcap_2s=True) for i in range(32)]
    sess = lst.Session(g2.modules, device=local)
    db = [to_device(evs, dev)]
    ms, st = time_device_batches(sess, db, 32, stream, flush, 10, 3)
    objs = sum(st[k] for k in OBJ_KEYS)
    phys = sampled_candidates(sess, db[0][0], 32, evs, [3], stream, "endcap_2s_1000trk_batch32", g2.modules, pending)
    out["endcap_2s_1000trk_batch32"] = {"events_per_s": 32 / (ms * 1e-3), "objects_per_s": objs / (ms * 1e-3),
                                        "ms_per_batch": ms, "objects_per_batch": {k: st[k] for k in OBJ_KEYS},
                                        "mean_hits_per_event": float(np.mean([e.n_hits for e in evs])),
                                        "physics": phys,
                                        "geometry": "2S endcap rings (r >= 60 cm), 1000 tracks per event"}
    sess.close()
    return out


def serving_sweep(local, rates=(1e3, 5e3, 10e3, 20e3), budgets_gb=(1, 8, 64), n_events=2200, warm=200):
    """Serving workload (U{2000..8000} tracks, 20 % noise): Poisson arrivals at each offered
    rate, under each device-memory budget, with the slots' batches queued one after another
    on the device or sharing it.  Events cycle over a pool of 64 generated events."""
    import lst_synth as S
    import paper_2407_18231_gb300 as lst
    g = S.geometry(False)
    pool = [S.make_event("serving", i) for i in range(64)]
    # per-event baseline on a context that only runs single events (sized by one pass)
    sess_e = lst.Session(g.modules, device=local)
    for e in pool[:24]:
        sess_e.release(sess_e.run_event(e))
    lat = []
    for e in pool[:24]:
        t0 = time.perf_counter()
        rid = sess_e.run_event(e)
        sess_e.candidates(rid)
        lat.append(time.perf_counter() - t0)
        sess_e.release(rid)
    sess_e.close()
    lat = np.array(lat[4:])
    sess = lst.Session(g.modules, device=local)
    for i in sess.run_batch(pool[:32]):
        sess.release(i)
    per_event = {"events_per_s": float(1.0 / lat.mean()), "p50_ms": float(np.median(lat) * 1e3),
                 "p99_ms": float(np.percentile(lat, 99) * 1e3)}
    points = []
    rng = np.random.default_rng(11)
    evs = [pool[i % len(pool)] for i in range(n_events)]
    for budget in budgets_gb:
        for share in (False, True):
            for rate in rates:
                arrival = np.cumsum(rng.exponential(1.0 / rate, n_events))
                lt, ntc, _, wall = sess.serve_replay(evs, arrival, n_slots=SERVE_SLOTS, max_batch=SERVE_BATCH,
                                                     memory_budget=int(budget) << 30, share_device=share)
                st = sess.stats()
                l = lt[warm:]
                points.append({"offered_hz": rate, "budget_gb": budget, "share_device": int(share),
                               "events_per_s": n_events / wall, "p50_ms": float(np.median(l) * 1e3),
                               "p99_ms": float(np.percentile(l, 99) * 1e3), "batches": st["served_batches"],
                               "max_batch": st["served_max_batch"],
                               "peak_device_gb": st["served_peak_bytes"] / 2 ** 30})
    sess.close()
    return {"workload": "serving: U{2000..8000} tracks, 20 % noise, no seeds", "events_per_point": n_events,
            "warmup_events": warm, "pool": "64 generated events, cycled", "slots": SERVE_SLOTS, "max_batch": SERVE_BATCH,
            "per_event": per_event, "points": points}


# Algorithmic bytes of the MD and LS stages per unit (the minimum each must move): MD =
# 20 B per hit read (x, y, z, r, index) + 32 B per MD written (two hit indices, anchor
# point, direction) + 100 B per module of geometry; LS = 32 B per MD read once + 4 B per
# connection-map entry of the batch + 16 B per LS written.
def stage_hbm(st, n_ev, n_mod, map_edges, ms_md, ms_ls, peak):
    md_bytes = 20 * st["n_hits"] + 32 * st["n_md"] + 100 * n_mod
    ls_bytes = 32 * st["n_md"] + 4 * map_edges * n_ev + 16 * st["n_ls"]
    out = {}
    for name, b, ms in (("md", md_bytes, ms_md), ("ls", ls_bytes, ms_ls)):
        gbs = b / (ms * 1e-3) / 1e9
        out[name] = {"algorithmic_bytes": int(b), "ms": ms, "achieved_gbs": gbs, "peak_gbs": peak, "frac": gbs / peak}
    return out


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
    events = make_events(B * P, 100_000 * rank, args.workload)
    batches = [events[i * B:(i + 1) * B] for i in range(P)]
    t5_weights = lst.load_t5_mlp() if args.t5 == "learned" else None
    dev_batches = [to_device(b, dev) for b in batches]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2
    tuning = {}
    if args.config:
        bs, bps, cap = (int(v) for v in args.config.split(","))
        tuning = {"block_size": bs, "blocks_per_sm": bps, "ls_list_cap": cap}
    elif args.tune:
        from paper_2407_18231_gb300 import autotune
        space = {"block_size": [128, 256], "blocks_per_sm": [4, 8, 12], "ls_list_cap": [512, 1024]}
        tuning = autotune.tune(geom.modules, events[:B], device=local, space=space, reps=5)["best"]
    sess = lst.Session(geom.modules, device=local, **tuning)
    sess.set_t5_selection(t5_weights)
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
        # sustained: the same step for --sustain seconds right after the timed steps, so
        # that the clock samples cover the device under this load
        sustained = None
        if args.sustain > 0:
            n_s, ms_s = 0, 0.0
            t_wall = time.perf_counter()
            while time.perf_counter() - t_wall < args.sustain:
                flush.zero_()
                t_start.record(stream)
                sess.run_batch_device(dev_batches[n_s % P][0], stream.cuda_stream)
                t_end.record(stream)
                sess.batch_finish(B, timeout_ms=120000)
                ms_s += t_start.elapsed_time(t_end)
                n_s += 1
            sustained = {"steps": n_s, "seconds": time.perf_counter() - t_wall, "ms_per_step": ms_s / n_s,
                         "events_per_s": n_s * B / (ms_s * 1e-3)}
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

    # ---- what was timed, kept for the oracle check of the CPU leg: sampled events of a
    # timed batch (the same resident inputs, graph and launch configuration)
    pending = []
    if args.parity:
        picks = sorted(set(np.linspace(0, B - 1, args.parity).astype(int).tolist()))
        sampled_candidates(sess, dev_batches[0][0], B, batches[0], picks, stream, "headline", geom.modules, pending,
                           t5_weights)

    # ---- end to end: host buffers through the asynchronous batch API (lst_submit_batch /
    # lst_collect_batch): one batch in flight while the next is packed and uploaded; every
    # step's H2D copy and the read-back of its candidates fall inside the timed region
    sess_h = lst.Session(geom.modules, device=local, **tuning)
    sess_h.set_t5_selection(t5_weights)
    for k in range(max(args.warmup, P) + 1):  # both slots: buffers sized, graphs captured
        t_w = sess_h.submit_batch(batches[k % P])
        for i in sess_h.collect_batch(sess_h.submit_batch(batches[(k + 1) % P])) + sess_h.collect_batch(t_w):
            sess_h.release(i)
    torch.cuda.synchronize()
    # twice the timed steps: the first upload and the last read-back overlap nothing, so a
    # short run understates the sustained rate
    e2e_steps = max(3, 2 * args.steps)
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

    # ---- LST as a seeder (Sec. 2, Table 1): PU200-like events whose seeds are 20 %
    # triplets; LST's tracks (pT5, pT3, T5) plus the seeds it leaves unlinked, quads only or
    # quads and triplets, as the recovery iteration would receive them (not timed)
    seed_evs = [S.make_event("pu200", 500 + i, with_pls=True, triplet_frac=0.2) for i in range(8)]
    seed_ids = sess_h.run_batch(seed_evs)
    cover = {"quads": [0, 0], "quads_triplets": [0, 0]}
    n_seeds = {"quads": 0, "quads_triplets": 0}
    for rid, e in zip(seed_ids, seed_evs):
        tc = sess_h.candidates(rid)
        sel = (e.tracks["pt"] >= 0.9) & (np.abs(e.tracks["eta"]) < 2.4)
        tracks = V.match_candidates(tc[tc["type"] != lst.TC_PLS], e.sim, e.pls_sim)
        for name, mode in (("quads", lst.SEEDS_QUADS), ("quads_triplets", lst.SEEDS_QUADS_TRIPLETS)):
            sd = sess_h.seeds(rid, mode)
            n_seeds[name] += len(sd)
            rec = np.zeros(len(sd), lst.TC_DTYPE)
            rec["ot"] = lst.NONE
            rec["pix"] = sd["pix"]
            found = set(tracks[tracks >= 0].tolist()) | set(V.match_candidates(rec, e.sim, e.pls_sim).tolist())
            cover[name][0] += int(sel.sum())
            cover[name][1] += int(sum(1 for k in np.nonzero(sel)[0] if int(k) in found))
        sess_h.release(rid)
    seeding = {"events": len(seed_evs), "triplet_fraction_of_seeds": 0.2,
               "seeds_per_event": {k: v / len(seed_evs) for k, v in n_seeds.items()},
               "tracks_covered": {k: v[1] / max(v[0], 1) for k, v in cover.items()},
               "covered": "simulated tracks with pT >= 0.9 GeV and |eta| < 2.4 matched (75 % rule) by an LST "
                          "pT5, pT3 or T5 or by a seed handed on"}

    # ---- per-event launch: latency of single events
    per_event = None
    if args.per_event:
        # a context that only ever runs single events (as a per-event deployment would):
        # every timed event once first, so that its buffers hold the largest of them
        sess_e = lst.Session(geom.modules, device=local, **tuning)
        sess_e.set_t5_selection(t5_weights)
        for e in events[: args.per_event]:
            sess_e.release(sess_e.run_event(e))
        lat = []
        for e in events[: args.per_event]:
            t0 = time.perf_counter()
            rid = sess_e.run_event(e)
            sess_e.candidates(rid)
            lat.append(time.perf_counter() - t0)
            sess_e.release(rid)
        sess_e.close()
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
        # the slots' batches share the device (measured faster than queueing them one after
        # another at every offered rate of the serving sweep)
        lat, ntc, _, wall = sess_h.serve_replay(evs, arrival, n_slots=SERVE_SLOTS, max_batch=SERVE_BATCH,
                                                share_device=True)
        served = {"offered_hz": rate, "events_per_s": args.served / wall, "p50_ms": float(np.percentile(lat, 50) * 1e3),
                  "p99_ms": float(np.percentile(lat, 99) * 1e3), "events": args.served, "slots": SERVE_SLOTS,
                  "max_batch": SERVE_BATCH, "share_device": 1}
    sess_h.close()

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
    prof_sess.close()
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
    # the MD and LS stages against the HBM roof, with the minimal bytes of each stage
    map_edges = int(pst["map_edges"])
    per = lambda k: acc.get(k, [1, 0.0])[1] / reps  # noqa: E731
    stages = stage_hbm(pst, B, geom.n_modules, map_edges, per("md_count") + per("md_fill"),
                       per("ls_count") + per("ls_fill"), hbm_peak)
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
                "kernel_share": share, "hbm": hbm, "md_ls_stages_hbm": stages}
    elif hbm is not None:
        roof = {"bound": "hbm", "kernel": kname, "traffic": recorded_traffic(kname), "ms_per_launch": per_launch_ms,
                "kernel_share": share, **hbm, "md_ls_stages_hbm": stages}
    kernel_times = {k: round(v[1] / reps, 4) for k, v in sorted(acc.items(), key=lambda kv: -kv[1][1])}

    # ---- the other workloads and the serving sweep (not timed with the headline)
    legs = workload_legs(local, dev, flush, stream, pending) if args.legs else None
    sweep = serving_sweep(local) if args.sweep else None

    # ---- CPU leg: the oracle on a bounded sample of the same events, and the oracle check
    # of every GPU result kept above
    cpu, parity = None, None
    if args.cpu_sample:
        cpu = cpu_oracle_rates(events, geom.modules)
        checked = check_pending(pending)
        parity = checked.pop("headline", None)
        for label, r in checked.items():
            if legs and label in legs:
                legs[label]["parity"] = r

    clocks = clk.summary()
    clocks["window"] = (f"{args.steps} timed steps + the sustained run ({sustained['seconds']:.1f} s)"
                        if sustained else f"{args.steps} timed steps")
    line = {
        "metric": METRIC, "value": value, "unit": "events/s", "n_gpus": ws, "steps": args.steps,
        "warmup": n_warm, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD if args.workload == "pu200" else "highocc_12000trk_30pct_noise_with_pixel_seeds",
                   "t5_selection": "curvature cuts" if t5_weights is None else "learned (shipped network)",
                   "events_per_step": B, "mean_hits_per_event": float(np.mean([e.n_hits for e in events])),
                   "mean_pls_per_event": float(np.mean([e.n_pls for e in events])),
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                   "mode": "batched persistent kernels, CUDA graph replay",
                   "tuning": tuning or "defaults",
                   "l2": "256 MB buffer written between timed steps; inputs rotate over "
                         f"{P} resident batches"},
        "parity": parity, "sustained": sustained,
        "e2e": e2e, "per_event": per_event, "served": served, "serving_sweep": sweep, "workloads": legs,
        "physics": physics, "seeding": seeding,
        "objects_per_step": {k: stats[k] for k in OBJ_KEYS},
        "roofline": roof, "kernel_ms_per_step": kernel_times, "cpu_baseline": cpu, "clocks": clocks,
        "gpu_launches": kernels_per_step * args.steps,
    }
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
