#!/usr/bin/env python
"""Benchmark of the GB300 HOP hot path: end-to-end particles/s at 512^3.

One step is one complete HOP pass (cell build, kNN + density, hops, chains,
boundaries, merge, results in the caller's order) over the 512^3 synthetic
NFW + 40% background box, through the batched call (one subvolume, the pass
captured once into a CUDA graph and replayed).  The headline value uses the
learned first search radius; the plain-radius path is timed beside it and
must give identical output.  Inputs are resident in HBM for `value`; `e2e`
passes host (pinned) buffers through the same C-ABI call, copies included.
The `batch` object times the 64-subvolume workload (graph pass, the same
pass enqueued kernel by kernel, and one hop_run per subvolume); the
`halo_stats` and `subhalos` objects time the halo statistics and the
ADAPTAHOP subhalo call (five thresholds) on the learned run's output.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Multi-GPU runs (torchrun) are replicas: every rank runs its own box, and
the value is all particles over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particles/s end-to-end HOP at 512^3: learned-radius vs plain GPU, same output"
N_DENS, N_HOP, N_MERGE = 64, 16, 4
DELTAS = (80.0, 200.0, 240.0)
FLOP_PER_CANDIDATE = 8          # d^2 of one candidate: 3 sub + 1 mul + 2 fma, an fma counted as 2
IDEAL_CANDIDATES = N_DENS * 6.0 / math.pi   # stencil sized to the ball


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="nfw512")
    ap.add_argument("--scale", type=int, default=None, help="override particle count (testing)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--tune-top", type=int, default=0,
                    help="autotune over the first K candidates of each policy (0: all)")
    ap.add_argument("--no-batch", action="store_true", help="skip the 64-subvolume section")
    ap.add_argument("--no-subhalos", action="store_true", help="skip the ADAPTAHOP subhalo section")
    # single-case mode: one box, a few passes, one JSON line of stage times
    # and counters per pass (the command the profiles/ summaries run under ncu)
    ap.add_argument("--case", action="store_true", help="run one case and print per-pass stage times")
    ap.add_argument("--n", type=int, default=16777216, help="--case: particles of the NFW box")
    ap.add_argument("--radius", default="learned", help="--case: plain, count or learned (comma list)")
    ap.add_argument("--lists", default="64:16", help="--case: Ndens:Nhop pairs, comma separated")
    ap.add_argument("--qpw", type=int, default=4, help="--case: queries per warp")
    ap.add_argument("--cpr", type=int, default=1, help="--case: search cells per radius")
    ap.add_argument("--buf", type=int, default=0,
                    help="--case: candidate-buffer factor (0: count-then-gather kNN kernel; 2-6: "
                         "single-scan kernel with that many Ndens of buffer per query)")
    ap.add_argument("--path", choices=["batch", "eager", "single"], default="batch",
                    help="--case: graph-captured batched pass, the same pass enqueued kernel by "
                         "kernel, or hop_run")
    ap.add_argument("--halo", action="store_true", help="--case: also time the halo statistics")
    ap.add_argument("--subhalos", action="store_true", help="--case: also time ADAPTAHOP subhalos")
    return ap.parse_args()


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except FileNotFoundError:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p:
            self.p.terminate()
            try:
                self.p.wait(5)
            except subprocess.TimeoutExpired:
                self.p.kill()

    def summary(self):
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.count(",") >= 8]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = max(float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit())
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].strip() == "Active"})
        pw = [float(r[3]) for r in rows if r[3].strip().replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": reasons, "samples": len(rows), "power_w_max": max(pw) if pw else None}


def gpu_index(local_rank: int) -> int:
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    parts = [p for p in vis.split(",") if p.strip()]
    if parts and parts[min(local_rank, len(parts) - 1)].strip().isdigit():
        return int(parts[min(local_rank, len(parts) - 1)])
    return local_rank


TRAFFIC_RECORD = os.path.join(ROOT, "profiles", "knn_traffic.json")


def source_hashes(files):
    """sha256 (first 16 hex digits) of each source file, by repo-relative path."""
    import hashlib
    out = {}
    for f in files:
        with open(os.path.join(ROOT, f), "rb") as fh:
            out[f] = hashlib.sha256(fh.read()).hexdigest()[:16]
    return out


def knn_traffic_per_particle():
    """DRAM bytes per particle of the kNN kernel from the committed ncu
    capture record, or None when any source file the kernel is compiled from
    changed since that capture."""
    try:
        rec = json.load(open(TRAFFIC_RECORD))
        now = source_hashes(rec["sources"].keys())
    except (OSError, ValueError, KeyError):
        return None, "no capture"
    if now != rec["sources"]:
        return None, "kernel sources changed since the ncu capture"
    return float(rec["traffic_bytes_per_particle"]), rec["basis"]


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# ---------------------------------------------------------------- oracle
def oracle_rate(pos, seconds: float, seed: int = 7):
    """The CPU oracle as it stands, on a bounded sample of the workload:
    brute-force kNN + density of S random particles against the whole box
    (the oracle's per-particle cost), plus its linking, boundary and merge
    stages timed per particle on the 32,768-particle Plummer set."""
    import numpy as np

    import oracle
    import synth
    n = len(pos)
    pos64 = np.ascontiguousarray(pos, dtype=np.float64)
    rng = np.random.default_rng(seed)
    threads = oracle.num_threads()
    q = rng.choice(n, size=max(threads, 4), replace=False)
    t0 = time.perf_counter()
    _, d2 = oracle.knn(pos64, N_DENS, 1.0, queries=q)
    oracle.density(d2, n)
    t_cal = (time.perf_counter() - t0) / len(q)
    s = int(max(threads, min(4096, seconds * 0.9 / max(t_cal, 1e-9))))
    s = max(threads, (s // threads) * threads)
    q = rng.choice(n, size=s, replace=False)
    t0 = time.perf_counter()
    _, d2 = oracle.knn(pos64, N_DENS, 1.0, queries=q)
    oracle.density(d2, n)
    t_knn = time.perf_counter() - t0
    small = synth.workload("plummer32k")
    nbr_s, d2_s = oracle.knn(small, N_DENS)
    dens_s = oracle.density(d2_s, len(small))
    t0 = time.perf_counter()
    _, ch = oracle.link(dens_s, nbr_s, N_HOP)
    lo, hi, sm = oracle.boundaries(ch, dens_s, nbr_s, N_MERGE, DELTAS[0])
    oracle.merge(ch, dens_s, lo, hi, sm, *DELTAS)
    t_rest = time.perf_counter() - t0
    per_particle = t_knn / s + t_rest / len(small)
    return {"value": 1.0 / per_particle, "unit": "particles/s", "cores": threads, "kind": "oracle",
            "sample": (f"fp64 brute-force kNN + M4 density of {s} random particles of the {n}-particle "
                       f"box ({t_knn:.1f} s), plus link/boundaries/merge timed per particle on the "
                       f"32,768-particle Plummer set ({t_rest * 1e3:.0f} ms)"),
            "seconds": t_knn + t_rest}


def oracle_rate_single_thread(seconds: float):
    """The oracle on one host core, on a sample of the 256^3 box: the
    per-core figure of the CPU baseline."""
    import oracle
    import synth
    pos = synth.workload("nfw256")
    before = oracle.num_threads()
    oracle.set_threads(1)
    try:
        r = oracle_rate(pos, seconds, seed=11)
    finally:
        oracle.set_threads(before)
    return {"value": r["value"], "unit": "particles/s", "cores": 1, "sample": r["sample"]}


# ------------------------------------------------------------- gb300 arm
_MODELS = None


def load_models(hop):
    """Loads the stored network of every queries-per-warp setting into the
    context (one network per setting)."""
    global _MODELS
    from paper_1001_3411_gb300 import radius_model
    if _MODELS is None:
        _MODELS = radius_model.load()
    saved = hop.get_tuning()
    for q, (params, margin) in _MODELS.items():
        hop.set_tuning(q, 1)
        hop.hop_mlp_load(params, margin)
    hop.apply_tuning(saved["qpw"], saved["cpr"], saved["buf_factor"])


def ensure_model(hop):
    """Trained weights ship with the package; if absent, train them here
    (untimed) on the 256^3 set exactly as radius_model.main() does."""
    import torch

    from paper_1001_3411_gb300 import radius_model
    import synth
    if os.path.exists(radius_model.DEFAULT_PATH):
        return "stored"
    pos, _ = synth.nfw_box(256 ** 3, synth.workload_seed(2))
    dpos = torch.from_numpy(pos).cuda()
    models = {}
    for q in (4, 8, 16):
        feat, tgt = radius_model.samples(hop, dpos, q)
        params, margin, _ = radius_model.train(hop, feat, tgt)
        models[q] = (params, margin)
    radius_model.save(radius_model.DEFAULT_PATH, models, {"train_n": 256 ** 3})
    del dpos
    torch.cuda.empty_cache()
    return "trained now"


def timed(fn, steps, dist, hop):
    """Runs fn() `steps` times between CUDA events on torch's current stream
    (the stream the library enqueues on), barrier + synchronize around."""
    import torch
    st = torch.cuda.current_stream()
    stats = []
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(steps):
        fn()
        stats.append(hop.stats())
    e1.record(st)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    if dist:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, stats


def knn_kernel_name(t):
    """The kNN kernel a (queries per warp, cells per radius, buffer factor)
    tuning runs (float32 positions)."""
    qpw, _, buf = t
    if qpw == 32:
        return "knn32_kernel"
    if buf:
        return "knn_kernel (single scan)"
    return "knn_wq_kernel (one warp per query)" if qpw == 4 else "knn_cg_kernel (grouped queries)"


def stage(st):
    keys = ("ms_sort", "ms_radius", "ms_knn", "ms_link", "ms_boundaries", "ms_merge", "ms_total")
    return {k[3:]: round(statistics.median(s[k] for s in st), 3) for k in keys}


# (queries per warp, cells per radius, buffer factor): 4 queries per warp runs
# the one-warp-per-query kernel, 8 and 16 the grouped count-then-gather
# kernel, 32 one query per lane; a buffer factor selects the single-scan
# kernel with that candidate buffer
CANDS = {"learned": [(4, 2, 0), (4, 1, 0), (4, 3, 0), (8, 1, 0), (8, 2, 0), (16, 1, 0), (4, 1, 3), (32, 1, 3)],
         "count": [(4, 2, 0), (4, 1, 0), (8, 1, 0), (16, 1, 0), (4, 1, 3), (32, 1, 3)],
         "plain": [(4, 2, 0), (8, 2, 0), (32, 1, 0), (32, 1, 3)]}


def batch_section(hop, args, dist):
    """The 64-subvolume workload (N_b log-uniform in [16^3, 128^3], NFW + 30%
    background): one graph-captured batched pass against the same pass
    enqueued kernel by kernel and against one hop_run call per subvolume."""
    import numpy as np
    import torch

    import synth
    from paper_1001_3411_gb300 import default_params
    from paper_1001_3411_gb300.shard import shard_subvolumes, subset
    pos, off = synth.workload("batch64")
    n_all = int(off[-1])
    world = dist.get_world_size() if dist else 1
    rank = dist.get_rank() if dist else 0
    # several ranks: each runs its balanced share of the subvolumes (no data
    # crosses ranks); the step time is the slowest rank's
    share = shard_subvolumes(np.diff(off), world)[rank]
    pos, off, boxes = subset(pos, off, np.ones(len(off) - 1), share)
    B = len(off) - 1
    n = int(off[-1])
    d = torch.from_numpy(pos).cuda()
    subs = [d[off[b]:off[b + 1]] for b in range(B)]
    out = {"group": torch.empty(n, dtype=torch.int32, device="cuda"),
           "dens": torch.empty(n, dtype=torch.float32, device="cuda")}
    res = {"workload": "batch64", "n_subvolumes": 64, "n_particles": n_all,
           "sizes": [int(x) for x in (np.diff(off).min(), np.median(np.diff(off)), np.diff(off).max())],
           "ranks": world, "scaling": "strong (subvolumes shared out by particle count)" if world > 1 else None}
    for name, mode in (("learned", 2), ("plain", 0)):
        p = default_params(radius_mode=mode)
        best, tr = hop.hop_autotune(d, off, boxes, p, CANDS[name], reps=2)
        t = hop.get_tuning()
        kinds = (("graph", lambda: hop.hop_run_batch(d, off, boxes, p, out=out)),)
        if name == "learned":
            kinds += (("eager", lambda: hop.hop_run_batch(d, off, boxes, p, out=out, eager=True)),
                      ("per_subvolume", lambda: [hop.hop_run(sb, p) for sb in subs]))
        r = {"tuning": [t["qpw"], t["cpr"], t["buf_factor"]],
             "autotune_ms": {str(tuple(c)): round(x["ms"], 2) for c, x in zip(CANDS[name], tr)}}
        for kind, fn in kinds:
            for _ in range(args.warmup):
                fn()
            ms, st = timed(fn, args.steps, dist, hop)
            r[kind] = {"value": n_all / (ms / args.steps * 1e-3), "ms_per_step": ms / args.steps}
            if kind == "graph":
                r[kind]["stages_ms"] = stage(st)
                r[kind]["gpu_launches_per_step"] = int(st[-1]["launches"])
                r[kind]["n_groups"] = int(st[-1]["n_groups"])
        res[name] = r
    res["speedup_graph_vs_per_subvolume"] = (res["learned"]["per_subvolume"]["ms_per_step"] /
                                            res["learned"]["graph"]["ms_per_step"])
    res["speedup_learned_vs_plain"] = (res["plain"]["graph"]["ms_per_step"] /
                                      res["learned"]["graph"]["ms_per_step"])
    del d, subs, out
    torch.cuda.empty_cache()
    return res


def run_gb300(args):
    import numpy as np
    import torch

    import synth
    from paper_1001_3411_gb300 import Hop, build_library, default_params

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl", device_id=torch.device("cuda", local))
        dist = tdist
    torch.cuda.set_device(local)
    build_library()
    hop = Hop(local)
    model_src = ensure_model(hop)
    load_models(hop)

    if args.scale:
        pos, _ = synth.nfw_box(args.scale, synth.workload_seed(3, rank))
        wl = f"nfw{args.scale}"
    else:
        pos = synth.workload(args.workload, sub=rank)
        wl = args.workload
    n = len(pos)
    off, boxes = [0, n], [1.0]
    dpos = torch.from_numpy(pos).cuda()
    out = {"group": torch.empty(n, dtype=torch.int32, device="cuda"),
           "dens": torch.empty(n, dtype=torch.float32, device="cuda")}
    params = {"learned": default_params(radius_mode=2), "plain": default_params(radius_mode=0),
              "count": default_params(radius_mode=1)}
    # the autotuner (graph replays, untimed) picks each policy's tuning;
    # output does not depend on it
    tuned, tuned_from = {}, {}
    for name in ("learned", "count", "plain"):
        cs = CANDS[name][:1] if args.no_tune else (CANDS[name][:args.tune_top] if args.tune_top > 0 else CANDS[name])
        best, tr = hop.hop_autotune(dpos, off, boxes, params[name], cs, reps=1)
        tuned[name] = tuple(cs[best])
        tuned_from[name] = [list(c) for c in cs]

    def configure(name):
        hop.apply_tuning(*tuned[name])

    def call(name, pos_in, o):
        return int(hop.hop_run_batch(pos_in, off, boxes, params[name], out=o)["n_groups"][0])

    def step(name):
        return lambda: call(name, dpos, out)

    # identical output across radius policies (untimed check): group ids,
    # densities and (below 2^29 particles, where three copies fit beside the
    # pass's own buffers) the Nhop neighbour lists, element by element
    ld_check = N_HOP if n < (1 << 29) else 0
    ref = {}
    for name in ("plain", "learned", "count"):
        configure(name)
        r = hop.hop_run_batch(dpos, off, boxes, params[name], ld_nbr=ld_check)
        ng = int(r["n_groups"][0])
        ref[name] = (r["group"], r["dens"], r["nbr"] if ld_check else None, ng)
        del r
    same = all(torch.equal(ref["plain"][0], ref[k][0]) and torch.equal(ref["plain"][1], ref[k][1])
               and (not ld_check or torch.equal(ref["plain"][2], ref[k][2])) and ref["plain"][3] == ref[k][3]
               for k in ("learned", "count"))
    group_ref = ref["plain"][0].cpu()
    n_groups_ref = ref["learned"][3]
    del ref
    torch.cuda.empty_cache()

    results = {}
    clocks = {}
    for name in ("plain", "count", "learned"):
        configure(name)
        for _ in range(args.warmup):
            step(name)()
        if name == "learned":
            with ClockSampler(gpu_index(local)) as cs:
                ms, stats = timed(step(name), args.steps, dist, hop)
            clocks = cs.summary()
        else:
            ms, stats = timed(step(name), args.steps, dist, hop)
        results[name] = (ms / args.steps, stats)

    # halo statistics (mass, centre of mass, maximum radius) of the learned
    # run's groups: HBM-bound passes, timed alone
    configure("learned")
    ng_l = call("learned", dpos, out)
    halo = None
    if ng_l > 0:
        for _ in range(2):
            hop.hop_halo_stats(dpos, out["dens"], out["group"], ng_l)
        hms, _ = timed(lambda: hop.hop_halo_stats(dpos, out["dens"], out["group"], ng_l), args.steps, dist, hop)
        hms /= args.steps
        members = int((out["group"] >= 0).sum())
        # group ids read in three passes; density and two position reads per member
        hbytes = 12 * n + 28 * members
        hbm = measured_peaks().get("hbm_gbs", 6800.0)
        halo = {"ms": hms, "n_groups": ng_l, "members": members,
                "roofline": {"bound": "hbm", "achieved": hbytes / (hms * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
                             "frac": hbytes / (hms * 1e-3) / 1e9 / hbm, "traffic": None,
                             "basis": "12 B per particle (group id, 3 passes) + 28 B per member "
                                      "(density, position twice); peak = measured copy bandwidth"}}

    # ADAPTAHOP subhalos (symmetric boundaries, one labelling per threshold)
    # on the learned run's chains and lists: timed alone
    sub = None
    if not args.no_subhalos:
        r = hop.hop_run(dpos, params["learned"], ld_nbr=N_HOP, want_chain=True)
        levels = [80.0, 160.0, 320.0, 640.0, 1280.0]
        subs, n_sub = hop.hop_subhalos(r["chain"], r["dens"], r["nbr"], 4, 80.0, levels)
        del subs
        sms, _ = timed(lambda: hop.hop_subhalos(r["chain"], r["dens"], r["nbr"], 4, 80.0, levels), args.steps,
                       dist, hop)
        sms /= args.steps
        st = hop.stats()
        ms_lv = st["ms_merge"] / len(levels)
        # per level: key + chain id per particle in the member pass and the
        # labelling pass, plus the label write
        lbytes = 28 * n
        hbm = measured_peaks().get("hbm_gbs", 6800.0)
        sub = {"ms": sms, "levels": levels, "n_sub": [int(x) for x in n_sub],
               "ms_boundaries": st["ms_boundaries"], "ms_per_level": ms_lv,
               "symmetric_boundaries": st["n_edges"], "chains": st["n_chains"],
               "roofline_level": {"bound": "hbm", "achieved": lbytes / (ms_lv * 1e-3) / 1e9, "peak": hbm,
                                  "unit": "GB/s", "frac": lbytes / (ms_lv * 1e-3) / 1e9 / hbm, "traffic": None,
                                  "basis": "28 B per particle per level (density key and chain id read twice, "
                                           "label written); the level time includes its component "
                                           "rounds, whose convergence the host reads once per four rounds"}}
        del r
        torch.cuda.empty_cache()

    # the single-volume call (hop_run, host round trips between stages) on
    # the same box and tuning, for comparison
    configure("learned")
    for _ in range(max(1, args.warmup - 1)):
        hop.hop_run(dpos, params["learned"], out=out)
    ms_single, _ = timed(lambda: hop.hop_run(dpos, params["learned"], out=out), args.steps, dist, hop)
    ms_single /= args.steps

    # end to end through the same C-ABI call with host (pinned) buffers
    hpos = torch.from_numpy(pos).pin_memory()
    hout = {"group": torch.empty(n, dtype=torch.int32).pin_memory(),
            "dens": torch.empty(n, dtype=torch.float32).pin_memory()}
    call("learned", hpos, hout)
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        call("learned", hpos, hout)
    e2e_s = (time.perf_counter() - t0) / args.steps
    if dist:
        t = torch.tensor([e2e_s], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    assert torch.equal(hout["group"], group_ref), "host-buffer run differs"
    del hpos, hout

    batch = batch_section(hop, args, dist) if not args.no_batch else None

    ms_l, st_l = results["learned"]
    ms_p, st_p = results["plain"]
    ms_c, st_c = results["count"]
    last = st_l[-1]
    knn_ms = statistics.median(s["ms_knn"] for s in st_l)
    peaks = measured_peaks()
    sm_mhz = clocks.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    fp32_peak = sms * 128 * 2 * sm_mhz * 1e6 / 1e12           # TFLOP/s at the sampled clock
    alg_flop = n * IDEAL_CANDIDATES * FLOP_PER_CANDIDATE
    achieved = alg_flop / (knn_ms * 1e-3) / 1e12
    tpp, tsrc = knn_traffic_per_particle()

    line = {
        "metric": METRIC,
        "value": n * world / (ms_l * 1e-3),
        "unit": "particles/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_l,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": wl, "n_particles": n, "n_dens": N_DENS, "n_hop": N_HOP,
                   "n_merge": N_MERGE, "deltas": list(DELTAS), "radius": "learned",
                   "path": "hop_run_batch (one subvolume), graph-captured pass",
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2": "inputs (12 B/particle, %.2f GB) larger than L2; no flush" % (n * 12 / 1e9),
                   "tuning": {k: {"queries_per_warp": v[0], "cells_per_radius": v[1], "buf_factor": v[2]}
                              for k, v in tuned.items()},
                   "tuning_candidates": tuned_from,
                   "radius_model": model_src},
        "identical_output": bool(same),
        "identical_output_compares": "group ids, densities" + (", Nhop neighbour lists" if ld_check else ""),
        "n_groups": n_groups_ref,
        "plain": {"value": n * world / (ms_p * 1e-3), "ms_per_step": ms_p, "stages_ms": stage(st_p),
                  "candidates_per_particle": st_p[-1]["candidates"] / n,
                  "retries": st_p[-1]["retries"], "searches": st_p[-1]["searches"]},
        "count": {"value": n * world / (ms_c * 1e-3), "ms_per_step": ms_c, "stages_ms": stage(st_c),
                  "candidates_per_particle": st_c[-1]["candidates"] / n,
                  "retries": st_c[-1]["retries"], "searches": st_c[-1]["searches"]},
        "learned": {"stages_ms": stage(st_l), "candidates_per_particle": last["candidates"] / n,
                    "retries": last["retries"], "searches": last["searches"]},
        "single_call_hop_run": {"value": n * world / (ms_single * 1e-3), "ms_per_step": ms_single},
        "speedup_learned_vs_plain": ms_p / ms_l,
        "speedup_learned_vs_count": ms_c / ms_l,
        "ablation": ("plain: the first radius is the mean-density Ndens-th-neighbour distance, "
                     "then certified stencil expansion; count: the closed-form radius from the 27 "
                     "stencil counts, the non-learned policy closest to the network"),
        "roofline": {"kernel": knn_kernel_name(tuned["learned"]) + " (kNN + M4 density)", "bound": "alu",
                     "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                     "frac": achieved / fp32_peak, "traffic": (tpp * n if tpp else None),
                     "traffic_basis": tsrc,
                     "basis": ("algorithmic flop = N x 64 x 6/pi candidates x 8 flop; peak = SMs x 128 "
                               "FP32 lanes x 2 x sampled median SM clock"),
                     "knn_ms": knn_ms},
        "gpu_launches": int(sum(s["launches"] for s in st_l)),
        "gpu_launches_per_step": int(last["launches"]),
        "clocks": clocks,
        "e2e": {"value": n * world / e2e_s, "unit": "particles/s",
                "h2d_bytes_per_step": n * 12, "d2h_bytes_per_step": n * 8},
        "batch": batch,
        "halo_stats": halo,
        "subhalos": sub,
    }
    if rank == 0:
        line["cpu_baseline"] = oracle_rate(pos, args.cpu_seconds)
        line["cpu_baseline"]["single_thread_nfw256"] = oracle_rate_single_thread(args.cpu_seconds / 4)
        print(json.dumps(line), flush=True)
    hop.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()


# ------------------------------------------------------- single case
def run_case(args):
    """One NFW box (the 512^3 generator and seed at --n particles), each
    radius policy and list length in turn, --steps passes each; one JSON line
    of stage times and counters per pass.  This is the command the ncu
    summaries under profiles/ were captured with: --path eager enqueues the
    batched pass kernel by kernel (ncu cannot look inside a graph with
    conditional nodes), --path batch replays the graph, --path single calls
    hop_run."""
    import torch

    import synth
    from paper_1001_3411_gb300 import Hop, build_library, default_params, radius_model
    build_library()
    pos, _ = synth.nfw_box(args.n, synth.workload_seed(3))
    d = torch.from_numpy(pos).cuda()
    h = Hop(0)
    h.apply_tuning(args.qpw, args.cpr, args.buf)
    modes = {"plain": 0, "count": 1, "learned": 2}
    radii = args.radius.split(",")
    if "learned" in radii:
        w, m = radius_model.load()[args.qpw]
        h.hop_mlp_load(w, m)
    for radius in radii:
        for lst in args.lists.split(","):
            nd, nh = (int(x) for x in lst.split(":"))
            p = default_params(radius_mode=modes[radius], n_dens=nd, n_hop=nh)
            for i in range(args.steps):
                if args.path == "single":
                    r = h.hop_run(d, p)
                    ng = int(r["n_groups"])
                else:
                    r = h.hop_run_batch(d, [0, args.n], [1.0], p, eager=args.path == "eager")
                    ng = int(r["n_groups"][0])
                line = dict(step=i, radius=radius, n_dens=nd, n_hop=nh, **h.stats())
                if args.halo:
                    h.hop_halo_stats(d, r["dens"], r["group"], ng)
                    line["halo_ms"] = h.stats()["ms_total"]
                if args.subhalos:
                    rs = h.hop_run(d, p, ld_nbr=p.n_hop, want_chain=True)
                    _, n_sub = h.hop_subhalos(rs["chain"], rs["dens"], rs["nbr"], p.n_merge, p.delta_outer,
                                              [80.0, 160.0, 320.0, 640.0, 1280.0])
                    st = h.stats()
                    line.update(sub_ms=st["ms_total"], sub_boundaries_ms=st["ms_boundaries"],
                                sub_edges=st["n_edges"], sub_chains=st["n_chains"], n_sub=n_sub.tolist())
                    del rs
                print(json.dumps(line), flush=True)
    h.close()


# --------------------------------------------------------- reference arm
def run_reference(args):
    """The oracle (the plain CPU definition of the method) as the reference
    arm: each step is a bounded sample of the same workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import synth
    if args.scale:
        pos, _ = synth.nfw_box(args.scale, synth.workload_seed(3))
        wl = f"nfw{args.scale}"
    else:
        pos = synth.workload(args.workload)
        wl = args.workload
    per_step = max(2.0, min(20.0, 150.0 / max(1, args.steps + args.warmup)))
    for i in range(args.warmup):
        oracle_rate(pos, per_step * 0.25, seed=100 + i)
    rates = [oracle_rate(pos, per_step, seed=i) for i in range(args.steps)]
    v = statistics.median(r["value"] for r in rates)
    # a step is the whole box: its time at the sampled rate
    line = {"metric": METRIC, "value": v, "unit": "particles/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": len(pos) * 1e3 / v,
            "ms_per_step_basis": "particles of the box / sampled rate (the sample itself took "
                                 f"{statistics.median(r['seconds'] for r in rates):.1f} s per step)",
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": wl, "n_particles": len(pos), "n_dens": N_DENS, "n_hop": N_HOP,
                       "n_merge": N_MERGE, "deltas": list(DELTAS)},
            "cpu_baseline": {"value": v, "unit": "particles/s", "cores": rates[0]["cores"],
                             "kind": "oracle", "sample": rates[0]["sample"]},
            "e2e": {"value": v, "unit": "particles/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    a = parse()
    if a.case:
        run_case(a)
    elif a.impl == "reference":
        run_reference(a)
    else:
        run_gb300(a)
