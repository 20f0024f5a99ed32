"""Runs HOP on one synthetic box a few times and prints each call's stage
times and counters: a small driver for profilers (ncu) and quick timing.

  python -m paper_1001_3411_gb300.run_case --n 16777216 --radius learned \
      --qpw 4 --cpr 1 --steps 2 [--path batch|eager|single] [--lists 64:16,65:65]

``--subhalos`` adds the ADAPTAHOP subhalo call (five thresholds) on the
same box after each pass.  ``--path batch`` (the default) runs the box as a one-subvolume batched pass
(the CUDA-graph path the benchmark times); ``--path eager`` runs the same
pass with its kernels enqueued one by one (the same kernels on the same
data; profilers that cannot look inside a graph with conditional nodes see
them this way); ``--path single`` calls hop_run.

The box is the NFW + 40% background generator with the 512^3 workload's
seed (``synth.nfw_box``), so any --n is a smaller copy of the benchmark box.
"""
from __future__ import annotations

import argparse
import json
import os
import sys


def main(argv=None):
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import torch

    import synth
    from paper_1001_3411_gb300 import Hop, build_library, default_params, radius_model

    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=16777216)
    ap.add_argument("--radius", default="learned",
                    help="plain, count or learned; a comma list runs each in turn on the same box")
    ap.add_argument("--lists", default="64:16",
                    help="Ndens:Nhop pairs, comma separated (65:65 is the paper's default, Table 2)")
    ap.add_argument("--qpw", type=int, default=4)
    ap.add_argument("--cpr", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--path", choices=["batch", "eager", "single"], default="batch")
    ap.add_argument("--halo", action="store_true", help="also compute the halo statistics of each pass")
    ap.add_argument("--subhalos", action="store_true",
                    help="also run hop_run with chains and lists, then ADAPTAHOP subhalos at five thresholds")
    a = ap.parse_args(argv)
    build_library()
    pos, _ = synth.nfw_box(a.n, synth.workload_seed(3))
    d = torch.from_numpy(pos).cuda()
    h = Hop(0)
    h.set_tuning(a.qpw, a.cpr)
    modes = {"plain": 0, "count": 1, "learned": 2}
    radii = a.radius.split(",")
    if "learned" in radii:
        w, m = radius_model.load()[a.qpw]
        h.hop_mlp_load(w, m)
    for radius in radii:
        for lst in a.lists.split(","):
            nd, nh = (int(x) for x in lst.split(":"))
            p = default_params(radius_mode=modes[radius], n_dens=nd, n_hop=nh)
            run(a, h, d, p, dict(radius=radius, n_dens=nd, n_hop=nh) if len(radii) > 1 or "," in a.lists else {})
    h.close()


def run(a, h, d, p, tag):
    for i in range(a.steps):
        if a.path in ("batch", "eager"):
            r = h.hop_run_batch(d, [0, a.n], [1.0], p, eager=a.path == "eager")
            ng = int(r["n_groups"][0])
        else:
            r = h.hop_run(d, p)
            ng = r["n_groups"]
        line = dict(step=i, **tag, **h.stats())
        if a.halo:
            h.hop_halo_stats(d, r["dens"], r["group"], ng)
            line["halo_ms"] = h.stats()["ms_total"]
        if a.subhalos:
            rs = h.hop_run(d, p, ld_nbr=p.n_hop, want_chain=True)
            _, n_sub = h.hop_subhalos(rs["chain"], rs["dens"], rs["nbr"], p.n_merge, p.delta_outer,
                                      [80.0, 160.0, 320.0, 640.0, 1280.0])
            st = h.stats()
            line.update(sub_ms=st["ms_total"], sub_boundaries_ms=st["ms_boundaries"],
                        sub_edges=st["n_edges"], sub_chains=st["n_chains"], n_sub=n_sub.tolist())
            del rs
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
