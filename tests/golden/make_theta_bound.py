"""Writes theta_bound.json: the accuracy bound of the Barnes-Hut approximation.

Calls only the CPU oracle (and the seeded generators).  For each workload and
opening angle it compares the oracle's Barnes-Hut field and force (single
precision tree, leaf_max = 1) with its FP64 all-pairs sum, per particle as
err_k = |x_k - ref_k| / max(|ref_k|, 0.1 rms|ref|), and records the RMS and
99th percentile.  The bound at each theta is the larger of the two workloads
times 1.2 (20 % headroom); a power law a theta^p is fitted for reference.

Run from the repository root:  python tests/golden/make_theta_bound.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1212_2934_gb300 import synth  # noqa: E402

THETAS = [0.3, 0.5, 0.7]


def metrics(x, ref):
    nr = np.linalg.norm(ref, axis=1)
    den = np.maximum(nr, 0.1 * np.sqrt((nr ** 2).mean()))
    e = np.linalg.norm(x - ref, axis=1) / den
    return float(np.sqrt((e ** 2).mean())), float(np.percentile(e, 99)), float(e.max())


def main():
    work = {
        "dense4096": synth.make_ensemble("dense4096"),
        "phi05_n20000": synth.make_ensemble("phi05", n=20000),
    }
    out = {"thetas": THETAS, "headroom": 1.2, "workloads": {}, "bound": {}}
    for name, e in work.items():
        pos = e["pos"].astype(np.float32).astype(np.float64)
        u = e["u"]
        h_ap, f_ap, _ = oracle.allpairs(pos, u, 1.0, 1.0, 1.0, 2.5, True, "f32")
        rows = {}
        for th in THETAS:
            r = oracle.bh(pos, u, th, 1, "f32", 1.0, 1.0, 1.0, 2.5, True)
            rows[str(th)] = dict(h=metrics(r["h"], h_ap), f=metrics(r["f"], f_ap),
                                 interactions_per_particle=float((r["nacc"] + r["npair"]).mean()))
        out["workloads"][name] = rows
    for th in THETAS:
        b = {}
        for q in ("h", "f"):
            rms = max(out["workloads"][w][str(th)][q][0] for w in work)
            p99 = max(out["workloads"][w][str(th)][q][1] for w in work)
            b[q] = dict(rms=1.2 * rms, p99=1.2 * p99)
        out["bound"][str(th)] = b
    for q in ("h", "f"):
        ys = [out["bound"][str(t)][q]["rms"] / 1.2 for t in THETAS]
        p, loga = np.polyfit(np.log(THETAS), np.log(ys), 1)
        out["fit_rms_" + q] = dict(a=float(np.exp(loga)), p=float(p))
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "theta_bound.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1, sort_keys=True)
    print(json.dumps(out["bound"], indent=1))


if __name__ == "__main__":
    main()
