"""Magnetisation curve of batched dilute ensembles against the Langevin function (Sec. 5,
Figs. 3-4, Eq. Langevin).

The paper compares the mean magnetisation of a dilute ferrofluid with the Langevin
function L(alpha) = coth(alpha) - 1/alpha, alpha = m mu0 H / kT, and plots the mean
dipolar field <h_dip_z> against alpha.  Here 256 independent systems (sizes log-uniform
from 1,024 to 65,536, volume fraction 0.02, applied fields 0..5 along z on a linear grid)
are advanced together in one context (one forest, one CUDA graph per step) for `steps`
steps; each system's <u_z> and <h_dip_z> are averaged over the steps after `equil`.

Standard errors: the per-system means are read every `stride` steps; the integrated
autocorrelation time of those window means is estimated from the autocorrelation function
pooled over all systems (each system's series normalised by its own variance), and each
system's standard error is sqrt(var * (1 + 2 sum rho) / windows).

  python -m paper_1212_2934_gb300.magnetisation [--steps 2000] [--equil 1000] \
      [--stride 10] [--out profiles/magnetisation_c4.md]
"""
import argparse
import math
import time

import numpy as np

from . import ff, synth


def langevin(a):
    """L(a) = coth a - 1/a (Sec. 5, Eq. Langevin); its series a/3 - a^3/45 near 0."""
    a = np.asarray(a, dtype=np.float64)
    small = np.abs(a) < 1e-3
    safe = np.where(small, 1.0, a)
    return np.where(small, a / 3.0 - a ** 3 / 45.0, 1.0 / np.tanh(safe) - 1.0 / safe)


def pooled_tau(series, max_lag=None):
    """Integrated autocorrelation time (in windows) of the rows of `series` (systems x
    windows), from the autocorrelation function averaged over rows, summed up to the first
    non-positive value."""
    x = series - series.mean(axis=1, keepdims=True)
    var = (x * x).mean(axis=1)
    ok = var > 0
    x = x[ok] / np.sqrt(var[ok])[:, None]
    w = x.shape[1]
    max_lag = max_lag or w // 3
    rho = []
    for lag in range(1, max_lag):
        r = float((x[:, :-lag] * x[:, lag:]).mean())
        if r <= 0:
            break
        rho.append(r)
    return 1.0 + 2.0 * sum(rho), len(rho)


def run(steps=2000, equil=1000, stride=10, seed=1, theta=0.5, tune=True, device=0):
    """Runs the batched ensembles; returns a dict of per-system results and run facts."""
    b = synth.batched_ensembles(256, 0.02, 5.0, seed)
    sizes = np.asarray(b["sizes"], dtype=np.int64)
    n = int(sizes.sum())
    p = ff.ff_params_default(n=n, precision="f32", theta=theta, leaf_max=1, dip_scale=0.125,
                             gamma_t=1.0, gamma_r=1.0, kT=1.0, walls=1, box_lo=(0, 0, 0),
                             box_hi=(1, 1, 1), seed=seed, device=device)
    ctx = ff.ff_create(p)
    ff.ff_set_systems(ctx, sizes, b["fields"], b["box_lo"], b["box_hi"])
    ff.ff_set_particles(ctx, b["pos"].astype(np.float32), b["u"].astype(np.float32))
    tuning = None
    if tune:
        scheds = ff.ff_schedules()
        best, ms = ff.ff_tune_schedule(ctx, reps=3)
        name = lambda i: "group %d, %d threads x %d blocks/SM" % scheds[i]
        tuning = {"chosen": name(best), "ms": {name(i): m for i, m in ms.items()}}
    ff.ff_step(ctx, equil)
    ff.ff_system_moments(ctx, reset=True)
    windows = (steps - equil) // stride
    uz = np.zeros((len(sizes), windows))
    hz = np.zeros((len(sizes), windows))
    ff.ff_synchronize(ctx)
    t0 = time.perf_counter()
    for w in range(windows):
        ff.ff_step(ctx, stride)
        sums, st = ff.ff_system_moments(ctx, reset=True)
        uz[:, w] = sums[:, 2] / (st * sizes)
        hz[:, w] = sums[:, 3] / (st * sizes)
    wall = time.perf_counter() - t0
    ff.ff_destroy(ctx)
    tau_u, lags_u = pooled_tau(uz)
    tau_h, lags_h = pooled_tau(hz)
    alpha = np.abs(b["fields"][:, 2]) / 1.0
    mu = uz.mean(axis=1)
    mh = hz.mean(axis=1)
    se_u = np.sqrt(uz.var(axis=1, ddof=1) * tau_u / windows)
    se_h = np.sqrt(hz.var(axis=1, ddof=1) * tau_h / windows)
    return dict(sizes=sizes, alpha=alpha, uz=mu, se_u=se_u, hz=mh, se_h=se_h, L=langevin(alpha),
                tau_u=tau_u, tau_h=tau_h, lags_u=lags_u, windows=windows, stride=stride,
                steps=steps, equil=equil, n=n, wall_s=wall,
                rate=n * (steps - equil) / wall, tuning=tuning, theta=theta, seed=seed)


def report(r, out="profiles/magnetisation_c4.md"):
    """Markdown summary with one row per system (sorted by alpha)."""
    dev = (r["uz"] - r["L"]) / np.where(r["se_u"] > 0, r["se_u"], np.inf)
    nz = r["alpha"] > 0
    lines = []
    lines.append("# Magnetisation of 256 batched dilute ensembles against the Langevin function")
    lines.append("")
    lines.append("Command: `python -m paper_1212_2934_gb300.magnetisation --steps %d --equil %d "
                 "--stride %d --out %s` (one GB300)." % (r["steps"], r["equil"], r["stride"], out))
    lines.append("")
    lines.append("Workload: 256 independent systems, sizes round(1024 * 64^((i+1/2)/256)) "
                 "(%d particles), hard-core gases at volume fraction 0.02 with walls on each "
                 "system's cube, isotropic initial moments, applied fields 5 i / 255 along z "
                 "(alpha = h / kT, kT = 1) assigned to the sizes by a seeded permutation; "
                 "dip_scale 1/8 (coupling constant lambda = 0.25), Gamma_t = Gamma_r = 1, "
                 "dt = 1e-3, LJ eps = sigma = 1, rcut = 2.5, Barnes-Hut theta = %.1f, FP32." %
                 (r["n"], r["theta"]))
    lines.append("")
    lines.append("Averages over steps %d..%d, read every %d steps (%d windows).  Standard errors "
                 "from the window means with the pooled integrated autocorrelation time "
                 "(%.2f windows for u_z, %.2f for h_dip_z)." %
                 (r["equil"], r["steps"], r["stride"], r["windows"], r["tau_u"], r["tau_h"]))
    lines.append("")
    lines.append("Production rate: %.3g particle-steps/s (wall clock over the production steps, "
                 "including the per-window reads of the system sums)." % r["rate"])
    if r["tuning"]:
        lines.append("")
        lines.append("Traversal schedule chosen by the autotuner: %s (ms per candidate: %s)." %
                     (r["tuning"]["chosen"], ", ".join("%s: %.3f" % (k, v)
                                                       for k, v in r["tuning"]["ms"].items())))
    lines.append("")
    lines.append("Summary over the %d systems with alpha > 0:" % int(nz.sum()))
    d = dev[nz]
    lines.append("")
    lines.append("| quantity | value |")
    lines.append("|---|---|")
    lines.append("| mean of (<u_z> - L) / SE | %.2f |" % d.mean())
    lines.append("| RMS of (<u_z> - L) / SE | %.2f |" % math.sqrt((d ** 2).mean()))
    lines.append("| fraction within 2 SE | %.3f |" % (np.abs(d) <= 2).mean())
    lines.append("| fraction within 3 SE | %.3f |" % (np.abs(d) <= 3).mean())
    lines.append("| mean of <u_z> - L | %.4g |" % (r["uz"] - r["L"])[nz].mean())
    lines.append("| largest abs(<u_z> - L) | %.4g |" % np.abs(r["uz"] - r["L"])[nz].max())
    lines.append("")
    lines.append("| system | N | alpha | <u_z> | SE | L(alpha) | (<u_z> - L) / SE | <h_dip_z> | SE |")
    lines.append("|---|---|---|---|---|---|---|---|---|")
    for i in np.argsort(r["alpha"], kind="stable"):
        lines.append("| %d | %d | %.4f | %.5f | %.5f | %.5f | %+.2f | %.5f | %.5f |" %
                     (i, r["sizes"][i], r["alpha"][i], r["uz"][i], r["se_u"][i], r["L"][i],
                      dev[i], r["hz"][i], r["se_h"][i]))
    return "\n".join(lines) + "\n"


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--equil", type=int, default=1000)
    ap.add_argument("--stride", type=int, default=10)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    r = run(a.steps, a.equil, a.stride, a.seed)
    text = report(r, a.out or "(stdout)")
    if a.out:
        with open(a.out, "w") as fh:
            fh.write(text)
    print(text)


if __name__ == "__main__":
    main()
