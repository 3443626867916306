"""Batched ensembles (ff_set_systems): several independent systems advanced together.

A batch is by definition the same systems run one by one, so the reference
is the oracle applied to each system separately:
  * keys, order and the forest of per-system trees bit-exact (the oracle's
    trees concatenated with particle and cell offsets);
  * per-system field and force within the single-system bars, interaction
    counts bit-exact;
  * FP64 trajectories with per-system applied fields and boxes;
  * the per-system sums of u and h_dip_z accumulated on the GPU;
  * the magnetisation of dilute, weakly coupled ensembles against the
    Langevin function (Sec. 5, Eq. Langevin) at several field amplitudes.
"""
import numpy as np
import pytest

from conftest import rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ff():
    from paper_1212_2934_gb300 import _build, ff

    _build.build()
    ff.lib()
    return ff


def _batch(sizes, phi, seed):
    from paper_1212_2934_gb300 import synth

    pos, u, sides = [], [], []
    for i, n in enumerate(sizes):
        side = synth.box_side_for_fraction(n, phi)
        pos.append(synth.rsa_cube(n, side, seed + i))
        u.append(synth.isotropic_moments(n, seed + 100 + i))
        sides.append(side)
    return pos, u, sides


SIZES = [1, 37, 500, 2048, 3001]


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_batch_forest_and_fields_match_per_system_oracle(ff, ora, prec):
    pos, u, sides = _batch(SIZES, 0.05, 7)
    dt = np.float32 if prec == "f32" else np.float64
    P = np.concatenate(pos).astype(dt)
    U = np.concatenate(u).astype(dt)
    n = P.shape[0]
    ctx = ff.ff_create(ff.ff_params_default(n=n, precision=prec, count_interactions=1))
    ff.ff_set_systems(ctx, SIZES)
    ff.ff_set_particles(ctx, P, U)
    h, f = ff.ff_dipolar_field(ctx, ff.FF_ALGO_BH, 0.5, True)
    g = ff.ff_get_tree(ctx)
    acc, pairs, opened = ff.ff_get_counts(ctx)
    keys, order, lev, leaf, pb, pe, skip = [], [], [], [], [], [], []
    p_off = c_off = 0
    tol = 1e-5 if prec == "f32" else 1e-10
    for i, m in enumerate(SIZES):
        Ps = P[p_off:p_off + m].astype(np.float64)
        Us = U[p_off:p_off + m].astype(np.float64)
        t = ora.tree(Ps, Us, prec, 1)
        keys.append(t["keys"])
        order.append(t["order"] + p_off)
        lev.append(t["level"])
        leaf.append(t["leaf"])
        pb.append(t["pbegin"] + p_off)
        pe.append(t["pend"] + p_off)
        skip.append(t["skip"] + c_off)
        r = ora.bh(Ps, Us, 0.5, 1, prec, 1.0, 1.0, 1.0, 2.5, True)
        sl = slice(p_off, p_off + m)
        if m > 1:
            assert rel_err(h[sl], r["h"]).max() <= tol
            assert rel_err(f[sl], r["f"]).max() <= tol
        else:
            assert np.all(h[sl] == 0) and np.all(f[sl] == 0)
        assert np.array_equal(acc[sl], r["nacc"]) and np.array_equal(pairs[sl], r["npair"])
        assert np.array_equal(opened[sl], r["nopen"])
        p_off += m
        c_off += len(t["level"])
    assert np.array_equal(g["keys"], np.concatenate(keys))
    assert np.array_equal(g["order"].astype(np.int64), np.concatenate(order))
    assert np.array_equal(g["level"], np.concatenate(lev))
    assert np.array_equal(g["leaf"], np.concatenate(leaf))
    assert np.array_equal(g["pbegin"], np.concatenate(pb))
    assert np.array_equal(g["pend"], np.concatenate(pe))
    assert np.array_equal(g["skip"], np.concatenate(skip))


def test_batch_trajectories_and_moments(ff, ora):
    sizes = [300, 700, 1200]
    pos, u, sides = _batch(sizes, 0.05, 11)
    fields = np.array([[0.0, 0.0, 0.5], [0.3, 0.0, 1.0], [0.0, -0.7, 2.0]])
    lo = np.zeros((3, 3))
    hi = np.array([[s, s, s] for s in sides])
    P = np.concatenate(pos)
    U = np.concatenate(u)
    n = P.shape[0]
    steps = 30
    big = max(sides)
    p = ff.ff_params_default(n=n, precision="f64", walls=1, seed=3, kT=1.0, gamma_t=0.5,
                             gamma_r=0.5, box_lo=(0, 0, 0), box_hi=(big, big, big))
    ctx = ff.ff_create(p)
    ff.ff_set_systems(ctx, sizes, fields, lo, hi)
    ff.ff_set_particles(ctx, P, U)
    ff.ff_step(ctx, steps)
    x, uu, v, w = ff.ff_get_particles(ctx)
    sums, nst = ff.ff_system_moments(ctx)
    assert nst == steps
    off = 0
    for s_, m in enumerate(sizes):
        st = dict(pos=P[off:off + m].copy(), vel=np.zeros((m, 3)), u=U[off:off + m].copy(),
                  om=np.zeros((m, 3)), id=np.arange(off, off + m, dtype=np.int64))
        dyn = ora.make_dyn(kT=1.0, gamma_t=0.5, gamma_r=0.5, h_ext=fields[s_], box_lo=lo[s_],
                           box_hi=hi[s_], walls=True, seed=3)
        acc = np.zeros(4)
        for k in range(steps):
            hd, fi, _ = ora.fields(st, "bh", theta=0.5, leaf_max=1, prec="f64", lj_eps=1.0)
            acc[:3] += st["u"].sum(axis=0)
            acc[3] += hd[:, 2].sum()
            ora.em_step(st, hd, fi, dyn, k)
        sl = slice(off, off + m)
        assert np.abs(x[sl] - st["pos"]).max() <= 1e-9 * np.abs(st["pos"]).max()
        assert rel_err(v[sl], st["vel"]).max() <= 1e-9
        assert np.abs(uu[sl] - st["u"]).max() <= 1e-9
        np.testing.assert_allclose(sums[s_], acc, rtol=1e-9, atol=1e-9 * m * steps)
        off += m


def test_batch_rejects_bad_input(ff):
    ctx = ff.ff_create(ff.ff_params_default(n=100))
    with pytest.raises(ff.FFError):
        ff.ff_set_systems(ctx, [50, 49])  # counts must add up to n
    with pytest.raises(ff.FFError):
        ff.ff_set_systems(ctx, [100, 0])
    ff.ff_set_systems(ctx, [60, 40])
    with pytest.raises(ff.FFError):
        ff.ff_dipolar_field(ctx, ff.FF_ALGO_AP, 0.0, True)  # systems must not see each other


@pytest.mark.slow
def test_langevin_magnetisation_curve(ff, ora):
    """Dilute (phi = 0.02), weakly coupled (dip_scale = 1/8, lambda = 0.25) ensembles at
    alpha = h/kT = 0, 1, 2, 3, 5: the time-averaged <u_z> follows L(alpha) (Sec. 5)."""
    alphas = np.array([0.0, 1.0, 2.0, 3.0, 5.0])
    m = 2000
    sizes = [m] * len(alphas)
    pos, u, sides = _batch(sizes, 0.02, 21)
    fields = np.stack([np.zeros_like(alphas), np.zeros_like(alphas), alphas], axis=1)
    hi = np.array([[s, s, s] for s in sides])
    P = np.concatenate(pos).astype(np.float32)
    U = np.concatenate(u).astype(np.float32)
    big = max(sides)
    p = ff.ff_params_default(n=P.shape[0], precision="f32", walls=1, kT=1.0, gamma_t=1.0,
                             gamma_r=1.0, dip_scale=0.125, seed=9, box_lo=(0, 0, 0),
                             box_hi=(big, big, big))
    ctx = ff.ff_create(p)
    ff.ff_set_systems(ctx, sizes, fields, np.zeros((len(alphas), 3)), hi)
    ff.ff_set_particles(ctx, P, U)
    ff.ff_step(ctx, 3000)  # relaxation (about 2.5 time units are needed from an isotropic start)
    ff.ff_system_moments(ctx, reset=True)
    from paper_1212_2934_gb300 import magnetisation

    windows, stride = 200, 20
    uz = np.zeros((len(alphas), windows))
    for w in range(windows):
        ff.ff_step(ctx, stride)
        sums, nst = ff.ff_system_moments(ctx, reset=True)
        uz[:, w] = sums[:, 2] / (nst * m)
    mz = uz.mean(axis=1)
    # the run's own standard error: window means with the integrated autocorrelation time
    # of the window series (pooled over the systems)
    tau, _ = magnetisation.pooled_tau(uz)
    se = np.sqrt(uz.var(axis=1, ddof=1) * tau / windows)
    L = ora.langevin(alphas)
    # 4 standard errors, plus 0.005 for the weak coupling: in the modified mean-field
    # picture <u_z> = L(alpha + chi L(alpha)), chi = 8 lambda phi = 0.02 (lambda = 1/8 in the
    # usual units), a shift below 0.002 at every alpha
    assert np.all(np.abs(mz - L) <= 4 * se + 0.005), (mz, L, se)
    assert np.all(np.diff(mz) > 0)
