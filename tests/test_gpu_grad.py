"""Gradient of the dipolar energy on the GPU (ff_energy_grad) against the oracle.

E = -1/2 sum u.h (Sec. 5).  All pairs: dE/du = -h, dE/drho = -f.  Barnes-Hut:
the exact gradient with the opening decisions frozen, whose oracle is pinned
by central differences (tests/test_oracle_grad.py); it is evaluated here with
the decision tree's own centres, as the GPU places its pseudo-particles
(single-precision centres are rounded means).  Bars: FP64 1e-10,
FP32 1e-5 (err_k = |x_k - ref_k| / max(|ref_k|, 0.1 rms|ref|)).  The energy
is a sum of terms of both signs, so its bar is the same relative error of the
sum of their magnitudes, 1/2 sum |u_k| |h_k| (with |h_k| ~ |dE/du_k|).  Position
gradients are sums of forces, which cancel between touching neighbours, so in
single precision they are measured against the sum of the magnitudes of the
force terms (the oracle's fabs) where that exceeds the result.
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


def _gas(n, seed, phi=0.05):
    from paper_1212_2934_gb300 import synth

    side = synth.box_side_for_fraction(n, phi)
    return synth.rsa_cube(n, side, seed), synth.isotropic_moments(n, seed + 1)


def _energy_ok(e, e0, gu0, tol):
    return abs(e - e0) <= tol * 0.5 * np.linalg.norm(gu0, axis=1).sum()


def _grad(ff, prec, pos, u, algo, theta, **kw):
    dt = np.float64 if prec == "f64" else np.float32
    ctx = ff.ff_create(ff.ff_params_default(n=len(pos), precision=prec, **kw))
    ff.ff_set_particles(ctx, pos.astype(dt), u.astype(dt))
    return ff.ff_energy_grad(ctx, algo, theta)


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_allpairs_gradient_is_minus_field_and_force(ff, ora, prec):
    pos, u = _gas(3001, 2)
    pos = pos.astype(np.float32).astype(np.float64)
    u = u.astype(np.float32).astype(np.float64)
    e, gp, gu = _grad(ff, prec, pos, u, ff.FF_ALGO_AP, 0.0)
    e0, gp0, gu0 = ora.bh_energy_grad(pos, u, 0.0, 1, "f64")
    tol = 1e-10 if prec == "f64" else 1e-5
    assert rel_err(gu, gu0).max() <= tol
    assert rel_err(gp, gp0).max() <= tol
    assert _energy_ok(e, e0, gu0, tol)


@pytest.mark.parametrize("prec,leaf_max", [("f64", 1), ("f64", 4), ("f32", 1), ("f32", 4)])
@pytest.mark.parametrize("theta", [0.3, 0.6])
def test_bh_gradient_matches_oracle(ff, ora, prec, leaf_max, theta):
    pos, u = _gas(6007, 5)
    pos = pos.astype(np.float32).astype(np.float64)
    u = u.astype(np.float32).astype(np.float64)
    e, gp, gu = _grad(ff, prec, pos, u, ff.FF_ALGO_BH, theta, leaf_max=leaf_max, dip_scale=0.8)
    e0, gp0, gu0 = ora.bh_energy_grad(pos, u, theta, leaf_max, prec, dip_scale=0.8, lj_eps=1.0,
                                      tree_centres=True)
    tol = 1e-10 if prec == "f64" else 1e-5
    scale = None
    if prec != "f64":
        scale = ora.bh(pos, u, theta, leaf_max, prec, 0.8, 1.0, 1.0, 2.5, False)["fabs"]
    assert rel_err(gu, gu0).max() <= tol, rel_err(gu, gu0).max()
    assert rel_err(gp, gp0, scale=scale).max() <= tol, rel_err(gp, gp0, scale=scale).max()
    assert _energy_ok(e, e0, gu0, tol)


def test_bh_gradient_batched_systems(ff, ora):
    from paper_1212_2934_gb300 import synth

    sizes = [1, 700, 2300]
    pos, u = [], []
    for i, m in enumerate(sizes):
        side = synth.box_side_for_fraction(m, 0.05)
        pos.append(synth.rsa_cube(m, side, 60 + i))
        u.append(synth.isotropic_moments(m, 70 + i))
    P, U = np.concatenate(pos), np.concatenate(u)
    ctx = ff.ff_create(ff.ff_params_default(n=len(P), precision="f64"))
    ff.ff_set_systems(ctx, sizes)
    ff.ff_set_particles(ctx, P, U)
    e, gp, gu = ff.ff_energy_grad(ctx, ff.FF_ALGO_BH, 0.5)
    off, etot = 0, 0.0
    for m in sizes:
        sl = slice(off, off + m)
        if m > 1:
            e0, gp0, gu0 = ora.bh_energy_grad(P[sl], U[sl], 0.5, 1, "f64", lj_eps=1.0)
            assert rel_err(gu[sl], gu0).max() <= 1e-10
            assert rel_err(gp[sl], gp0).max() <= 1e-10
            etot += e0
        else:
            assert not gu[sl].any() and not gp[sl].any()
        off += m
    assert e == pytest.approx(etot, rel=1e-12)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_bh_gradient_regrows_its_source_lists(ff, ora, prec):
    """A small opening angle makes nearly every source an exact pair (about n per
    particle), more than the source lists' first allocation (9 chunks of 128 per
    particle) holds: the walk is redone with room for what it took.  The result
    must match the oracle, and a second call (room from the start) must give
    the same bits."""
    pos, u = _gas(2500, 9, phi=0.2)
    pos = pos.astype(np.float32).astype(np.float64)
    u = u.astype(np.float32).astype(np.float64)
    dt = np.float64 if prec == "f64" else np.float32
    ctx = ff.ff_create(ff.ff_params_default(n=len(pos), precision=prec, leaf_max=1))
    ff.ff_set_particles(ctx, pos.astype(dt), u.astype(dt))
    e, gp, gu = ff.ff_energy_grad(ctx, ff.FF_ALGO_BH, 0.05)
    e2, gp2, gu2 = ff.ff_energy_grad(ctx, ff.FF_ALGO_BH, 0.05)
    assert e == e2 and np.array_equal(gp, gp2) and np.array_equal(gu, gu2)
    e0, gp0, gu0 = ora.bh_energy_grad(pos, u, 0.05, 1, prec, lj_eps=1.0, tree_centres=True)
    tol = 1e-10 if prec == "f64" else 1e-5
    scale = None
    if prec != "f64":
        scale = ora.bh(pos, u, 0.05, 1, prec, 1.0, 1.0, 1.0, 2.5, False)["fabs"]
    assert rel_err(gu, gu0).max() <= tol, rel_err(gu, gu0).max()
    assert rel_err(gp, gp0, scale=scale).max() <= tol, rel_err(gp, gp0, scale=scale).max()
    assert _energy_ok(e, e0, gu0, tol)


def test_bh_gradient_tasks_with_many_sources(ff, ora):
    """5000 particles at theta = 0.05: every 32-particle task has about 5000 distinct
    sources, more than the shared-memory table that collects a task's sources holds, so
    the tasks' source lists are merged warp by warp instead; the result must still match."""
    pos, u = _gas(5000, 13, phi=0.2)
    e, gp, gu = _grad(ff, "f64", pos, u, ff.FF_ALGO_BH, 0.05)
    e0, gp0, gu0 = ora.bh_energy_grad(pos, u, 0.05, 1, "f64", lj_eps=1.0, tree_centres=True)
    assert rel_err(gu, gu0).max() <= 1e-10
    assert rel_err(gp, gp0).max() <= 1e-10
    assert _energy_ok(e, e0, gu0, 1e-10)


@pytest.mark.parametrize("n", [2, 3])
def test_bh_gradient_fewest_entries(ff, ora, n):
    """Two and three particles: the smallest entry lists the source sort sees."""
    from paper_1212_2934_gb300 import synth

    pos = np.array([[0.0, 0.0, 0.0], [1.5, 0.2, -0.3], [3.1, 1.0, 0.4]])[:n]
    u = synth.isotropic_moments(n, 4)
    e, gp, gu = _grad(ff, "f64", pos, u, ff.FF_ALGO_BH, 0.5)
    e0, gp0, gu0 = ora.bh_energy_grad(pos, u, 0.5, 1, "f64", lj_eps=1.0, tree_centres=True)
    assert rel_err(gu, gu0).max() <= 1e-10
    assert rel_err(gp, gp0).max() <= 1e-10
    assert _energy_ok(e, e0, gu0, 1e-10)


def test_autograd_function(ff):
    import torch

    pos, u = _gas(2000, 8)
    p = torch.tensor(pos, dtype=torch.float64, device="cuda", requires_grad=True)
    q = torch.tensor(u, dtype=torch.float64, device="cuda", requires_grad=True)
    ctx = ff.ff_create(ff.ff_params_default(n=2000, precision="f64"))
    l0 = ff.ff_profile_read(ctx)["launches"]
    e = ff.dipolar_energy(p, q, ctx, ff.FF_ALGO_BH, 0.5)
    l_forward = ff.ff_profile_read(ctx)["launches"] - l0
    (3.0 * e).backward()
    ctx2 = ff.ff_create(ff.ff_params_default(n=2000, precision="f64"))
    ff.ff_set_particles(ctx2, pos, u)
    l1 = ff.ff_profile_read(ctx2)["launches"]
    e2, gp, gu = ff.ff_energy_grad(ctx2, ff.FF_ALGO_BH, 0.5)
    l_grad = ff.ff_profile_read(ctx2)["launches"] - l1
    # the forward pass evaluates the field only; the gradient pass waits for backward
    assert l_forward < l_grad
    assert float(e) == pytest.approx(e2, rel=1e-14)
    assert np.array_equal(p.grad.cpu().numpy(), 3.0 * gp)
    assert np.array_equal(q.grad.cpu().numpy(), 3.0 * gu)


def test_gradient_rejects_bad_input(ff):
    pos, u = _gas(100, 1)
    ctx = ff.ff_create(ff.ff_params_default(n=100))
    with pytest.raises(ff.FFError):
        ff.ff_energy_grad(ctx)  # no particles yet
    ff.ff_set_particles(ctx, pos.astype(np.float32), u.astype(np.float32))
    with pytest.raises(ff.FFError):
        ff.ff_energy_grad(ctx, 7, 0.5)
    with pytest.raises(ff.FFError):
        ff.ff_energy_grad(ctx, ff.FF_ALGO_BH, -1.0)
    e, gp, gu = ff.ff_energy_grad(ctx, ff.FF_ALGO_BH, 0.5)  # still usable
    assert np.isfinite(e) and np.isfinite(gp).all()


@pytest.mark.slow
def test_full_size_gradient_sampled(ff, ora):
    """N = 262,144 at volume fraction 0.05, FP32, theta = 0.5 (the size the gradient is
    measured at): every particle's gradient against the oracle's."""
    pos, u = _gas(262144, 3)
    pos = pos.astype(np.float32).astype(np.float64)
    u = u.astype(np.float32).astype(np.float64)
    e, gp, gu = _grad(ff, "f32", pos, u, ff.FF_ALGO_BH, 0.5)
    e0, gp0, gu0 = ora.bh_energy_grad(pos, u, 0.5, 1, "f32", lj_eps=1.0, tree_centres=True)
    fabs = ora.bh(pos, u, 0.5, 1, "f32", 1.0, 1.0, 1.0, 2.5, False)["fabs"]
    assert rel_err(gu, gu0).max() <= 1e-5
    assert rel_err(gp, gp0, scale=fabs).max() <= 1e-5
    assert _energy_ok(e, e0, gu0, 1e-5)
