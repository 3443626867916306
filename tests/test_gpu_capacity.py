"""Cell arrays that grow with the tree.

A context starts with room for 2 n + 8192 cells (gases, chains and dense packings need 1.2
to 1.8 per particle).  Pairs of nearly coincident particles split only deep in the tree,
every level of the way down costing a cell, so such a state needs several times more.  The
build then raises a flag instead of writing past the arrays; the step that needed the room
and every step after it leave the state alone, and the next call that waits for results
grows the arrays, runs the held-back steps again and redoes its own work.  The results must
equal, bit for bit, those of a context whose arrays were already large enough.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ff():
    from paper_1212_2934_gb300 import _build, ff

    _build.build()
    ff.lib()
    return ff


def _close_pairs(npairs, seed=4, side=100.0, gap=1e-4):
    """npairs pairs of particles gap apart, the pairs spread over a cube."""
    rng = np.random.default_rng(seed)
    a = rng.uniform(0.0, side, (npairs, 3))
    d = rng.standard_normal((npairs, 3))
    d *= gap / np.linalg.norm(d, axis=1, keepdims=True)
    pos = np.concatenate([a, a + d]).astype(np.float32)
    g = rng.standard_normal((2 * npairs, 3))
    u = (g / np.linalg.norm(g, axis=1, keepdims=True)).astype(np.float32)
    return pos, u


def test_tree_grows_past_the_initial_cells(ff, ora):
    pos, u = _close_pairs(2000)
    n = pos.shape[0]
    ctx = ff.ff_create(ff.ff_params_default(n=n, precision="f32", count_interactions=1))
    ff.ff_set_particles(ctx, pos, u)
    ff.ff_dipolar_field(ctx, ff.FF_ALGO_BH, 0.5, True)
    info = ff.ff_tree_info(ctx)
    assert info["ncells"] > 2 * n + 8192  # the arrays had to grow
    g = ff.ff_get_tree(ctx)
    t = ora.tree(pos.astype(np.float64), u.astype(np.float64), "f32", 1)
    assert np.array_equal(g["keys"], t["keys"])
    for k in ("pbegin", "pend", "skip", "level", "leaf"):
        assert np.array_equal(g[k].astype(np.int64), t[k].astype(np.int64)), k
    assert np.array_equal(g["centre"], t["centre"])


def test_held_back_steps_run_again(ff):
    pos, u = _close_pairs(3000, seed=5)
    n = pos.shape[0]
    kw = dict(n=n, precision="f32", dip_scale=0.0, lj_eps=0.0, seed=11)
    grown = ff.ff_create(ff.ff_params_default(**kw))
    ff.ff_set_particles(grown, pos, u)
    ff.ff_dipolar_field(grown, ff.FF_ALGO_BH, 0.5, True)  # grows its arrays first
    fresh = ff.ff_create(ff.ff_params_default(**kw))
    ff.ff_set_particles(fresh, pos, u)
    ff.ff_set_particles(grown, pos, u)
    # the first step of `fresh` needs more cells than it has: it and the next two are held
    # back, then grown and run again when the state is read
    ff.ff_step(fresh, 3)
    ff.ff_step(grown, 3)
    a = ff.ff_get_particles(fresh)
    b = ff.ff_get_particles(grown)
    assert ff.ff_get_step(fresh) == ff.ff_get_step(grown) == 3
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    assert not np.array_equal(a[2], 0.0)  # the steps moved the particles
    # stepping on afterwards: still the same trajectory
    ff.ff_step(fresh, 2)
    ff.ff_step(grown, 2)
    for x, y in zip(ff.ff_get_particles(fresh), ff.ff_get_particles(grown)):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("prec", ["f64", "mixed"])
def test_growth_in_double_and_mixed_precision(ff, ora, prec):
    pos, u = _close_pairs(1500, seed=6)
    n = pos.shape[0]
    dt = np.float64 if prec == "f64" else np.float32
    ctx = ff.ff_create(ff.ff_params_default(n=n, precision=prec, count_interactions=1))
    ff.ff_set_particles(ctx, pos.astype(dt), u.astype(dt))
    ff.ff_dipolar_field(ctx, ff.FF_ALGO_BH, 0.5, True)
    assert ff.ff_tree_info(ctx)["ncells"] > 2 * n + 8192
    g = ff.ff_get_tree(ctx)
    t = ora.tree(pos.astype(np.float64), u.astype(np.float64), prec, 1)
    for k in ("pbegin", "pend", "skip", "level", "leaf"):
        assert np.array_equal(g[k].astype(np.int64), t[k].astype(np.int64)), k


def test_growth_with_batched_systems(ff):
    """Systems of close pairs next to a plain gas: the forest grows; every system's field
    equals that of a context that had room from the start."""
    from paper_1212_2934_gb300 import synth

    a, ua = _close_pairs(2500, seed=7)
    m = 4000
    side = synth.box_side_for_fraction(m, 0.05)
    b = synth.rsa_cube(m, side, 8).astype(np.float32)
    ub = synth.isotropic_moments(m, 9).astype(np.float32)
    P = np.concatenate([a, b])
    U = np.concatenate([ua, ub])
    sizes = [a.shape[0], m]
    fresh = ff.ff_create(ff.ff_params_default(n=len(P)))
    ff.ff_set_systems(fresh, sizes)
    ff.ff_set_particles(fresh, P, U)
    # the LJ force of pairs 1e-4 apart overflows single precision: dipolar terms only
    h1, f1 = ff.ff_dipolar_field(fresh, ff.FF_ALGO_BH, 0.5, False)
    assert np.isfinite(h1).all() and np.isfinite(f1).all()
    assert ff.ff_tree_info(fresh)["ncells"] > 2 * len(P) + 8192
    again = ff.ff_dipolar_field(fresh, ff.FF_ALGO_BH, 0.5, False)
    assert np.array_equal(again[0], h1) and np.array_equal(again[1], f1)
    # each system alone (its own context) gives the same bits
    off = 0
    for i, k in enumerate(sizes):
        one = ff.ff_create(ff.ff_params_default(n=k))
        ff.ff_set_particles(one, P[off:off + k], U[off:off + k])
        h, f = ff.ff_dipolar_field(one, ff.FF_ALGO_BH, 0.5, False)
        assert np.array_equal(h, h1[off:off + k]) and np.array_equal(f, f1[off:off + k]), i
        off += k
