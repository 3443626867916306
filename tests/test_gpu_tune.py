"""Traversal schedule autotuner (ff_tune_traversal).

Every lane group gives bit-identical results (each lane makes its own
particle's decisions in depth-first order), so the tuner may only change
speed: the fields before and after tuning, and trajectories stepped with the
chosen schedule, must match an untuned context bit for bit.  The choice is the
fastest of the times it reports.
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


def _gas(n, seed=3):
    from paper_1212_2934_gb300 import synth

    side = synth.box_side_for_fraction(n, 0.05)
    return synth.rsa_cube(n, side, seed), synth.isotropic_moments(n, seed + 1), side


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_tuner_picks_the_fastest_and_changes_no_bit(ff, prec):
    pos, u, side = _gas(20000)
    dt = np.float32 if prec == "f32" else np.float64
    P, U = pos.astype(dt), u.astype(dt)
    kw = dict(n=len(P), precision=prec, walls=1, box_lo=(0, 0, 0), box_hi=(side,) * 3, seed=4)
    tuned = ff.ff_create(ff.ff_params_default(**kw))
    ff.ff_set_particles(tuned, P, U)
    h0, f0 = ff.ff_dipolar_field(tuned, ff.FF_ALGO_BH, 0.5, True)
    groups = None if prec == "f32" else [32, 1]
    best, ms = ff.ff_tune_traversal(tuned, groups, reps=2)
    assert best in (ff.TRAVERSE_GROUPS if groups is None else groups)
    assert len(ms) == (6 if groups is None else 2)
    assert all(m > 0 for m in ms.values())
    assert ms[best] == min(ms.values())
    h1, f1 = ff.ff_dipolar_field(tuned, ff.FF_ALGO_BH, 0.5, True)
    assert np.array_equal(h0, h1) and np.array_equal(f0, f1)
    # steps with the chosen schedule equal steps of a context left at one lane per walk
    ref = ff.ff_create(ff.ff_params_default(traverse_group=1, **kw))
    ff.ff_set_particles(ref, P, U)
    ff.ff_dipolar_field(ref, ff.FF_ALGO_BH, 0.5, True)  # same internal order as the tuned one
    ff.ff_step(tuned, 5)
    ff.ff_step(ref, 5)
    for a, b in zip(ff.ff_get_particles(tuned), ff.ff_get_particles(ref)):
        assert np.array_equal(a, b)


def test_tuner_on_batched_systems(ff):
    from paper_1212_2934_gb300 import synth

    sizes = [500, 3000, 12000]
    pos, u = [], []
    for i, m in enumerate(sizes):
        side = synth.box_side_for_fraction(m, 0.02)
        pos.append(synth.rsa_cube(m, side, 40 + i))
        u.append(synth.isotropic_moments(m, 50 + i))
    P = np.concatenate(pos).astype(np.float32)
    U = np.concatenate(u).astype(np.float32)
    ctx = ff.ff_create(ff.ff_params_default(n=len(P)))
    ff.ff_set_systems(ctx, sizes)
    ff.ff_set_particles(ctx, P, U)
    h0, f0 = ff.ff_dipolar_field(ctx, ff.FF_ALGO_BH, 0.5, True)
    best, ms = ff.ff_tune_traversal(ctx, [1, 4, 32], reps=1)
    assert best in (1, 4, 32) and ms[best] == min(ms.values())
    h1, f1 = ff.ff_dipolar_field(ctx, ff.FF_ALGO_BH, 0.5, True)
    assert np.array_equal(h0, h1) and np.array_equal(f0, f1)


def test_tuner_rejects_bad_input(ff):
    pos, u, _ = _gas(1000)
    ctx = ff.ff_create(ff.ff_params_default(n=1000))
    with pytest.raises(ff.FFError):
        ff.ff_tune_traversal(ctx)  # no particles yet
    ff.ff_set_particles(ctx, pos.astype(np.float32), u.astype(np.float32))
    for groups, reps in (([3], 1), ([1, 64], 1), ([1], 0), ([1], 101), ([], 1)):
        with pytest.raises(ff.FFError):
            ff.ff_tune_traversal(ctx, groups, reps=reps)
    ap = ff.ff_create(ff.ff_params_default(n=1000, algo="ap"))
    ff.ff_set_particles(ap, pos.astype(np.float32), u.astype(np.float32))
    with pytest.raises(ff.FFError):
        ff.ff_tune_traversal(ap)
    # the context stays usable after rejected calls
    best, _ = ff.ff_tune_traversal(ctx, [2], reps=1)
    assert best == 2


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_every_schedule_gives_the_same_bits(ff, prec):
    """The launch schedules (block shapes of the plain FP32 walk, lane groups) change speed
    only: fields, forces and steps are bit-identical, and the tuner keeps the fastest."""
    pos, u, side = _gas(30000, 5)
    dt = np.float32 if prec == "f32" else np.float64
    P, U = pos.astype(dt), u.astype(dt)
    kw = dict(n=len(P), precision=prec, walls=1, box_lo=(0, 0, 0), box_hi=(side,) * 3, seed=6)
    ctx = ff.ff_create(ff.ff_params_default(**kw))
    ff.ff_set_particles(ctx, P, U)
    h0, f0 = ff.ff_dipolar_field(ctx, ff.FF_ALGO_BH, 0.5, True)
    scheds = ff.ff_schedules()
    assert len(scheds) >= 8 and all(g in ff.TRAVERSE_GROUPS for g, _, _ in scheds.values())
    for i in scheds:
        ff.ff_set_schedule(ctx, i)
        h, f = ff.ff_dipolar_field(ctx, ff.FF_ALGO_BH, 0.5, True)
        assert np.array_equal(h, h0) and np.array_equal(f, f0), i
    best, ms = ff.ff_tune_schedule(ctx, reps=2)
    assert best in scheds and ms[best] == min(ms.values())
    ref = ff.ff_create(ff.ff_params_default(traverse_group=1, **kw))
    ff.ff_set_particles(ref, P, U)
    ff.ff_dipolar_field(ref, ff.FF_ALGO_BH, 0.5, True)
    ff.ff_step(ctx, 4)
    ff.ff_step(ref, 4)
    for a, b in zip(ff.ff_get_particles(ctx), ff.ff_get_particles(ref)):
        assert np.array_equal(a, b)
    with pytest.raises(ff.FFError):
        ff.ff_set_schedule(ctx, len(scheds) + 1)
