"""GPU parity: the CUDA library through its C interface against the CPU oracle.

Bars (each stated where it is checked):
  * Morton keys, sort order and tree topology: bit-exact; cell centres
    bit-exact in the tree precision.
  * Interaction counts (accepted cells, exact pairs, opened cells): bit-exact.
  * FP32 Barnes-Hut field and force: err_k <= 1e-5 with
    err_k = |x_k - ref_k| / max(|ref_k|, 0.1 rms|ref|) against the oracle's
    Barnes-Hut with the same single-precision tree (FP64 sums).
  * FP64 path: err_k <= 1e-10.
  * Barnes-Hut against FP64 all-pairs: RMS and 99th percentile within the
    theta bound measured on the oracle (tests/golden/theta_bound.json).
"""
import json
import os

import numpy as np
import pytest

from conftest import rel_err

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
TOL32 = 1e-5
TOL64 = 1e-10


@pytest.fixture(scope="module")
def ff():
    from paper_1212_2934_gb300 import _build, ff

    _build.build()
    ff.lib()
    return ff


def _system(n, seed, phi=0.05):
    from paper_1212_2934_gb300 import synth

    side = synth.box_side_for_fraction(n, phi)
    return synth.rsa_cube(n, side, seed), synth.isotropic_moments(n, seed), side


def _ctx(ff, n, prec, leaf_max=1, **kw):
    p = ff.ff_params_default(n=n, precision=prec, leaf_max=leaf_max, count_interactions=1, **kw)
    return ff.ff_create(p)


def _cast(prec, *arrs):
    dt = np.float64 if prec == "f64" else np.float32  # f32 and mixed store single
    return [np.ascontiguousarray(a, dtype=dt) for a in arrs]


@pytest.mark.parametrize("prec", ["f32", "f64", "mixed"])
@pytest.mark.parametrize("n,leaf_max", [(1, 1), (2, 1), (33, 1), (1000, 1), (5003, 1),
                                        (5003, 4), (4099, 16)])
def test_keys_and_tree_bit_exact(ff, ora, prec, n, leaf_max):
    pos, u, _ = _system(n, 11 + n)
    pos, u = _cast(prec, pos, u)
    ctx = _ctx(ff, n, prec, leaf_max)
    ff.ff_set_particles(ctx, pos, u)
    ff.ff_dipolar_field(ctx, ff.FF_ALGO_BH, 0.5, True)
    g = ff.ff_get_tree(ctx)
    t = ora.tree(pos.astype(np.float64), u.astype(np.float64), prec, leaf_max)
    assert np.array_equal(g["keys"], t["keys"])
    assert np.array_equal(g["order"].astype(np.int64), t["order"])
    for k in ("pbegin", "pend", "skip", "level", "leaf"):
        assert np.array_equal(g[k].astype(np.int64), t[k].astype(np.int64)), k
    assert np.array_equal(g["centre"], t["centre"])  # exact in the tree precision
    if prec == "mixed":
        # FP64 sums in the oracle's order, rounded once: exact
        assert np.array_equal(g["moment"], t["U"].astype(np.float32).astype(np.float64))
    else:
        np.testing.assert_allclose(g["moment"], t["U"], rtol=0, atol=(2e-5 if prec == "f32" else 1e-12) * max(1, np.abs(t["U"]).max()))
    info = g["info"]
    assert info["ncells"] == len(t["level"])
    assert np.allclose(info["root"], t["root"])


def _bh_case(ff, ora, prec, pos, u, theta, leaf_max=1, **kw):
    n = pos.shape[0]
    pos, u = _cast(prec, pos, u)
    ctx = _ctx(ff, n, prec, leaf_max, **kw)
    ff.ff_set_particles(ctx, pos, u)
    h, f = ff.ff_dipolar_field(ctx, ff.FF_ALGO_BH, theta, True)
    ref = ora.bh(pos.astype(np.float64), u.astype(np.float64), theta, leaf_max, prec,
                 kw.get("dip_scale", 1.0), kw.get("lj_eps", 1.0), kw.get("lj_sigma", 1.0),
                 kw.get("lj_rcut", 2.5), True)
    # results may not depend on the traversal group size
    
    return ctx, h, f, ref


@pytest.mark.parametrize("prec", ["f32", "f64", "mixed"])
@pytest.mark.parametrize("theta", [0.3, 0.5, 0.7])
@pytest.mark.parametrize("leaf_max", [1, 8])
@pytest.mark.parametrize("group", [1, 4, 8, 16, 32])
def test_bh_field_matches_oracle(ff, ora, prec, theta, leaf_max, group):
    if group not in (8, 32) and (theta != 0.5 or leaf_max != 1):
        pytest.skip("group sizes other than 8 and 32 are checked at theta 0.5, leaf_max 1")
    if prec == "mixed" and group not in (1, 32):
        pytest.skip("mixed precision is checked with groups 1 and 32")
    pos, u, _ = _system(6007, 21)
    ctx, h, f, ref = _bh_case(ff, ora, prec, pos, u, theta, leaf_max, traverse_group=group)
    tol = TOL64 if prec == "f64" else TOL32
    eh, ef = rel_err(h, ref["h"]), rel_err(f, ref["f"])
    assert eh.max() <= tol, eh.max()
    assert ef.max() <= tol, ef.max()
    acc, pairs, opened = ff.ff_get_counts(ctx)
    assert np.array_equal(acc, ref["nacc"])
    assert np.array_equal(pairs, ref["npair"])
    assert np.array_equal(opened, ref["nopen"])


def test_bh_dense_cube(ff, ora):
    from paper_1212_2934_gb300 import synth

    e = synth.make_ensemble("dense4096")
    for prec in ("f32", "f64"):
        ctx, h, f, ref = _bh_case(ff, ora, prec, e["pos"], e["u"], 0.5)
        tol = TOL32 if prec == "f32" else TOL64
        assert rel_err(h, ref["h"]).max() <= tol
        assert rel_err(f, ref["f"]).max() <= tol


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("n", [1, 2, 257, 3001])
def test_allpairs_matches_oracle(ff, ora, prec, n):
    pos, u, _ = _system(n, 31 + n, phi=0.1)
    pos, u = _cast(prec, pos, u)
    ctx = _ctx(ff, n, prec)
    ff.ff_set_particles(ctx, pos, u)
    h, f = ff.ff_dipolar_field(ctx, ff.FF_ALGO_AP, 0.0, True)
    rh, rf, _ = ora.allpairs(pos.astype(np.float64), u.astype(np.float64), 1.0, 1.0, 1.0, 2.5, True,
                             prec)
    tol = TOL32 if prec == "f32" else TOL64
    if n == 1:
        assert np.all(h == 0) and np.all(f == 0)
        return
    assert rel_err(h, rh).max() <= tol
    assert rel_err(f, rf).max() <= tol


def test_bh_theta0_equals_allpairs_on_gpu(ff):
    pos, u, _ = _system(2500, 41)
    ctx = _ctx(ff, 2500, "f64")
    ff.ff_set_particles(ctx, pos, u)
    hb, fb = ff.ff_dipolar_field(ctx, ff.FF_ALGO_BH, 0.0, True)
    ha, fa = ff.ff_dipolar_field(ctx, ff.FF_ALGO_AP, 0.0, True)
    assert rel_err(hb, ha).max() <= 1e-12
    assert rel_err(fb, fa).max() <= 1e-12


@pytest.mark.parametrize("theta", [0.3, 0.5, 0.7])
@pytest.mark.parametrize("work", ["dense4096", "phi05_n20000"])
def test_bh_within_theta_bound_of_allpairs(ff, ora, theta, work):
    # the workloads on which the bound was measured (tests/golden/make_theta_bound.py)
    from paper_1212_2934_gb300 import synth

    bound = json.load(open(os.path.join(GOLDEN, "theta_bound.json")))["bound"][str(theta)]
    e = synth.make_ensemble("dense4096") if work == "dense4096" else synth.make_ensemble("phi05", n=20000)
    pos32, u32 = _cast("f32", e["pos"], e["u"])
    n = pos32.shape[0]
    ctx = _ctx(ff, n, "f32")
    ff.ff_set_particles(ctx, pos32, u32)
    h, f = ff.ff_dipolar_field(ctx, ff.FF_ALGO_BH, theta, True)
    rh, rf, _ = ora.allpairs(pos32.astype(np.float64), u32.astype(np.float64), 1.0, 1.0, 1.0, 2.5,
                             True, "f32")
    for got, ref, q in ((h, rh, "h"), (f, rf, "f")):
        e_ = rel_err(got, ref)
        assert np.sqrt((e_ ** 2).mean()) <= bound[q]["rms"], q
        assert np.percentile(e_, 99) <= bound[q]["p99"], q


def test_device_buffers_match_host(ff):
    torch = pytest.importorskip("torch")
    pos, u, _ = _system(3000, 61)
    ctx = _ctx(ff, 3000, "f32")
    ff.ff_set_particles(ctx, torch.tensor(pos, dtype=torch.float32, device="cuda"),
                        torch.tensor(u, dtype=torch.float32, device="cuda"))
    hd = torch.empty((3000, 3), dtype=torch.float64, device="cuda")
    fd = torch.empty_like(hd)
    ff.ff_dipolar_field(ctx, ff.FF_ALGO_BH, 0.5, True, hd, fd)
    ff.ff_set_particles(ctx, pos.astype(np.float32), u.astype(np.float32))
    h, f = ff.ff_dipolar_field(ctx, ff.FF_ALGO_BH, 0.5, True)
    assert np.array_equal(hd.cpu().numpy(), h) and np.array_equal(fd.cpu().numpy(), f)


def test_two_dipoles_closed_form(ff):
    ctx = _ctx(ff, 2, "f64")
    pos = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, 1.5]])
    u = np.array([[0.0, 0.0, 1.0], [0.0, 0.0, 1.0]])
    ff.ff_set_particles(ctx, pos, u)
    for algo in (ff.FF_ALGO_BH, ff.FF_ALGO_AP):
        h, f = ff.ff_dipolar_field(ctx, algo, 0.5, False)
        np.testing.assert_allclose(h, [[0, 0, 2 / 1.5 ** 3]] * 2, rtol=1e-14)
        np.testing.assert_allclose(f, [[0, 0, 6 / 1.5 ** 4], [0, 0, -6 / 1.5 ** 4]], rtol=1e-14)


@pytest.mark.parametrize("prec", ["f32", "f64", "mixed"])
@pytest.mark.parametrize("leaf_max", [1, 8])
def test_plain_walk_equals_counting_walk(ff, ora, prec, leaf_max):
    """The walk without counts (the one every step runs) settles the opening rule lazily where
    the outcome cannot change a term; its field and force (LJ included) equal the counting
    walk's bit for bit at every theta, and the oracle's within the bar."""
    pos, u, _ = _system(6007, 21)
    pos, u = _cast(prec, pos, u)
    plain = ff.ff_create(ff.ff_params_default(n=len(pos), precision=prec, leaf_max=leaf_max,
                                              count_interactions=0))
    ff.ff_set_particles(plain, pos, u)
    counted = _ctx(ff, len(pos), prec, leaf_max)
    ff.ff_set_particles(counted, pos, u)
    for theta in (0.3, 0.5, 0.7):
        hp, fp = ff.ff_dipolar_field(plain, ff.FF_ALGO_BH, theta, True)
        hc, fc = ff.ff_dipolar_field(counted, ff.FF_ALGO_BH, theta, True)
        assert np.array_equal(hp, hc) and np.array_equal(fp, fc), theta
    ref = ora.bh(pos.astype(np.float64), u.astype(np.float64), 0.7, leaf_max, prec, 1.0, 1.0,
                 1.0, 2.5, True)
    tol = TOL64 if prec == "f64" else TOL32
    assert rel_err(hp, ref["h"]).max() <= tol
    assert rel_err(fp, ref["f"]).max() <= tol


def test_plain_walk_chains(ff):
    """Touching chains (every neighbour at contact, LJ bracket near zero): the plain walk still
    equals the counting walk bit for bit."""
    from paper_1212_2934_gb300 import synth

    side = synth.box_side_for_fraction(64 * 100, 0.01)
    pos, u = synth.chains_cube(100, 64, side, 5)
    pos, u = pos.astype(np.float32), u.astype(np.float32)
    plain = ff.ff_create(ff.ff_params_default(n=len(pos), precision="f32", count_interactions=0))
    counted = ff.ff_create(ff.ff_params_default(n=len(pos), precision="f32", count_interactions=1))
    for c in (plain, counted):
        ff.ff_set_particles(c, pos, u)
    hp, fp = ff.ff_dipolar_field(plain, ff.FF_ALGO_BH, 0.5, True)
    hc, fc = ff.ff_dipolar_field(counted, ff.FF_ALGO_BH, 0.5, True)
    assert np.array_equal(hp, hc) and np.array_equal(fp, fc)


@pytest.mark.parametrize("n", [3072 * 5, 3072 * 5 + 1, 100003])
def test_sort_many_tiles_with_repeated_keys(ff, ora, n):
    """Keys and the stable order (equal keys by input index) over many sort tiles, including
    an exact multiple of the tile and a ragged last tile: positions drawn with repeats from a
    small set of lattice points, so most keys occur several times.  The reference is the
    oracle's keys in input order, ordered by numpy's stable argsort."""
    from paper_1212_2934_gb300 import synth

    rng = np.random.default_rng(n)
    pts = rng.integers(0, 64, size=(max(n // 5, 1), 3)).astype(np.float64) * 1.5
    pos = pts[rng.integers(0, len(pts), size=n)].astype(np.float32)
    u = synth.isotropic_moments(n, 3).astype(np.float32)
    ctx = _ctx(ff, n, "f32")
    ff.ff_set_particles(ctx, pos, u)
    ff.ff_dipolar_field(ctx, ff.FF_ALGO_BH, 0.5, False)
    g = ff.ff_get_tree(ctx)
    keys, _ = ora.morton(pos.astype(np.float64), "f32")
    order = np.argsort(keys, kind="stable")
    assert len(np.unique(keys)) < n // 2  # the case has many repeated keys
    assert np.array_equal(g["keys"], keys[order])
    assert np.array_equal(g["order"].astype(np.int64), order)


def test_coincident_particles(ff, ora):
    pos, u, _ = _system(500, 71)
    pos[10] = pos[20]
    pos[30] = pos[20]
    for prec in ("f32", "f64"):
        ctx, h, f, ref = _bh_case(ff, ora, prec, pos, u, 0.5)
        assert np.isfinite(h).all() and np.isfinite(f).all()
        tol = TOL32 if prec == "f32" else TOL64
        assert rel_err(h, ref["h"]).max() <= tol
        g = ff.ff_get_tree(ctx)
        assert g["level"].max() == 21  # the three coincident particles share a level-21 leaf


def test_errors_reported(ff):
    ctx = _ctx(ff, 100, "f32")
    with pytest.raises(ff.FFError) as ei:
        ff.ff_step(ctx, 1)
    assert ei.value.status == ff.FF_ESTATE
    pos, u, _ = _system(100, 81)
    pos = pos.astype(np.float32)
    pos[5, 1] = np.nan
    ff.ff_set_particles(ctx, pos, u.astype(np.float32))
    with pytest.raises(ff.FFError) as ei:
        ff.ff_dipolar_field(ctx, ff.FF_ALGO_BH, 0.5, True)
    assert ei.value.status == ff.FF_ENONFINITE
    with pytest.raises(ff.FFError) as ei:
        ff.ff_step(ctx, 1)
    assert ei.value.status == ff.FF_ESTATE  # poisoned until new particles are set
    pos[5, 1] = 1.0
    ff.ff_set_particles(ctx, pos, u.astype(np.float32))
    ff.ff_dipolar_field(ctx, ff.FF_ALGO_BH, 0.5, True)
    with pytest.raises(ff.FFError):
        ff.ff_dipolar_field(ctx, ff.FF_ALGO_BH, -1.0, True)


@pytest.mark.slow
def test_full_size_sampled(ff, ora):
    """The bench workload (N = 1,048,576, phi = 0.05, FP32, theta = 0.5, leaf_max = 1) in the
    bench's launch configuration: keys bit-exact for every particle; field, force and
    interaction counts of 3000 sampled particles against the oracle's Barnes-Hut; the walk
    without counts equal to the counting walk for every particle."""
    from paper_1212_2934_gb300 import synth

    e = synth.make_ensemble("phi05")
    n = e["n"]
    pos32, u32 = _cast("f32", e["pos"], e["u"])
    side = e["side"]
    p = ff.ff_params_default(n=n, precision="f32", theta=0.5, leaf_max=1, count_interactions=1,
                             h_ext=(0, 0, 1.0), walls=1, box_lo=(0, 0, 0), box_hi=(side, side, side))
    ctx = ff.ff_create(p)
    ff.ff_set_particles(ctx, pos32, u32)
    h, f = ff.ff_dipolar_field(ctx, ff.FF_ALGO_BH, 0.5, True)
    keys, root = ora.morton(pos32.astype(np.float64), "f32")
    g = ff.ff_get_tree(ctx)
    assert np.array_equal(g["keys"], np.sort(keys))
    idx = np.random.default_rng(9).choice(n, 3000, replace=False)
    ref = ora.bh(pos32.astype(np.float64), u32.astype(np.float64), 0.5, 1, "f32", 1.0, 1.0, 1.0,
                 2.5, True, only=idx)
    assert rel_err(h[idx], ref["h"][idx]).max() <= TOL32
    assert rel_err(f[idx], ref["f"][idx]).max() <= TOL32
    acc, pairs, opened = ff.ff_get_counts(ctx)
    assert np.array_equal(acc[idx], ref["nacc"][idx])
    assert np.array_equal(pairs[idx], ref["npair"][idx])
    assert np.array_equal(opened[idx], ref["nopen"][idx])
    assert ref["ncells"] == ff.ff_tree_info(ctx)["ncells"]
    # the walk every step runs (no counts) gives the same bits for every particle
    p.count_interactions = 0
    plain = ff.ff_create(p)
    ff.ff_set_particles(plain, pos32, u32)
    hp, fp = ff.ff_dipolar_field(plain, ff.FF_ALGO_BH, 0.5, True)
    assert np.array_equal(hp, h) and np.array_equal(fp, f)
