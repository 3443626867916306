"""Pins for the oracle's all-pairs and Barnes-Hut sums (Sec. 3.1, 3.2).

Conservation laws of a pair interaction (total force and total angular
momentum vanish), the total energy against the textbook pair energy,
Barnes-Hut at theta = 0 against all-pairs, every other particle reached
exactly once by the traversal, error decreasing with theta, and the LJ pairs
inside the cut-off always summed exactly.
"""
import numpy as np
import pytest

from paper_1212_2934_gb300 import synth


def _system(n, seed, phi=0.1):
    side = synth.box_side_for_fraction(n, phi)
    return synth.rsa_cube(n, side, seed), synth.isotropic_moments(n, seed)


def test_two_dipoles(ora):
    pos = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, 1.5]])
    u = np.array([[0.0, 0.0, 1.0], [0.0, 0.0, 1.0]])
    h, f, _ = ora.allpairs(pos, u)
    np.testing.assert_allclose(h, [[0, 0, 2 / 1.5 ** 3]] * 2, rtol=1e-15)
    np.testing.assert_allclose(f, [[0, 0, 6 / 1.5 ** 4], [0, 0, -6 / 1.5 ** 4]], rtol=1e-15)


def test_conservation(ora):
    pos, u = _system(300, 3)
    h, f, _ = ora.allpairs(pos, u, lj_eps=1.0)
    fs = np.abs(f).sum()
    assert np.abs(f.sum(axis=0)).max() < 1e-13 * fs
    # total angular momentum: sum u x h + rho x f = 0 for rotation-invariant pair energies
    L = np.cross(u, h).sum(axis=0) + np.cross(pos, f).sum(axis=0)
    scale = np.abs(np.cross(u, h)).sum() + np.abs(np.cross(pos, f)).sum()
    assert np.abs(L).max() < 1e-12 * scale


def test_energy_matches_pair_energy(ora):
    pos, u = _system(120, 4)
    h, _, _ = ora.allpairs(pos, u)
    e_field = -0.5 * np.einsum("ij,ij->", u, h)
    e_pairs = 0.0
    for k in range(len(pos)):
        for j in range(k + 1, len(pos)):
            r = pos[k] - pos[j]
            rn = np.linalg.norm(r)
            e_pairs += u[k] @ u[j] / rn ** 3 - 3 * (u[k] @ r) * (u[j] @ r) / rn ** 5
    np.testing.assert_allclose(e_field, e_pairs, rtol=1e-12)


def test_dip_scale_and_self_skip(ora):
    pos, u = _system(50, 5)
    h1, f1, _ = ora.allpairs(pos, u, dip_scale=1.0)
    h2, f2, _ = ora.allpairs(pos, u, dip_scale=0.125)
    np.testing.assert_allclose(h2, 0.125 * h1, rtol=1e-15)
    np.testing.assert_allclose(f2, 0.125 * f1, rtol=1e-15)
    # brute force over ordered pairs with the pair routine
    hb = np.zeros_like(h1)
    for k in range(len(pos)):
        for j in range(len(pos)):
            if j != k:
                hb[k] += ora.pair_dipole(pos[k] - pos[j], u[k], u[j])[0]
    np.testing.assert_allclose(h1, hb, rtol=1e-13)


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("leaf_max", [1, 8])
def test_bh_theta0_equals_allpairs(ora, prec, leaf_max):
    pos, u = _system(700, 6)
    if prec == "f32":
        pos = pos.astype(np.float32).astype(np.float64)
    h, f, e = ora.allpairs(pos, u, lj_eps=1.0)
    r = ora.bh(pos, u, 0.0, leaf_max, prec, lj_eps=1.0)
    assert np.all(r["nacc"] == 0) and np.all(r["npair"] == len(pos) - 1)
    np.testing.assert_allclose(r["h"], h, rtol=1e-12, atol=1e-14 * np.abs(h).max())
    np.testing.assert_allclose(r["f"], f, rtol=1e-12, atol=1e-14 * np.abs(f).max())
    np.testing.assert_allclose(r["e_sr"], e, rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("theta", [0.3, 0.5, 0.7, 1.2])
@pytest.mark.parametrize("leaf_max", [1, 4])
def test_bh_reaches_every_particle_once(ora, theta, leaf_max):
    pos, u = _system(1500, 7)
    r = ora.bh(pos, u, theta, leaf_max, "f32", lj_eps=1.0)
    assert np.all(r["ncover"] + r["npair"] == len(pos) - 1)
    assert r["nacc"].sum() > 0


def test_bh_error_decreases_with_theta(ora):
    pos, u = _system(2000, 8, phi=0.05)
    h, f, _ = ora.allpairs(pos, u)
    from conftest import rel_err

    errs = []
    for th in (0.9, 0.7, 0.5, 0.3, 0.15):
        r = ora.bh(pos, u, th, 1, "f64")
        errs.append(np.sqrt((rel_err(r["h"], h) ** 2).mean()))
    assert all(a > b for a, b in zip(errs, errs[1:])), errs


def test_bh_lj_pairs_inside_cut_are_exact(ora):
    pos, u = _system(1500, 9, phi=0.2)
    _, f_ap, e_ap = ora.allpairs(pos, u, dip_scale=0.0, lj_eps=1.0, lj_rcut=2.5)
    r = ora.bh(pos, u, 0.9, 1, "f32", dip_scale=0.0, lj_eps=1.0, lj_rcut=2.5)
    np.testing.assert_allclose(r["f"], f_ap, rtol=1e-12, atol=1e-14 * np.abs(f_ap).max())
    np.testing.assert_allclose(r["e_sr"], e_ap, rtol=1e-12, atol=1e-14)


def test_bh_subset_rows(ora):
    pos, u = _system(900, 10)
    full = ora.bh(pos, u, 0.5, 1, "f32", lj_eps=1.0)
    idx = np.array([0, 17, 450, 899])
    part = ora.bh(pos, u, 0.5, 1, "f32", lj_eps=1.0, only=idx)
    np.testing.assert_array_equal(part["h"][idx], full["h"][idx])
    np.testing.assert_array_equal(part["nacc"][idx], full["nacc"][idx])


def test_allpairs_target_subset(ora, rng):
    """Rows of a target subset equal the same rows of the full sum (sources are all particles)."""
    n = 700
    pos = rng.uniform(0, 12, (n, 3))
    u = rng.normal(size=(n, 3))
    h, f, e = ora.allpairs(pos, u, lj_eps=1.0)
    idx = np.array([0, 5, 699, 123, 5])
    hs, fs, es = ora.allpairs(pos, u, lj_eps=1.0, only=idx)
    assert np.array_equal(hs[idx], h[idx]) and np.array_equal(fs[idx], f[idx])
    assert np.array_equal(es[idx], e[idx])
    rest = np.setdiff1d(np.arange(n), idx)
    assert not hs[rest].any() and not fs[rest].any()


def test_term_magnitude_sums(ora, rng):
    """habs/fabs: the sums of the magnitudes of the terms summed into h and f (the scale of
    the rounding error of a sum with cancellation)."""
    # three touching head-to-tail dipoles on a line: the middle one feels two pair forces of
    # magnitude 6 (collinear unit dipoles at unit distance: 6 / r^4) that cancel
    pos = np.array([[0.0, 0, 0], [1.0, 0, 0], [2.0, 0, 0]])
    u = np.array([[1.0, 0, 0]] * 3)
    r = ora.bh(pos, u, 0.0, 1, "f64")
    assert r["fabs"][1] == pytest.approx(12.0, rel=1e-14)
    assert np.abs(r["f"][1]).max() < 1e-12
    assert r["habs"][1] == pytest.approx(4.0, rel=1e-14)  # |h| of each neighbour: 2 / r^3
    assert np.linalg.norm(r["h"][1]) == pytest.approx(4.0, rel=1e-14)  # fields add here
    # a single pair: one term each
    r2 = ora.bh(pos[:2], u[:2], 0.0, 1, "f64", 0.5)
    np.testing.assert_allclose(r2["fabs"], np.linalg.norm(r2["f"], axis=1), rtol=1e-14)
    np.testing.assert_allclose(r2["habs"], np.linalg.norm(r2["h"], axis=1), rtol=1e-14)
    # brute force at theta = 0 with LJ, and the triangle inequality at theta = 0.5
    n = 24
    pos = synth.rsa_cube(n, 5.0, 8)
    u = rng.normal(size=(n, 3))
    u /= np.linalg.norm(u, axis=1)[:, None]
    r = ora.bh(pos, u, 0.0, 1, "f64", 0.7, 1.0, 1.0, 2.5, True)
    for k in range(n):
        hs = fs = 0.0
        for j in range(n):
            if j == k:
                continue
            h, f = ora.pair_dipole(pos[k] - pos[j], u[k], u[j])
            hs += 0.7 * np.linalg.norm(h)
            fs += 0.7 * np.linalg.norm(f)
            if np.linalg.norm(pos[k] - pos[j]) < 2.5:
                fs += np.linalg.norm(ora.pair_lj(pos[k] - pos[j])[0])
        assert r["habs"][k] == pytest.approx(hs, rel=1e-12)
        assert r["fabs"][k] == pytest.approx(fs, rel=1e-12)
    r = ora.bh(synth.rsa_cube(500, 12.0, 2), rng.normal(size=(500, 3)), 0.5, 1, "f32")
    assert np.all(r["habs"] >= np.linalg.norm(r["h"], axis=1) * (1 - 1e-12))
    assert np.all(r["fabs"] >= np.linalg.norm(r["f"], axis=1) * (1 - 1e-12))


# ------------------------------------------ dipole-position (quadrupole) cell terms


def _cluster_and_target(rng, dist, nc=6, spread=0.6):
    """A compact cluster of nc dipoles around the origin and one target at `dist`."""
    d = rng.uniform(-spread, spread, (nc, 3))
    direction = rng.normal(size=3)
    direction /= np.linalg.norm(direction)
    pos = np.vstack([d, dist * direction])
    u = rng.normal(size=(nc + 1, 3))
    u /= np.linalg.norm(u, axis=1)[:, None]
    return pos, u


def test_quadrupole_term_is_second_order(ora, rng):
    """A cluster accepted whole by a distant target: the monopole error falls like
    (size / distance)^1 relative to the field, the corrected one like (size / distance)^2."""
    pos0, u = _cluster_and_target(rng, 1.0)
    errs = {False: [], True: []}
    for dist in (40.0, 80.0, 160.0):
        pos = pos0.copy()
        pos[-1] *= dist
        exact, fexact, _ = ora.allpairs(pos, u, include_sr=False)
        for quad in (False, True):
            r = ora.bh(pos, u, 0.9, 1, "f64", include_sr=False, quad=quad)
            assert r["nacc"][-1] >= 1  # the cluster is taken through an accepted cell
            errs[quad].append(np.linalg.norm(r["h"][-1] - exact[-1]) / np.linalg.norm(exact[-1]))
    mono, quad = np.array(errs[False]), np.array(errs[True])
    # doubling the distance: relative error / 2 (monopole) and / 4 (with the correction)
    np.testing.assert_allclose(mono[:-1] / mono[1:], 2.0, rtol=0.15)
    np.testing.assert_allclose(quad[:-1] / quad[1:], 4.0, rtol=0.15)
    assert np.all(quad < 0.2 * mono)


def test_quadrupole_force_is_gradient_of_energy(ora, rng):
    """The corrected force on the target equals grad (u_k . h) of the corrected field, by central
    differences of the target's position (the cluster's cell stays accepted)."""
    pos, u = _cluster_and_target(rng, 30.0)
    r0 = ora.bh(pos, u, 0.9, 1, "f64", include_sr=False, quad=True)
    fd = np.zeros(3)
    for a in range(3):
        e = np.zeros_like(pos)
        e[-1, a] = 1e-4
        hp = ora.bh(pos + e, u, 0.9, 1, "f64", include_sr=False, quad=True)["h"][-1]
        hm = ora.bh(pos - e, u, 0.9, 1, "f64", include_sr=False, quad=True)["h"][-1]
        fd[a] = (u[-1] @ hp - u[-1] @ hm) / 2e-4
    np.testing.assert_allclose(r0["f"][-1], fd, rtol=1e-7, atol=1e-12)


def test_quadrupole_reduces_the_gas_error(ora):
    """On a gas the corrected Barnes-Hut error against all pairs is several times smaller, the
    more so the smaller theta; theta = 0 is all pairs either way."""
    side = synth.box_side_for_fraction(3000, 0.05)
    pos = synth.rsa_cube(3000, side, 4)
    u = synth.isotropic_moments(3000, 5)
    h0, _, _ = ora.allpairs(pos, u, include_sr=False)
    rms = lambda x: np.sqrt(np.mean(np.sum((x - h0) ** 2, axis=1)) / np.mean(np.sum(h0 ** 2, axis=1)))
    e = {(th, q): rms(ora.bh(pos, u, th, 1, "f64", include_sr=False, quad=q)["h"])
         for th in (0.3, 0.6) for q in (False, True)}
    # measured on this gas: 4.5x smaller at theta 0.3, 2.3x at 0.6; the gain grows as theta
    # shrinks, as for a term of higher order
    assert e[(0.3, True)] < 0.3 * e[(0.3, False)]
    assert e[(0.6, True)] < 0.5 * e[(0.6, False)]
    assert e[(0.6, False)] / e[(0.6, True)] < e[(0.3, False)] / e[(0.3, True)]
    r = ora.bh(pos, u, 0.0, 1, "f64", include_sr=False, quad=True)
    np.testing.assert_allclose(r["h"], h0, rtol=1e-12, atol=1e-12 * np.abs(h0).max())
