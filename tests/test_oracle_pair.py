"""Pins for the oracle's pair terms (Sec. 2, reduced Eqs. h_dip, f_dip and LJ).

Each check comes from outside the oracle's own formula: closed-form fields of
two dipoles, the force as minus the gradient of the textbook dipole-dipole
energy (central differences), the field being divergence- and curl-free away
from its source, Newton's third law bit for bit, and the LJ force vanishing at
sigma as the paper states.
"""
import numpy as np
import pytest

Z = np.array([0.0, 0.0, 1.0])
X = np.array([1.0, 0.0, 0.0])


@pytest.mark.parametrize("d", [1.0, 1.7, 3.25])
def test_head_to_tail_closed_form(ora, d):
    # k above j on the z axis, both moments along z: h = 2/d^3 z, f = -6/d^4 z (attraction)
    h, f = ora.pair_dipole(d * Z, Z, Z)
    np.testing.assert_allclose(h, [0, 0, 2.0 / d ** 3], rtol=1e-15, atol=1e-300)
    np.testing.assert_allclose(f, [0, 0, -6.0 / d ** 4], rtol=1e-15, atol=1e-300)


@pytest.mark.parametrize("d", [1.0, 2.0, 5.5])
def test_side_by_side_closed_form(ora, d):
    # side by side along x, both moments along z: h = -1/d^3 z, f = +3/d^4 x (repulsion)
    h, f = ora.pair_dipole(d * X, Z, Z)
    np.testing.assert_allclose(h, [0, 0, -1.0 / d ** 3], rtol=1e-15, atol=1e-300)
    np.testing.assert_allclose(f, [3.0 / d ** 4, 0, 0], rtol=1e-15, atol=1e-300)


def _pair_energy(r, uk, uj):
    # textbook dipole-dipole energy in the reduced units: (uk.uj)/r^3 - 3 (uk.r)(uj.r)/r^5
    rn = np.linalg.norm(r)
    return uk @ uj / rn ** 3 - 3.0 * (uk @ r) * (uj @ r) / rn ** 5


def test_force_is_minus_energy_gradient(ora, rng):
    for _ in range(20):
        r = rng.normal(size=3) * rng.uniform(1, 4)
        uk = rng.normal(size=3)
        uk /= np.linalg.norm(uk)
        uj = rng.normal(size=3)
        uj /= np.linalg.norm(uj)
        h, f = ora.pair_dipole(r, uk, uj)
        eps = 1e-6 * np.linalg.norm(r)
        grad = np.zeros(3)
        for a in range(3):
            dr = np.zeros(3)
            dr[a] = eps
            grad[a] = (_pair_energy(r + dr, uk, uj) - _pair_energy(r - dr, uk, uj)) / (2 * eps)
        np.testing.assert_allclose(f, -grad, rtol=1e-7, atol=1e-9 * np.abs(f).max())
        # the field is minus the derivative of the pair energy with respect to u_k
        np.testing.assert_allclose(-(uk @ h), _pair_energy(r, uk, uj), rtol=1e-13)


def test_field_divergence_and_curl_free(ora, rng):
    for _ in range(10):
        r0 = rng.normal(size=3) * 2.0
        uj = rng.normal(size=3)
        uj /= np.linalg.norm(uj)
        eps = 1e-5
        J = np.zeros((3, 3))  # J[a, b] = d h_a / d r_b
        for b in range(3):
            dr = np.zeros(3)
            dr[b] = eps
            hp, _ = ora.pair_dipole(r0 + dr, Z, uj)
            hm, _ = ora.pair_dipole(r0 - dr, Z, uj)
            J[:, b] = (hp - hm) / (2 * eps)
        scale = np.abs(J).max()
        assert abs(np.trace(J)) < 1e-7 * scale
        np.testing.assert_allclose(J, J.T, atol=1e-7 * scale)


def test_action_reaction_bit_exact(ora, rng):
    for _ in range(200):
        r = rng.normal(size=3) * rng.uniform(0.8, 30)
        uk = rng.normal(size=3)
        uj = rng.normal(size=3)
        _, fkj = ora.pair_dipole(r, uk, uj)
        _, fjk = ora.pair_dipole(-r, uj, uk)
        assert np.array_equal(fkj, -fjk)


def test_lj_force_vanishes_at_sigma_and_signs(ora):
    sigma, eps, rcut = 1.0, 1.0, 2.5
    f, _ = ora.pair_lj(sigma * X, eps, sigma, rcut)
    assert np.array_equal(f, np.zeros(3))
    f, _ = ora.pair_lj(0.9 * X, eps, sigma, rcut)
    assert f[0] > 0  # repulsive inside sigma (pushes k away from j)
    f, _ = ora.pair_lj(1.3 * X, eps, sigma, rcut)
    assert f[0] < 0  # attractive between sigma and the cut
    f, e = ora.pair_lj(2.5 * X, eps, sigma, rcut)
    assert np.array_equal(f, np.zeros(3)) and e == 0.0


def test_lj_force_is_minus_energy_gradient(ora, rng):
    for _ in range(20):
        r = rng.normal(size=3)
        r *= rng.uniform(0.85, 2.4) / np.linalg.norm(r)
        f, _ = ora.pair_lj(r, 1.3, 1.0, 2.5)
        eps = 1e-6
        g = np.zeros(3)
        for a in range(3):
            dr = np.zeros(3)
            dr[a] = eps
            g[a] = (ora.pair_lj(r + dr, 1.3, 1.0, 2.5)[1] - ora.pair_lj(r - dr, 1.3, 1.0, 2.5)[1]) / (2 * eps)
        np.testing.assert_allclose(f, -g, rtol=1e-6, atol=1e-8)
    # energy is shifted to zero at the cut and continuous there
    _, e_in = ora.pair_lj(np.nextafter(2.5, 0) * X, 1.0, 1.0, 2.5)
    assert abs(e_in) < 1e-12


def test_wall_force(ora):
    dyn = ora.make_dyn(box_lo=(0, 0, 0), box_hi=(10, 10, 10), walls=True, wall_eps=1.0)
    f, e = ora.wall(np.array([5.0, 5.0, 5.0]), dyn)
    assert np.array_equal(f, np.zeros(3)) and e == 0.0
    # the lower plane sits at -1/2: a centre at x = 0 just touches it (w = sigma_w)
    f, e = ora.wall(np.array([0.0, 5.0, 5.0]), dyn)
    assert np.array_equal(f, np.zeros(3))
    f, e = ora.wall(np.array([-0.1, 5.0, 10.05]), dyn)
    assert f[0] > 0 and f[2] < 0 and f[1] == 0 and e > 0
    # force = -dE/dx
    x0 = np.array([-0.13, 5.0, 5.0])
    d = 1e-7
    ep = ora.wall(x0 + [d, 0, 0], dyn)[1]
    em = ora.wall(x0 - [d, 0, 0], dyn)[1]
    np.testing.assert_allclose(ora.wall(x0, dyn)[0][0], -(ep - em) / (2 * d), rtol=1e-6)
