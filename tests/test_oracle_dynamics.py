"""Pins for the oracle's noise, Euler-Maruyama step and observables (Sec. 2, 4, 5).

Philox against its published known-answer vectors; Box-Muller normals by their
moments; closed forms of the noise-free recursion (exponential velocity decay,
rotation by atan(dt |w|) per step, relaxation of a moment toward the field);
the exact variance of the discrete Ornstein-Uhlenbeck recursion, which fixes
the translational and rotational noise strengths; the Langevin magnetisation
of a non-interacting ensemble (Sec. 5, Eq. Langevin); checkpoint/resume.
"""
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _state(n, seed=0):
    rng = np.random.default_rng(seed)
    u = rng.normal(size=(n, 3))
    u /= np.linalg.norm(u, axis=1)[:, None]
    return dict(pos=rng.uniform(0, 10, (n, 3)), vel=np.zeros((n, 3)), u=u, om=np.zeros((n, 3)),
                id=np.arange(n, dtype=np.int64))


def test_philox_known_answers(ora):
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        c, k, o = [[int(x, 16) for x in part.split()] for part in line.split("|")]
        assert [int(x) for x in ora.philox4x32_10(c, k)] == o


def test_normals_moments(ora):
    z = ora.normals(7, 3, np.arange(40000)).ravel()
    assert abs(z.mean()) < 4 * 1 / np.sqrt(z.size)
    assert abs(z.var() - 1) < 4 * np.sqrt(2 / z.size)
    assert abs((z ** 4).mean() - 3) < 4 * np.sqrt(96 / z.size)
    from scipy import stats

    assert stats.kstest(z, "norm").pvalue > 1e-3
    # distinct (step, id, seed) give distinct streams
    assert not np.array_equal(ora.normals(7, 3, [5]), ora.normals(7, 4, [5]))
    assert not np.array_equal(ora.normals(7, 3, [5]), ora.normals(8, 3, [5]))


def test_free_translation_closed_form(ora):
    s = _state(4)
    s["vel"][:] = [[1.0, -2.0, 0.5]] * 4
    v0, x0 = s["vel"].copy(), s["pos"].copy()
    dyn = ora.make_dyn(gamma_t=0.7, gamma_r=0.1, kT=0.0)
    n = 250
    zero = np.zeros((4, 3))
    for k in range(n):
        ora.em_step(s, zero, zero, dyn, k)
    a = 1 - 0.7 * 1e-3
    np.testing.assert_allclose(s["vel"], v0 * a ** n, rtol=1e-12)
    np.testing.assert_allclose(s["pos"], x0 + v0 * (1 - a ** n) / 0.7, rtol=1e-12)


def test_free_rotor_closed_form(ora):
    s = _state(1)
    s["u"][:] = [[1.0, 0.0, 0.0]]
    s["om"][:] = [[0.0, 0.0, 3.0]]
    dyn = ora.make_dyn(gamma_r=0.0, kT=0.0)
    n = 500
    zero = np.zeros((1, 3))
    for k in range(n):
        ora.em_step(s, zero, zero, dyn, k)
    # u + dt w x u with w perpendicular to u turns u by atan(dt |w|) about w
    ang = n * np.arctan(1e-3 * 3.0)
    np.testing.assert_allclose(s["u"][0], [np.cos(ang), np.sin(ang), 0.0], atol=1e-12)
    assert abs(np.linalg.norm(s["u"][0]) - 1) < 1e-15
    np.testing.assert_allclose(s["om"][0], [0, 0, 3.0], rtol=0, atol=0)


def test_rotational_damping_closed_form(ora):
    s = _state(1)
    s["om"][:] = [[0.3, -1.0, 2.0]]
    dyn = ora.make_dyn(gamma_r=0.9, kT=0.0)
    zero = np.zeros((1, 3))
    for k in range(300):
        ora.em_step(s, zero, zero, dyn, k)
    np.testing.assert_allclose(s["om"][0], np.array([0.3, -1.0, 2.0]) * (1 - 0.9e-3 / 0.4) ** 300,
                               rtol=1e-12)


def test_moment_relaxes_toward_field(ora):
    s = _state(1)
    s["u"][:] = [[1.0, 0.0, 0.0]]
    # overdamped (gamma_r > 2 sqrt(I |h|)): the tilt decays without overshoot
    dyn = ora.make_dyn(gamma_r=2.0, kT=0.0, h_ext=(0, 0, 2.0))
    zero = np.zeros((1, 3))
    uz = []
    for k in range(4000):
        ora.em_step(s, zero, zero, dyn, k)
        uz.append(s["u"][0, 2])
    uz = np.array(uz)
    assert uz[0] >= 0 and np.all(np.diff(uz) >= 0)
    assert uz[-1] > 0.999


@pytest.mark.slow
def test_ou_variance_fixes_noise_strengths(ora):
    n, steps = 20000, 1000
    s = _state(n, 1)
    gt, gr, kT, dt, I = 1.0, 0.5, 1.7, 1e-3, 0.4
    dyn = ora.make_dyn(gamma_t=gt, gamma_r=gr, kT=kT, seed=99)
    zero = np.zeros((n, 3))
    for k in range(steps):
        ora.em_step(s, zero, zero, dyn, k)
    # discrete OU: v' = a v + sigma xi  ->  Var v_n = sigma^2 (1 - a^2n) / (1 - a^2)
    a, sig2 = 1 - gt * dt, 2 * gt * kT * dt
    var_v = sig2 * (1 - a ** (2 * steps)) / (1 - a * a)
    ar, sig2r = 1 - gr * dt / I, 2 * gr * kT * dt / I ** 2
    var_w = sig2r * (1 - ar ** (2 * steps)) / (1 - ar * ar)
    se = np.sqrt(2.0 / (3 * n))
    assert abs(s["vel"].var() / var_v - 1) < 4 * se
    assert abs(s["om"].var() / var_w - 1) < 4 * se
    assert abs(s["vel"].mean()) < 4 * np.sqrt(var_v / (3 * n))


@pytest.mark.slow
@pytest.mark.parametrize("alpha", [1.0, 3.0])
def test_langevin_magnetisation(ora, alpha):
    # non-interacting moments in h_ext = alpha z at kT = 1: <u_z> = L(alpha) (Sec. 5)
    n = 3000
    s = _state(n, 2)
    dyn = ora.make_dyn(gamma_t=1.0, gamma_r=1.0, kT=1.0, h_ext=(0, 0, alpha), seed=5)
    zero = np.zeros((n, 3))
    acc = np.zeros(n)
    cnt = 0
    # about 2500 steps (2.5 time units) relax the isotropic start; average afterwards
    for k in range(7000):
        ora.em_step(s, zero, zero, dyn, k)
        if k >= 3000 and k % 50 == 0:
            acc += s["u"][:, 2]
            cnt += 1
    per = acc / cnt
    m, se = per.mean(), per.std(ddof=1) / np.sqrt(n)
    L = float(ora.langevin(np.array([alpha]))[0])
    assert abs(m - L) < 3 * se + 5e-3, (m, L, se)


def test_resume_is_bit_identical(ora):
    s1 = _state(50, 3)
    s1["vel"][:] = 0.1
    dyn = ora.make_dyn(gamma_t=0.3, gamma_r=0.2, kT=0.8, h_ext=(0.1, 0, 0.4), seed=11)
    h = np.tile([0.0, 0.2, 0.1], (50, 1))
    f = np.tile([0.05, 0.0, -0.1], (50, 1))
    for k in range(10):
        ora.em_step(s1, h, f, dyn, k)
    s2 = {k: v.copy() for k, v in s1.items()}
    for k in range(10, 20):
        ora.em_step(s1, h, f, dyn, k)
    for k in range(10, 20):
        ora.em_step(s2, h, f, dyn, k)
    for key in ("pos", "vel", "u", "om"):
        assert np.array_equal(s1[key], s2[key])


def test_energy_observables(ora):
    pos = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, 2.0]])
    u = np.array([[0.0, 0.0, 1.0], [0.0, 0.0, 1.0]])
    h, f, e = ora.allpairs(pos, u)
    s = dict(pos=pos, vel=np.array([[1.0, 0, 0], [0, 2.0, 0]]), u=u, om=np.array([[0, 0, 1.0], [0, 0, 0]]),
             id=np.arange(2))
    dyn = ora.make_dyn(h_ext=(0, 0, 3.0))
    E = ora.energy(s, h, e, dyn)
    assert E["e_dip"] == pytest.approx(-2 / 8)          # head to tail: -2/r^3
    assert E["e_zeeman"] == pytest.approx(-6.0)
    assert E["e_kin_t"] == pytest.approx(2.5)
    assert E["e_kin_r"] == pytest.approx(0.2)
    np.testing.assert_allclose(E["m"], [0, 0, 1.0])
    assert E["hdip_z_mean"] == pytest.approx(2 / 8)
    # side by side: +1/r^3
    pos2 = np.array([[0.0, 0.0, 0.0], [2.0, 0.0, 0.0]])
    h2, _, _ = ora.allpairs(pos2, u)
    s["pos"] = pos2
    assert ora.energy(s, h2, None, dyn)["e_dip"] == pytest.approx(1 / 8)


def test_langevin_function(ora):
    a = np.array([1e-6, 0.5, 2.0, 10.0])
    L = ora.langevin(a)
    np.testing.assert_allclose(L[1:], 1 / np.tanh(a[1:]) - 1 / a[1:], rtol=1e-14)
    assert L[0] == pytest.approx(a[0] / 3)


# ------------------------------------------- the printed angle equations (documented bias)


def test_literal_angle_step_by_hand(ora):
    """The printed reduced angle equations on one noise-free particle: u = x (theta = pi/2,
    phi = 0) in h = (0, 1, 0): the theta torque u_x h_y - u_y h_x = 1 and the phi torque
    -(u_y h_z - u_z h_y) sin phi + (u_z h_x - u_x h_z) cos phi = 0; the first step changes
    only the rates, the second moves theta by dt times the new rate."""
    s = dict(pos=np.zeros((1, 3)), vel=np.zeros((1, 3)), u=np.array([[1.0, 0, 0]]),
             om=np.zeros((1, 3)), id=np.zeros(1, dtype=np.int64))
    dt, g, inertia = 1e-3, 0.1, 0.4
    dyn = ora.make_dyn(dt=dt, gamma_r=g, inertia=inertia, kT=0.0, h_ext=(0, 1.0, 0),
                       literal=True)
    zero = np.zeros((1, 3))
    ora.em_step(s, zero, zero, dyn, 0)
    rate = dt * 1.0 / inertia
    np.testing.assert_allclose(s["om"][0], [rate, 0.0, 0.0], atol=1e-15)
    np.testing.assert_allclose(s["u"][0], [1.0, 0.0, 0.0], atol=1e-15)
    # second step: theta = pi/2 + dt * rate (the torque is now cos(theta') in x-y terms)
    ora.em_step(s, zero, zero, dyn, 1)
    th = np.pi / 2 + dt * rate
    np.testing.assert_allclose(s["u"][0], [np.sin(th), 0.0, np.cos(th)], atol=1e-14)
    tq = np.sin(np.pi / 2) * 1.0  # u_x h_y at the second step's start (u_x = sin(pi/2) = 1)
    np.testing.assert_allclose(s["om"][0, 0], rate + dt * (tq - g * rate) / inertia, rtol=1e-13)


@pytest.mark.slow
def test_literal_angles_do_not_magnetise(ora):
    """The documented bias of the printed angle equations: a field along z exerts no torque on
    theta, so a non-interacting ensemble does not magnetise (<u_z> stays near 0), where the
    vector rigid rotor gives L(alpha) (test_langevin_magnetisation)."""
    n = 2000
    s = _state(n, 3)
    dyn = ora.make_dyn(gamma_t=1.0, gamma_r=1.0, kT=1.0, h_ext=(0, 0, 3.0), seed=7, literal=True)
    zero = np.zeros((n, 3))
    acc, cnt = 0.0, 0
    for k in range(5000):
        ora.em_step(s, zero, zero, dyn, k)
        if k >= 3000 and k % 50 == 0:
            acc += s["u"][:, 2].mean()
            cnt += 1
    L3 = float(ora.langevin(np.array([3.0]))[0])
    assert abs(acc / cnt) < 0.1 < L3 - 0.5
