"""The oracle's gradient of the Barnes-Hut dipolar energy, pinned without itself.

E = -1/2 sum_k u_k . h_k (Sec. 5, e_dip) with h from the Barnes-Hut field
(Sec. 3.2).  The opening decisions are piecewise constant in the positions, so
the gradient is that of the smooth energy with the decisions frozen:
  * theta = 0 (every pair exact): dE/du = -h and dE/drho = -f_dip of the
    all-pairs sum (force = -dE/dx);
  * E equals -1/2 sum u.h of the oracle's own Barnes-Hut field;
  * central differences of E in the moments (E is quadratic in u: exact up to
    rounding) and in the positions with the decisions kept from the
    unperturbed configuration (O(h^2));
  * multi-particle leaves, single-precision decisions and dip_scale.
"""
import numpy as np
import pytest

from paper_1212_2934_gb300 import synth


def _gas(n, seed, phi=0.05):
    side = synth.box_side_for_fraction(n, phi)
    pos = synth.rsa_cube(n, side, seed)
    u = synth.isotropic_moments(n, seed + 1)
    return pos, u


def test_theta0_is_minus_field_and_force(ora):
    pos, u = _gas(400, 3)
    h, f, _ = ora.allpairs(pos, u, include_sr=False)
    e, gp, gu = ora.bh_energy_grad(pos, u, 0.0, 1, "f64")
    np.testing.assert_allclose(gu, -h, rtol=1e-12, atol=1e-12 * np.abs(h).max())
    np.testing.assert_allclose(gp, -f, rtol=1e-11, atol=1e-11 * np.abs(f).max())
    assert e == pytest.approx(-0.5 * np.sum(u * h), rel=1e-12)


@pytest.mark.parametrize("prec,leaf_max", [("f64", 1), ("f64", 4), ("f32", 1)])
def test_energy_is_that_of_the_bh_field(ora, prec, leaf_max):
    pos, u = _gas(900, 5)
    if prec == "f32":
        pos = pos.astype(np.float32).astype(np.float64)
    r = ora.bh(pos, u, 0.5, leaf_max, prec, 0.7, 1.0, 1.0, 2.5, False)
    e, gp, gu = ora.bh_energy_grad(pos, u, 0.5, leaf_max, prec, dip_scale=0.7, lj_eps=1.0)
    # a single-precision tree places its pseudo-particles at the rounded centres; the energy
    # being differentiated uses the exact means (the smooth function), one rounding apart
    assert e == pytest.approx(-0.5 * np.sum(u * r["h"]), rel=1e-12 if prec == "f64" else 1e-6)
    # with the tree's own centres the energy is the field's exactly (same sources, same order
    # of the pair kernel), and the gradient moves by rounding only
    e1, gp1, gu1 = ora.bh_energy_grad(pos, u, 0.5, leaf_max, prec, dip_scale=0.7, lj_eps=1.0,
                                      tree_centres=True)
    assert e1 == pytest.approx(-0.5 * np.sum(u * r["h"]), rel=1e-13)
    tol = 1e-12 if prec == "f64" else 1e-4
    assert np.abs(gu1 - gu).max() <= tol * np.abs(gu).max()
    assert np.abs(gp1 - gp).max() <= tol * np.abs(gp).max()
    # at theta > 0 the gradient is not simply -h: the reverse sums matter
    assert np.abs(gu + r["h"]).max() > 1e-6 * np.abs(r["h"]).max()


@pytest.mark.parametrize("prec,leaf_max,ds", [("f64", 1, 1.0), ("f64", 4, 1.0), ("f32", 1, 0.125)])
def test_central_differences(ora, prec, leaf_max, ds):
    pos, u = _gas(700, 9)
    if prec == "f32":
        pos = pos.astype(np.float32).astype(np.float64)
    kw = dict(dip_scale=ds, lj_eps=1.0)
    e0, gp, gu = ora.bh_energy_grad(pos, u, 0.5, leaf_max, prec, **kw)
    rng = np.random.default_rng(4)
    picks = [(int(k), int(a)) for k, a in zip(rng.choice(len(pos), 12, replace=False),
                                              rng.integers(0, 3, 12))]
    scale_u = np.sqrt(np.mean(gu ** 2))
    scale_p = np.sqrt(np.mean(gp ** 2))
    for k, a in picks:
        # moments: E is quadratic in u, so the central difference is exact up to rounding
        du = np.zeros_like(u)
        du[k, a] = 1e-3
        ep, _, _ = ora.bh_energy_grad(pos, u + du, 0.5, leaf_max, prec, **kw)
        em, _, _ = ora.bh_energy_grad(pos, u - du, 0.5, leaf_max, prec, **kw)
        assert (ep - em) / 2e-3 == pytest.approx(gu[k, a], abs=1e-9 * scale_u)
        # positions, with the decisions of the unperturbed configuration
        dx = np.zeros_like(pos)
        dx[k, a] = 1e-5
        ep, _, _ = ora.bh_energy_grad(pos + dx, u, 0.5, leaf_max, prec, pos_dec=pos, **kw)
        em, _, _ = ora.bh_energy_grad(pos - dx, u, 0.5, leaf_max, prec, pos_dec=pos, **kw)
        assert (ep - em) / 2e-5 == pytest.approx(gp[k, a], abs=1e-6 * scale_p)


# ---------------------------------------------------------------- reverse mode of the step


@pytest.mark.parametrize("prec,theta,leaf_max", [("f64", 0.5, 1), ("f64", 0.5, 4), ("f32", 0.6, 1)])
def test_field_force_vjp_central_differences(ora, prec, theta, leaf_max):
    """dL/dpos and dL/du of L = sum abar.h + bbar.f (dipolar field, dipolar + LJ force) with
    the decisions frozen, against central differences; the frozen forward equals the oracle's
    Barnes-Hut field and force."""
    pos, u = _gas(500, 13, phi=0.1)
    if prec == "f32":
        pos = pos.astype(np.float32).astype(np.float64)
    rng = np.random.default_rng(6)
    ab = rng.normal(size=pos.shape)
    bb = rng.normal(size=pos.shape)
    kw = dict(dip_scale=0.9, lj_eps=1.0)
    dp, du, h, f = ora.bh_vjp(pos, u, ab, bb, theta, leaf_max, prec, tree_centres=True, **kw)
    r = ora.bh(pos, u, theta, leaf_max, prec, 0.9, 1.0, 1.0, 2.5, True)
    np.testing.assert_allclose(h, r["h"], rtol=1e-13, atol=1e-13 * np.abs(r["h"]).max())
    np.testing.assert_allclose(f, r["f"], rtol=1e-12, atol=1e-12 * np.abs(r["f"]).max())

    def L(p_, u_):
        _, _, hh, ff_ = ora.bh_vjp(p_, u_, ab, bb, theta, leaf_max, prec, pos_dec=pos, **kw)
        return np.sum(ab * hh) + np.sum(bb * ff_)

    dp0, du0, _, _ = ora.bh_vjp(pos, u, ab, bb, theta, leaf_max, prec, **kw)
    sp, su = np.sqrt(np.mean(dp0 ** 2)), np.sqrt(np.mean(du0 ** 2))
    for k, a in zip(rng.choice(len(pos), 8, replace=False), rng.integers(0, 3, 8)):
        e = np.zeros_like(pos)
        e[k, a] = 1e-3
        assert (L(pos, u + e) - L(pos, u - e)) / 2e-3 == pytest.approx(du0[k, a], abs=1e-8 * su)
        e[k, a] = 1e-5
        assert (L(pos + e, u) - L(pos - e, u)) / 2e-5 == pytest.approx(dp0[k, a], abs=2e-6 * sp)


def test_vjp_reduces_to_the_energy_gradient(ora):
    """With abar = -1/2 u and bbar = 0, the VJP plus the energy's explicit -1/2 h is dE/du, and
    the VJP itself is dE/drho."""
    pos, u = _gas(600, 17)
    e, gp, gu = ora.bh_energy_grad(pos, u, 0.5, 1, "f64", dip_scale=0.7, lj_eps=1.0)
    dp, du, h, _ = ora.bh_vjp(pos, u, -0.5 * u, np.zeros_like(u), 0.5, 1, "f64", dip_scale=0.7,
                              lj_eps=1.0)
    np.testing.assert_allclose(du - 0.5 * h, gu, rtol=1e-10, atol=1e-12 * np.abs(gu).max())
    np.testing.assert_allclose(dp, gp, rtol=1e-10, atol=1e-12 * np.abs(gp).max())


def _state(n, seed):
    pos, u = _gas(n, seed, phi=0.08)
    rng = np.random.default_rng(seed)
    return dict(pos=pos, vel=0.3 * rng.normal(size=pos.shape), u=u,
                om=0.5 * rng.normal(size=pos.shape))


@pytest.mark.parametrize("theta,ds", [(0.0, 1.0), (0.5, 1.0), (0.5, 0.0)])
def test_mz_sensitivity_central_differences(ora, theta, ds):
    """d<M_z>/dh_ext over 40 steps by reverse mode against central differences (h = 1e-3,
    FP64) of the oracle's own trajectories with the same noise; with interactions (all pairs
    and Barnes-Hut, LJ and walls on) and without (dip_scale 0, LJ off).  The interactions move
    the derivative by ~2e-8 absolute, far above the agreement reached."""
    st = _state(120, 31)
    side = st["pos"].max() + 0.5
    kw = dict(kT=1.0, gamma_t=0.5, gamma_r=0.8, box_lo=(0, 0, 0), box_hi=(side, side, side),
              walls=True, seed=5)

    def mz(hz, hx=0.2):
        d = ora.make_dyn(h_ext=(hx, -0.1, hz), **kw)
        return ora.mz_grad(st, d, 40, theta, 1, "f64", ds, 1.0 if ds else 0.0)

    m0, g = mz(1.5)
    fd_z = (mz(1.5 + 1e-3)[0] - mz(1.5 - 1e-3)[0]) / 2e-3
    fd_x = (mz(1.5, 0.2 + 1e-3)[0] - mz(1.5, 0.2 - 1e-3)[0]) / 2e-3
    # reverse mode is exact; the central difference errs by O(h^2) (about 1e-11 here)
    assert g[2] == pytest.approx(fd_z, rel=1e-8)
    assert g[0] == pytest.approx(fd_x, rel=1e-7)
    assert g[2] > 0  # a stronger field aligns the moments
