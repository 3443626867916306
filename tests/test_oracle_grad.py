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
