"""Dipole-position (quadrupole) cell terms on the GPU (ff_params.quadrupole).

An accuracy option beyond the paper's pseudo-particles: every accepted cell also
contributes -grad Phi to the field and -H Phi u_k to the force, Phi from the
symmetric part of sum (rho_i - c) (x) u_i about the cell's centre.  Checked
against the oracle's quadrupole mode (decisions and counts unchanged; FP32 1e-5,
forces against the term magnitudes; FP64 1e-10), for multi-particle leaves, and
for the error against all pairs falling several-fold at the same theta.
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


def _gas(n, seed):
    from paper_1212_2934_gb300 import synth

    side = synth.box_side_for_fraction(n, 0.05)
    pos = synth.rsa_cube(n, side, seed).astype(np.float32).astype(np.float64)
    u = synth.isotropic_moments(n, seed + 1).astype(np.float32).astype(np.float64)
    return pos, u


@pytest.mark.parametrize("prec,leaf_max", [("f32", 1), ("f32", 4), ("f64", 1), ("f64", 4)])
def test_quadrupole_matches_oracle(ff, ora, prec, leaf_max):
    pos, u = _gas(6007, 9)
    dt = np.float64 if prec == "f64" else np.float32
    ctx = ff.ff_create(ff.ff_params_default(n=len(pos), precision=prec, leaf_max=leaf_max,
                                            quadrupole=1, count_interactions=1))
    ff.ff_set_particles(ctx, pos.astype(dt), u.astype(dt))
    h, f = ff.ff_dipolar_field(ctx, ff.FF_ALGO_BH, 0.5, True)
    ref = ora.bh(pos, u, 0.5, leaf_max, prec, 1.0, 1.0, 1.0, 2.5, True, quad=True)
    if prec == "f64":
        assert rel_err(h, ref["h"]).max() <= 1e-10
        assert rel_err(f, ref["f"]).max() <= 1e-10
    else:
        assert rel_err(h, ref["h"]).max() <= 1e-5
        assert rel_err(f, ref["f"]).max() <= 1e-5  # the plain bar (7.5e-6 measured on GB300)
    acc, pairs, opened = ff.ff_get_counts(ctx)
    assert np.array_equal(acc, ref["nacc"]) and np.array_equal(opened, ref["nopen"])


def test_quadrupole_reduces_error_against_allpairs(ff):
    pos, u = _gas(20000, 3)
    out = {}
    for q in (0, 1):
        ctx = ff.ff_create(ff.ff_params_default(n=len(pos), quadrupole=q))
        ff.ff_set_particles(ctx, pos.astype(np.float32), u.astype(np.float32))
        out[q] = ff.ff_dipolar_field(ctx, ff.FF_ALGO_BH, 0.5, False)[0]
    ap = ff.ff_create(ff.ff_params_default(n=len(pos), precision="f64"))
    ff.ff_set_particles(ap, pos, u)
    h0 = ff.ff_dipolar_field(ap, ff.FF_ALGO_AP, 0.0, False)[0]
    rms = lambda x: np.sqrt(np.mean(np.sum((x - h0) ** 2, axis=1)) / np.mean(np.sum(h0 ** 2, axis=1)))
    assert rms(out[1]) < 0.5 * rms(out[0])


def test_quadrupole_rejected_by_the_gradients(ff):
    pos, u = _gas(500, 2)
    ctx = ff.ff_create(ff.ff_params_default(n=500, quadrupole=1))
    ff.ff_set_particles(ctx, pos.astype(np.float32), u.astype(np.float32))
    with pytest.raises(ff.FFError):
        ff.ff_energy_grad(ctx, ff.FF_ALGO_BH, 0.5)
    with pytest.raises(ff.FFError):
        ff.ff_mz_sensitivity(ctx, 3, 1)
    ff.ff_step(ctx, 2)  # stepping with the option works
    assert ff.ff_get_step(ctx) == 2
