"""GPU parity of the integration step (Sec. 4) and observables (Sec. 5).

  * Noise: with zero forces, friction and a unit step the velocity update is
    v' = v + sig xi, so the GPU's normals are recovered from one FP64 step
    and must equal the oracle's Philox/Box-Muller normals to 1e-12 (the raw
    32-bit words therefore agree bit for bit).
  * 100-step trajectories of the dense 4096-particle cube (FP64, BH theta =
    0.5, h_ext = 0.5 z, seed 1): positions, velocities, moments and angular
    velocities within 1e-9 of the oracle; FP32 trajectories within 1e-4
    (per-particle error normalised as for the fields).
  * Energies and magnetisation against the oracle.
  * Resuming from a saved state gives bit-identical results.
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


def _params(ff, e, prec, **kw):
    side = e["side"]
    base = dict(n=e["n"], precision=prec, theta=e["theta"], leaf_max=e["leaf_max"],
                dt=e["dt"], gamma_t=e["gamma_t"], gamma_r=e["gamma_r"], inertia=e["inertia"],
                kT=e["kT"], rot_noise=e["rot_noise"], dip_scale=e["dip_scale"],
                lj_eps=e["lj_eps"], lj_sigma=e["lj_sigma"], lj_rcut=e["lj_rcut"],
                h_ext=e["h_ext"], box_lo=(0, 0, 0), box_hi=(side, side, side), walls=1,
                wall_eps=e["wall_eps"], seed=e["seed"])
    base.update(kw)
    return ff.ff_params_default(**base)


def _odyn(ora, e, **kw):
    side = e["side"]
    d = dict(dt=e["dt"], gamma_t=e["gamma_t"], gamma_r=e["gamma_r"], inertia=e["inertia"],
             kT=e["kT"], rot_noise=e["rot_noise"], h_ext=e["h_ext"], box_lo=(0, 0, 0),
             box_hi=(side, side, side), walls=True, wall_eps=e["wall_eps"], seed=e["seed"])
    d.update(kw)
    return ora.make_dyn(**d)


def test_noise_matches_oracle(ff, ora):
    n = 777
    ids = np.arange(n)
    pos = np.random.default_rng(1).uniform(0, 50, (n, 3))
    u = np.tile([0.0, 0.0, 1.0], (n, 1))
    # zero forces and field (dip_scale 0, LJ off, no walls), v = w = 0, dt = 1:
    # v' = sig_t xi_t and w' = sig_r xi_r with sig_t = sig_r = sqrt(2 * 0.5 * kT)
    p2 = ff.ff_params_default(n=n, precision="f64", dt=1.0, gamma_t=0.5, gamma_r=0.5, kT=1.0,
                              rot_noise=2.0, inertia=1.0, dip_scale=0.0, lj_eps=0.0,
                              seed=0xABCDEF12345, algo="ap")
    ctx = ff.ff_create(p2)
    ff.ff_set_particles(ctx, pos, u)
    ff.ff_set_step(ctx, 123456789012)
    ff.ff_step(ctx, 1)
    x, uu, v, w = ff.ff_get_particles(ctx)
    z = ora.normals(0xABCDEF12345, 123456789012, ids)
    sig = np.sqrt(2 * 0.5 * 1.0 * 1.0)
    np.testing.assert_allclose(v / sig, z[:, 0:3], rtol=0, atol=1e-12)
    np.testing.assert_allclose(w / sig, z[:, 3:6], rtol=0, atol=1e-12)


def _run_oracle(ora, e, nsteps, prec):
    """Oracle trajectory; in single precision the state is stored rounded to FP32 after every
    step, as the kernel stores it (the arithmetic of each step stays FP64)."""
    s = dict(pos=e["pos"].copy(), vel=np.zeros_like(e["pos"]), u=e["u"].copy(),
             om=np.zeros_like(e["pos"]), id=np.arange(e["n"], dtype=np.int64))
    dyn = _odyn(ora, e)
    kw = dict(theta=e["theta"], leaf_max=e["leaf_max"], prec=prec, dip_scale=e["dip_scale"],
              lj_eps=e["lj_eps"], lj_sigma=e["lj_sigma"], lj_rcut=e["lj_rcut"])
    for k in range(nsteps):
        if prec == "f32":
            for key in ("pos", "vel", "u", "om"):
                s[key] = np.ascontiguousarray(s[key].astype(np.float32).astype(np.float64))
        ora.run(s, 1, dyn, "bh", k, **kw)
    if prec == "f32":
        for key in ("pos", "vel", "u", "om"):
            s[key] = s[key].astype(np.float32).astype(np.float64)
    return s


@pytest.mark.slow
@pytest.mark.parametrize("prec,tol", [("f64", 1e-9), ("f32", 1e-4)])
def test_trajectory_matches_oracle(ff, ora, prec, tol):
    from paper_1212_2934_gb300 import synth

    e = synth.make_ensemble("dense4096")
    steps = 100
    ref = _run_oracle(ora, e, steps, prec)
    ctx = ff.ff_create(_params(ff, e, prec))
    dt = np.float32 if prec == "f32" else np.float64
    ff.ff_set_particles(ctx, e["pos"].astype(dt), e["u"].astype(dt))
    ff.ff_step(ctx, steps)
    assert ff.ff_get_step(ctx) == steps
    x, u, v, w = ff.ff_get_particles(ctx)
    # positions relative to the box scale (FP32 positions near 16 carry 1e-6 ulps)
    assert np.abs(x - ref["pos"]).max() <= tol * np.abs(ref["pos"]).max()
    assert rel_err(v, ref["vel"]).max() <= tol
    assert rel_err(w, ref["om"]).max() <= tol
    assert np.abs(u - ref["u"]).max() <= tol


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_energy_matches_oracle(ff, ora, prec):
    from paper_1212_2934_gb300 import synth

    e = synth.make_ensemble("dilute", n=3000)
    dt = np.float32 if prec == "f32" else np.float64
    pos = e["pos"].astype(dt)
    u = e["u"].astype(dt)
    rng = np.random.default_rng(3)
    vel = rng.normal(size=pos.shape).astype(dt)
    om = rng.normal(size=pos.shape).astype(dt)
    ctx = ff.ff_create(_params(ff, e, prec))
    ff.ff_set_particles(ctx, pos, u, vel, om)
    E = ff.ff_energy(ctx)
    p64 = pos.astype(np.float64)
    r = ora.bh(p64, u.astype(np.float64), e["theta"], 1, prec, 1.0, 1.0, 1.0, 2.5, True)
    s = dict(pos=p64, vel=vel.astype(np.float64), u=u.astype(np.float64), om=om.astype(np.float64),
             id=np.arange(e["n"]))
    R = ora.energy(s, r["h"], r["e_sr"], _odyn(ora, e))
    rtol = 1e-5 if prec == "f32" else 1e-10
    for k in ("e_dip", "e_zeeman", "e_kin_t", "e_kin_r", "hdip_z_mean"):
        assert E[k] == pytest.approx(R[k], rel=rtol, abs=rtol * abs(R["e_kin_t"]) * 1e-3), k
    assert E["e_sr"] == pytest.approx(R["e_sr"], rel=1e-4, abs=1e-6)
    np.testing.assert_allclose(E["m"], R["m"], atol=1e-7 if prec == "f32" else 1e-14)


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_resume_bit_identical(ff, prec):
    from paper_1212_2934_gb300 import synth

    e = synth.make_ensemble("dilute", n=2000)
    dt = np.float32 if prec == "f32" else np.float64
    a = ff.ff_create(_params(ff, e, prec))
    ff.ff_set_particles(a, e["pos"].astype(dt), e["u"].astype(dt))
    ff.ff_step(a, 20)
    xa = ff.ff_get_particles(a, dtype=dt)
    b = ff.ff_create(_params(ff, e, prec))
    ff.ff_set_particles(b, e["pos"].astype(dt), e["u"].astype(dt))
    ff.ff_step(b, 10)
    saved = ff.ff_get_particles(b, dtype=dt)
    c = ff.ff_create(_params(ff, e, prec))
    ff.ff_set_particles(c, *saved)
    ff.ff_set_step(c, 10)
    ff.ff_step(c, 10)
    xc = ff.ff_get_particles(c, dtype=dt)
    for p, q in zip(xa, xc):
        assert np.array_equal(p, q)


def test_walls_hold_particles(ff):
    from paper_1212_2934_gb300 import synth

    e = synth.make_ensemble("dilute", n=1500)
    ctx = ff.ff_create(_params(ff, e, "f32", kT=5.0, gamma_t=1.0))
    ff.ff_set_particles(ctx, e["pos"].astype(np.float32), e["u"].astype(np.float32))
    ff.ff_step(ctx, 300)
    x, u, v, w = ff.ff_get_particles(ctx)
    assert np.isfinite(x).all()
    assert x.min() > -0.6 and x.max() < e["side"] + 0.6
    np.testing.assert_allclose(np.linalg.norm(u, axis=1), 1.0, atol=1e-5)


def test_printed_angle_equations_match_oracle(ff, ora):
    """rotation = FF_ROT_PRINTED: the printed reduced angle equations, FP64, 40 steps of the
    dense cube with the field tilted off z, against the oracle's literal mode."""
    from paper_1212_2934_gb300 import synth

    e = synth.make_ensemble("dense4096")
    e["h_ext"] = (0.4, -0.3, 0.8)
    steps = 40
    s = dict(pos=e["pos"].copy(), vel=np.zeros_like(e["pos"]), u=e["u"].copy(),
             om=np.zeros_like(e["pos"]), id=np.arange(e["n"], dtype=np.int64))
    dyn = _odyn(ora, e, literal=True)
    kw = dict(theta=e["theta"], leaf_max=e["leaf_max"], prec="f64", dip_scale=e["dip_scale"],
              lj_eps=e["lj_eps"], lj_sigma=e["lj_sigma"], lj_rcut=e["lj_rcut"])
    for k in range(steps):
        ora.run(s, 1, dyn, "bh", k, **kw)
    ctx = ff.ff_create(_params(ff, e, "f64", rotation=ff.FF_ROT_PRINTED))
    ff.ff_set_particles(ctx, e["pos"], e["u"])
    ff.ff_step(ctx, steps)
    x, u, v, w = ff.ff_get_particles(ctx)
    assert np.abs(x - s["pos"]).max() <= 1e-9 * np.abs(s["pos"]).max()
    assert np.abs(u - s["u"]).max() <= 1e-9
    assert rel_err(w, s["om"]).max() <= 1e-9
    assert np.all(w[:, 2] == 0.0)  # the rates live in w_x, w_y


@pytest.mark.slow
def test_printed_angle_equations_do_not_magnetise(ff, ora):
    """The documented bias on the GPU: non-interacting moments in h = 3 z under the printed
    angle equations keep <u_z> near 0, while the vector rotor follows L(3) = 0.672."""
    n = 4000
    rng = np.random.default_rng(11)
    pos = rng.uniform(0, 200, (n, 3))
    u = rng.normal(size=(n, 3))
    u /= np.linalg.norm(u, axis=1)[:, None]
    out = {}
    for rot in (ff.FF_ROT_VECTOR, ff.FF_ROT_PRINTED):
        p = ff.ff_params_default(n=n, precision="f32", algo="ap", dip_scale=0.0, lj_eps=0.0,
                                 gamma_t=1.0, gamma_r=1.0, kT=1.0, h_ext=(0, 0, 3.0), seed=3,
                                 rotation=rot)
        ctx = ff.ff_create(p)
        ff.ff_set_particles(ctx, pos.astype(np.float32), u.astype(np.float32))
        ff.ff_step(ctx, 3000)
        acc = 0.0
        for _ in range(20):
            ff.ff_step(ctx, 100)
            acc += ff.ff_get_particles(ctx)[1][:, 2].mean()
        out[rot] = acc / 20
    L3 = float(ora.langevin(np.array([3.0]))[0])
    assert abs(out[ff.FF_ROT_VECTOR] - L3) < 0.05
    assert abs(out[ff.FF_ROT_PRINTED]) < 0.1
