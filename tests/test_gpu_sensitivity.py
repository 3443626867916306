"""d<M_z>/dh_ext by checkpointed reverse mode on the GPU (ff_mz_sensitivity).

<M_z> is the mean over the nsteps new states of 1/n sum u_z (Sec. 5).  The
reference is the oracle's reverse mode (ora_mz_grad), itself pinned by central
differences (tests/test_oracle_grad.py).  Checked here:
  * FP64: <M_z> and the gradient against the oracle;
  * the checkpoint interval changes nothing (bit-identical results);
  * central differences (h = 1e-3) of the GPU's own FP64 <M_z>, as the north
    star asks, within 1e-4 relative;
  * FP32 against the oracle;
  * the context ends at the advanced state, bit for bit as after ff_step.
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


def _state(n, seed):
    from paper_1212_2934_gb300 import synth

    side = synth.box_side_for_fraction(n, 0.08)
    pos = synth.rsa_cube(n, side, seed)
    u = synth.isotropic_moments(n, seed + 1)
    rng = np.random.default_rng(seed)
    return dict(pos=pos, vel=0.3 * rng.normal(size=pos.shape), u=u,
                om=0.5 * rng.normal(size=pos.shape), side=side)


DYN = dict(kT=1.0, gamma_t=0.5, gamma_r=0.8, seed=5)


def _ctx(ff, st, prec, hz, theta=0.5):
    side = st["side"] + 0.5
    dt = np.float64 if prec == "f64" else np.float32
    p = ff.ff_params_default(n=len(st["pos"]), precision=prec, theta=theta, walls=1,
                             box_lo=(0, 0, 0), box_hi=(side, side, side), h_ext=(0.2, -0.1, hz),
                             **DYN)
    c = ff.ff_create(p)
    ff.ff_set_particles(c, *[st[k].astype(dt) for k in ("pos", "u", "vel", "om")])
    return c


def _oracle(ora, st, hz, steps, theta=0.5, prec="f64"):
    side = st["side"] + 0.5
    d = ora.make_dyn(h_ext=(0.2, -0.1, hz), box_lo=(0, 0, 0), box_hi=(side, side, side),
                     walls=True, **DYN)
    s64 = {k: st[k].astype(np.float64) for k in ("pos", "vel", "u", "om")}
    return ora.mz_grad(s64, d, steps, theta, 1, prec, 1.0, 1.0)


def test_fp64_matches_oracle_and_checkpoints_change_nothing(ff, ora):
    st = _state(400, 3)
    m0, g0 = _oracle(ora, st, 1.5, 30)
    res = []
    for every in (7, 1, 30):
        c = _ctx(ff, st, "f64", 1.5)
        res.append(ff.ff_mz_sensitivity(c, 30, every))
    for mz, g in res:
        assert mz == pytest.approx(m0, rel=1e-11, abs=1e-14)
        np.testing.assert_allclose(g, g0, rtol=1e-7, atol=1e-9 * np.abs(g0).max())
    assert all(r[0] == res[0][0] and np.array_equal(r[1], res[0][1]) for r in res)


def test_fp64_central_differences(ff):
    st = _state(300, 8)
    c = _ctx(ff, st, "f64", 1.0)
    mz, g = ff.ff_mz_sensitivity(c, 40, 10)
    mp, _ = ff.ff_mz_sensitivity(_ctx(ff, st, "f64", 1.0 + 1e-3), 40, 10)
    mm, _ = ff.ff_mz_sensitivity(_ctx(ff, st, "f64", 1.0 - 1e-3), 40, 10)
    assert g[2] == pytest.approx((mp - mm) / 2e-3, rel=1e-4)


def test_fp32_matches_oracle(ff, ora):
    st = _state(400, 4)
    st32 = {k: (v.astype(np.float32).astype(np.float64) if k != "side" else v)
            for k, v in st.items()}
    m0, g0 = _oracle(ora, st32, 1.5, 30, prec="f32")
    mz, g = ff.ff_mz_sensitivity(_ctx(ff, st32, "f32", 1.5), 30, 10)
    assert mz == pytest.approx(m0, rel=1e-5, abs=1e-7)
    # measured on GB300: 4e-7 relative (three seeds: at most 1.1e-6 per component)
    np.testing.assert_allclose(g, g0, rtol=1e-5, atol=1e-6 * np.abs(g0).max())


def test_ends_at_the_advanced_state(ff):
    st = _state(250, 6)
    a = _ctx(ff, st, "f64", 0.7)
    ff.ff_mz_sensitivity(a, 12, 5)
    b = _ctx(ff, st, "f64", 0.7)
    ff.ff_step(b, 12)
    assert ff.ff_get_step(a) == ff.ff_get_step(b) == 12
    for x, y in zip(ff.ff_get_particles(a), ff.ff_get_particles(b)):
        assert np.array_equal(x, y)


def test_rejects_bad_input(ff):
    st = _state(100, 2)
    c = _ctx(ff, st, "f32", 1.0)
    for args in ((0, 5), (5, 0)):
        with pytest.raises(ff.FFError):
            ff.ff_mz_sensitivity(c, *args)
    ap = ff.ff_create(ff.ff_params_default(n=100, algo="ap"))
    ff.ff_set_particles(ap, st["pos"].astype(np.float32), st["u"].astype(np.float32))
    with pytest.raises(ff.FFError):
        ff.ff_mz_sensitivity(ap, 3, 1)
    b = ff.ff_create(ff.ff_params_default(n=100))
    ff.ff_set_systems(b, [50, 50])
    ff.ff_set_particles(b, st["pos"].astype(np.float32), st["u"].astype(np.float32))
    with pytest.raises(ff.FFError):
        ff.ff_mz_sensitivity(b, 3, 1)


@pytest.mark.slow
def test_full_size_200_step_unroll_central_differences(ff):
    """N = 262,144 at volume fraction 0.05, FP64: d<M_z>/dh_z through a 200-step unroll saved
    every 20 steps, against central differences (h = 1e-3) of the same FP64 trajectories."""
    from paper_1212_2934_gb300 import synth

    n = 262144
    side = synth.box_side_for_fraction(n, 0.05)
    pos = synth.rsa_cube(n, side, 3)
    u = synth.isotropic_moments(n, 4)

    def ctx(hz):
        p = ff.ff_params_default(n=n, precision="f64", walls=1, box_lo=(0, 0, 0),
                                 box_hi=(side, side, side), h_ext=(0.0, 0.0, hz), seed=1)
        c = ff.ff_create(p)
        ff.ff_set_particles(c, pos, u)
        return c

    def mean_mz(hz):
        # the plain trajectory: mean of u_z over the 200 new states
        c = ctx(hz)
        acc = 0.0
        for _ in range(200):
            ff.ff_step(c, 1)
            acc += ff.ff_get_particles(c)[1][:, 2].mean()
        return acc / 200

    mz, g = ff.ff_mz_sensitivity(ctx(1.0), 200, 20)
    assert mz == pytest.approx(mean_mz(1.0), rel=1e-10, abs=1e-13)
    assert g[2] == pytest.approx((mean_mz(1.0 + 1e-3) - mean_mz(1.0 - 1e-3)) / 2e-3, rel=1e-4)


@pytest.mark.slow
def test_full_size_fp32_against_fp64(ff):
    """N = 262,144 at volume fraction 0.05: the FP32 d<M_z>/dh_ext through a 200-step unroll
    saved every 20 steps against the FP64 one and against central differences (h = 1e-3) of
    FP64 trajectories (measured on GB300: 8e-7 relative for the z component)."""
    from paper_1212_2934_gb300 import synth

    n = 262144
    side = synth.box_side_for_fraction(n, 0.05)
    pos = synth.rsa_cube(n, side, 3).astype(np.float32)
    u = synth.isotropic_moments(n, 4).astype(np.float32)

    def ctx(hz, prec):
        p = ff.ff_params_default(n=n, precision=prec, walls=1, box_lo=(0, 0, 0),
                                 box_hi=(side, side, side), h_ext=(0.0, 0.0, hz), seed=1)
        c = ff.ff_create(p)
        dt = np.float64 if prec == "f64" else np.float32
        ff.ff_set_particles(c, pos.astype(dt), u.astype(dt))
        return c

    def mean_mz(hz):
        c = ctx(hz, "f64")
        acc = 0.0
        for _ in range(200):
            ff.ff_step(c, 1)
            acc += ff.ff_get_particles(c)[1][:, 2].mean()
        return acc / 200

    mz32, g32 = ff.ff_mz_sensitivity(ctx(1.0, "f32"), 200, 20)
    mz64, g64 = ff.ff_mz_sensitivity(ctx(1.0, "f64"), 200, 20)
    cd = (mean_mz(1.0 + 1e-3) - mean_mz(1.0 - 1e-3)) / 2e-3
    assert mz32 == pytest.approx(mz64, rel=1e-5)
    assert g32[2] == pytest.approx(g64[2], rel=1e-5)
    assert g32[2] == pytest.approx(cd, rel=1e-5)
    np.testing.assert_allclose(g32, g64, rtol=1e-4, atol=1e-5 * abs(g64[2]))
