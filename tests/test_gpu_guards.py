"""Device guards report instead of waiting forever (no GPU fault is provoked).

Two kernels have thread blocks that wait on one another: the key sort (each
tile adds up the digit counts that earlier tiles publish) and the gradient's
one-pass record scan (each tile adds up the entry counts of earlier tiles).
Both poll a bounded number of times and raise a device flag when the polls run
out.  ff_selftest_sort_wait and ff_selftest_record_wait withhold the first
tile's counts so that the second tile's wait must run out; each call checks
that the flag reached the host.  The GPU stays usable: a field evaluated
afterwards equals one evaluated before, bit for bit.
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


def _field(ff, pos, u):
    c = ff.ff_create(ff.ff_params_default(n=len(pos)))
    ff.ff_set_particles(c, pos, u)
    out = ff.ff_dipolar_field(c, ff.FF_ALGO_BH, 0.5, True)
    ff.ff_destroy(c)
    return out


def test_sort_wait_runs_out_and_is_reported(ff):
    from paper_1212_2934_gb300 import synth

    n = 5000
    side = synth.box_side_for_fraction(n, 0.05)
    pos = synth.rsa_cube(n, side, 2).astype(np.float32)
    u = synth.isotropic_moments(n, 3).astype(np.float32)
    h0, f0 = _field(ff, pos, u)
    for n_keys in (8192, 100003):
        ff.ff_selftest_sort_wait(n_keys)  # raises unless the wait ran out and was reported
    h1, f1 = _field(ff, pos, u)
    assert np.array_equal(h0, h1) and np.array_equal(f0, f1)


def test_sort_wait_selftest_rejects_one_tile(ff):
    with pytest.raises(ff.FFError) as ei:
        ff.ff_selftest_sort_wait(4096)
    assert ei.value.status == ff.FF_EINVAL


def test_record_scan_wait_runs_out_and_is_reported(ff):
    from paper_1212_2934_gb300 import synth

    n = 3000
    side = synth.box_side_for_fraction(n, 0.05)
    pos = synth.rsa_cube(n, side, 4).astype(np.float32)
    u = synth.isotropic_moments(n, 5).astype(np.float32)
    c = ff.ff_create(ff.ff_params_default(n=n))
    ff.ff_set_particles(c, pos, u)
    e0, gp0, gu0 = ff.ff_energy_grad(c, ff.FF_ALGO_BH, 0.5)
    for nrec in (4096, 100003):
        ff.ff_selftest_record_wait(nrec)  # raises unless the wait ran out and was reported
    e1, gp1, gu1 = ff.ff_energy_grad(c, ff.FF_ALGO_BH, 0.5)
    assert e0 == e1 and np.array_equal(gp0, gp1) and np.array_equal(gu0, gu1)


def test_record_wait_selftest_rejects_one_tile(ff):
    with pytest.raises(ff.FFError) as ei:
        ff.ff_selftest_record_wait(2048)
    assert ei.value.status == ff.FF_EINVAL
