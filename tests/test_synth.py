"""The seeded input generators (host only): the geometry each workload promises."""
import numpy as np
import pytest
from scipy.spatial import cKDTree

from paper_1212_2934_gb300 import synth


def test_chains_geometry():
    nch, length = 300, 64
    side = synth.box_side_for_fraction(nch * length, 0.01)
    pos, u = synth.chains_cube(nch, length, side, 3)
    assert pos.shape == (nch * length, 3) and u.shape == pos.shape
    assert pos.min() >= 0.0 and pos.max() <= side
    c = pos.reshape(nch, length, 3)
    m = u.reshape(nch, length, 3)
    step = np.diff(c, axis=1)
    # touching neighbours along a straight axis
    np.testing.assert_allclose(np.linalg.norm(step, axis=2), 1.0, rtol=0, atol=1e-12)
    axis = step[:, :1, :]
    np.testing.assert_allclose(step, np.broadcast_to(axis, step.shape), atol=1e-12)
    # head-to-tail unit moments along the axis, one sign per chain, both signs present
    np.testing.assert_allclose(np.linalg.norm(u, axis=1), 1.0, atol=1e-12)
    dots = np.einsum("cij,cij->ci", m[:, :-1], step)
    assert np.all(np.abs(np.abs(dots) - 1.0) < 1e-12)
    assert np.all(np.sign(dots) == np.sign(dots[:, :1]))
    assert 0.3 < np.mean(dots[:, 0] > 0) < 0.7
    # different chains never closer than one diameter
    pairs = cKDTree(pos).query_pairs(1.0 - 1e-9, output_type="ndarray")
    assert len(pairs) == 0
    # isotropic axes: mean of each squared component near 1/3
    a2 = (axis[:, 0, :] ** 2).mean(axis=0)
    assert np.all(np.abs(a2 - 1 / 3) < 0.08)


def test_chains_seeded_and_guarded():
    side = synth.box_side_for_fraction(64 * 50, 0.01)
    a = synth.chains_cube(50, 64, side, 9)
    b = synth.chains_cube(50, 64, side, 9)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    with pytest.raises(RuntimeError):
        synth.chains_cube(10, 64, 10.0, 1)  # a 63-long rod never fits a cube of side 10


def test_rsa_and_batched_shapes():
    side = synth.box_side_for_fraction(2000, 0.05)
    pos = synth.rsa_cube(2000, side, 4)
    assert len(cKDTree(pos).query_pairs(1.0 - 1e-9)) == 0
    assert pos.min() >= 0 and pos.max() <= side
    sizes = synth.batched_sizes(256)
    assert sizes[0] == round(1024 * 64 ** (0.5 / 256)) and sizes[-1] == round(1024 * 64 ** (255.5 / 256))
    assert int(sizes.sum()) == 3970997
    b = synth.batched_ensembles(8, 0.02, 5.0, 2)
    assert b["pos"].shape[0] == int(b["sizes"].sum())
    assert sorted(b["fields"][:, 2].tolist()) == pytest.approx(list(5.0 * np.arange(8) / 7))


def test_slab_monolayer():
    pos, side = synth.slab_monolayer(1500, 0.3, 2)
    assert pos.shape == (1500, 3)
    assert pos[:, 2].min() >= 0.0 and pos[:, 2].max() <= 0.05
    assert pos[:, :2].min() >= 0.0 and pos[:, :2].max() <= side
    assert len(cKDTree(pos).query_pairs(1.0 - 1e-9)) == 0
    assert 1500 * np.pi / 4 / side ** 2 == pytest.approx(0.3)
