"""Pins for the oracle's Morton keys, octree and cell aggregates (Sec. 3.2).

Hand-derived keys and trees on tiny inputs (corners, points on splitting
planes, coincident points, a degenerate line); an independent set-based
definition of the tree ("a level-L cell exists iff its parent holds more than
leaf_max particles") checked against the recursive build; structural
invariants; and the aggregates of Eq. magCenter against plain sums.
"""
import itertools

import numpy as np
import pytest

Z3 = np.zeros(3)
ALL = (8 ** 21 - 1) // 7  # a 63-bit key whose every 3-bit digit is 001


def _u(n):
    u = np.zeros((n, 3))
    u[:, 2] = 1.0
    return u


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_hand_keys(ora, prec):
    # box [0,1]^3 fixed by the two corners; a coordinate c maps to q = floor(c 2^21)
    pos = np.array([[0, 0, 0], [1, 1, 1], [0.5, 0, 0], [0, 0.5, 0], [0, 0, 0.5], [0.25, 0, 0]],
                   dtype=np.float64)
    keys, root = ora.morton(pos, prec)
    assert list(root) == [0, 0, 0, 1]
    # (1,1,1) clamps to q = 2^21 - 1 on every axis -> all 63 bits set
    expect = [0, 2 ** 63 - 1, 2 ** 62, 2 ** 61, 2 ** 60, 2 ** 59]
    assert [int(k) for k in keys] == expect


def test_octant_centres_tree(ora):
    # eight points at {0.25, 0.75}^3, given in reverse octant order
    pts = [np.array(p) for p in itertools.product([0.25, 0.75], repeat=3)][::-1]
    pos = np.array(pts)
    t = ora.tree(pos, _u(8), "f32", 1)
    # root cube: origin 0.25, side 0.5; 0.75 quantises to 2^21 -> clamped to 2^21-1
    assert list(t["root"]) == [0.25, 0.25, 0.25, 0.5]
    # every digit of a key equals the point's octant number (x*4 + y*2 + z)
    assert [int(k) for k in t["keys"]] == [d * ALL for d in range(8)]
    assert list(t["order"]) == [7 - d for d in range(8)]
    assert list(t["level"]) == [0] + [1] * 8
    assert list(t["leaf"]) == [0] + [1] * 8
    assert list(t["pbegin"]) == [0] + list(range(8))
    assert list(t["pend"]) == [8] + list(range(1, 9))
    assert list(t["skip"]) == [9] + list(range(2, 10))


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_split_plane_tree(ora, prec):
    # points on the x axis at 1.0, 0.0, 0.5: 0.5 falls in the upper half (floor)
    pos = np.array([[1.0, 0, 0], [0.0, 0, 0], [0.5, 0, 0]])
    t = ora.tree(pos, _u(3), prec, 1)
    assert [int(k) for k in t["keys"]] == [0, 2 ** 62, 4 * ALL]
    assert list(t["order"]) == [1, 2, 0]
    assert list(t["level"]) == [0, 1, 1, 2, 2]
    assert list(t["leaf"]) == [0, 1, 0, 1, 1]
    assert list(t["pbegin"]) == [0, 0, 1, 1, 2]
    assert list(t["pend"]) == [3, 1, 3, 2, 3]
    assert list(t["skip"]) == [5, 2, 5, 4, 5]
    np.testing.assert_array_equal(t["lo"][:, 0], [0, 0, 0.5, 0.5, 0.75])
    np.testing.assert_array_equal(t["side"], [1, 0.5, 0.5, 0.25, 0.25])


def test_coincident_points_leaf_at_level_21(ora):
    pos = np.array([[0, 0, 0], [1, 1, 1], [0, 0, 0], [0, 0, 0]], dtype=np.float64)
    t = ora.tree(pos, _u(4), "f32", 1)
    assert list(t["order"]) == [0, 2, 3, 1]  # ties keep input order
    nc = len(t["level"])
    assert nc == 23
    assert list(t["level"]) == list(range(22)) + [1]
    assert list(t["leaf"]) == [0] * 21 + [1, 1]
    assert list(t["pend"]) == [4] + [3] * 21 + [4]
    assert list(t["skip"]) == [23] + [22] * 21 + [23]


def test_single_particle(ora):
    t = ora.tree(np.array([[3.0, -2.0, 7.0]]), _u(1), "f32", 1)
    assert list(t["level"]) == [0] and list(t["leaf"]) == [1] and list(t["skip"]) == [1]
    np.testing.assert_array_equal(t["centre"][0], [3.0, -2.0, 7.0])


def test_degenerate_line(ora):
    # all x equal, z equal: the root side is set by the y extent (3)
    pos = np.array([[5.0, y, 0.0] for y in (3.0, 0.0, 2.0, 1.0)])
    t = ora.tree(pos, _u(4), "f32", 1)
    assert list(t["root"]) == [5.0, 0.0, 0.0, 3.0]
    assert list(t["order"]) == [1, 3, 2, 0]
    assert list(t["level"]) == [0, 1, 2, 2, 1, 2, 2]
    assert list(t["leaf"]) == [0, 0, 1, 1, 0, 1, 1]
    assert list(t["skip"]) == [7, 4, 3, 4, 7, 6, 7]


def _definition_cells(keys, leaf_max):
    """Cells by definition: (L, prefix) exists iff L = 0 or its parent holds > leaf_max
    particles and sits above level 21.  Returned in (first particle, level) order,
    which is depth-first preorder."""
    n = len(keys)
    keys = [int(k) for k in keys]
    cells = [(0, 0, n)]
    frontier = [(0, 0, n)]
    for L in range(0, 21):
        nxt = []
        for (lv, b, e) in frontier:
            if e - b <= leaf_max:
                continue
            shift = 3 * (21 - (L + 1))
            s = b
            while s < e:
                p = keys[s] >> shift
                s2 = s
                while s2 < e and keys[s2] >> shift == p:
                    s2 += 1
                nxt.append((L + 1, s, s2))
                s = s2
        cells.extend(nxt)
        frontier = nxt
    cells.sort(key=lambda c: (c[1], c[0]))
    return cells


@pytest.mark.parametrize("leaf_max", [1, 3, 16])
@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_tree_matches_definition_and_invariants(ora, rng, leaf_max, prec):
    n = 3000
    pos = rng.uniform(-7, 11, (n, 3))
    pos[:50] = pos[50:100]  # some coincident pairs
    pos[200:260, 1] = 0.125  # a plane of points
    u = rng.normal(size=(n, 3))
    t = ora.tree(pos, u, prec, leaf_max)
    keys = t["keys"]
    assert np.all(keys[1:] >= keys[:-1])
    assert sorted(t["order"]) == list(range(n))
    cells = _definition_cells(keys, leaf_max)
    assert [(c[0], c[1], c[2]) for c in cells] == list(zip(t["level"], t["pbegin"], t["pend"]))
    nc = len(cells)
    lvl, pb, pe, skip, leaf = t["level"], t["pbegin"], t["pend"], t["skip"], t["leaf"]
    for c in range(nc):
        cnt = pe[c] - pb[c]
        assert cnt >= 1
        assert leaf[c] == (cnt <= leaf_max or lvl[c] == 21)
        if leaf[c]:
            assert skip[c] == c + 1
        else:
            # children partition the parent's range in octant (key) order
            ch = c + 1
            cur = pb[c]
            while ch < skip[c]:
                assert lvl[ch] == lvl[c] + 1 and pb[ch] == cur
                cur = pe[ch]
                ch = skip[ch]
            assert ch == skip[c] and cur == pe[c]
    # every particle is in exactly one leaf
    cover = np.zeros(n, dtype=int)
    for c in np.nonzero(leaf)[0]:
        cover[pb[c]:pe[c]] += 1
    assert np.all(cover == 1)


def test_aggregates(ora, rng):
    n = 2000
    pos = rng.uniform(0, 40, (n, 3))
    u = rng.normal(size=(n, 3))
    for prec in ("f32", "f64"):
        p = pos.astype(np.float32).astype(np.float64) if prec == "f32" else pos
        t = ora.tree(p, u, prec, 2)
        np.testing.assert_allclose(t["U"][0], u.sum(axis=0), rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(t["centre64"][0], p.mean(axis=0), rtol=1e-13)
        order = t["order"]
        for c in rng.choice(len(t["level"]), 200, replace=False):
            idx = order[t["pbegin"][c]:t["pend"][c]]
            np.testing.assert_allclose(t["U"][c], u[idx].sum(axis=0), rtol=1e-12, atol=1e-12)
            np.testing.assert_allclose(t["centre64"][c], p[idx].mean(axis=0), rtol=1e-13)
            # the tree-precision centre is the single-precision rounding of the same sum
            tol = (1e-15 if prec == "f64" else 2.0 ** -24 * 24) * np.abs(p).max()
            assert np.all(np.abs(t["centre"][c] - t["centre64"][c]) <= tol)
            # every particle lies in its cell's cube (up to one quantisation step)
            q = t["side"][c] * 1e-6 + 2 ** -21 * t["root"][3]
            assert np.all(p[idx] >= t["lo"][c] - q) and np.all(p[idx] <= t["lo"][c] + t["side"][c] + q)


def test_mixed_precision_tree(ora, rng):
    """Mixed precision: keys, topology and cube geometry are those of the single-precision
    tree; each centre is the FP64 mean of the cell's particles rounded once to single."""
    n = 3000
    pos = rng.uniform(0, 40, (n, 3)).astype(np.float32).astype(np.float64)
    u = rng.normal(size=(n, 3))
    s = ora.tree(pos, u, "f32", 1)
    m = ora.tree(pos, u, "mixed", 1)
    for k in ("keys", "order", "level", "leaf", "pbegin", "pend", "skip", "lo", "side", "root"):
        assert np.array_equal(s[k], m[k]), k
    order = m["order"]
    for c in range(len(m["level"])):
        idx = order[m["pbegin"][c]:m["pend"][c]]
        mean = pos[idx].mean(axis=0)
        np.testing.assert_allclose(m["centre64"][c], mean, rtol=1e-13)
    assert np.array_equal(m["centre"], m["centre64"].astype(np.float32).astype(np.float64))
    # one-particle leaves: the particle itself in both modes
    one = (m["pend"] - m["pbegin"]) == 1
    assert np.array_equal(m["centre"][one], s["centre"][one])
    # cells of many particles: single-precision sums drift, the rounded FP64 mean does not
    big = (m["pend"] - m["pbegin"]) >= 256
    err_s = np.abs(s["centre"][big] - m["centre64"][big]).max()
    err_m = np.abs(m["centre"][big] - m["centre64"][big]).max()
    assert err_m <= 2.0 ** -24 * 40 and err_m <= err_s


def test_mixed_precision_bh(ora, rng):
    """Mixed-precision Barnes-Hut: theta = 0 is all-pairs; at theta = 0.5 it agrees with the
    single-precision tree to rounding (only the centres differ, by a few single ulps)."""
    n = 1500
    pos = rng.uniform(0, 25, (n, 3)).astype(np.float32).astype(np.float64)
    u = rng.normal(size=(n, 3))
    u /= np.linalg.norm(u, axis=1)[:, None]
    ap_h, ap_f, _ = ora.allpairs(pos, u, include_sr=False)
    r0 = ora.bh(pos, u, 0.0, 1, "mixed")
    np.testing.assert_allclose(r0["h"], ap_h, rtol=1e-12, atol=1e-12 * np.abs(ap_h).max())
    rs = ora.bh(pos, u, 0.5, 1, "f32")
    rm = ora.bh(pos, u, 0.5, 1, "mixed")
    scale = np.sqrt((rs["h"] ** 2).sum(axis=1)).mean()
    assert np.abs(rm["h"] - rs["h"]).max() <= 1e-4 * scale
    assert (rm["ncover"] + rm["npair"] == n - 1).all()
