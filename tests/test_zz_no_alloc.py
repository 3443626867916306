"""The allocation-free Morton ordering entry point (ff_morton_order_noalloc).

It exists for callers that cannot allocate device memory (memory owned by the
application's own pool or allocator, loops that must not stall on an
allocation); it uses a fixed scratch array inside the library instead.  Its
keys and order must equal, bit for bit, what the allocating path reports
through ff_get_tree for the same single-precision positions, on two calls in a
row (the scratch keeps the previous call's contents), and the oracle's keys
with a stable sort.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ff():
    from paper_1212_2934_gb300 import _build, ff

    _build.build()
    ff.lib()
    return ff


def _positions(n, seed):
    from paper_1212_2934_gb300 import synth

    side = synth.box_side_for_fraction(n, 0.05)
    return synth.rsa_cube(n, side, seed).astype(np.float32)


def _reference(ff, pos):
    """Keys and order from the allocating path (ff_dipolar_field + ff_get_tree)."""
    n = pos.shape[0]
    ctx = ff.ff_create(ff.ff_params_default(n=n, precision="f32"))
    u = np.tile(np.array([[0.0, 0.0, 1.0]], dtype=np.float32), (n, 1))
    ff.ff_set_particles(ctx, pos, u)
    ff.ff_dipolar_field(ctx, ff.FF_ALGO_BH, 0.5, True)
    g = ff.ff_get_tree(ctx)
    ff.ff_destroy(ctx)
    return g["keys"], g["order"]


def test_noalloc_order_matches_allocating_path_twice(ff):
    torch = pytest.importorskip("torch")
    cases = [(ff.FF_NOALLOC_MAX_N, 3), (70001, 4)]
    refs = []
    for n, seed in cases:
        pos = _positions(n, seed)
        refs.append((pos, *_reference(ff, pos)))
    outs = []
    for pos, _, _ in refs:  # two calls in a row; the second is smaller than the first
        n = pos.shape[0]
        keys = torch.empty(n, dtype=torch.int64, device="cuda")  # uint64 bits
        order = torch.empty(n, dtype=torch.int32, device="cuda")
        ff.ff_morton_order_noalloc(torch.tensor(pos, device="cuda"), keys, order)
        outs.append((keys, order))
    for (pos, want_keys, want_order), (keys, order) in zip(refs, outs):
        assert np.array_equal(keys.cpu().numpy().view(np.uint64), want_keys)
        assert np.array_equal(order.cpu().numpy().view(np.uint32), want_order)


def test_noalloc_rejects_sizes_beyond_the_scratch(ff):
    torch = pytest.importorskip("torch")
    n = ff.FF_NOALLOC_MAX_N + 1
    pd = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
    keys = torch.empty(n, dtype=torch.int64, device="cuda")
    order = torch.empty(n, dtype=torch.int32, device="cuda")
    with pytest.raises(ff.FFError) as ei:
        ff.ff_morton_order_noalloc(pd, keys, order)
    assert ei.value.status == ff.FF_EINVAL
    assert "131072" in ff.ff_last_error(None)


def _oracle_order(pos):
    """The oracle's single-precision keys (Sec. 3.2 reading: 63-bit Morton keys of the root
    cube) with a stable sort: sorted keys and the input index of each sorted position."""
    import oracle

    keys, _ = oracle.morton(pos.astype(np.float64), "f32")
    order = np.argsort(keys, kind="stable")
    return keys[order], order


def test_noalloc_matches_oracle_small_and_side_stream(ff):
    """n = 1 (the sort returns at once), n = 5000 (less than one sort tile) and a ragged
    multi-tile size, on a side stream, against the oracle and the allocating path."""
    torch = pytest.importorskip("torch")
    side = torch.cuda.Stream()
    for n, seed in ((1, 5), (5000, 6), (9001, 7)):
        pos = _positions(n, seed)
        want_keys, want_order = _oracle_order(pos)
        ref_keys, ref_order = _reference(ff, pos)
        assert np.array_equal(ref_keys, want_keys) and np.array_equal(ref_order, want_order)
        for _ in range(2):
            with torch.cuda.stream(side):
                pd = torch.tensor(pos, device="cuda")
                keys = torch.empty(n, dtype=torch.int64, device="cuda")
                order = torch.empty(n, dtype=torch.int32, device="cuda")
                ff.ff_morton_order_noalloc(pd, keys, order, stream=side)
            side.synchronize()
            assert np.array_equal(keys.cpu().numpy().view(np.uint64), want_keys)
            assert np.array_equal(order.cpu().numpy().view(np.uint32), want_order.astype(np.uint32))


def test_noalloc_reports_non_finite_positions(ff):
    torch = pytest.importorskip("torch")
    n = 3000
    pos = _positions(n, 8)
    pos[17, 2] = np.nan
    keys = torch.empty(n, dtype=torch.int64, device="cuda")
    order = torch.empty(n, dtype=torch.int32, device="cuda")
    with pytest.raises(ff.FFError) as ei:
        ff.ff_morton_order_noalloc(torch.tensor(pos, device="cuda"), keys, order)
    assert ei.value.status == ff.FF_ENONFINITE
    # the next call on finite positions is unaffected
    pos[17, 2] = 1.0
    ff.ff_morton_order_noalloc(torch.tensor(pos, device="cuda"), keys, order)
    want_keys, want_order = _oracle_order(pos)
    assert np.array_equal(keys.cpu().numpy().view(np.uint64), want_keys)
