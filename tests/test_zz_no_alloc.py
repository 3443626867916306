"""The allocation-free Morton ordering entry point (ff_morton_order_noalloc).

It exists for callers that cannot allocate device memory (stream capture in
progress, memory owned by the application's pool, loops that must not stall
on an allocation); it uses a fixed scratch array inside the library instead.
Its keys and order must equal, bit for bit, what the allocating path reports
through ff_get_tree for the same single-precision positions, on two calls in a
row (the scratch keeps the previous call's contents).  This file is collected
last on purpose.
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
