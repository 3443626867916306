"""Host-side checks of the C library boundary (no GPU needed).

The library builds for sm_103a and loads; it exports every function that
include/ff.h declares and nothing else; parameter validation in ff_create rejects bad input
before touching a device and reports why through ff_last_error(NULL).
"""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libff():
    from paper_1212_2934_gb300 import _build, ff

    _build.build()
    return ff


def declared_functions():
    src = open(os.path.join(ROOT, "include", "ff.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ff_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("ff_create", "ff_destroy", "ff_set_particles", "ff_dipolar_field", "ff_step",
                     "ff_energy"):
        assert required in names


def test_library_exports_every_declared_symbol(libff):
    L = ctypes.CDLL(libff.LIB_PATH)
    for name in declared_functions():
        assert hasattr(L, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", libff.LIB_PATH], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r"\bT (ff_\w+)", out))
    assert set(declared_functions()) <= exported
    # and nothing else: internal launchers and the static CUDA runtime stay local
    defined = {ln.split()[-1] for ln in out.splitlines() if len(ln.split()) >= 3}
    assert defined == set(declared_functions()), sorted(defined ^ set(declared_functions()))
    # the binding covers the same names
    assert set(libff.exported_symbols()) == set(declared_functions())


def test_params_default_and_validation(libff):
    p = libff.ff_params_default(n=100)
    assert p.struct_size == ctypes.sizeof(libff.ff_params)
    assert p.theta == 0.5 and p.leaf_max == 1 and p.dt == 1e-3 and p.rot_noise == 2.0
    bad = [dict(n=0), dict(leaf_max=0), dict(leaf_max=65), dict(theta=-1.0), dict(dt=0.0),
           dict(inertia=0.0), dict(precision=7), dict(algo=3),
           dict(walls=1, box_lo=(0, 0, 0), box_hi=(1, 0, 1)), dict(lj_eps=1.0, lj_rcut=0.0)]
    for kw in bad:
        q = libff.ff_params_default(n=100, **{k: v for k, v in kw.items() if k != "n"})
        if "n" in kw:
            q.n = kw["n"]
        with pytest.raises(libff.FFError) as ei:
            libff.ff_create(q)
        assert ei.value.status == libff.FF_EINVAL
        assert libff.ff_last_error(None)
    q = libff.ff_params_default(n=100)
    q.struct_size = 8
    with pytest.raises(libff.FFError):
        libff.ff_create(q)


def test_status_strings(libff):
    assert libff.ff_status_string(0) == "FF_OK"
    assert libff.ff_status_string(5) == "FF_ENONFINITE"


def test_struct_layout_matches_header(libff, tmp_path):
    # compile a tiny C program against include/ff.h and compare sizes/offsets
    prog = tmp_path / "lay.c"
    prog.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "ff.h"\n'
        'int main(void){printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(ff_params),'
        ' offsetof(ff_params, seed), offsetof(ff_params, stream), sizeof(ff_energy_t),'
        ' sizeof(ff_tree_info_t), offsetof(ff_params, h_ext));return 0;}\n')
    exe = tmp_path / "lay"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)],
                   check=True)
    vals = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    P = libff.ff_params
    assert vals == [ctypes.sizeof(P), P.seed.offset, P.stream.offset,
                    ctypes.sizeof(libff.ff_energy_t), ctypes.sizeof(libff.ff_tree_info_t),
                    P.h_ext.offset]


def test_noalloc_binding_rejects_bad_tensors(libff):
    """The allocation-free entry point sees raw pointers only; its binding refuses tensors
    whose bytes the library would misread (host memory, wrong dtype, shape or length)."""
    torch = pytest.importorskip("torch")
    n = 64
    pos = torch.zeros((n, 3), dtype=torch.float32)
    keys = torch.zeros(n, dtype=torch.int64)
    order = torch.zeros(n, dtype=torch.int32)
    cases = [(pos, keys, order),                      # host tensors
             (pos.double(), keys, order),
             (pos[:, :2], keys, order),
             (pos.t(), keys, order)]
    for p, k, o in cases:
        with pytest.raises(ValueError):
            libff.ff_morton_order_noalloc(p, k, o)
