"""CPU oracle for the dipolar Barnes-Hut ferrofluid step (FP64).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only code allowed to import this
package.  The CUDA library never calls it and shares nothing with it.

The arithmetic lives in ``ora.c`` (plain C, FP64, OpenMP over target
particles); this module only marshals numpy arrays through ctypes.  Paper
passages (Polyakov et al., arXiv:1212.2934):
  * pair field / force: Sec. 2, reduced Eqs. h_dip and f_dip;
  * LJ force: Sec. 2, Eq. LJ;
  * all-pairs: Sec. 3.1, Algorithm 1;
  * octree, pseudo-particle (Eq. magCenter), traversal: Sec. 3.2;
  * Euler-Maruyama step: Sec. 4;
  * magnetisation and the Langevin function: Sec. 5, Eqs. Langevin, alpha.
Functions whose parity has no external pin are marked in their docstring.
"""
import ctypes as C
import math

import numpy as np

from . import build as _build

_lib = None

_i64 = C.c_int64
_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_u64p = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")
_u32p = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")


class BHParams(C.Structure):
    _fields_ = [("theta", C.c_double), ("leaf_max", C.c_int32), ("prec", C.c_int32),
                ("dip_scale", C.c_double), ("lj_eps", C.c_double), ("lj_sigma", C.c_double),
                ("lj_rcut", C.c_double), ("include_sr", C.c_int32), ("quad", C.c_int32)]


class Dyn(C.Structure):
    _fields_ = [("dt", C.c_double), ("gamma_t", C.c_double), ("gamma_r", C.c_double),
                ("inertia", C.c_double), ("kT", C.c_double), ("rot_noise", C.c_double),
                ("h_ext", C.c_double * 3), ("box_lo", C.c_double * 3),
                ("box_hi", C.c_double * 3), ("walls", C.c_int32), ("literal", C.c_int32),
                ("wall_eps", C.c_double), ("seed", C.c_uint64)]


def lib():
    global _lib
    if _lib is None:
        _lib = bind(_build.build())
    return _lib


def bind(path):
    """Load an oracle library at `path` and declare its functions (the tests also
    bind deliberately broken copies of the oracle to show that the pins catch them)."""
    L = C.CDLL(path)
    L.ora_set_threads.argtypes = [C.c_int]
    L.ora_get_threads.restype = C.c_int
    L.ora_pair_dipole.argtypes = [_dp, _dp, _dp, _dp, _dp]
    L.ora_pair_lj.argtypes = [_dp, C.c_double, C.c_double, C.c_double, _dp]
    L.ora_pair_lj.restype = C.c_double
    L.ora_allpairs.argtypes = [_i64, _dp, _dp, C.c_double, C.c_double, C.c_double,
                               C.c_double, C.c_int32, C.c_int32, C.c_void_p, _i64, _dp, _dp,
                               C.c_void_p]
    L.ora_bh_energy_grad.argtypes = [_i64, _dp, _dp, C.POINTER(BHParams), C.c_void_p,
                                     C.c_int32, _dp, _dp]
    L.ora_bh_energy_grad.restype = C.c_double
    L.ora_bh_vjp.argtypes = [_i64, _dp, _dp, C.POINTER(BHParams), C.c_void_p, C.c_int32,
                             _dp, _dp, _dp, _dp, C.c_void_p, C.c_void_p]
    L.ora_mz_grad.argtypes = [_i64, _dp, _dp, _dp, _dp, C.POINTER(Dyn), C.POINTER(BHParams),
                              _i64, _dp]
    L.ora_mz_grad.restype = C.c_double
    L.ora_morton.argtypes = [_i64, _dp, C.c_int32, _u64p, _dp]
    L.ora_tree.argtypes = [_i64, _dp, _dp, C.c_int32, C.c_int32, _u64p, _i64p, _dp, _i64,
                           _i32p, _i32p, _i64p, _i64p, _i64p, _dp, _dp, _dp, _dp, _dp]
    L.ora_tree.restype = _i64
    L.ora_bh.argtypes = [_i64, _dp, _dp, C.POINTER(BHParams), C.c_void_p, _i64,
                         _dp, _dp, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                         C.c_void_p, _dp, _dp]
    L.ora_bh.restype = _i64
    L.ora_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
    L.ora_normals.argtypes = [C.c_uint64, C.c_uint64, C.c_uint32, _dp]
    L.ora_wall.argtypes = [_dp, C.POINTER(Dyn), _dp, C.POINTER(C.c_double)]
    L.ora_em_step.argtypes = [_i64, _dp, _dp, _dp, _dp, _i64p, _dp, _dp, C.POINTER(Dyn),
                              C.c_uint64]
    L.ora_energy.argtypes = [_i64, _dp, _dp, _dp, _dp, _dp, C.c_void_p, C.POINTER(Dyn), _dp]
    L.ora_bh_sources.argtypes = [_i64, _dp, _dp, C.POINTER(BHParams), _i64, _i64p, _i64p,
                                 _i64]
    L.ora_bh_sources.restype = _i64
    return L


def set_threads(n: int) -> None:
    lib().ora_set_threads(int(n))


def get_threads() -> int:
    return int(lib().ora_get_threads())


def _vec3(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.ndim != 2 or a.shape[1] != 3:
        raise ValueError("expected an (n, 3) array")
    return a


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def pair_dipole(r, uk, uj):
    """Reduced dipolar field of j at k and force on k for separation r = rho_k - rho_j."""
    h = np.zeros(3)
    f = np.zeros(3)
    lib().ora_pair_dipole(np.ascontiguousarray(r, dtype=np.float64),
                          np.ascontiguousarray(uk, dtype=np.float64),
                          np.ascontiguousarray(uj, dtype=np.float64), h, f)
    return h, f


def pair_lj(r, eps=1.0, sigma=1.0, rcut=2.5):
    """Printed LJ force on k (Sec. 2) and its pair energy shifted to zero at rcut."""
    f = np.zeros(3)
    e = lib().ora_pair_lj(np.ascontiguousarray(r, dtype=np.float64), eps, sigma, rcut, f)
    return f, e


def allpairs(pos, u, dip_scale=1.0, lj_eps=0.0, lj_sigma=1.0, lj_rcut=2.5, include_sr=True,
             cut_prec="f64", only=None):
    """Exact O(N^2) field and force (Sec. 3.1).  Returns (h, f, e_sr), FP64.

    cut_prec: precision of the LJ cut-off test (the single-precision kernel
    takes it in single precision).  With ``only`` (indices), only those rows are
    computed (all particles remain sources); other rows are zero."""
    pos, u = _vec3(pos), _vec3(u)
    n = pos.shape[0]
    h = np.zeros((n, 3))
    f = np.zeros((n, 3))
    e = np.zeros(n)
    if only is not None:
        only = np.ascontiguousarray(only, dtype=np.int64)
        if only.size and (only.min() < 0 or only.max() >= n):
            raise ValueError("only: index out of range")
        optr, nonly = C.c_void_p(only.ctypes.data), int(only.size)
    else:
        optr, nonly = None, 0
    lib().ora_allpairs(n, pos, u, dip_scale, lj_eps, lj_sigma, lj_rcut, int(bool(include_sr)),
                       _prec(cut_prec), optr, nonly, h, f, _ptr(e))
    return h, f, e


def _prec(p):
    if p in (0, "f32", "float32", np.float32):
        return 0
    if p in (1, "f64", "float64", np.float64):
        return 1
    if p in (2, "mixed"):
        return 2
    raise ValueError(p)


def morton(pos, prec="f32"):
    """63-bit Morton keys in input order and the root cube (origin xyz, side)."""
    pos = _vec3(pos)
    n = pos.shape[0]
    keys = np.zeros(n, dtype=np.uint64)
    root = np.zeros(4)
    lib().ora_morton(n, pos, _prec(prec), keys, root)
    return keys, root


def tree(pos, u, prec="f32", leaf_max=1):
    """Sorted keys, order and the full DFS-preorder octree with aggregates."""
    pos, u = _vec3(pos), _vec3(u)
    n = pos.shape[0]
    skeys = np.zeros(n, dtype=np.uint64)
    order = np.zeros(n, dtype=np.int64)
    root = np.zeros(4)
    cap = 0
    args = None
    while True:
        level = np.zeros(max(cap, 1), dtype=np.int32)
        leaf = np.zeros(max(cap, 1), dtype=np.int32)
        pb = np.zeros(max(cap, 1), dtype=np.int64)
        pe = np.zeros(max(cap, 1), dtype=np.int64)
        skip = np.zeros(max(cap, 1), dtype=np.int64)
        lo = np.zeros((max(cap, 1), 3))
        side = np.zeros(max(cap, 1))
        cen = np.zeros((max(cap, 1), 3))
        c64 = np.zeros((max(cap, 1), 3))
        U64 = np.zeros((max(cap, 1), 3))
        nc = lib().ora_tree(n, pos, u, _prec(prec), int(leaf_max), skeys, order, root, cap,
                            level, leaf, pb, pe, skip, lo, side, cen, c64, U64)
        if nc <= cap:
            args = dict(keys=skeys, order=order, root=root, level=level[:nc], leaf=leaf[:nc],
                        pbegin=pb[:nc], pend=pe[:nc], skip=skip[:nc], lo=lo[:nc],
                        side=side[:nc], centre=cen[:nc], centre64=c64[:nc], U=U64[:nc])
            return args
        cap = nc


def bh(pos, u, theta, leaf_max=1, prec="f32", dip_scale=1.0, lj_eps=0.0, lj_sigma=1.0,
       lj_rcut=2.5, include_sr=True, only=None, quad=False):
    """Barnes-Hut field and force (Sec. 3.2) with the opening rule stated in ora.c.

    Returns a dict with h, f, e_sr (n x 3 / n, FP64, input order), nacc, npair,
    nopen, ncover (per-particle counts), habs, fabs (sums of the magnitudes of the
    terms summed into h and f) and ncells.  With ``only`` (indices), rows of other
    particles are zero.  quad: add each accepted cell's dipole-position term.
    """
    pos, u = _vec3(pos), _vec3(u)
    n = pos.shape[0]
    p = BHParams(theta=float(theta), leaf_max=int(leaf_max), prec=_prec(prec),
                 dip_scale=float(dip_scale), lj_eps=float(lj_eps), lj_sigma=float(lj_sigma),
                 lj_rcut=float(lj_rcut), include_sr=int(bool(include_sr)), quad=int(bool(quad)))
    h = np.zeros((n, 3))
    f = np.zeros((n, 3))
    e = np.zeros(n)
    nacc = np.zeros(n, dtype=np.int64)
    npair = np.zeros(n, dtype=np.int64)
    nopen = np.zeros(n, dtype=np.int64)
    ncover = np.zeros(n, dtype=np.int64)
    habs = np.zeros(n)
    fabs = np.zeros(n)
    if only is not None:
        only = np.ascontiguousarray(only, dtype=np.int64)
        n_only = only.shape[0]
    else:
        n_only = 0
    nc = lib().ora_bh(n, pos, u, C.byref(p), _ptr(only), n_only, h, f, _ptr(e), _ptr(nacc),
                      _ptr(npair), _ptr(nopen), _ptr(ncover), habs, fabs)
    return dict(h=h, f=f, e_sr=e, nacc=nacc, npair=npair, nopen=nopen, ncover=ncover,
                habs=habs, fabs=fabs, ncells=int(nc))


def bh_sources(pos, u, k, theta, leaf_max=1, prec="f32", lj_eps=0.0, lj_sigma=1.0,
               lj_rcut=2.5, L=None):
    """The sources of particle k (input index) in the order the Barnes-Hut traversal of
    ``bh`` visits them (Sec. 3.2): a list of ("cell", frozenset of input indices) for a
    cell used as its pseudo-particle and ("pair", frozenset({j})) for a particle summed
    exactly.  L: an oracle library from ``bind`` (default: the oracle itself)."""
    L = lib() if L is None else L
    pos, u = _vec3(pos), _vec3(u)
    n = pos.shape[0]
    p = BHParams(theta=float(theta), leaf_max=int(leaf_max), prec=_prec(prec), dip_scale=1.0,
                 lj_eps=float(lj_eps), lj_sigma=float(lj_sigma), lj_rcut=float(lj_rcut),
                 include_sr=1, quad=0)
    order = np.zeros(n, dtype=np.int64)
    cap = 4 * n + 8
    while True:
        src = np.zeros(3 * cap, dtype=np.int64)
        cnt = int(L.ora_bh_sources(n, pos, u, C.byref(p), int(k), order, src, cap))
        if cnt <= cap:
            break
        cap = cnt
    out = []
    for q in range(cnt):
        kind, a, b = src[3 * q: 3 * q + 3]
        out.append(("cell" if kind == 0 else "pair", frozenset(int(j) for j in order[a:b])))
    return out


def bh_energy_grad(pos, u, theta, leaf_max=1, prec="f64", dip_scale=1.0, lj_eps=0.0,
                   lj_sigma=1.0, lj_rcut=2.5, pos_dec=None, tree_centres=False):
    """Barnes-Hut dipolar energy E = -1/2 sum u.h and its exact gradient with the opening
    decisions taken on pos_dec (default: pos) and frozen.  Returns (E, grad_pos, grad_u).
    tree_centres: place each cell at the decision tree's centre in its own precision (as
    the Barnes-Hut field does) instead of the exact mean of the current positions."""
    pos, u = _vec3(pos), _vec3(u)
    n = pos.shape[0]
    p = BHParams(theta=float(theta), leaf_max=int(leaf_max), prec=_prec(prec),
                 dip_scale=float(dip_scale), lj_eps=float(lj_eps), lj_sigma=float(lj_sigma),
                 lj_rcut=float(lj_rcut), include_sr=0, quad=0)
    gp = np.zeros((n, 3))
    gu = np.zeros((n, 3))
    keep = None
    if pos_dec is not None:
        keep = _vec3(pos_dec)
        if keep.shape != pos.shape:
            raise ValueError("pos_dec must match pos")
    e = lib().ora_bh_energy_grad(n, pos, u, C.byref(p),
                                 None if keep is None else C.c_void_p(keep.ctypes.data),
                                 int(bool(tree_centres)), gp, gu)
    return float(e), gp, gu


def bh_vjp(pos, u, abar, bbar, theta, leaf_max=1, prec="f64", dip_scale=1.0, lj_eps=0.0,
           lj_sigma=1.0, lj_rcut=2.5, include_sr=True, pos_dec=None, tree_centres=False):
    """Vector-Jacobian product of the Barnes-Hut field h and force f (decisions of pos_dec,
    default pos, frozen): for L = sum abar.h + bbar.f returns (dL/dpos, dL/du, h, f), with h
    and f of the same frozen evaluation."""
    pos, u, abar, bbar = _vec3(pos), _vec3(u), _vec3(abar), _vec3(bbar)
    n = pos.shape[0]
    p = BHParams(theta=float(theta), leaf_max=int(leaf_max), prec=_prec(prec),
                 dip_scale=float(dip_scale), lj_eps=float(lj_eps), lj_sigma=float(lj_sigma),
                 lj_rcut=float(lj_rcut), include_sr=int(bool(include_sr)), quad=0)
    dp, du, h, f = (np.zeros((n, 3)) for _ in range(4))
    keep = None if pos_dec is None else _vec3(pos_dec)
    lib().ora_bh_vjp(n, pos, u, C.byref(p), None if keep is None else C.c_void_p(keep.ctypes.data),
                     int(bool(tree_centres)), abar, bbar, dp, du, C.c_void_p(h.ctypes.data),
                     C.c_void_p(f.ctypes.data))
    return dp, du, h, f


def mz_grad(state, dyn, nsteps, theta=0.5, leaf_max=1, prec="f64", dip_scale=1.0, lj_eps=1.0,
            lj_sigma=1.0, lj_rcut=2.5, include_sr=True):
    """Mean magnetisation <M_z> over nsteps steps from `state` (pos, vel, u, om; ids 0..n-1,
    Philox steps 0..nsteps-1) and its derivative with respect to h_ext by reverse mode.
    Returns (Mz, dMz/dh_ext[3])."""
    if dyn.literal:
        raise ValueError("the sensitivity is defined for the vector rotor form only")
    pos, vel, u, om = (_vec3(state[k]) for k in ("pos", "vel", "u", "om"))
    n = pos.shape[0]
    p = BHParams(theta=float(theta), leaf_max=int(leaf_max), prec=_prec(prec),
                 dip_scale=float(dip_scale), lj_eps=float(lj_eps), lj_sigma=float(lj_sigma),
                 lj_rcut=float(lj_rcut), include_sr=int(bool(include_sr)), quad=0)
    g = np.zeros(3)
    mz = lib().ora_mz_grad(n, pos, vel, u, om, C.byref(dyn), C.byref(p), int(nsteps), g)
    return float(mz), g


def philox4x32_10(ctr, key):
    """Philox4x32 with 10 rounds (Salmon et al., SC'11) on one counter block."""
    out = np.zeros(4, dtype=np.uint32)
    lib().ora_philox4x32_10(np.ascontiguousarray(ctr, dtype=np.uint32),
                            np.ascontiguousarray(key, dtype=np.uint32), out)
    return out


def normals(seed, step, ids):
    """Eight Box-Muller normals per id for (seed, step): array (len(ids), 8)."""
    ids = np.atleast_1d(np.asarray(ids, dtype=np.uint64))
    out = np.zeros((ids.shape[0], 8))
    z = np.zeros(8)
    for i, idv in enumerate(ids):
        lib().ora_normals(int(seed), int(step), int(idv), z)
        out[i] = z
    return out


def make_dyn(dt=1e-3, gamma_t=0.1, gamma_r=0.1, inertia=0.4, kT=1.0, rot_noise=2.0,
             h_ext=(0.0, 0.0, 0.0), box_lo=(0.0, 0.0, 0.0), box_hi=(0.0, 0.0, 0.0),
             walls=False, wall_eps=1.0, seed=1, literal=False):
    d = Dyn()
    d.dt, d.gamma_t, d.gamma_r, d.inertia, d.kT, d.rot_noise = (
        float(dt), float(gamma_t), float(gamma_r), float(inertia), float(kT), float(rot_noise))
    for a in range(3):
        d.h_ext[a] = float(h_ext[a])
        d.box_lo[a] = float(box_lo[a])
        d.box_hi[a] = float(box_hi[a])
    d.walls = int(bool(walls))
    d.literal = int(bool(literal))
    d.wall_eps = float(wall_eps)
    d.seed = int(seed)
    return d


def wall(x, dyn):
    """Wall force and energy on a particle at x (planes at box_lo - 1/2 and box_hi + 1/2)."""
    fw = np.zeros(3)
    e = C.c_double(0.0)
    lib().ora_wall(np.ascontiguousarray(x, dtype=np.float64), C.byref(dyn), fw, C.byref(e))
    return fw, e.value


def em_step(state, hdip, fint, dyn, step):
    """One Euler-Maruyama step (Sec. 4) in place on state = dict(pos, vel, u, om, id)."""
    n = state["pos"].shape[0]
    lib().ora_em_step(n, state["pos"], state["vel"], state["u"], state["om"],
                      np.ascontiguousarray(state["id"], dtype=np.int64), _vec3(hdip), _vec3(fint),
                      C.byref(dyn), int(step))


def energy(state, hdip, e_sr, dyn):
    """FP64 energies and observables: dict with e_dip, e_zeeman, e_sr, e_wall,
    e_kin_t, e_kin_r, m (3), hdip_z_mean."""
    n = state["pos"].shape[0]
    out = np.zeros(10)
    es = None if e_sr is None else np.ascontiguousarray(e_sr, dtype=np.float64)
    lib().ora_energy(n, state["pos"], state["vel"], state["u"], state["om"], _vec3(hdip),
                     _ptr(es), C.byref(dyn), out)
    return dict(e_dip=out[0], e_zeeman=out[1], e_sr=out[2], e_wall=out[3], e_kin_t=out[4],
                e_kin_r=out[5], m=out[6:9].copy(), hdip_z_mean=out[9])


def fields(state, algo, theta=0.5, leaf_max=1, prec="f64", dip_scale=1.0, lj_eps=0.0,
           lj_sigma=1.0, lj_rcut=2.5):
    """Dipolar field and interaction force for a state: AP or BH (tree precision prec)."""
    if algo == "ap":
        h, f, e = allpairs(state["pos"], state["u"], dip_scale, lj_eps, lj_sigma, lj_rcut, True,
                           prec)
        return h, f, e
    r = bh(state["pos"], state["u"], theta, leaf_max, prec, dip_scale, lj_eps, lj_sigma, lj_rcut,
           True)
    return r["h"], r["f"], r["e_sr"]


def run(state, nsteps, dyn, algo="bh", step0=0, **fkw):
    """Integrate nsteps Euler-Maruyama steps from step index step0 (in place)."""
    for s in range(nsteps):
        h, f, _ = fields(state, algo, **fkw)
        em_step(state, h, f, dyn, step0 + s)
    return state


def langevin(alpha):
    """Langevin function L(a) = coth a - 1/a (Sec. 5, Eq. Langevin), series near 0."""
    a = np.asarray(alpha, dtype=np.float64)
    out = np.empty_like(a)
    small = np.abs(a) < 1e-4
    out[small] = a[small] / 3.0
    big = ~small
    out[big] = 1.0 / np.tanh(a[big]) - 1.0 / a[big]
    return out
