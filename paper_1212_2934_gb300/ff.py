"""Python binding of libff (include/ff.h): argument marshalling only.

Every entry point has the name of its C counterpart and passes plain pointers
and sizes.  Arrays may be numpy arrays (host memory) or torch CUDA tensors
(device memory, the context's GPU), shaped (n, 3), C-contiguous, float32 or
float64.  All compute runs in the CUDA library; if libff.so is missing or
cannot be loaded this module raises instead of falling back to anything.
"""
import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libff.so")

FF_OK, FF_EINVAL, FF_ENOMEM, FF_ECUDA, FF_EDEVICE, FF_ENONFINITE, FF_ESTATE = range(7)
FF_FP32, FF_FP64, FF_MIXED = 0, 1, 2
FF_ROT_VECTOR, FF_ROT_PRINTED = 0, 1
FF_ALGO_BH, FF_ALGO_AP = 0, 1
FF_DTYPE_F32, FF_DTYPE_F64 = 0, 1
FF_HOST, FF_DEVICE = 0, 1


class FFError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (_STATUS.get(status, status), msg))
        self.status = status


_STATUS = {0: "FF_OK", 1: "FF_EINVAL", 2: "FF_ENOMEM", 3: "FF_ECUDA", 4: "FF_EDEVICE",
           5: "FF_ENONFINITE", 6: "FF_ESTATE"}


class ff_params(C.Structure):
    _fields_ = [("struct_size", C.c_uint32), ("precision", C.c_int32), ("n", C.c_int64),
                ("algo", C.c_int32), ("leaf_max", C.c_int32), ("theta", C.c_double),
                ("dt", C.c_double), ("gamma_t", C.c_double), ("gamma_r", C.c_double),
                ("inertia", C.c_double), ("kT", C.c_double), ("rot_noise", C.c_double),
                ("dip_scale", C.c_double), ("lj_eps", C.c_double), ("lj_sigma", C.c_double),
                ("lj_rcut", C.c_double), ("h_ext", C.c_double * 3), ("box_lo", C.c_double * 3),
                ("box_hi", C.c_double * 3), ("walls", C.c_int32), ("device", C.c_int32),
                ("wall_eps", C.c_double), ("seed", C.c_uint64),
                ("count_interactions", C.c_int32), ("traverse_group", C.c_int32),
                ("stream", C.c_void_p), ("rotation", C.c_int32), ("quadrupole", C.c_int32)]


class ff_energy_t(C.Structure):
    _fields_ = [("e_dip", C.c_double), ("e_zeeman", C.c_double), ("e_sr", C.c_double),
                ("e_wall", C.c_double), ("e_kin_t", C.c_double), ("e_kin_r", C.c_double),
                ("m", C.c_double * 3), ("hdip_z_mean", C.c_double)]

    def as_dict(self):
        return dict(e_dip=self.e_dip, e_zeeman=self.e_zeeman, e_sr=self.e_sr, e_wall=self.e_wall,
                    e_kin_t=self.e_kin_t, e_kin_r=self.e_kin_r, m=np.array(self.m[:]),
                    hdip_z_mean=self.hdip_z_mean)


class ff_tree_info_t(C.Structure):
    _fields_ = [("ncells", C.c_int64), ("depth", C.c_int32), ("reserved", C.c_int32),
                ("root", C.c_double * 4), ("interactions", C.c_int64), ("accepted", C.c_int64),
                ("pairs", C.c_int64), ("opened", C.c_int64)]


class ff_profile_t(C.Structure):
    _fields_ = [("ms", C.c_double * 8), ("calls", C.c_int64 * 8), ("launches", C.c_int64)]


STAGES = ("keys", "sort", "gather", "build", "aggregate", "field", "integrate", "output")

_lib = None
_vp = C.c_void_p
_st = C.c_int
_SIGS = {
    "ff_params_default": (None, [C.POINTER(ff_params)]),
    "ff_create": (_st, [C.POINTER(ff_params), C.POINTER(_vp)]),
    "ff_destroy": (_st, [_vp]),
    "ff_set_particles": (_st, [_vp, _vp, _vp, _vp, _vp, C.c_int32, C.c_int32]),
    "ff_get_particles": (_st, [_vp, _vp, _vp, _vp, _vp, C.c_int32, C.c_int32]),
    "ff_dipolar_field": (_st, [_vp, C.c_int32, C.c_double, C.c_int32, _vp, _vp, C.c_int32,
                               C.c_int32]),
    "ff_step": (_st, [_vp, C.c_int64]),
    "ff_energy": (_st, [_vp, C.POINTER(ff_energy_t)]),
    "ff_get_step": (_st, [_vp, C.POINTER(C.c_int64)]),
    "ff_set_step": (_st, [_vp, C.c_int64]),
    "ff_synchronize": (_st, [_vp]),
    "ff_tree_info": (_st, [_vp, C.POINTER(ff_tree_info_t)]),
    "ff_get_tree": (_st, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, C.c_int32]),
    "ff_get_counts": (_st, [_vp, _vp, _vp, _vp]),
    "ff_set_systems": (_st, [_vp, C.c_int32, _vp, _vp, _vp, _vp]),
    "ff_system_moments": (_st, [_vp, _vp, C.POINTER(C.c_int64), C.c_int32]),
    "ff_tune_traversal": (_st, [_vp, _vp, C.c_int32, C.c_int32, C.POINTER(C.c_int32), _vp]),
    "ff_energy_grad": (_st, [_vp, C.c_int32, C.c_double, C.POINTER(C.c_double), _vp, _vp,
                             C.c_int32, C.c_int32]),
    "ff_mz_sensitivity": (_st, [_vp, C.c_int64, C.c_int64, C.POINTER(C.c_double), _vp]),
    "ff_profile": (_st, [_vp, C.c_int32]),
    "ff_profile_read": (_st, [_vp, C.POINTER(ff_profile_t)]),
    "ff_morton_order_noalloc": (_st, [_vp, C.c_int64, _vp, _vp, _vp]),
    "ff_selftest_sort_wait": (_st, [C.c_int64, _vp]),
    "ff_selftest_record_wait": (_st, [C.c_int64, _vp]),
    "ff_schedule_count": (C.c_int32, []),
    "ff_schedule_info": (_st, [C.c_int32, _vp, _vp, _vp]),
    "ff_set_schedule": (_st, [_vp, C.c_int32]),
    "ff_tune_schedule": (_st, [_vp, C.c_int32, _vp, _vp]),
    "ff_last_error": (C.c_char_p, [_vp]),
    "ff_status_string": (C.c_char_p, [C.c_int]),
}


def lib():
    """The loaded libff.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libff.so not found at %s; build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`" % LIB_PATH)
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(ctx, status):
    if status != FF_OK:
        msg = lib().ff_last_error(ctx)
        raise FFError(status, msg.decode() if msg else "")


def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _arr_in(a, n):
    """(pointer, dtype, loc, keepalive) for an (n, 3) input array."""
    if a is None:
        return None, None, None, None
    if _is_torch(a):
        import torch

        if a.dtype not in (torch.float32, torch.float64) or tuple(a.shape) != (n, 3):
            raise ValueError("expected an (n, 3) float32/float64 tensor")
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        dt = FF_DTYPE_F64 if a.dtype == torch.float64 else FF_DTYPE_F32
        if a.is_cuda:
            return C.c_void_p(a.data_ptr()), dt, FF_DEVICE, a
        a = a.numpy()
    a = np.ascontiguousarray(a)
    if a.dtype not in (np.float32, np.float64):
        a = a.astype(np.float64)
    if a.shape != (n, 3):
        raise ValueError("expected shape (%d, 3), got %s" % (n, a.shape))
    dt = FF_DTYPE_F64 if a.dtype == np.float64 else FF_DTYPE_F32
    return C.c_void_p(a.ctypes.data), dt, FF_HOST, a


class Context:
    """Owns one ff_ctx handle; destroyed with the object."""

    def __init__(self, handle, n, precision):
        self.handle = handle
        self.n = n
        self.precision = precision

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.ff_destroy(self.handle)
            self.handle = None

    @property
    def _as_parameter_(self):
        return self.handle


def ff_params_default(**overrides):
    """Default parameters (ff_params_default) with keyword overrides; lists fill arrays."""
    p = ff_params()
    lib().ff_params_default(C.byref(p))
    for k, v in overrides.items():
        if k in ("h_ext", "box_lo", "box_hi"):
            arr = getattr(p, k)
            for i in range(3):
                arr[i] = float(v[i])
        elif k == "precision" and isinstance(v, str):
            names = {"f32": FF_FP32, "fp32": FF_FP32, "float32": FF_FP32, "f64": FF_FP64,
                     "fp64": FF_FP64, "float64": FF_FP64, "mixed": FF_MIXED}
            if v not in names:
                raise ValueError("precision must be one of %s" % sorted(names))
            p.precision = names[v]
        elif k == "algo" and isinstance(v, str):
            p.algo = FF_ALGO_AP if v == "ap" else FF_ALGO_BH
        else:
            setattr(p, k, v)
    return p


def ff_create(params):
    h = C.c_void_p()
    st = lib().ff_create(C.byref(params), C.byref(h))
    _check(None, st)
    return Context(h, int(params.n), int(params.precision))


def ff_destroy(ctx):
    if ctx.handle:
        _check(None, lib().ff_destroy(ctx.handle))
        ctx.handle = None


def ff_set_particles(ctx, pos, u, vel=None, omega=None):
    args = [_arr_in(a, ctx.n) for a in (pos, u, vel, omega)]
    dts = {a[1] for a in args if a[0] is not None}
    locs = {a[2] for a in args if a[0] is not None}
    if len(dts) != 1 or len(locs) != 1:
        raise ValueError("all arrays must share dtype and location")
    _check(ctx.handle, lib().ff_set_particles(ctx.handle, args[0][0], args[1][0], args[2][0],
                                              args[3][0], dts.pop(), locs.pop()))


def _out_pair(out, n):
    if out is None:
        return None, None, None
    p, dt, loc, keep = _arr_in(out, n)
    if loc == FF_HOST and keep is not out:
        raise ValueError("host outputs must be C-contiguous float32/float64 numpy arrays")
    return p, dt, loc


def _alloc_out(n, dtype, like):
    if like is not None and _is_torch(like) and like.is_cuda:
        import torch

        return torch.empty((n, 3), dtype=torch.float64 if dtype == np.float64 else torch.float32,
                           device=like.device)
    return np.empty((n, 3), dtype=dtype)


def ff_get_particles(ctx, dtype=np.float64, device_like=None):
    """Returns (pos, u, vel, omega) in the caller's order (numpy unless device_like is a CUDA tensor)."""
    outs = [_alloc_out(ctx.n, dtype, device_like) for _ in range(4)]
    ptrs = [_out_pair(o, ctx.n) for o in outs]
    _check(ctx.handle, lib().ff_get_particles(ctx.handle, ptrs[0][0], ptrs[1][0], ptrs[2][0],
                                              ptrs[3][0], ptrs[0][1], ptrs[0][2]))
    return tuple(outs)


def ff_dipolar_field(ctx, algo=FF_ALGO_BH, theta=0.5, include_sr=True, h_out=None, f_out=None,
                     dtype=np.float64):
    """Field and force in the caller's order; allocates host outputs when none are given."""
    if h_out is None and f_out is None:
        h_out = np.empty((ctx.n, 3), dtype=dtype)
        f_out = np.empty((ctx.n, 3), dtype=dtype)
    ph = _out_pair(h_out, ctx.n)
    pf = _out_pair(f_out, ctx.n)
    ref = ph if ph[0] is not None else pf
    if ph[0] is not None and pf[0] is not None and ph[1:] != pf[1:]:
        raise ValueError("h_out and f_out must share dtype and location")
    _check(ctx.handle, lib().ff_dipolar_field(ctx.handle, int(algo), float(theta),
                                              int(bool(include_sr)), ph[0], pf[0], ref[1], ref[2]))
    return h_out, f_out


def ff_energy_grad(ctx, algo=FF_ALGO_BH, theta=0.5, dtype=np.float64, device_like=None,
                   grads=True):
    """(E, dE/dpos, dE/du) of the dipolar energy E = -1/2 sum u.h of the current state; the
    Barnes-Hut gradient is exact with this evaluation's opening decisions frozen.  Gradients
    are numpy arrays unless device_like is a CUDA tensor.  grads=False: (E, None, None) at
    the cost of one field evaluation."""
    if not grads:
        e = C.c_double()
        _check(ctx.handle, lib().ff_energy_grad(ctx.handle, int(algo), float(theta), C.byref(e),
                                                None, None, FF_DTYPE_F64, FF_HOST))
        return e.value, None, None
    gp = _alloc_out(ctx.n, dtype, device_like)
    gu = _alloc_out(ctx.n, dtype, device_like)
    pp, pu = _out_pair(gp, ctx.n), _out_pair(gu, ctx.n)
    e = C.c_double()
    _check(ctx.handle, lib().ff_energy_grad(ctx.handle, int(algo), float(theta), C.byref(e),
                                            pp[0], pu[0], pp[1], pp[2]))
    return e.value, gp, gu


def ff_mz_sensitivity(ctx, nsteps, every=20):
    """Advances nsteps steps and returns (<M_z>, d<M_z>/dh_ext[3]) by checkpointed reverse
    mode (the state is saved every `every` steps)."""
    mz = C.c_double()
    g = np.zeros(3)
    _check(ctx.handle, lib().ff_mz_sensitivity(ctx.handle, int(nsteps), int(every), C.byref(mz),
                                               C.c_void_p(g.ctypes.data)))
    return mz.value, g


def dipolar_energy(pos, u, ctx, algo=FF_ALGO_BH, theta=0.5):
    """Differentiable dipolar energy of (pos, u) (CUDA tensors of shape (n, 3) in the
    context's precision) under torch.autograd.  The context's state is replaced by (pos, u)
    with zero velocities.  The forward pass evaluates the field once; backward sets the same
    state again and takes the gradient from ff_energy_grad."""
    return _energy_fn().apply(pos, u, ctx, int(algo), float(theta))


_ENERGY_FN = None


def _energy_fn():
    global _ENERGY_FN
    if _ENERGY_FN is None:
        import torch

        class DipolarEnergy(torch.autograd.Function):
            @staticmethod
            def forward(fctx, pos, u, ctx, algo, theta):
                # the energy only; the gradient pass runs in backward, if it is asked for
                ff_set_particles(ctx, pos.detach(), u.detach())
                e, _, _ = ff_energy_grad(ctx, algo, theta, grads=False)
                fctx.save_for_backward(pos.detach(), u.detach())
                fctx.args = (ctx, algo, theta)
                return torch.tensor(e, dtype=torch.float64, device=pos.device)

            @staticmethod
            def backward(fctx, grad_e):
                pos, u = fctx.saved_tensors
                ctx, algo, theta = fctx.args
                # the same state again: the same tree, decisions and energy
                ff_set_particles(ctx, pos, u)
                _, gp, gu = ff_energy_grad(ctx, algo, theta, dtype=_np_dtype(pos),
                                           device_like=pos)
                g = grad_e.to(gp.dtype)
                return g * gp, g * gu, None, None, None

        _ENERGY_FN = DipolarEnergy
    return _ENERGY_FN


def _np_dtype(t):
    import torch

    return np.float64 if t.dtype == torch.float64 else np.float32


def ff_step(ctx, nsteps=1):
    _check(ctx.handle, lib().ff_step(ctx.handle, int(nsteps)))


def ff_energy(ctx):
    e = ff_energy_t()
    _check(ctx.handle, lib().ff_energy(ctx.handle, C.byref(e)))
    return e.as_dict()


def ff_get_step(ctx):
    s = C.c_int64()
    _check(ctx.handle, lib().ff_get_step(ctx.handle, C.byref(s)))
    return s.value


def ff_set_step(ctx, step):
    _check(ctx.handle, lib().ff_set_step(ctx.handle, int(step)))


def ff_synchronize(ctx):
    _check(ctx.handle, lib().ff_synchronize(ctx.handle))


def ff_tree_info(ctx):
    t = ff_tree_info_t()
    _check(ctx.handle, lib().ff_tree_info(ctx.handle, C.byref(t)))
    return dict(ncells=t.ncells, depth=t.depth, root=np.array(t.root[:]),
                interactions=t.interactions, accepted=t.accepted, pairs=t.pairs, opened=t.opened)


def ff_get_tree(ctx, dtype=np.float64):
    """The last Barnes-Hut tree: dict of keys, order, pbegin, pend, skip, level, leaf, centre, moment."""
    info = ff_tree_info(ctx)
    n, nc = ctx.n, int(info["ncells"])
    keys = np.empty(n, dtype=np.uint64)
    order = np.empty(n, dtype=np.uint32)
    ints = {k: np.empty(max(nc, 1), dtype=np.int32) for k in ("pbegin", "pend", "skip", "level", "leaf")}
    cen = np.empty((max(nc, 1), 3), dtype=dtype)
    mom = np.empty((max(nc, 1), 3), dtype=dtype)
    p = lambda a: C.c_void_p(a.ctypes.data)
    _check(ctx.handle, lib().ff_get_tree(ctx.handle, p(keys), p(order), p(ints["pbegin"]),
                                         p(ints["pend"]), p(ints["skip"]), p(ints["level"]),
                                         p(ints["leaf"]), p(cen), p(mom),
                                         FF_DTYPE_F64 if dtype == np.float64 else FF_DTYPE_F32))
    out = dict(keys=keys, order=order, centre=cen[:nc], moment=mom[:nc], info=info)
    for k, v in ints.items():
        out[k] = v[:nc]
    return out


def ff_get_counts(ctx):
    """Per-particle (accepted, pairs, opened) of the last Barnes-Hut evaluation, caller order."""
    a, b, c = (np.empty(ctx.n, dtype=np.int32) for _ in range(3))
    p = lambda x: C.c_void_p(x.ctypes.data)
    _check(ctx.handle, lib().ff_get_counts(ctx.handle, p(a), p(b), p(c)))
    return a, b, c


def ff_set_systems(ctx, counts, h_ext=None, box_lo=None, box_hi=None):
    """Batched ensembles: consecutive particle ranges of the given counts become independent
    systems with per-system applied fields and boxes ((nsys, 3) arrays or None)."""
    counts = np.ascontiguousarray(counts, dtype=np.int64)
    nsys = counts.shape[0]

    def arr(a):
        if a is None:
            return None, None
        a = np.ascontiguousarray(a, dtype=np.float64).reshape(nsys, 3)
        return C.c_void_p(a.ctypes.data), a

    ph, kh = arr(h_ext)
    pl, kl = arr(box_lo)
    pu, ku = arr(box_hi)
    _check(ctx.handle, lib().ff_set_systems(ctx.handle, nsys, C.c_void_p(counts.ctypes.data),
                                            ph, pl, pu))
    ctx.nsys = nsys


def ff_system_moments(ctx, reset=False):
    """(sums (nsys, 4): u_x, u_y, u_z, h_dip_z summed over steps and particles, steps)."""
    out = np.zeros((ctx.nsys, 4))
    st = C.c_int64()
    _check(ctx.handle, lib().ff_system_moments(ctx.handle, C.c_void_p(out.ctypes.data),
                                               C.byref(st), int(bool(reset))))
    return out, st.value


TRAVERSE_GROUPS = (1, 2, 4, 8, 16, 32)


def ff_schedules():
    """{index: (group, threads per block, blocks per SM)} of the traversal launch schedules."""
    out = {}
    for i in range(1, int(lib().ff_schedule_count()) + 1):
        g, t, b = C.c_int32(), C.c_int32(), C.c_int32()
        _check(None, lib().ff_schedule_info(i, C.byref(g), C.byref(t), C.byref(b)))
        out[i] = (g.value, t.value, b.value)
    return out


def ff_set_schedule(ctx, index):
    _check(ctx.handle, lib().ff_set_schedule(ctx.handle, int(index)))


def ff_tune_schedule(ctx, reps=3):
    """Times the traversal with every launch schedule, keeps the fastest for the context and
    returns (best index, {index: ms})."""
    k = int(lib().ff_schedule_count())
    ms = np.zeros(k, dtype=np.float32)
    best = C.c_int32()
    _check(ctx.handle, lib().ff_tune_schedule(ctx.handle, int(reps), C.byref(best),
                                              C.c_void_p(ms.ctypes.data)))
    return best.value, {i + 1: float(m) for i, m in enumerate(ms)}


def ff_tune_traversal(ctx, groups=None, reps=3):
    """Times the traversal with each lane group (all six when groups is None), keeps the
    fastest for the context and returns (best_group, {group: ms})."""
    cand = list(TRAVERSE_GROUPS if groups is None else groups)
    ms = np.zeros(len(cand), dtype=np.float32)
    best = C.c_int32()
    if groups is None:
        gp, ng = None, 0
    else:
        garr = (C.c_int32 * len(cand))(*cand)
        gp, ng = C.cast(garr, C.c_void_p), len(cand)
    _check(ctx.handle, lib().ff_tune_traversal(ctx.handle, gp, ng, int(reps), C.byref(best),
                                               C.c_void_p(ms.ctypes.data)))
    return best.value, {g: float(m) for g, m in zip(cand, ms)}


def ff_profile(ctx, enable=True):
    _check(ctx.handle, lib().ff_profile(ctx.handle, int(bool(enable))))


def ff_profile_read(ctx):
    """Accumulated stage times (ms), timed executions per stage and kernel launches."""
    p = ff_profile_t()
    _check(ctx.handle, lib().ff_profile_read(ctx.handle, C.byref(p)))
    return dict(ms={k: p.ms[i] for i, k in enumerate(STAGES)},
                calls={k: p.calls[i] for i, k in enumerate(STAGES)}, launches=p.launches)


FF_NOALLOC_MAX_N = 131072


def ff_morton_order_noalloc(pos, keys_out, order_out, stream=None):
    """Allocation-free Morton ordering of an (n, 3) float32 CUDA tensor into uint64 keys and
    int32 order tensors (device); see include/ff.h.  stream: a torch CUDA stream or None.
    The tensors are checked before the call (the library sees only raw pointers)."""
    def need(ok, what):
        if not ok:
            raise ValueError("ff_morton_order_noalloc: " + what)

    import torch

    need(getattr(pos, "is_cuda", False) and pos.dtype == torch.float32 and pos.dim() == 2
         and pos.shape[1] == 3 and pos.is_contiguous(),
         "pos must be a contiguous (n, 3) float32 CUDA tensor")
    n = int(pos.shape[0])
    for t, size, name in ((keys_out, 8, "keys_out"), (order_out, 4, "order_out")):
        need(getattr(t, "is_cuda", False) and t.is_contiguous() and t.element_size() == size
             and not t.is_floating_point() and not t.is_complex() and t.numel() >= n
             and t.device == pos.device,
             "%s must be a contiguous %d-byte integer CUDA tensor on pos's device with at "
             "least n elements" % (name, size))
    sp = None if stream is None else C.c_void_p(stream.cuda_stream)
    _check(None, lib().ff_morton_order_noalloc(C.c_void_p(pos.data_ptr()), n,
                                               C.c_void_p(keys_out.data_ptr()),
                                               C.c_void_p(order_out.data_ptr()), sp))
    return keys_out, order_out


def ff_selftest_sort_wait(n=20000, stream=None):
    """Runs the sort with its first tile withholding its counts (include/ff.h); raises FFError
    unless the bounded wait ran out and reported its flag."""
    sp = None if stream is None else C.c_void_p(stream.cuda_stream)
    _check(None, lib().ff_selftest_sort_wait(int(n), sp))


def ff_selftest_record_wait(nrec=20000, stream=None):
    """Runs the gradient's one-pass record scan with its first tile withholding its count
    (include/ff.h); raises FFError unless the bounded wait ran out and reported its flag."""
    sp = None if stream is None else C.c_void_p(stream.cuda_stream)
    _check(None, lib().ff_selftest_record_wait(int(nrec), sp))


def ff_last_error(ctx=None):
    m = lib().ff_last_error(ctx.handle if ctx is not None else None)
    return m.decode() if m else ""


def ff_status_string(status):
    return lib().ff_status_string(int(status)).decode()


def exported_symbols():
    """Names of the functions include/ff.h declares (as bound here)."""
    return sorted(_SIGS)
