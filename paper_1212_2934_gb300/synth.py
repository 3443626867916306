"""Seeded synthetic ensembles shaped like the paper's workloads.

Geometry and random numbers only: this module holds none of the method's
arithmetic (no field, force, tree or integrator code), so the CUDA path and
the CPU oracle can both be fed from it.  Every generator takes an explicit
seed and uses numpy's PCG64, whose streams are identical on x86-64 and
aarch64.

Workloads (the paper, Sec. 4-5: particles placed at random in a cubic
container, N from 1e3 to 1e6, volume fraction of a few per cent):
  * ``dense_cube``  - N = 4096 centres in [0, 16]^3, minimum separation 1.0
    (packing fraction 0.52, above the random-sequential-addition jamming
    limit): a 16^3 lattice of spacing 16/15, jittered, then relaxed by
    hard-sphere Monte Carlo sweeps;
  * ``rsa_cube``    - random sequential addition with a hard core of 1.0 in
    a cube sized for a given volume fraction (cell-grid neighbour search);
  * ``dilute_cubes`` / ``batched_ensembles`` - many dilute hard-core gases at
    once (uniform centres, overlapping ones redrawn) for batched ensembles of
    log-uniform sizes and a linear grid of applied fields;
  * ``isotropic_moments`` - unit moments from normalised Gaussian triples.
Lengths are in units of the hard-core diameter.
"""
import math

import numpy as np

__all__ = ["box_side_for_fraction", "isotropic_moments", "rsa_cube", "dense_cube",
           "uniform_cube", "chains_cube", "slab_monolayer", "batched_sizes", "batched_ensembles",
           "Ensemble", "make_ensemble"]


def box_side_for_fraction(n: int, phi: float, diameter: float = 1.0) -> float:
    """Edge of the cube holding n spheres of the given diameter at volume fraction phi."""
    return (n * (math.pi / 6.0) * diameter ** 3 / phi) ** (1.0 / 3.0)


def isotropic_moments(n: int, seed: int) -> np.ndarray:
    """n unit vectors, isotropic on the sphere (normalised Gaussian triples)."""
    rng = np.random.default_rng([seed, 0xC0FFEE])
    g = rng.standard_normal((n, 3))
    nrm = np.sqrt((g * g).sum(axis=1))
    bad = nrm < 1e-12
    while bad.any():
        g[bad] = rng.standard_normal((int(bad.sum()), 3))
        nrm = np.sqrt((g * g).sum(axis=1))
        bad = nrm < 1e-12
    return g / nrm[:, None]


def uniform_cube(n: int, side: float, seed: int) -> np.ndarray:
    """n centres uniform in [0, side]^3 with no hard core."""
    rng = np.random.default_rng([seed, 0xBEEF])
    return rng.uniform(0.0, side, (n, 3))


def _drop_later_conflicts(cand: np.ndarray, dmin: float) -> np.ndarray:
    """Mask of candidates kept when every later member of a close pair is dropped."""
    from scipy.spatial import cKDTree

    keep = np.ones(cand.shape[0], dtype=bool)
    if cand.shape[0] < 2:
        return keep
    pairs = cKDTree(cand).query_pairs(np.nextafter(dmin, 0.0), output_type="ndarray")
    if pairs.size:
        keep[np.maximum(pairs[:, 0], pairs[:, 1])] = False
    return keep


def rsa_cube(n: int, side: float, seed: int, dmin: float = 1.0) -> np.ndarray:
    """Random sequential addition of n centres in [0, side]^3, pairwise >= dmin apart.

    Candidates are drawn in batches; a candidate is rejected if it lies closer
    than dmin to an accepted centre (found through a grid of cells small
    enough to hold one centre each) or to an earlier candidate of its batch.
    """
    rng = np.random.default_rng([seed, 0x5EED])
    G = max(1, int(math.ceil(side * math.sqrt(3.0) / dmin)))
    a = side / G
    reach = int(math.ceil(dmin / a))
    offs = []
    for dx in range(-reach, reach + 1):
        for dy in range(-reach, reach + 1):
            for dz in range(-reach, reach + 1):
                gap = [max(abs(d) - 1, 0) * a for d in (dx, dy, dz)]
                if gap[0] ** 2 + gap[1] ** 2 + gap[2] ** 2 < dmin * dmin:
                    offs.append((dx, dy, dz))
    offs = np.array(offs, dtype=np.int64)
    grid = np.full(G * G * G, -1, dtype=np.int32)
    pos = np.empty((n, 3))
    cnt = 0
    d2min = dmin * dmin
    stall = 0
    while cnt < n:
        m = int(min(max(4096, 2 * (n - cnt)), 1 << 17))
        cand = rng.uniform(0.0, side, (m, 3))
        cell = np.minimum((cand / a).astype(np.int64), G - 1)
        ok = np.ones(m, dtype=bool)
        for o in offs:
            c = cell + o
            inb = np.all((c >= 0) & (c < G), axis=1)
            rows = np.nonzero(inb & ok)[0]
            if rows.size == 0:
                continue
            cc = c[rows]
            idx = grid[(cc[:, 0] * G + cc[:, 1]) * G + cc[:, 2]]
            has = idx >= 0
            if not has.any():
                continue
            r = rows[has]
            d = cand[r] - pos[idx[has]]
            close = (d * d).sum(axis=1) < d2min
            ok[r[close]] = False
        surv = np.nonzero(ok)[0]
        if surv.size:
            surv = surv[_drop_later_conflicts(cand[surv], dmin)]
        take = surv[: n - cnt]
        if take.size == 0:
            stall += 1
            if stall > 50:
                raise RuntimeError("random sequential addition jammed at %d of %d" % (cnt, n))
            continue
        stall = 0
        pos[cnt: cnt + take.size] = cand[take]
        tc = cell[take]
        grid[(tc[:, 0] * G + tc[:, 1]) * G + tc[:, 2]] = np.arange(cnt, cnt + take.size,
                                                                    dtype=np.int32)
        cnt += take.size
    return pos


def dense_cube(n_side: int = 16, side: float = 16.0, seed: int = 1, sweeps: int = 200,
               max_step: float = 0.1, dmin: float = 1.0) -> np.ndarray:
    """n_side^3 centres in [0, side]^3 at minimum separation dmin, beyond RSA jamming.

    A cubic lattice of spacing side/(n_side-1) is jittered by at most
    (spacing - dmin)/2 per axis, then `sweeps` hard-sphere Monte Carlo sweeps
    move every centre at once by a uniform step in [-max_step, max_step]^3; a
    move is kept only if the new centre stays in the cube and is at least dmin
    from the old and the proposed centres of every other particle (so any set
    of kept moves is overlap-free).
    """
    from scipy.spatial import cKDTree

    rng = np.random.default_rng([seed, 0xD15C])
    sp = side / (n_side - 1)
    g = np.arange(n_side) * sp
    pos = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3)
    jit = max(sp - dmin, 0.0) / 2.0
    pos = np.clip(pos + rng.uniform(-jit, jit, pos.shape), 0.0, side)
    n = pos.shape[0]
    r = np.nextafter(dmin, 0.0)
    for _ in range(sweeps):
        new = pos + rng.uniform(-max_step, max_step, pos.shape)
        ok = np.all((new >= 0.0) & (new <= side), axis=1)
        allp = np.concatenate([pos, new])
        pairs = cKDTree(allp).query_pairs(r, output_type="ndarray")
        if pairs.size:
            a, b = pairs[:, 0], pairs[:, 1]
            ia, ib = a % n, b % n
            a_new, b_new = a >= n, b >= n
            diff = ia != ib
            # new_i against old_j or new_j (j != i) rejects i
            ok[ia[diff & a_new]] = False
            ok[ib[diff & b_new]] = False
        pos = np.where(ok[:, None], new, pos)
    return pos


def chains_cube(nchains: int, length: int, side: float, seed: int,
                spacing: float = 1.0, dmin: float = 1.0):
    """Straight chains of touching particles with isotropic axes, overlap-free.

    Returns (pos, u): moments lie along each chain's axis with a random sign
    per chain (head-to-tail).  Chains are drawn in batches (uniform start,
    isotropic axis) and a chain is rejected if any of its centres leaves the
    cube or comes closer than dmin to a centre of an accepted chain or of an
    earlier chain of its batch (random sequential addition of rods).  Accepted
    centres are searched through two k-d trees, a large one rebuilt rarely and
    a small one holding the chains accepted since, so that a batch costs time
    in proportion to its own size.
    """
    from scipy.spatial import cKDTree

    rng = np.random.default_rng([seed, 0xC4A1])
    placed = []
    placed_u = []
    t = np.arange(length) * spacing
    main_pts = np.empty((0, 3))
    main_tree = None
    recent = []
    recent_tree = None
    count = 0
    idle = 0
    while count < nchains:
        if idle > 200:
            raise RuntimeError("chains_cube: no chain fits any more (%d of %d placed); the "
                               "cube is too small for isotropic rods" % (count, nchains))
        m = max(1024, min(8192, 2 * (nchains - count)))
        axis = rng.standard_normal((m, 3))
        axis /= np.linalg.norm(axis, axis=1)[:, None]
        start = rng.uniform(0.0, side, (m, 3))
        pts = start[:, None, :] + t[None, :, None] * axis[:, None, :]
        ok = np.all((pts >= 0.0) & (pts <= side), axis=(1, 2))
        flat_q = pts.reshape(-1, 3)
        for tree in (main_tree, recent_tree):
            if tree is not None:
                d, _ = tree.query(flat_q, k=1, distance_upper_bound=dmin)
                ok &= ~np.any((d < dmin).reshape(m, length), axis=1)
        idx = np.nonzero(ok)[0]
        if idx.size:
            flat = pts[idx].reshape(-1, 3)
            owner = np.repeat(np.arange(idx.size), length)
            pairs = cKDTree(flat).query_pairs(np.nextafter(dmin, 0.0), output_type="ndarray")
            keep = np.ones(idx.size, dtype=bool)
            if pairs.size:
                oa, ob = owner[pairs[:, 0]], owner[pairs[:, 1]]
                cross = oa != ob
                keep[np.maximum(oa[cross], ob[cross])] = False
            idx = idx[keep][: nchains - count]
        if idx.size == 0:
            idle += 1
            continue
        idle = 0
        sgn = np.where(rng.uniform(size=idx.size) < 0.5, 1.0, -1.0)
        placed.append(pts[idx].reshape(-1, 3))
        placed_u.append(np.repeat(sgn[:, None] * axis[idx], length, axis=0))
        count += idx.size
        recent.append(pts[idx].reshape(-1, 3))
        rpts = np.concatenate(recent)
        if rpts.shape[0] > max(0.25 * main_pts.shape[0], 65536):
            main_pts = np.concatenate([main_pts, rpts])
            main_tree = cKDTree(main_pts)
            recent, recent_tree = [], None
        else:
            recent_tree = cKDTree(rpts)
    pos = np.concatenate(placed)
    u = np.concatenate(placed_u)
    return pos, u


def slab_monolayer(n: int, area_fraction: float, seed: int, gap: float = 0.05,
                   dmin: float = 1.0):
    """A monolayer between two walls (Sec. 4: a parallelepiped of height 2.1 R as the
    confinement).  In diameters the wall planes are 2.1 R = 1.05 apart; with planes half a
    diameter beyond the box (the walls' convention) the centres lie in z in [0, gap],
    gap = 0.05.  In the plane: random sequential addition in a square of side
    sqrt(n (pi/4) / area_fraction), centres >= dmin apart (3-d distances).
    Returns (pos, side)."""
    from scipy.spatial import cKDTree

    side = math.sqrt(n * (math.pi / 4.0) / area_fraction)
    rng = np.random.default_rng([seed, 0x51AB])
    placed = np.empty((0, 3))
    tree = None
    idle = 0
    while placed.shape[0] < n:
        if idle > 200:
            raise RuntimeError("slab_monolayer jammed at %d of %d" % (placed.shape[0], n))
        m = max(1024, 2 * (n - placed.shape[0]))
        cand = np.column_stack([rng.uniform(0.0, side, m), rng.uniform(0.0, side, m),
                                rng.uniform(0.0, gap, m)])
        ok = np.ones(m, dtype=bool)
        if tree is not None:
            d, _ = tree.query(cand, k=1, distance_upper_bound=dmin)
            ok &= ~(d < dmin)
        idx = np.nonzero(ok)[0]
        if idx.size:
            idx = idx[_drop_later_conflicts(cand[idx], dmin)][: n - placed.shape[0]]
        if idx.size == 0:
            idle += 1
            continue
        idle = 0
        placed = np.concatenate([placed, cand[idx]])
        tree = cKDTree(placed)
    return placed, side


def batched_sizes(nsys: int = 256, nmin: int = 1024, nmax: int = 65536):
    """Deterministic log-uniform quantiles: N_i = round(nmin (nmax/nmin)^((i + 1/2) / nsys))."""
    r = nmax / nmin
    return np.array([int(round(nmin * r ** ((i + 0.5) / nsys))) for i in range(nsys)],
                    dtype=np.int64)


def dilute_cubes(sizes, sides, seed: int, dmin: float = 1.0, rounds: int = 200):
    """Hard-core gases for many dilute systems at once: uniform centres in each
    system's cube, then the later member of every pair closer than dmin is drawn
    again until no such pair is left.  Systems are placed side by side along x
    (gap > dmin) so one neighbour search serves them all.  Returns the
    concatenated centres, each system in its own [0, side]^3."""
    from scipy.spatial import cKDTree

    rng = np.random.default_rng([seed, 0xD11E])
    sizes = np.asarray(sizes, dtype=np.int64)
    sides = np.asarray(sides, dtype=np.float64)
    owner = np.repeat(np.arange(sizes.shape[0]), sizes)
    shift = np.concatenate([[0.0], np.cumsum(sides + 2.0 * dmin)[:-1]])
    side_of = sides[owner]
    pos = rng.uniform(0.0, 1.0, (owner.shape[0], 3)) * side_of[:, None]
    for _ in range(rounds):
        glob = pos.copy()
        glob[:, 0] += shift[owner]
        pairs = cKDTree(glob).query_pairs(np.nextafter(dmin, 0.0), output_type="ndarray")
        if pairs.size == 0:
            return pos
        redo = np.unique(np.maximum(pairs[:, 0], pairs[:, 1]))
        pos[redo] = rng.uniform(0.0, 1.0, (redo.shape[0], 3)) * side_of[redo, None]
    raise RuntimeError("dilute_cubes did not converge; the systems are too dense")


def batched_ensembles(nsys: int = 256, phi: float = 0.02, hmax: float = 5.0, seed: int = 1):
    """Independent dilute systems of log-uniform sizes with applied fields 0 .. hmax (along z)
    on a linear grid, assigned to the sizes by a seeded permutation.  Returns dict with the
    concatenated positions and moments, sizes, sides, fields (nsys, 3), box_lo, box_hi."""
    sizes = batched_sizes(nsys)
    amps = hmax * np.arange(nsys) / max(nsys - 1, 1)
    perm = np.random.default_rng([seed, 0xF1E1D]).permutation(nsys)
    fields = np.zeros((nsys, 3))
    fields[:, 2] = amps[perm]
    sides = np.array([box_side_for_fraction(int(n), phi) for n in sizes])
    pos = dilute_cubes(sizes, sides, seed)
    u = isotropic_moments(int(sizes.sum()), seed * 100003 + 7)
    return dict(pos=pos, u=u, sizes=sizes, sides=sides,
                fields=fields, box_lo=np.zeros((nsys, 3)),
                box_hi=np.repeat(sides[:, None], 3, axis=1))


class Ensemble(dict):
    """A synthetic workload: positions, moments and the run parameters (plain dict)."""


def make_ensemble(name: str, seed: int = 1, n: int = None) -> Ensemble:
    """The named workloads, sizes and parameters as used by the tests and the benchmark.

    'dense4096'  : N = 4096 in [0,16]^3 (min separation 1), FP64, h_ext = 0.5 z.
    'phi05'      : N = 1,048,576 (or n) at volume fraction 0.05, FP32, h_ext = z.
    'dilute'     : N = n at volume fraction 0.02 (batched-ensemble member shape).
    """
    e = Ensemble(name=name, seed=seed)
    common = dict(dt=1e-3, gamma_t=0.1, gamma_r=0.1, inertia=0.4, kT=1.0, rot_noise=2.0,
                  dip_scale=1.0, lj_eps=1.0, lj_sigma=1.0, lj_rcut=2.5, wall_eps=1.0,
                  theta=0.5, leaf_max=1, seed=seed)
    e.update(common)
    if name == "dense4096":
        side = 16.0
        pos = dense_cube(16, side, seed)
        e.update(precision="f64", h_ext=(0.0, 0.0, 0.5), side=side)
    elif name == "phi05":
        n = 1048576 if n is None else int(n)
        side = box_side_for_fraction(n, 0.05)
        pos = rsa_cube(n, side, seed)
        e.update(precision="f32", h_ext=(0.0, 0.0, 1.0), side=side)
    elif name == "dilute":
        n = 4096 if n is None else int(n)
        side = box_side_for_fraction(n, 0.02)
        pos = rsa_cube(n, side, seed)
        e.update(precision="f32", h_ext=(0.0, 0.0, 1.0), side=side)
    else:
        raise ValueError(name)
    e["pos"] = pos
    e["u"] = isotropic_moments(pos.shape[0], seed)
    e["n"] = pos.shape[0]
    e["box_lo"] = (0.0, 0.0, 0.0)
    e["box_hi"] = (side, side, side)
    return e
