"""Pins for the oracle's opening rule (Sec. 3.2: a cell stands in for its particles
when it is "far enough"; Eq. magCenter places its pseudo-particle at the geometric
centre).

The rule the oracle implements (the paper states no criterion): particle k uses cell
C as its pseudo-particle iff k is not in C, side_C^2 < theta^2 |rho_k - c_C|^2 with
c_C the geometric centre of C's particles and side_C the dyadic cube side (strict),
and, with the LJ term on, the distance from rho_k to C's cube is at least r_cut.

Each case below is a handful of particles at small integer coordinates, so every
quantity of the rule is exact in single and double precision; the expected source
lists were worked out by hand from that rule (the derivation is in each comment) and
are compared with the sources the oracle's own traversal visits
(``oracle.bh_sources``).  The cases are chosen so that each plausible misreading of
the rule changes at least one list: `<=` for `<`, the cube centre for the geometric
centre, side for side^2, theta for theta^2, no LJ clause, and the LJ clause on the
centre distance instead of the cube distance; ``test_misreadings_are_caught`` builds
the oracle with each misreading planted and checks exactly that.
"""
import os
import subprocess
import tempfile

import numpy as np
import pytest

CELL, PAIR = "cell", "pair"


def _src(*items):
    return [(kind, frozenset(ids)) for kind, ids in items]


# Each case: positions, theta, LJ on?, {target input index: expected sources in order}.
CASES = {
    # Root cube: origin (0,1,1), side 8 (largest extent, along x).  Level 1: p0 in
    # octant 0; p1 (8,1,1) and p2 (8,3,3) share the x-high octant F (x = 8 clamps into
    # the top half), side 4, side^2 = 16, geometric centre (8,2,2).
    # For p0 = (0,2,2): |p0 - c_F|^2 = 64, theta^2 d^2 = 16 = side^2, so the strict test
    # fails and F is opened.  Its children (level 2, side 2) are one-particle leaves
    # (p1 relative (8,0,0) and p2 relative (8,2,2) differ in their y and z digits), each
    # at d^2 = 66: 4 < 16.5, accepted.
    # (<= instead of <, side instead of side^2 (4 < 16) or theta instead of theta^2
    # (16 < 32) would all accept F whole.)
    "tie": (
        [[0, 2, 2], [8, 1, 1], [8, 3, 3]], 0.5, False,
        {0: _src((CELL, [1]), (CELL, [2])),
         # p1: the octant-0 cell {p0} (side 4, centre (0,2,2), d^2 = 66: 16 < 16.5) is
         # accepted; its sibling leaf p2 (side 2, d^2 = 8: 4 < 2 fails) is a pair.
         1: _src((CELL, [0]), (PAIR, [2])),
         2: _src((CELL, [0]), (PAIR, [1]))},
    ),
    # Same root as "tie" (origin (0,1,1), side 8).  F = {p1 (8,1,1), p2 (8,3,1)}: cube
    # [4,8] x [1,5] x [1,5], cube centre (6,3,3), geometric centre (8,2,1).
    # For p0 = (0,2,2): to the geometric centre d^2 = 64 + 0 + 1 = 65, theta^2 d^2 =
    # 16.25 > 16: F is accepted whole.  (To the cube centre d^2 = 38, 9.5 < 16: F would be
    # opened into its two leaves.)
    "geometric_centre": (
        [[0, 2, 2], [8, 1, 1], [8, 3, 1]], 0.5, False,
        {0: _src((CELL, [1, 2]))},
    ),
    # LJ on (r_cut = 2.5, r_cut^2 = 6.25), theta = 1.  Root: origin (0,1,1), side 8.
    # Octant 0 holds p0 (0,2,2) and p1 (3,2,2), split at level 2 (x digit 0 and 1);
    # the x-high octant F holds p2 (8,1,1) and p3 (8,3,3) (cube [4,8] x [1,5] x [1,5],
    # geometric centre (8,2,2)).  For p1 = (3,2,2):
    #  * leaf p0: cube [0,2] x [1,3] x [1,3], side^2 4 < d^2 9 passes, but the cube is 1
    #    away (1 < 6.25): not accepted, summed as a pair;
    #  * F: 16 < 25 passes, but its cube is 1 away: opened (its centre is 5 away, beyond
    #    r_cut, so a clause on the centre distance would accept it);
    #  * leaf p2: cube [6,8] x [1,3] x [1,3], 4 < 27, cube 3 away (9 >= 6.25): accepted;
    #  * leaf p3: cube [6,8] x [3,5] x [3,5], 4 < 27, cube distance^2 9 + 1 + 1 = 11:
    #    accepted.
    "lj_clause": (
        [[0, 2, 2], [3, 2, 2], [8, 1, 1], [8, 3, 3]], 1.0, True,
        {1: _src((PAIR, [0]), (CELL, [2]), (CELL, [3]))},
    ),
    # Eight particles at the octant centres of [2,6]^3 (root origin (2,2,2), side 4):
    # eight one-particle leaves of side 2 (side^2 4), visited in octant order
    # 4x + 2y + z (the x digit highest).  For p4 = (2,2,2), octant 0: the face
    # neighbours are at d^2 = 16, theta^2 d^2 = 4 = side^2 (strict test fails: pairs),
    # the edge neighbours at 32 and the corner at 48 (accepted).  Input order is
    # scrambled so the list order is the octant order, not the input order.
    "octants": (
        [[6, 6, 6], [2, 2, 6], [6, 2, 2], [2, 6, 2], [2, 2, 2], [6, 6, 2], [2, 6, 6],
         [6, 2, 6]], 0.5, False,
        {4: _src((PAIR, [1]), (PAIR, [3]), (CELL, [6]), (PAIR, [2]), (CELL, [7]),
                 (CELL, [5]), (CELL, [0]))},
    ),
}


def _run_case(ora, name, prec, L=None):
    pos, theta, lj, expect = CASES[name]
    pos = np.array(pos, dtype=np.float64)
    u = np.tile([0.0, 0.0, 1.0], (pos.shape[0], 1))
    got = {}
    for k in expect:
        got[k] = ora.bh_sources(pos, u, k, theta, prec=prec, lj_eps=1.0 if lj else 0.0,
                                lj_rcut=2.5, L=L)
    return got, expect


@pytest.mark.parametrize("prec", ["f32", "f64", "mixed"])
@pytest.mark.parametrize("name", sorted(CASES))
def test_hand_derived_sources(ora, name, prec):
    got, expect = _run_case(ora, name, prec)
    assert got == expect


def test_sources_match_counts(ora):
    """The listed sources are the ones the field sums count (bh's nacc / npair)."""
    from paper_1212_2934_gb300 import synth

    n = 300
    pos = synth.rsa_cube(n, synth.box_side_for_fraction(n, 0.1), 5)
    u = synth.isotropic_moments(n, 5)
    ref = ora.bh(pos, u, 0.6, 1, "f32", lj_eps=1.0)
    for k in (0, 17, 123, 299):
        src = ora.bh_sources(pos, u, k, 0.6, prec="f32", lj_eps=1.0)
        assert sum(kind == CELL for kind, _ in src) == ref["nacc"][k]
        assert sum(kind == PAIR for kind, _ in src) == ref["npair"][k]
        # every other particle appears in exactly one source
        seen = [j for _, ids in src for j in ids]
        assert sorted(seen) == sorted(set(range(n)) - {k})


# One-line misreadings of the rule, planted in a copy of the oracle's source.
MUTANTS = {
    "le_for_lt": [("if (!(s2 < td)) return 0;", "if (!(s2 <= td)) return 0;"),
                  ("if (!(s2 < theta2 * d2)) return 0;", "if (!(s2 <= theta2 * d2)) return 0;")],
    "cube_centre": [
        ("float dx = xk[0] - c[0], dy = xk[1] - c[1], dz = xk[2] - c[2];",
         "float dx = xk[0] - (lo[0] + 0.5f * side), dy = xk[1] - (lo[1] + 0.5f * side), "
         "dz = xk[2] - (lo[2] + 0.5f * side);"),
        ("double dx = xk[0] - c[0], dy = xk[1] - c[1], dz = xk[2] - c[2];",
         "double dx = xk[0] - (lo[0] + 0.5 * side), dy = xk[1] - (lo[1] + 0.5 * side), "
         "dz = xk[2] - (lo[2] + 0.5 * side);")],
    "side_for_side2": [("float s2 = side * side;", "float s2 = side;"),
                       ("double s2 = side * side;", "double s2 = side;")],
    "theta_for_theta2": [("theta2_d = p->theta * p->theta;", "theta2_d = p->theta;")],
    "no_lj_clause": [("    if (use_rcut) {\n        float t[3];", "    if (0) {\n        float t[3];"),
                     ("    if (use_rcut) {\n        double t[3];", "    if (0) {\n        double t[3];")],
    "lj_on_centre_distance": [("if (b2 < rcut2) return 0;", "if (d2 < rcut2) return 0;")],
}


def _build_mutants(tmp):
    from oracle import build as obuild

    src = open(obuild.SRC).read()
    procs = {}
    for name, edits in MUTANTS.items():
        text = src
        for old, new in edits:
            assert text.count(old) >= 1, (name, old)
            text = text.replace(old, new)
        path = os.path.join(tmp, name + ".c")
        with open(path, "w") as fh:
            fh.write(text)
        lib = os.path.join(tmp, "lib" + name + ".so")
        procs[name] = (lib, subprocess.Popen(["gcc", *obuild.CFLAGS, "-o", lib, path, "-lm"],
                                             stdout=subprocess.PIPE, stderr=subprocess.STDOUT))
    libs = {}
    for name, (lib, p) in procs.items():
        out, _ = p.communicate()
        assert p.returncode == 0, out.decode(errors="replace")
        libs[name] = lib
    return libs


def test_misreadings_are_caught(ora):
    """Every planted misreading changes at least one hand-derived source list."""
    with tempfile.TemporaryDirectory() as tmp:
        libs = _build_mutants(tmp)
        for name, path in libs.items():
            L = ora.bind(path)
            caught = []
            for case in CASES:
                for prec in ("f32", "f64"):
                    got, expect = _run_case(ora, case, prec, L=L)
                    if got != expect:
                        caught.append((case, prec))
            assert caught, "misreading %s is not caught by any case" % name
