"""The unstructured mesh variants of the input generator, and the oracle on them (no GPU).

The method applies to any triangulation (the mesh arrays of Section 2 and Eqs. 1-3 make no
assumption on valences or angles). The jittered grid alone has interior valence 6, so the
generator also cuts each cell along a random diagonal (closed fans of 4 to 8 triangles), removes
a block of cells (a hole: open fans, unused vertices, empty rows) together with two cells that
leave one vertex in two fans touching only at it, and can stretch the square (angles from about
4 to 168 degrees). These tests pin the generator's promises and check the oracle on such meshes
against exact-rational brute force and the integral identities of the unit (or stretched)
square.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1305_3122_gb300 import meshgen
from tests import exact_fe


def _signed_double_areas(m):
    x, y = m.q
    me = m.me
    return (x[me[1]] - x[me[0]]) * (y[me[2]] - y[me[0]]) - (x[me[2]] - x[me[0]]) * (y[me[1]] - y[me[0]])


def _fans(m, v):
    """The triangle fans around vertex v: connected groups of its triangles, two triangles being
    connected when they share an edge at v."""
    tris = [k for k in range(m.nme) if v in m.me[:, k]]
    adj = {k: set(int(u) for u in m.me[:, k] if u != v) for k in tris}
    seen, groups = set(), []
    for k in tris:
        if k in seen:
            continue
        stack, grp = [k], []
        seen.add(k)
        while stack:
            t = stack.pop()
            grp.append(t)
            for o in tris:
                if o not in seen and adj[o] & adj[t]:
                    seen.add(o)
                    stack.append(o)
        groups.append(grp)
    return groups


def test_default_mesh_is_unchanged_by_the_options():
    a = meshgen.square_mesh(16, 7)
    b = meshgen.square_mesh(16, 7, random_diagonals=False, hole=False, stretch=1.0)
    np.testing.assert_array_equal(a.q, b.q)
    np.testing.assert_array_equal(a.me, b.me)


@pytest.mark.parametrize("kw", [dict(random_diagonals=True), dict(random_diagonals=True, hole=True),
                                dict(random_diagonals=True, stretch=7.0), dict(hole=True)])
def test_variants_are_valid_triangulations(kw):
    m = meshgen.square_mesh(24, 3, **kw)
    assert np.all(_signed_double_areas(m) > 0)                     # counter-clockwise, none inverted
    assert m.me.min() >= 0 and m.me.max() < m.nq
    assert np.all((m.me[0] != m.me[1]) & (m.me[1] != m.me[2]) & (m.me[0] != m.me[2]))
    # every interior edge is shared by exactly two triangles, the others by one (a manifold mesh)
    e = np.sort(np.concatenate([m.me[[0, 1]], m.me[[1, 2]], m.me[[2, 0]]], axis=1), axis=0)
    _, counts = np.unique(e, axis=1, return_counts=True)
    assert set(counts.tolist()) <= {1, 2}


def test_random_diagonals_give_every_fan_size():
    m = meshgen.square_mesh(40, 9, random_diagonals=True, permute=False)
    val = np.bincount(m.me.ravel(), minlength=m.nq)
    n1 = m.N + 1
    ii, jj = np.arange(m.nq) % n1, np.arange(m.nq) // n1
    interior = (ii > 0) & (ii < m.N) & (jj > 0) & (jj < m.N)
    assert set(val[interior].tolist()) == {4, 5, 6, 7, 8}           # closed fans of every size 4..8
    edge = ~interior & ~(((ii == 0) | (ii == m.N)) & ((jj == 0) | (jj == m.N)))
    assert set(val[edge].tolist()) == {2, 3, 4}                     # open fans along the sides
    corner = ~interior & ~edge
    assert set(val[corner].tolist()) <= {1, 2}


def test_hole_gives_empty_rows_and_a_pinch_vertex():
    N = 16
    m = meshgen.square_mesh(N, 4, random_diagonals=True, hole=True, permute=False)
    val = np.bincount(m.me.ravel(), minlength=m.nq)
    n1 = N + 1
    lo, hi, p = N // 4, N // 2, (3 * N) // 4
    inside = [j * n1 + i for j in range(lo + 1, hi) for i in range(lo + 1, hi)]
    assert np.all(val[inside] == 0) and int((val == 0).sum()) == len(inside)
    pinch = (p + 1) * n1 + (p + 1)
    assert len(_fans(m, pinch)) == 2                                # two fans touch at one vertex
    assert m.nme == 2 * (N * N - (hi - lo) ** 2 - 2)


def test_stretch_spreads_the_angles():
    m = meshgen.square_mesh(30, 5, random_diagonals=True, stretch=7.0)
    x, y = m.q
    P = [np.stack([x[m.me[k]], y[m.me[k]]]) for k in range(3)]
    ang = []
    for k in range(3):
        u, v = P[(k + 1) % 3] - P[k], P[(k + 2) % 3] - P[k]
        ang.append(np.degrees(np.arccos((u * v).sum(0) / np.sqrt((u * u).sum(0) * (v * v).sum(0)))))
    ang = np.array(ang)
    assert ang.min() < 8.0 and ang.max() > 160.0
    assert x.max() == 7.0


@pytest.mark.parametrize("kw", [dict(random_diagonals=True, hole=True), dict(random_diagonals=True, stretch=5.0)])
def test_oracle_brute_force_on_unstructured_meshes(kw):
    """The oracle's CSR equals exact dense accumulation (rationals) on a mesh with fans of every
    size, empty rows and a pinch vertex: pattern structural and complete, values to 1e-13 of
    the row maximum."""
    m = meshgen.square_mesh(8, 21, **kw)
    w = meshgen.vertex_weights(m, 21)
    pts = [(Fraction(float(m.q[0, i])), Fraction(float(m.q[1, i]))) for i in range(m.nq)]
    tris = [tuple(int(v) for v in m.me[:, k]) for k in range(m.nme)]
    wf = [Fraction(float(v)) for v in w]
    for kind, name in ((oracle.MASS, "mass"), (oracle.WMASS, "wmass"), (oracle.STIFF, "stiff"),
                       (oracle.ELAS, "elas")):
        rp, ci, va = oracle.assemble(kind, m.q, m.me, w, lam=1.0, mu=0.5)
        G = exact_fe.assemble_dense(name, pts, tris, wf, lam=1, mu=Fraction(1, 2))
        n = len(G)
        dense = oracle.csr_to_dense(rp, ci, va, n)
        share = np.zeros((m.nq, m.nq), bool)
        for t in tris:
            share[np.ix_(t, t)] = True
        if name == "elas":
            share = np.kron(share, np.ones((2, 2), bool))
        for i in range(n):
            want = np.array([float(v) for v in G[i]])
            cols = ci[rp[i]:rp[i + 1]]
            np.testing.assert_array_equal(cols, np.nonzero(share[i])[0])
            if len(cols):
                assert np.abs(dense[i] - want).max() <= 1e-13 * np.abs(want).max()
            else:
                assert not np.any(want)


def _quad(rp, ci, va, u):
    rows = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
    return np.bincount(rows, weights=va * u[ci], minlength=len(rp) - 1)


@pytest.mark.parametrize("s", [1.0, 3.0])
def test_oracle_identities_on_random_diagonals(s):
    """On [0, s] x [0, 1]: sum of M = s; S 1 = 0; for u = a + bx + cy (exact in P1),
    u'Su = (b^2 + c^2) s and u'Mu = a^2 s + b^2 s^3/3 + c^2 s/3 + ab s^2 + ac s + bc s^2/2."""
    m = meshgen.square_mesh(20, 8, random_diagonals=True, stretch=s)
    rpm, cim, vam = oracle.assemble(oracle.MASS, m.q, m.me)
    assert vam.sum() == pytest.approx(s, rel=1e-13)
    rp, ci, va = oracle.assemble(oracle.STIFF, m.q, m.me)
    rm = np.maximum.reduceat(np.abs(va), rp[:-1])
    assert np.all(np.abs(_quad(rp, ci, va, np.ones(m.nq))) <= 1e-13 * rm)
    a, b, c = 0.3, -1.7, 0.6
    u = a + b * m.q[0] + c * m.q[1]
    assert u @ _quad(rp, ci, va, u) == pytest.approx((b * b + c * c) * s, rel=1e-12)
    want = a * a * s + b * b * s ** 3 / 3 + c * c * s / 3 + a * b * s * s + a * c * s + b * c * s * s / 2
    assert u @ _quad(rpm, cim, vam, u) == pytest.approx(want, rel=1e-12)


@pytest.mark.parametrize("points", ["poisson", "lattice"])
def test_disk_meshes_are_valid_delaunay_triangulations(points):
    """The unit-disk recipe: counter-clockwise triangles, a manifold mesh whose boundary edges are
    exactly the nb chords of the circle, every vertex used, the empty-circumcircle property, and
    the valences each point set promises."""
    m = meshgen.disk_mesh(3000, 5, points=points, permute=False)
    assert np.all(_signed_double_areas(m) > 0)
    e = np.sort(np.concatenate([m.me[[0, 1]], m.me[[1, 2]], m.me[[2, 0]]], axis=1), axis=0)
    ue, counts = np.unique(e, axis=1, return_counts=True)
    assert set(counts.tolist()) <= {1, 2}
    r = np.hypot(*m.q)
    bnd = ue[:, counts == 1]
    nb = int(np.sum(np.isclose(r, 1.0, rtol=0, atol=1e-15)))
    assert bnd.shape[1] == nb and np.allclose(r[bnd], 1.0, rtol=0, atol=1e-15)
    assert np.all(np.bincount(m.me.ravel(), minlength=m.nq) > 0)
    # empty circumcircles (Delaunay): no vertex strictly inside any triangle's circumcircle
    x, y = m.q
    P = m.q[:, m.me]                                        # [2, 3, nme]
    ax, ay, bx, by, cx, cy = P[0, 0], P[1, 0], P[0, 1], P[1, 1], P[0, 2], P[1, 2]
    d = 2 * (ax * (by - cy) + bx * (cy - ay) + cx * (ay - by))
    ux = ((ax * ax + ay * ay) * (by - cy) + (bx * bx + by * by) * (cy - ay) + (cx * cx + cy * cy) * (ay - by)) / d
    uy = ((ax * ax + ay * ay) * (cx - bx) + (bx * bx + by * by) * (ax - cx) + (cx * cx + cy * cy) * (bx - ax)) / d
    R2 = (ax - ux) ** 2 + (ay - uy) ** 2
    for k in range(0, m.nme, 7):                            # a sample of the triangles
        dist2 = (x - ux[k]) ** 2 + (y - uy[k]) ** 2
        assert np.all(dist2 >= R2[k] * (1 - 1e-9))
    val = np.bincount(m.me.ravel(), minlength=m.nq)
    inner = r < 1 - 1e-12
    if points == "lattice":
        assert np.mean(val[inner] == 6) > 0.9
    else:
        assert 0.01 < np.mean(val > 8) < 0.1 and val.max() >= 10


def test_oracle_identities_on_the_disk():
    """On the disk recipe (a polygon with nb vertices on the unit circle): sum of M = its area
    (nb/2) sin(2 pi/nb); S 1 = 0; u'Su = (b^2 + c^2) area for u = a + bx + cy; and x'Mx = the
    integral of x^2 over the polygon, summed over its nb triangles from the centre."""
    m = meshgen.disk_mesh(2000, 6, points="poisson")
    nb = int(np.sum(np.isclose(np.hypot(*m.q), 1.0, rtol=0, atol=1e-15)))
    area = nb / 2 * np.sin(2 * np.pi / nb)
    rpm, cim, vam = oracle.assemble(oracle.MASS, m.q, m.me)
    assert vam.sum() == pytest.approx(area, rel=1e-13)
    rp, ci, va = oracle.assemble(oracle.STIFF, m.q, m.me)
    rm = np.maximum.reduceat(np.abs(va), rp[:-1])
    assert np.all(np.abs(_quad(rp, ci, va, np.ones(m.nq))) <= 1e-13 * rm)
    a, b, c = 0.3, -1.7, 0.6
    u = a + b * m.q[0] + c * m.q[1]
    assert u @ _quad(rp, ci, va, u) == pytest.approx((b * b + c * c) * area, rel=1e-12)
    # int x^2 over the polygon: the sum over its nb triangles (0, p_k, p_k+1) of |T|/6 (x_k^2 +
    # x_k x_k+1 + x_k+1^2), the exact integral of a quadratic over a triangle with a vertex at 0
    t = 2 * np.pi * np.arange(nb) / nb
    xk, xk1 = np.cos(t), np.cos(t + 2 * np.pi / nb)
    ix2 = np.sum(0.5 * np.sin(2 * np.pi / nb) / 6 * (xk * xk + xk * xk1 + xk1 * xk1))
    x = m.q[0]
    assert x @ _quad(rpm, cim, vam, x) == pytest.approx(ix2, rel=1e-12)


def test_oracle_brute_force_on_a_small_disk():
    """A Poisson disk of about 60 vertices (valences 3 to 9) against exact dense accumulation."""
    m = meshgen.disk_mesh(60, 12, points="poisson")
    w = meshgen.vertex_weights(m, 12)
    pts = [(Fraction(float(m.q[0, i])), Fraction(float(m.q[1, i]))) for i in range(m.nq)]
    tris = [tuple(int(v) for v in m.me[:, k]) for k in range(m.nme)]
    wf = [Fraction(float(v)) for v in w]
    for kind, name in ((oracle.MASS, "mass"), (oracle.WMASS, "wmass"), (oracle.STIFF, "stiff")):
        rp, ci, va = oracle.assemble(kind, m.q, m.me, w)
        G = exact_fe.assemble_dense(name, pts, tris, wf)
        dense = oracle.csr_to_dense(rp, ci, va, m.nq)
        want = np.array([[float(v) for v in row] for row in G])
        for i in range(m.nq):
            assert np.abs(dense[i] - want[i]).max() <= 1e-13 * np.abs(want[i]).max()
