"""Pins of the oracle's ZZ estimator (Eq. 1.6), Doerfler marking (Eq. 2.6) and
newest-vertex bisection (Fig. 3) against brute force and invariants."""
import collections
import itertools
import math

import numpy as np
import pytest

import oracle as O
from paper_1901_08393_gb300 import inputs
from tests._golden import capacity_reference


def _edges(tris):
    c = collections.Counter()
    for t in tris:
        for k in range(3):
            a, b = int(t[k]), int(t[(k + 1) % 3])
            c[(min(a, b), max(a, b))] += 1
    return c


def _normals(v, t):
    return np.cross(v[t[:, 1]] - v[t[:, 0]], v[t[:, 2]] - v[t[:, 0]])


# ------------------------------------------------------------------ ZZ
def test_zz_brute_force():
    m = inputs.workload_polycube_adaptive()
    t = O.canonical(m.verts, m.tris)
    rng = np.random.default_rng(1)
    x = rng.random(m.N)
    eta2 = O.zz(m.verts, t, x)
    area, diam = O.geometry(m.verts, t)
    # independent: nodal averages by dictionary, L2 norm by the edge-midpoint rule
    num = collections.defaultdict(float)
    den = collections.defaultdict(float)
    for i, tri in enumerate(t):
        for z in tri:
            num[int(z)] += area[i] * x[i]
            den[int(z)] += area[i]
    for i, tri in enumerate(t):
        d = [num[int(z)] / den[int(z)] - x[i] for z in tri]
        mids = [(d[k] + d[(k + 1) % 3]) / 2 for k in range(3)]
        l2 = area[i] / 3 * sum(q * q for q in mids)
        P = m.verts[tri]
        h = max(np.linalg.norm(P[k] - P[(k + 1) % 3]) for k in range(3))
        assert abs(eta2[i] - h * l2) <= 1e-13 * max(h * l2, 1e-300) + 1e-300
    e1 = O.zz(m.verts, t, x, h_mode=1)
    assert np.allclose(e1, eta2 * np.sqrt(area) / diam, rtol=1e-14, atol=0)


def test_zz_constant_is_zero():
    m = inputs.cube_mesh(2)
    t = O.canonical(m.verts, m.tris)
    eta2 = O.zz(m.verts, t, np.full(m.N, 0.37))
    assert np.max(eta2) < 1e-30


def test_zz_permutation_equivariant():
    m = inputs.cube_mesh(2)
    t = O.canonical(m.verts, m.tris)
    x = np.random.default_rng(3).random(m.N)
    # relabel vertices: same geometry, same eta2
    perm = np.random.default_rng(4).permutation(m.M)
    inv = np.argsort(perm)
    v2 = m.verts[perm]
    t2 = inv[t].astype(np.int32)
    assert np.allclose(O.zz(v2, t2, x), O.zz(m.verts, t, x), rtol=1e-13)


# ------------------------------------------------------------------ Doerfler
def _min_card(eta2, theta):
    tot = math.fsum(eta2)
    for k in range(len(eta2) + 1):
        for S in itertools.combinations(range(len(eta2)), k):
            if math.fsum(eta2[list(S)]) >= theta * tot * (1 - 1e-12):
                return k
    return len(eta2)


def test_dorfler_minimal_brute_force():
    rng = np.random.default_rng(5)
    for trial in range(40):
        n = int(rng.integers(1, 11))
        eta2 = rng.random(n) ** 3
        theta = float(rng.choice([0.2, 0.5, 0.8]))
        m = O.dorfler(eta2, theta).astype(bool)
        key = eta2.astype(np.float32)
        assert math.fsum(eta2[m]) >= theta * math.fsum(eta2) * (1 - 1e-12)
        kmin = _min_card(eta2, theta)
        cut = key[m].min()
        ties = int(np.sum(key == cut))
        assert kmin <= m.sum() <= kmin + ties - 1
        # marked set is upward closed in the ordering
        assert np.all(key[~m] < cut) if (~m).any() else True


def test_dorfler_ties_and_extremes():
    eta2 = np.array([1.0, 1.0, 1.0, 1.0, 0.5])
    assert O.dorfler(eta2, 0.5).tolist() == [1, 1, 1, 1, 0]
    eta2 = np.array([0.1, 0.4, 0.2, 0.3])
    assert O.dorfler(eta2, 0.5).tolist() == [0, 1, 0, 1]
    assert O.dorfler(eta2, 1.0).tolist() == [1, 1, 1, 1]
    assert O.dorfler(np.zeros(5), 0.5).tolist() == [0] * 5
    assert O.dorfler(np.zeros(0), 0.5).tolist() == []


# ------------------------------------------------------------------ NVB
def test_canonical_longest_edge_first():
    m = inputs.tetra_mesh(2)
    v = m.verts + np.random.default_rng(6).normal(scale=0.05, size=m.verts.shape)
    t = O.canonical(v, m.tris)
    for a, b in zip(t, m.tris):
        assert sorted(a) == sorted(b)
        assert tuple(a) in {tuple(np.roll(b, -k)) for k in range(3)}  # rotation only
        L = [np.linalg.norm(v[a[k]] - v[a[(k + 1) % 3]]) for k in range(3)]
        assert L[0] >= L[1] and L[0] >= L[2]


def _check_conforming(v, t, old_M):
    E = _edges(t)
    assert all(c % 2 == 0 for c in E.values())
    # no hanging node: no vertex strictly inside another edge
    for (a, b) in E:
        pa, pb = v[a], v[b]
        d = pb - pa
        L2 = d @ d
        w = v - pa
        s = (w @ d) / L2
        perp = np.linalg.norm(w - np.outer(s, d), axis=1)
        inside = (s > 1e-12) & (s < 1 - 1e-12) & (perp < 1e-12 * math.sqrt(L2))
        assert not inside.any()


def test_nvb_uniform_refinement():
    m = inputs.cube_mesh(1)
    v, t = m.verts, O.canonical(m.verts, m.tris)
    area0 = O.geometry(v, t)[0].sum()
    for level in range(3):
        M, N = v.shape[0], t.shape[0]
        n0 = _normals(v, t)
        v, t, parent, kept = O.refine(v, t, np.ones(N, dtype=np.uint8))
        assert t.shape[0] == 2 * N and not kept.any()
        assert np.all(t[:, 2] >= M)  # the newest vertex is opposite the reference edge
        assert np.all(np.einsum("ij,ij->i", _normals(v, t), n0[parent]) > 0)
        _check_conforming(v, t, M)
        assert abs(O.geometry(v, t)[0].sum() / area0 - 1) < 1e-14
        # all descendants of the right isosceles triangles stay right isosceles
        L = np.sort(np.stack([np.linalg.norm(v[t[:, k]] - v[t[:, (k + 1) % 3]], axis=1)
                              for k in range(3)], 1), 1)
        assert np.allclose(L[:, 0], L[:, 1]) and np.allclose(L[:, 2], L[:, 0] * math.sqrt(2))


def test_nvb_closure_and_patterns():
    m = inputs.workload_polycube_adaptive()
    v, t = m.verts, O.canonical(m.verts, m.tris)
    rng = np.random.default_rng(7)
    seen = set()
    for trial in range(4):
        N, M = t.shape[0], v.shape[0]
        marked = (rng.random(N) < 0.15).astype(np.uint8)
        v2, t2, parent, kept = O.refine(v, t, marked)
        counts = np.bincount(parent, minlength=N)
        seen |= set(counts.tolist())
        assert np.all(counts[marked.astype(bool)] >= 2)  # every marked element bisected
        assert np.all(kept == (counts[parent] == 1))
        K = int(kept.sum())
        assert kept[:K].all() and not kept[K:].any()  # unrefined triangles first
        assert np.all(np.diff(parent[:K]) > 0) and np.all(np.diff(parent[K:]) >= 0)
        assert np.array_equal(t2[:K], t[parent[:K]])
        _check_conforming(v2, t2, M)
        assert abs(O.geometry(v2, t2)[0].sum() / O.geometry(v, t)[0].sum() - 1) < 1e-13
        # new vertices are edge midpoints, numbered by first appearance
        assert np.all(v2[:M] == v)
        v, t = v2, t2
    assert {1, 2, 3, 4} <= seen


def test_nvb_bisec3_marks_all_edges():
    m = inputs.cube_mesh(1)
    t = O.canonical(m.verts, m.tris)
    marked = np.zeros(m.N, dtype=np.uint8)
    marked[0] = 1
    v2, t2, parent, kept = O.refine(m.verts, t, marked, bisec3=True)
    assert np.sum(parent == 0) == 4
    _check_conforming(v2, t2, m.M)


def test_adaptive_loop_monotone():
    """Alg. 1 on the primal P0 space: nested meshes -> non-decreasing Cap_l
    (Corollary, App. A) up to the quadrature error of the entries (a few 1e-6
    relative on coarse meshes), bounded by the reference value of Sec. 3.1.
    The 12-triangle cube starts with a constant solution (all indicators vanish
    up to rounding), so the first steps refine uniformly."""
    ref = capacity_reference()["unit_cube_capacity"]
    m = inputs.cube_mesh(1)
    hist = O.adaptive_run(m.verts, m.tris, theta=0.5, max_N=500)
    caps = [h["cap"] for h in hist]
    assert len(hist) >= 5
    assert all(b > a * (1 - 1e-5) for a, b in zip(caps, caps[1:]))
    assert caps[-1] - caps[0] > 5e-3
    assert caps[-1] < ref
    assert hist[0]["marked"].all()  # vanishing estimator -> uniform step
    adaptive = [h for h in hist[:-1] if h["eta2_total"] > 1e-10]
    assert adaptive and all(h["marked"].sum() > 0 for h in adaptive)
    assert any(h["marked"].sum() < h["N"] for h in adaptive)  # symmetric tie groups may be whole


def test_dorfler_large_sets_meet_eq_2_6_minimally():
    """Beyond one summation block (128 sorted elements): the marked set satisfies
    theta * sum(eta^2) <= sum over the set with exact sums, and dropping its last
    tie group of single-precision keys breaks the inequality (minimality up to the
    rounding of the running sums)."""
    rng = np.random.default_rng(17)
    for N in (129, 1000, 5000):
        for theta in (0.2, 0.5, 0.9):
            eta2 = rng.random(N) ** 4
            eta2[: N // 7] = eta2[N // 7]  # exact ties across block boundaries
            m = O.dorfler(eta2, theta).astype(bool)
            tot = math.fsum(eta2)
            assert math.fsum(eta2[m]) >= theta * tot * (1 - 1e-12)
            key = eta2.astype(np.float32)
            cut = key[m].min()
            assert not np.any(key[~m] > cut) and not np.any(key[~m] == cut)  # upward closed, ties closed
            rest = m & (key > cut)
            assert math.fsum(eta2[rest]) < theta * tot * (1 + 1e-12)
