"""Seeded input generators: closed, outward-oriented surfaces of the stated sizes."""
import collections

import numpy as np

from paper_1901_08393_gb300 import inputs


def _closed(m):
    c = collections.Counter()
    for t in m.tris:
        for k in range(3):
            a, b = int(t[k]), int(t[(k + 1) % 3])
            c[(min(a, b), max(a, b))] += 1
    return all(v % 2 == 0 for v in c.values())


def _volume(m):
    v, t = m.verts, m.tris
    return np.einsum("ij,ij->i", v[t[:, 0]], np.cross(v[t[:, 1]], v[t[:, 2]])).sum() / 6


def test_sizes_and_closedness():
    assert inputs.cube_mesh(4).N == 192
    assert inputs.fichera_mesh().N == 48  # the paper's initial Fichera mesh size (Sec. 3.2)
    assert inputs.graded_cube_mesh(71).N == 60492
    assert inputs.icosphere_mesh(3).N == 180 and inputs.tetra_mesh(3).N == 36
    for m in (inputs.cube_mesh(3), inputs.workload_polycube_adaptive(), inputs.fichera_mesh(2),
              inputs.graded_cube_mesh(6), inputs.tetra_mesh(3), inputs.icosphere_mesh(2)):
        assert _closed(m), m.name
        assert _volume(m) > 0, m.name  # outward orientation
        assert m.tris.dtype == np.int32 and m.verts.dtype == np.float64
    assert abs(_volume(inputs.fichera_mesh()) - 7.0) < 1e-12
    assert abs(_volume(inputs.graded_cube_mesh(7)) - 1.0) < 1e-12


def test_polycube_deterministic_and_seeded():
    a = inputs.polycube_mesh(6, 0.5, 1)
    b = inputs.polycube_mesh(6, 0.5, 1)
    c = inputs.polycube_mesh(6, 0.5, 2)
    assert np.array_equal(a.tris, b.tris) and np.array_equal(a.verts, b.verts)
    assert a.N != c.N or not np.array_equal(a.verts, c.verts)
    occ = inputs.polycube_occupancy(6, 0.5, 1)
    from scipy import ndimage
    lab, n = ndimage.label(occ, structure=ndimage.generate_binary_structure(3, 1))
    assert n == 1  # one face-connected component
    lab2, _ = ndimage.label(np.pad(~occ, 1, constant_values=True),
                            structure=ndimage.generate_binary_structure(3, 1))
    assert lab2.max() == 1  # no enclosed cavity


def test_splitmix_uniform():
    r = inputs.SplitMix64(123)
    u = r.uniforms(20000)
    assert 0 <= u.min() and u.max() < 1 and abs(u.mean() - 0.5) < 0.01
    r2 = inputs.SplitMix64(123)
    assert r2.uniform() == u[0]


def test_batch_and_requests_shapes():
    ms = inputs.batch_meshes(count=4, n_hi=3000)
    assert len(ms) == 4 and all(_closed(m) for m in ms)
    reqs = inputs.serving_requests(count=6)
    assert all(3 <= r["steps"] <= 6 for r in reqs)
    assert all(5000 <= r["target"] <= 40000 for r in reqs)
    # the start mesh is the shape subdivided toward target / 1.13^(steps - 1), never
    # coarser than the shape's description
    for r in reqs:
        start = r["target"] / 1.13 ** (r["steps"] - 1)
        assert r["mesh"].N >= r["coarse"] and 0.4 * start <= r["mesh"].N <= 2.5 * start, r
    assert all(b["t_arrive"] > a["t_arrive"] for a, b in zip(reqs, reqs[1:]))
    assert all(_closed(r["mesh"]) and _volume(r["mesh"]) > 0 for r in reqs)
