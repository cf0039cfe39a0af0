"""Seeded synthetic surface meshes: the inputs shared by the CUDA path, the oracle,
the tests and the benchmark.

This module builds geometry only.  It holds none of the boundary-element method's
arithmetic (no quadrature, no operator, no estimator, no refinement), so both sides
of a parity check can take their input from here without sharing any of the code
under test.

Workloads follow the shapes the paper computes on (Section 3): the unit cube
(Section 3.1), Fichera-like polycubes with re-entrant edges and corners
(Section 3.2), plus a sphere family for the Cap = r limit (Section 1.2) and
tetrahedra / rotated, scaled cubes for mixed request streams.

Conventions
-----------
* vertices: float64 array (M, 3); triangles: int32 array (N, 3), 0-based,
  counter-clockwise seen from outside (outward normal).
* Voxel surfaces: every unit face between an occupied and an empty voxel is one
  quad; vertices are merged by integer coordinates and numbered in lexicographic
  order of (x, y, z); each quad is rotated so that its lexicographically smallest
  corner comes first and is split along the diagonal from that corner.
* Faces are emitted direction by direction (-x, +x, -y, +y, -z, +z), voxels in
  C order of ``occ[x, y, z]`` within a direction.
* Random numbers come from SplitMix64 (Steele, Lea, Flood 2014): state advances by
  0x9E3779B97F4A7C15, output mixed by the 30/27/31 xor-shift-multiply finaliser;
  a uniform double is the top 53 bits times 2**-53.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

_M64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 generator (Steele, Lea and Flood, OOPSLA 2014)."""

    def __init__(self, seed: int):
        self.state = seed & _M64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _M64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def uniforms(self, n: int) -> np.ndarray:
        return np.array([self.uniform() for _ in range(n)], dtype=np.float64)

    def randint(self, lo: int, hi: int) -> int:
        """Uniform integer in [lo, hi] (inclusive)."""
        return lo + int(self.uniform() * (hi - lo + 1))

    def normal(self) -> float:
        u1 = max(self.uniform(), 1e-300)
        u2 = self.uniform()
        return math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2)


@dataclass
class Mesh:
    verts: np.ndarray  # (M, 3) float64
    tris: np.ndarray   # (N, 3) int32
    name: str = ""

    @property
    def M(self) -> int:
        return int(self.verts.shape[0])

    @property
    def N(self) -> int:
        return int(self.tris.shape[0])


# Outward quads of a unit voxel at the origin, per direction, counter-clockwise
# seen from outside.  Order of directions: -x, +x, -y, +y, -z, +z.
_DIRS = [(-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)]
_QUADS = [
    [(0, 0, 0), (0, 0, 1), (0, 1, 1), (0, 1, 0)],  # -x
    [(1, 0, 0), (1, 1, 0), (1, 1, 1), (1, 0, 1)],  # +x
    [(0, 0, 0), (1, 0, 0), (1, 0, 1), (0, 0, 1)],  # -y
    [(0, 1, 0), (0, 1, 1), (1, 1, 1), (1, 1, 0)],  # +y
    [(0, 0, 0), (0, 1, 0), (1, 1, 0), (1, 0, 0)],  # -z
    [(0, 0, 1), (1, 0, 1), (1, 1, 1), (0, 1, 1)],  # +z
]


def voxel_surface_int(occ: np.ndarray, sub: int = 1):
    """Boundary of a voxel set as triangles on integer coordinates.

    ``sub`` splits every voxel face into sub x sub squares (a uniform mesh of the
    same surface).  Returns (ivert (M,3) int64, tris (N,3) int32).
    """
    occ = np.asarray(occ, dtype=bool)
    pad = np.pad(occ, 1, constant_values=False)
    quads = []
    for d, (dx, dy, dz) in enumerate(_DIRS):
        nb = pad[1 + dx:pad.shape[0] - 1 + dx, 1 + dy:pad.shape[1] - 1 + dy,
                 1 + dz:pad.shape[2] - 1 + dz]
        face = occ & ~nb
        vox = np.argwhere(face)  # C order of occ[x, y, z]
        if vox.size == 0:
            continue
        base = np.array(_QUADS[d], dtype=np.int64)  # (4, 3)
        q = vox[:, None, :].astype(np.int64) * sub + base[None, :, :] * sub  # (F,4,3)
        if sub > 1:
            # split each face into sub x sub squares, spanned by the quad edges
            e1 = (base[1] - base[0])
            e3 = (base[3] - base[0])
            parts = []
            for a in range(sub):
                for b in range(sub):
                    o = vox.astype(np.int64) * sub + base[0] * sub + a * e1 + b * e3
                    parts.append(np.stack([o, o + e1, o + e1 + e3, o + e3], axis=1))
            q = np.stack(parts, axis=1).reshape(-1, 4, 3)
        quads.append(q)
    if not quads:
        return np.zeros((0, 3), np.int64), np.zeros((0, 3), np.int32)
    Q = np.concatenate(quads, axis=0)
    # rotate each quad so that its lexicographically smallest corner is first
    G = int(Q.max()) + 2
    key = (Q[:, :, 0] * G + Q[:, :, 1]) * G + Q[:, :, 2]
    first = np.argmin(key, axis=1)
    idx = (first[:, None] + np.arange(4)[None, :]) % 4
    Q = np.take_along_axis(Q, idx[:, :, None], axis=1)
    corners = Q.reshape(-1, 3)
    uniq, inv = np.unique(corners, axis=0, return_inverse=True)
    inv = inv.reshape(-1, 4)
    tris = np.empty((2 * inv.shape[0], 3), dtype=np.int32)
    tris[0::2] = inv[:, [0, 1, 2]]
    tris[1::2] = inv[:, [0, 2, 3]]
    return uniq.astype(np.int64), tris


def cube_mesh(n: int = 4) -> Mesh:
    """Unit cube [0,1]^3, every face split into an n x n grid of squares, each cut
    into 2 triangles: 12 n^2 triangles (n = 4 gives 192)."""
    occ = np.ones((1, 1, 1), dtype=bool)
    iv, tris = voxel_surface_int(occ, sub=n)
    return Mesh(iv.astype(np.float64) / n, tris, f"cube{n}")


def graded_cube_mesh(n: int = 71) -> Mesh:
    """Unit cube with a tensor grid on each face graded toward the face edges and
    corners: node k of n on every axis sits at g(k/n), g(u) = 2u^2 for u <= 1/2 and
    1 - 2(1-u)^2 above.  12 n^2 triangles (n = 71 gives 60,492)."""
    occ = np.ones((1, 1, 1), dtype=bool)
    iv, tris = voxel_surface_int(occ, sub=n)
    u = iv.astype(np.float64) / n
    g = np.where(u <= 0.5, 2.0 * u * u, 1.0 - 2.0 * (1.0 - u) * (1.0 - u))
    return Mesh(g, tris, f"graded_cube{n}")


def polycube_occupancy(g: int, p: float, seed: int) -> np.ndarray:
    """Bernoulli(p) voxels of a g^3 grid (draws in C order of occ[x,y,z]), largest
    6-connected component (ties: the one holding the smallest flat index), enclosed
    cavities filled.  Guaranteed non-empty: an all-empty draw keeps voxel 0."""
    from scipy import ndimage

    rng = SplitMix64(seed)
    u = rng.uniforms(g * g * g).reshape(g, g, g)
    occ = u < p
    if not occ.any():
        occ.flat[0] = True
    st = ndimage.generate_binary_structure(3, 1)
    lab, nlab = ndimage.label(occ, structure=st)
    if nlab > 1:
        sizes = np.bincount(lab.ravel())[1:]
        best = sizes.max()
        cands = [c + 1 for c in range(nlab) if sizes[c] == best]
        flat = lab.ravel()
        firsts = [int(np.flatnonzero(flat == c)[0]) for c in cands]
        keep = cands[int(np.argmin(firsts))]
        occ = lab == keep
    # fill cavities: empty voxels not face-connected to the padded outside
    pad = np.pad(~occ, 1, constant_values=True)
    elab, _ = ndimage.label(pad, structure=st)
    outside = elab == elab[0, 0, 0]
    inner_empty = ~outside[1:-1, 1:-1, 1:-1] & ~occ
    return occ | inner_empty


def polycube_mesh(g: int = 6, p: float = 0.5, seed: int = 1, sub: int = 1,
                  scale: float = 1.0) -> Mesh:
    """Seeded random polycube surface (unit voxels times ``scale``)."""
    occ = polycube_occupancy(g, p, seed)
    iv, tris = voxel_surface_int(occ, sub=sub)
    return Mesh(iv.astype(np.float64) * (scale / sub), tris, f"polycube{g}_p{p}_s{seed}")


def fichera_mesh(sub: int = 1) -> Mesh:
    """Fichera cube [-1,1]^3 minus [0,1]^3 as 7 unit voxels (Section 3.2 shape)."""
    occ = np.ones((2, 2, 2), dtype=bool)
    occ[1, 1, 1] = False
    iv, tris = voxel_surface_int(occ, sub=sub)
    return Mesh(iv.astype(np.float64) / sub - 1.0, tris, f"fichera{sub}")


def _subdivided_polyhedron(corners: np.ndarray, faces, k: int):
    """Split every triangular face (a,b,c) into k^2 triangles; vertices merged by
    their exact integer barycentric weights on the polyhedron's corners."""
    keymap = {}
    verts = []

    def vid(weights):
        key = tuple(sorted((v, w) for v, w in weights if w))
        if key not in keymap:
            keymap[key] = len(verts)
            verts.append(sum(w * corners[v] for v, w in weights) / k)
        return keymap[key]

    tris = []
    for (a, b, c) in faces:
        def P(i, j):
            return vid([(a, k - i - j), (b, i), (c, j)])
        for i in range(k):
            for j in range(k - i):
                tris.append((P(i, j), P(i + 1, j), P(i, j + 1)))
                if i + j + 1 < k:
                    tris.append((P(i + 1, j), P(i + 1, j + 1), P(i, j + 1)))
    return np.array(verts, dtype=np.float64), np.array(tris, dtype=np.int32)


def _orient_outward(verts: np.ndarray, tris: np.ndarray, center) -> np.ndarray:
    t = tris.copy()
    a, b, c = verts[t[:, 0]], verts[t[:, 1]], verts[t[:, 2]]
    nrm = np.cross(b - a, c - a)
    flip = np.einsum("ij,ij->i", nrm, (a + b + c) / 3.0 - np.asarray(center)) < 0
    t[flip] = t[flip][:, [0, 2, 1]]
    return t


def tetra_mesh(k: int = 4, edge: float = 1.0) -> Mesh:
    """Regular tetrahedron with the given edge length, each face split into k^2."""
    c = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], dtype=np.float64)
    c *= edge / (2.0 * math.sqrt(2.0))
    faces = [(0, 1, 2), (0, 3, 1), (0, 2, 3), (1, 3, 2)]
    v, t = _subdivided_polyhedron(c, faces, k)
    return Mesh(v, _orient_outward(v, t, [0, 0, 0]), f"tetra{k}")


def icosphere_mesh(k: int = 4, r: float = 1.0) -> Mesh:
    """Polyhedron inscribed in the sphere of radius r: icosahedron faces split into
    k^2 triangles, vertices pushed to the sphere (20 k^2 triangles)."""
    ph = (1.0 + math.sqrt(5.0)) / 2.0
    c = np.array([[-1, ph, 0], [1, ph, 0], [-1, -ph, 0], [1, -ph, 0],
                  [0, -1, ph], [0, 1, ph], [0, -1, -ph], [0, 1, -ph],
                  [ph, 0, -1], [ph, 0, 1], [-ph, 0, -1], [-ph, 0, 1]], dtype=np.float64)
    faces = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
             (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
             (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
             (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    v, t = _subdivided_polyhedron(c, faces, k)
    v = v / np.linalg.norm(v, axis=1, keepdims=True) * r
    return Mesh(v, _orient_outward(v, t, [0, 0, 0]), f"icosphere{k}")


def random_rotation(rng: SplitMix64) -> np.ndarray:
    """Uniform random rotation from a normalised Gaussian quaternion."""
    q = np.array([rng.normal() for _ in range(4)])
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


def transformed(mesh: Mesh, R: np.ndarray, scale: float = 1.0, shift=(0.0, 0.0, 0.0)) -> Mesh:
    v = (mesh.verts @ np.asarray(R).T) * scale + np.asarray(shift, dtype=np.float64)
    return Mesh(np.ascontiguousarray(v), mesh.tris.copy(), mesh.name + "_xf")


# ---------------------------------------------------------------- workloads
def workload_cube192() -> Mesh:
    """Unit cube, 4x4 squares per face, 2 triangles per square: 192 triangles."""
    return cube_mesh(4)


def workload_polycube_adaptive() -> Mesh:
    """Initial mesh of the adaptive polycube run: 6^3 grid, p = 0.5, seed 1."""
    return polycube_mesh(6, 0.5, 1)


def workload_graded_cube_60k() -> Mesh:
    """Unit cube, tensor-graded toward edges and corners, 60,492 triangles."""
    return graded_cube_mesh(71)


def batch_meshes(count: int = 256, seed: int = 4, n_lo: int = 500, n_hi: int = 30000):
    """Batch of uniform polycube meshes: grid g ~ U{3..10}, p ~ U[0.3, 0.7], a
    target size log-uniform in [n_lo, n_hi]; every voxel face is split into s x s
    squares with s the smallest integer reaching the target."""
    rng = SplitMix64(seed)
    out = []
    for b in range(count):
        g = rng.randint(3, 10)
        p = 0.3 + 0.4 * rng.uniform()
        target = math.exp(math.log(n_lo) + (math.log(n_hi) - math.log(n_lo)) * rng.uniform())
        s_seed = rng.next_u64() & 0xFFFFFFFF
        occ = polycube_occupancy(g, p, s_seed)
        iv1, t1 = voxel_surface_int(occ, 1)
        faces = t1.shape[0] // 2
        s = max(1, int(math.ceil(math.sqrt(target / (2.0 * faces)))))
        iv, tris = voxel_surface_int(occ, sub=s)
        out.append(Mesh(iv.astype(np.float64) / s, tris, f"batch{b}_g{g}_s{s}"))
    return out


def serving_requests(count: int = 2000, seed: int = 5, rate: float = 50.0, n_lo: int = 5000,
                     n_hi: int = 40000, growth: float = 1.13):
    """Poisson stream of capacity requests with 3..6 adaptive steps ending at 5k..40k
    triangles from shapes described by 100..2000 triangles.

    Per request, in this order of draws: the inter-arrival gap (exponential, ``rate``
    per second); the shape kind (a third each: seeded polycubes with g in 3..6 and
    p in [0.3, 0.7], cubes with a uniform random rotation and a scale log-uniform in
    [0.5, 2], regular tetrahedra); the coarse size N0 in [100, 2000] of the shape's
    description (polycube faces / cube and tetrahedron face grids split into about N0
    triangles); the number of adaptive steps L in 3..6; the target size N_T
    log-uniform in [n_lo, n_hi]; then the shape's own draws.  Dorfler marking with
    theta = 0.5 grows a uniform start mesh of these shapes by about ``growth`` per
    level (1.13, measured on this stream: the first levels mark mostly elements at
    edges and corners), so L steps cannot take 100..2000 triangles to 5k..40k; the request
    therefore starts from the same shape uniformly subdivided to about
    N_T / growth^(L-1) triangles (at least its N0), runs at most L levels and stops at
    the first level with N >= N_T.  Returned per request: id, arrival time, start
    mesh, steps (L), target (N_T), coarse size (N0)."""
    rng = SplitMix64(seed)
    t = 0.0
    reqs = []
    for r in range(count):
        t += -math.log(max(1.0 - rng.uniform(), 1e-300)) / rate
        kind = rng.randint(0, 2)
        n0 = rng.randint(100, 2000)
        steps = rng.randint(3, 6)
        target = int(round(math.exp(math.log(n_lo) + (math.log(n_hi) - math.log(n_lo)) * rng.uniform())))
        start = target / growth ** (steps - 1)
        if kind == 0:
            g = rng.randint(3, 6)
            p = 0.3 + 0.4 * rng.uniform()
            occ = polycube_occupancy(g, p, rng.next_u64() & 0xFFFFFFFF)
            _, t1 = voxel_surface_int(occ, 1)
            s0 = max(1, int(round(math.sqrt(n0 / t1.shape[0]))))
            s = max(s0, int(round(math.sqrt(start / t1.shape[0]))))
            iv, tris = voxel_surface_int(occ, sub=s)
            m = Mesh(iv.astype(np.float64) / s, tris, f"req{r}_polycube")
            coarse = t1.shape[0] * s0 * s0
        elif kind == 1:
            n_c = max(1, int(round(math.sqrt(n0 / 12.0))))
            n = max(n_c, int(round(math.sqrt(start / 12.0))))
            sc = math.exp(math.log(0.5) + (math.log(2.0) - math.log(0.5)) * rng.uniform())
            m = transformed(cube_mesh(n), random_rotation(rng), sc)
            m.name = f"req{r}_cube"
            coarse = 12 * n_c * n_c
        else:
            k_c = max(1, int(round(math.sqrt(n0 / 4.0))))
            k = max(k_c, int(round(math.sqrt(start / 4.0))))
            m = tetra_mesh(k)
            m.name = f"req{r}_tetra"
            coarse = 4 * k_c * k_c
        reqs.append({"id": r, "t_arrive": t, "mesh": m, "steps": steps, "target": target, "coarse": coarse})
    return reqs
