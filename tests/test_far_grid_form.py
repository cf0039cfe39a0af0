"""The double-float far field's grid form, emulated on the CPU in FP32 (numpy float32
arithmetic is IEEE single precision, round to nearest; an FMA is its exact product and
sum, rounded once).

The form splits the centroid difference D = c_i - c_j and the two points' offsets from
their centroids on one power-of-two grid per pair, so that the hi part of every point
difference x_a - y_b is a single exact FP32 subtraction.  These tests pin the two
properties the kernel relies on: (1) that subtraction is exact for every pair the form
takes (|D| >= 1.12 (R_i + R_j)), and (2) the entry sums stay within 1e-11 of FP64 on
seeded meshes with needle triangles, far from the 1e-10 bound of the FP64 paths.
"""
import numpy as np
import pytest

from paper_1901_08393_gb300 import inputs

F = np.float32
SQ15 = np.sqrt(15.0)
_A, _B = (6.0 - SQ15) / 21.0, (6.0 + SQ15) / 21.0
BARY = np.array([[1 / 3, 1 / 3, 1 / 3], [_A, _A, 1 - 2 * _A], [_A, 1 - 2 * _A, _A], [1 - 2 * _A, _A, _A],
                 [_B, _B, 1 - 2 * _B], [_B, 1 - 2 * _B, _B], [1 - 2 * _B, _B, _B]])
W = np.array([9 / 40] + [(155 - SQ15) / 1200] * 3 + [(155 + SQ15) / 1200] * 3)
WH = W.astype(F)
WL = (W - WH.astype(np.float64)).astype(F)


def fma(a, b, c):
    return (np.asarray(a, np.float64) * np.asarray(b, np.float64) + np.asarray(c, np.float64)).astype(F)


def two_sum(a, b):
    s = (a + b).astype(F)
    bb = (s - a).astype(F)
    return s, ((a - (s - bb)) + (b - bb)).astype(F)


def fast_two_sum(a, b):
    s = (a + b).astype(F)
    return s, (b - (s - a)).astype(F)


def pos_two_sum(a, b):
    s = (a + b).astype(F)
    return s, (np.minimum(a, b) - (s - np.maximum(a, b))).astype(F)


def snap(v, big):
    return ((v + big).astype(F) - big).astype(F)


def tables(m):
    """The per-triangle double-float table of the kernel: offsets (hi, lo), the centroid
    as three floats, the largest |hi| offset coordinate and the largest point distance."""
    P = m.verts[m.tris]
    c = P.mean(axis=1)
    off = np.einsum("ak,nkc->nac", BARY, P - c[:, None, :])
    oh = off.astype(F)
    ol = (off - oh.astype(np.float64)).astype(F)
    c0 = c.astype(F)
    r1 = c - c0.astype(np.float64)
    c1 = r1.astype(F)
    c2 = (r1 - c1.astype(np.float64)).astype(F)
    rmax = np.abs(oh).max(axis=(1, 2))
    Rd = np.nextafter(np.linalg.norm(off, axis=2).max(axis=1).astype(F), F(np.inf))
    x = c[:, None, :] + off  # FP64 quadrature points, for the reference
    return oh, ol, (c0, c1, c2), rmax, Rd, x


def grid_pairs(m, n_rand, seed):
    """Far pairs (no shared vertex) within 6 h of each other plus random ones."""
    t = m.tris
    c = m.verts[t].mean(axis=1)
    h = np.sqrt(np.linalg.norm(np.cross(m.verts[t[:, 1]] - m.verts[t[:, 0]], m.verts[t[:, 2]] - m.verts[t[:, 0]]),
                               axis=1))
    sets = [set(x) for x in t.tolist()]
    out = []
    for i in range(len(t)):
        d = np.linalg.norm(c - c[i], axis=1)
        for j in np.nonzero(d < 6 * h[i])[0]:
            if j > i and not (sets[i] & sets[j]):
                out.append((i, j))
    rng = np.random.default_rng(seed)
    while n_rand > 0:
        i, j = rng.integers(0, len(t), 2)
        if i != j and not (sets[i] & sets[j]):
            out.append((min(i, j), max(i, j)))
            n_rand -= 1
    return np.array(out)


def grid_form(m, pairs):
    """Entry sums sum_a w_a sum_b w_b / |x_a - y_b| of the pairs the grid form takes,
    the FP64 reference of the same sums, and whether every hi-part subtraction was exact."""
    oh, ol, (c0, c1, c2), rmax, Rd, x = tables(m)
    I, J = pairs[:, 0], pairs[:, 1]
    # centroid difference in double-float from the three-float centroids
    s1, e1 = two_sum(c0[I], -c0[J])
    s2, e2 = two_sum(c1[I], -c1[J])
    s3 = (c2[I] - c2[J]).astype(F)
    hh, ll = two_sum(s1, s2)
    ll = (ll + ((e1 + e2).astype(F) + s3).astype(F)).astype(F)
    Dh, Dl = fast_two_sum(hh, ll)
    Rs = (Rd[I] + Rd[J]).astype(F)
    D2 = (Dh * Dh).sum(axis=1, dtype=F)
    bound = np.maximum(np.abs(Dh).max(axis=1), np.maximum(rmax[I], rmax[J]))
    eb = (bound.view(np.uint32) >> 23) | 1
    take = (D2 >= F(1.26) * (Rs * Rs)) & (eb >= 93) & (eb <= 185)
    I, J, Dh, Dl, eb = I[take], J[take], Dh[take], Dl[take], eb[take]
    big = (((eb + 2) << 23) | 0x400000).astype(np.uint32).view(F)[:, None]
    Dg = snap(Dh, big)
    Dl2 = (F(2) * ((Dh - Dg).astype(F) + Dl).astype(F)).astype(F)
    og = snap(oh[J].reshape(len(J), -1), big).reshape(len(J), 7, 3)
    ol2 = (F(2) * ((oh[J] - og).astype(F) + ol[J]).astype(F)).astype(F)
    exact = True
    acc_h = np.zeros(len(I), F)
    acc_l = np.zeros(len(I), F)
    for a in range(7):
        rg = snap(oh[I, a], big)
        eh = (Dg + rg).astype(F)
        el2 = fma(F(2), ((oh[I, a] - rg).astype(F) + ol[I, a]).astype(F), Dl2)
        sh = np.zeros(len(I), F)
        sl = np.zeros(len(I), F)
        for b in range(7):
            dh = (eh - og[:, b]).astype(F)
            exact &= bool(np.array_equal(dh.astype(np.float64), eh.astype(np.float64) - og[:, b].astype(np.float64)))
            dl2 = (el2 - ol2[:, b]).astype(F)
            p = (dh * dh).astype(F)
            pe = fma(dh, dh, -p)
            pe = fma(dl2, fma(F(0.25), dl2, dh), pe)
            t1, u1 = pos_two_sum(p[:, 0], p[:, 1])
            S, u2 = pos_two_sum(t1, p[:, 2])
            Sl = ((pe[:, 0] + pe[:, 1]).astype(F) + (pe[:, 2] + (u1 + u2).astype(F)).astype(F)).astype(F)
            y = (1.0 / np.sqrt(S.astype(np.float64))).astype(F) * F(1 + 2.0 ** -22)  # a MUFU-sized error
            y2 = (y * y).astype(F)
            y2e = fma(y, y, -y2)
            tt = fma(-S, y2, F(1))
            tt = fma(-S, y2e, tt)
            tt = fma(-Sl, y2, tt)
            yl = ((F(0.5) * y).astype(F) * tt).astype(F)
            ph = (WH[b] * y).astype(F)
            q = fma(WH[b], y, -ph)
            q = fma(WH[b], yl, q)
            q = fma(WL[b], y, q)
            u, ue = pos_two_sum(sh, ph)
            sh, sl = u, (sl + (q + ue).astype(F)).astype(F)
        ph = (WH[a] * sh).astype(F)
        q = fma(WH[a], sh, -ph)
        q = fma(WH[a], sl, q)
        q = fma(WL[a], sh, q)
        u, ue = pos_two_sum(acc_h, ph)
        acc_h, acc_l = u, (acc_l + (q + ue).astype(F)).astype(F)
    h, l = fast_two_sum(acc_h, acc_l)
    d = x[I][:, :, None, :] - x[J][:, None, :, :]
    ref = np.einsum("a,b,nab->n", W, W, 1.0 / np.linalg.norm(d, axis=3))
    return h.astype(np.float64) + l.astype(np.float64), ref, exact, take.mean()


@pytest.mark.parametrize("make", [lambda: inputs.graded_cube_mesh(8), lambda: inputs.cube_mesh(6),
                                  lambda: inputs.fichera_mesh(2), lambda: inputs.workload_polycube_adaptive()],
                         ids=["graded-needles", "cube6", "fichera2", "polycube"])
def test_grid_form_exact_hi_differences_and_entry_error(make):
    m = make()
    got, ref, exact, frac = grid_form(m, grid_pairs(m, 4000, 3))
    assert exact, "a hi-part point difference was rounded"
    assert frac > 0.3 and len(got) > 1000, (frac, len(got))
    assert np.max(np.abs(got / ref - 1)) < 1e-11, np.max(np.abs(got / ref - 1))
