"""Parity of the dual-basis path (Sec. 2.1, 2.6, Eq. 1.6, 2.8) with the oracle.

Tolerances: barycentric meshes, dual ZZ indicators and marks bit-exact (both sides
evaluate the same IEEE operations on the same bytes); V^dual 1e-10 relative
elementwise (the entries of V^bary carry the assembly's 1e-10 and are all positive,
so their sums keep it); Cap 1e-9 relative; iterates 1e-7 relative to max |x|.
"""
import numpy as np
import pytest

import oracle as O
from oracle import dual as D
from paper_1901_08393_gb300 import bem, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    c = bem.Context()
    yield c
    c.close()


def _upload(ctx, m):
    mesh = bem.Mesh.upload(ctx, m.verts, m.tris)
    v, t, _, _ = mesh.download()
    return mesh, v, t


SMALL = [inputs.cube_mesh(1), inputs.cube_mesh(2), inputs.tetra_mesh(2), inputs.fichera_mesh(1),
         inputs.icosphere_mesh(1)]
MESHES = SMALL + [inputs.cube_mesh(4), inputs.workload_polycube_adaptive(), inputs.fichera_mesh(2)]


@pytest.mark.parametrize("m", MESHES, ids=lambda m: m.name)
def test_barycentric_refinement_bitexact(ctx, m):
    mesh, v, t = _upload(ctx, m)
    b = mesh.barycentric()
    vb, tb, _, _ = b.download()
    ov, ot = D.barycentric(v, t)
    assert np.array_equal(vb, ov)
    assert np.array_equal(tb, O.canonical(ov, ot))
    ab, db = b.geometry()
    ar, dr = O.geometry(ov, O.canonical(ov, ot))
    assert np.array_equal(ab, ar) and np.array_equal(db, dr)


@pytest.mark.parametrize("prec", [bem.PREC_F64, bem.PREC_DF64], ids=["f64", "df64"])
@pytest.mark.parametrize("m", SMALL, ids=lambda m: m.name)
def test_dual_operator_and_capacity_match_oracle(ctx, m, prec):
    mesh, v, t = _upload(ctx, m)
    bop = bem.Operator.assemble(mesh.barycentric(), precision=prec)
    dop = bem.Operator.dual(bop, mesh)
    N, p = dop.info()
    assert N == m.M and p == prec
    Vd = dop.read()
    cap_r, x_r, _, Vd_r = D.solve_dual(v, t, tol=1e-13)
    assert np.max(np.abs(Vd - Vd_r) / np.abs(Vd_r)) < 1e-10
    assert np.array_equal(Vd, Vd.T)
    # the block preconditioner belongs to the persistent solver of DF64/FP32 operators
    pcs = (bem.PRECOND_NONE, bem.PRECOND_JACOBI) + ((bem.PRECOND_BLOCK,) if prec == bem.PREC_DF64 else ())
    for pc in pcs:
        cap, x, info = bem.solve_capacity(dop, tol=1e-12, precond=pc)
        assert info["converged"]
        assert abs(cap / cap_r - 1) < 1e-9, (pc, cap, cap_r)
        assert np.max(np.abs(x - x_r)) < 1e-7 * np.max(np.abs(x_r))


def test_dual_operator_sums_the_barycentric_operator(ctx):
    """At a size the oracle's assembly is not needed for: V^dual = P^T V^bary P with the
    library's own V^bary, P built from the primal triangles on the host."""
    m = inputs.workload_polycube_adaptive()
    mesh, v, t = _upload(ctx, m)
    bop = bem.Operator.assemble(mesh.barycentric(), precision=bem.PREC_F64)
    Vd = bem.Operator.dual(bop, mesh).read()
    ref = D.dual_operator(bop.read(), D.child_cell(t), m.M)
    assert np.max(np.abs(Vd - ref) / np.abs(ref)) < 1e-13
    dop = bem.Operator.dual(bem.Operator.assemble(mesh.barycentric(), precision=bem.PREC_DF64), mesh)
    cap, _, _ = bem.solve_capacity(dop, tol=1e-12)
    cap_r = O.capacity(D.dual_areas(v, t), np.linalg.solve(ref, D.dual_areas(v, t)))
    assert abs(cap / cap_r - 1) < 1e-9


@pytest.mark.parametrize("h_mode", [0, 1])
@pytest.mark.parametrize("m", [inputs.cube_mesh(2), inputs.workload_polycube_adaptive(), inputs.fichera_mesh(2)],
                         ids=lambda m: m.name)
def test_zz_dual_bitexact(ctx, m, h_mode):
    mesh, v, t = _upload(ctx, m)
    x = np.random.default_rng(7).random(m.M) + 0.5
    eta2, tot, scale = bem.zz_estimate_dual(mesh, x, h_mode)
    ref = D.zz_dual(v, t, x, h_mode)
    assert np.array_equal(eta2, ref)
    area, diam = O.geometry(v, t)
    h = np.sqrt(area) if h_mode == 1 else diam
    xm = (x[t[:, 0]] + x[t[:, 1]] + x[t[:, 2]]) / 3.0
    assert abs(tot / ref.sum() - 1) < 1e-12
    assert abs(scale / np.sum(h * area * xm * xm / 12.0) - 1) < 1e-12
    # a constant density has no jumps: every indicator vanishes
    e0, t0, _ = bem.zz_estimate_dual(mesh, np.full(m.M, 2.5), h_mode)
    assert t0 == 0.0 and not e0.any()


@pytest.mark.parametrize("prec", [bem.PREC_F64, bem.PREC_DF64], ids=["f64", "df64"])
def test_dual_adaptive_loop_matches_oracle(ctx, prec):
    m = inputs.workload_polycube_adaptive()
    mesh = bem.Mesh.upload(ctx, m.verts, m.tris)
    recs, fin = bem.adaptive_run(mesh, theta=0.5, max_N=1500, tol=1e-12, precision=prec, want_final=True,
                                 basis=bem.BASIS_DUAL)
    hist = D.adaptive_run_dual(m.verts, m.tris, theta=0.5, max_N=1500, tol=1e-12)
    assert len(recs) == len(hist)
    for r, h in zip(recs, hist):
        assert r["N"] == h["N"] and r["M"] == h["M"]
        assert abs(r["cap"] / h["cap"] - 1) < 1e-9
        assert abs(r["eta2_total"] / h["eta2_total"] - 1) < 1e-6
        if "marked" in h:
            assert r["n_marked"] == int(h["marked"].sum())
    v, t, _, _ = fin.download()
    assert np.array_equal(v, hist[-1]["verts"]) and np.array_equal(t, hist[-1]["tris"])


def test_dual_levels_match_oracle_levelwise_on_a_symmetric_mesh(ctx):
    """On the cube the indicators come in symmetric groups whose order is decided by
    rounding, so each level is compared with the oracle on the library's own mesh."""
    m = inputs.cube_mesh(1)
    mesh = bem.Mesh.upload(ctx, m.verts, m.tris)
    caps = []
    for _ in range(6):
        v, t, _, _ = mesh.download()
        dop = bem.Operator.dual(bem.Operator.assemble(mesh.barycentric(), precision=bem.PREC_DF64), mesh)
        cap, x, _ = bem.solve_capacity(dop, tol=1e-12)
        cap_r, x_r, _, _ = D.solve_dual(v, t, tol=1e-13)
        assert abs(cap / cap_r - 1) < 1e-9
        eta2, _, _ = bem.zz_estimate_dual(mesh, x)
        assert np.array_equal(eta2, D.zz_dual(v, t, x))
        caps.append(cap)
        _, _, mesh = bem.mark_refine(mesh, eta2, 0.5)
    assert all(b > a for a, b in zip(caps, caps[1:]))


def test_dual_errors_are_reported(ctx):
    m = inputs.cube_mesh(1)
    mesh = bem.Mesh.upload(ctx, m.verts, m.tris)
    primal = bem.Operator.assemble(mesh)
    with pytest.raises(bem.BemError) as e:  # not the operator of the barycentric refinement
        bem.Operator.dual(primal, mesh)
    assert e.value.code == bem.BEM_ERR_INVALID
    dop = bem.Operator.dual(bem.Operator.assemble(mesh.barycentric()), mesh)
    with pytest.raises(bem.BemError) as e:
        bem.solve_capacity(dop, inexact_lambda=1e-3)
    assert e.value.code == bem.BEM_ERR_INVALID
    fine = bem.refine(mesh, np.ones(m.N, dtype=np.uint8))
    with pytest.raises(bem.BemError) as e:
        bem.Operator.update(fine, dop)
    assert e.value.code == bem.BEM_ERR_INVALID
    with pytest.raises(bem.BemError) as e:
        bem.adaptive_run(mesh, max_N=100, basis=bem.BASIS_DUAL, inexact_lambda=1e-3)
    assert e.value.code == bem.BEM_ERR_INVALID
    with pytest.raises(bem.BemError) as e:
        bem.adaptive_run(mesh, max_N=100, basis=7)
    assert e.value.code == bem.BEM_ERR_INVALID
