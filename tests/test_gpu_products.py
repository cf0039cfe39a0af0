"""Sources of the persistent solver's iteration products (bem_solve_opts.products).

Whatever the products, the residual that decides convergence is formed with the
operator's own product, so every mode must reach the same solution to the solve's
tolerance: the Caps agree with each other and with the oracle, and the reported
relative residual is the operator's."""
import numpy as np
import pytest

import oracle as O
from paper_1901_08393_gb300 import bem, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    return bem.Context()


MESHES = [inputs.workload_polycube_adaptive(), inputs.cube_mesh(13), inputs.graded_cube_mesh(12)]


@pytest.mark.parametrize("prec", [bem.PREC_DF64, bem.PREC_F32], ids=["df64", "f32"])
@pytest.mark.parametrize("precond", [bem.PRECOND_JACOBI, bem.PRECOND_BLOCK], ids=["jacobi", "block"])
def test_fp16_products_reach_the_same_solution(ctx, prec, precond):
    tol = 1e-11
    for m in MESHES:
        mesh = bem.Mesh.upload(ctx, m.verts, m.tris)
        op = bem.Operator.assemble(mesh, precision=prec)
        cap32, x32, i32 = bem.solve_capacity(op, tol=tol, precond=precond, products=bem.PRODUCTS_FP32)
        cap16, x16, i16 = bem.solve_capacity(op, tol=tol, precond=precond, products=bem.PRODUCTS_FP16)
        assert i16["converged"] and i16["relres"] <= tol, (m.name, i16)
        # the two solutions differ by at most the tolerance times the conditioning
        assert abs(cap16 / cap32 - 1) < 1e-9, (m.name, cap16, cap32)
        if prec == bem.PREC_DF64 and m.N <= 1000:
            t = O.canonical(m.verts, m.tris)
            assert abs(cap16 / O.solve_capacity(m.verts, t, tol=1e-12)[0] - 1) < 1e-9
        # the FP16 copy costs iterations, not convergence
        assert i16["iterations"] <= 2 * i32["iterations"] + 20, (m.name, i16, i32)
        op.close()
        mesh.close()


def test_default_products_follow_the_operator(ctx):
    """DEFAULT = the FP32 copy for DF64 operators (bit for bit), the FP16 copy for FP32 ones."""
    m = inputs.cube_mesh(10)
    mesh = bem.Mesh.upload(ctx, m.verts, m.tris)
    op = bem.Operator.assemble(mesh, precision=bem.PREC_DF64)
    c0, _, _ = bem.solve_capacity(op, tol=1e-11, precond=bem.PRECOND_BLOCK)
    c32, _, _ = bem.solve_capacity(op, tol=1e-11, precond=bem.PRECOND_BLOCK, products=bem.PRODUCTS_FP32)
    assert c0 == c32
    op.close()
    op = bem.Operator.assemble(mesh, precision=bem.PREC_F32)
    c0, _, _ = bem.solve_capacity(op, tol=1e-11, precond=bem.PRECOND_BLOCK)
    c16, _, _ = bem.solve_capacity(op, tol=1e-11, precond=bem.PRECOND_BLOCK, products=bem.PRODUCTS_FP16)
    assert c0 == c16
    op.close()
    mesh.close()


def test_adaptive_loop_with_fp16_products_matches_oracle(ctx):
    m = inputs.workload_polycube_adaptive()
    mesh = bem.Mesh.upload(ctx, m.verts, m.tris)
    recs, _ = bem.adaptive_run(mesh, theta=0.5, max_N=2500, tol=1e-11, precision=bem.PREC_DF64,
                               precond=bem.PRECOND_BLOCK, products=bem.PRODUCTS_FP16)
    hist = O.adaptive_run(m.verts, m.tris, theta=0.5, max_N=2500, tol=1e-12)
    assert [r["N"] for r in recs] == [h["N"] for h in hist]
    for r, h in zip(recs, hist):
        assert abs(r["cap"] / h["cap"] - 1) < 1e-9


@pytest.mark.parametrize("prec", [bem.PREC_DF64, bem.PREC_F32], ids=["df64", "f32"])
def test_batch_with_fp16_products_matches_single_solves(ctx, prec):
    """A batch takes the FP16 copy like a single solve (DF64 problems pack it inside the
    cooperative launch, FP32 ones before it): every problem's Cap equals its single
    solve's with the same products."""
    ms = [inputs.cube_mesh(4), inputs.workload_polycube_adaptive(), inputs.fichera_mesh(2), inputs.icosphere_mesh(3)]
    meshes = [bem.Mesh.upload(ctx, m.verts, m.tris) for m in ms]
    b = bem.Batch(ctx, meshes, precision=prec, precond=bem.PRECOND_BLOCK, tol=1e-11, products=bem.PRODUCTS_FP16)
    res = b.run()
    for m, mesh, r in zip(ms, meshes, res):
        op = bem.Operator.assemble(mesh, precision=prec)
        cap, _, info = bem.solve_capacity(op, tol=1e-11, precond=bem.PRECOND_BLOCK, products=bem.PRODUCTS_FP16)
        assert r["converged"] and r["relres"] <= 1e-11, (m.name, r)
        assert abs(r["cap"] / cap - 1) < 1e-9, (m.name, r["cap"], cap)
        op.close()
    b.close()
