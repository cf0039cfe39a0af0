"""Batched assembly and solve (bem_batch_*): every problem of a batch gets the
result of its own single solve, runs are reproducible bit for bit (the second run
replays the captured CUDA graph), and the batch frees what it allocated."""
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


def _meshes():
    return [inputs.cube_mesh(2), inputs.tetra_mesh(3), inputs.cube_mesh(4), inputs.icosphere_mesh(2),
            inputs.workload_polycube_adaptive(), inputs.fichera_mesh(2)]


@pytest.mark.parametrize("precond", [bem.PRECOND_JACOBI, bem.PRECOND_BLOCK], ids=["jacobi", "block"])
@pytest.mark.parametrize("prec", [bem.PREC_DF64, bem.PREC_F32], ids=["df64", "f32"])
def test_batch_matches_single_solves(ctx, prec, precond):
    ms = _meshes()
    meshes = [bem.Mesh.upload(ctx, m.verts, m.tris) for m in ms]
    b = bem.Batch(ctx, meshes, precision=prec, precond=precond, tol=1e-11)
    r1 = b.run()
    assert b.info()["graph_used"] == 1
    r2 = b.run()
    assert b.info()["graph_used"] == 1
    assert [r["cap"] for r in r1] == [r["cap"] for r in r2]  # graph replay: the same bits
    for m, mesh, r in zip(ms, meshes, r1):
        op = bem.Operator.assemble(mesh, precision=prec)
        cap, _, info = bem.solve_capacity(op, tol=1e-11, precond=precond)
        assert r["converged"] and r["status"] == 0 and r["relres"] <= 1e-11, (m.name, r)
        assert abs(r["cap"] / cap - 1) < 1e-9, (m.name, r["cap"], cap)  # other CTA counts: other sum orders
        assert abs(r["iterations"] - info["iterations"]) <= 2 + info["iterations"] // 10, (m.name, r, info)
        op.close()
    if prec == bem.PREC_DF64:
        for m, r in list(zip(ms, r1))[:3]:
            t = O.canonical(m.verts, m.tris)
            assert abs(r["cap"] / O.solve_capacity(m.verts, t, tol=1e-12)[0] - 1) < 1e-10
    b.close()


def test_batch_direct_launches_same_results(ctx):
    ms = _meshes()[:4]
    meshes = [bem.Mesh.upload(ctx, m.verts, m.tris) for m in ms]
    g = bem.Batch(ctx, meshes, precision=bem.PREC_DF64, precond=bem.PRECOND_BLOCK, use_graph=True).run()
    d = bem.Batch(ctx, meshes, precision=bem.PREC_DF64, precond=bem.PRECOND_BLOCK, use_graph=False)
    rd = d.run()
    assert d.info()["graph_used"] == 0
    assert [r["cap"] for r in rd] == [r["cap"] for r in g]
    d.close()


def test_batch_errors_and_memory(ctx):
    m = inputs.cube_mesh(2)
    mesh = bem.Mesh.upload(ctx, m.verts, m.tris)
    before = ctx.memory_in_use()
    with pytest.raises(bem.BemError) as e:
        bem.Batch(ctx, [mesh], precision=bem.PREC_F64)
    assert e.value.code == bem.BEM_ERR_INVALID
    b = bem.Batch(ctx, [mesh, mesh], precision=bem.PREC_DF64)
    b.run()
    b.close()
    assert ctx.memory_in_use() == before


def _wave_meshes():
    return [inputs.cube_mesh(14), inputs.polycube_mesh(4, 0.5, 3, sub=3), inputs.cube_mesh(2),
            inputs.fichera_mesh(6), inputs.tetra_mesh(24), inputs.cube_mesh(12)]


@pytest.mark.parametrize("prec", [bem.PREC_F32, bem.PREC_DF64], ids=["f32", "df64"])
def test_batch_waves_under_a_budget(prec):
    """A context budget that holds about half of the batch: the problems run in two or
    more waves through one arena, every Cap equals the one-wave batch's (other CTA
    shares only change the order of the sums) and the FP64 oracle's within the
    tolerance of the precision (1e-6 for the FP32 operator, 1e-10 for DF64)."""
    ms = _wave_meshes()
    big = bem.Context()
    one = bem.Batch(big, [bem.Mesh.upload(big, m.verts, m.tris) for m in ms], precision=prec,
                    precond=bem.PRECOND_BLOCK, tol=1e-10)
    w1, arena1, _ = one.waves()
    r1 = one.run()
    one.close()
    assert w1 == 1
    small = bem.Context(hbm_budget_bytes=1 << 40)  # probe the meshes' own bytes first
    probe = [bem.Mesh.upload(small, m.verts, m.tris) for m in ms]
    base = small.memory_in_use()
    for mh in probe:
        mh.close()
    small.close()
    ctx = bem.Context(hbm_budget_bytes=base + arena1 // 2 + (8 << 20))
    meshes = [bem.Mesh.upload(ctx, m.verts, m.tris) for m in ms]
    b = bem.Batch(ctx, meshes, precision=prec, precond=bem.PRECOND_BLOCK, tol=1e-10)
    nw, arena, wave_of = b.waves()
    assert nw >= 2 and arena < arena1, (nw, arena, arena1)
    assert list(wave_of) == sorted(wave_of)  # waves follow the given order
    ra = b.run()
    rb = b.run()  # graph replay of every wave: the same bits
    assert b.info()["graph_used"] == 1
    assert [r["cap"] for r in ra] == [r["cap"] for r in rb]
    assert ctx.memory_in_use() <= base + arena1 // 2 + (8 << 20)
    tol = 1e-6 if prec == bem.PREC_F32 else 1e-10
    for m, x, y in zip(ms, ra, r1):
        assert x["status"] == 0 and x["converged"], (m.name, x)
        assert abs(x["cap"] / y["cap"] - 1) < 1e-11, (m.name, x["cap"], y["cap"])
        ref = O.solve_capacity(m.verts, O.canonical(m.verts, m.tris), tol=1e-12)[0]
        assert abs(x["cap"] / ref - 1) < tol, (m.name, x["cap"], ref)
    b.close()
