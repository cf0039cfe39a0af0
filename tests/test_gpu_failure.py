"""Failure detection of the persistent solver, without faulting the GPU.

The CTAs of the persistent PCG meet at grid barriers whose wait is bounded in
time.  Here one CTA is told to leave at its first barrier without arriving, as a
CTA that stopped would; the others' waits run out after a short limit set from
the host, they raise the error flag and return, and the call reports
BEM_ERR_CUDA.  The context must still work afterwards: the next solve gives the
same Cap bit for bit as before the injected failure.  Nothing here traps, faults
or hangs: every wait has a limit and the kernel returns a status the host reads.
"""
import time

import pytest

from paper_1901_08393_gb300 import bem, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    return bem.Context()


@pytest.mark.parametrize("precond", [bem.PRECOND_JACOBI, bem.PRECOND_BLOCK], ids=["jacobi", "block"])
def test_barrier_timeout_reports_error_and_context_survives(ctx, precond):
    m = inputs.workload_polycube_adaptive()  # 604 triangles: a grid of at least 8 CTAs
    mesh = bem.Mesh.upload(ctx, m.verts, m.tris)
    op = bem.Operator.assemble(mesh, precision=bem.PREC_DF64)
    cap0, _, info0 = bem.solve_capacity(op, tol=1e-10, precond=precond)
    ctx.barrier_fault(wait_limit_ns=2_000_000, absent_cta=1)  # 2 ms limit, CTA 1 leaves
    try:
        t0 = time.perf_counter()
        with pytest.raises(bem.BemError) as e:
            bem.solve_capacity(op, tol=1e-10, precond=precond)
        dt = time.perf_counter() - t0
    finally:
        ctx.barrier_fault(0, -1)
    assert e.value.code == bem.BEM_ERR_CUDA
    assert "grid barrier timed out" in str(e.value)
    assert dt < 5.0  # the limit, not the default 2 s per barrier, ended the wait
    cap1, _, info1 = bem.solve_capacity(op, tol=1e-10, precond=precond)
    assert cap1 == cap0 and info1["iterations"] == info0["iterations"]
    op.close()
    mesh.close()


def test_barrier_limit_alone_changes_nothing(ctx):
    """A short limit without an absent CTA: the solve completes as usual (every wait
    of a healthy solve is far below a millisecond at this size)."""
    m = inputs.cube_mesh(4)
    mesh = bem.Mesh.upload(ctx, m.verts, m.tris)
    op = bem.Operator.assemble(mesh, precision=bem.PREC_DF64)
    cap0, _, _ = bem.solve_capacity(op, tol=1e-10)
    ctx.barrier_fault(wait_limit_ns=50_000_000, absent_cta=-1)
    try:
        cap1, _, _ = bem.solve_capacity(op, tol=1e-10)
    finally:
        ctx.barrier_fault(0, -1)
    assert cap1 == cap0
    op.close()
    mesh.close()


def test_fault_hook_rejects_bad_arguments(ctx):
    with pytest.raises(bem.BemError) as e:
        ctx.barrier_fault(0, -2)
    assert e.value.code == bem.BEM_ERR_INVALID
