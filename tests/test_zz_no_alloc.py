"""The no-allocation product bem_operator_matvec_noalloc, through the C ABI.

It exists for callers that must not have device memory allocated during a call
(code being captured into a CUDA graph, serving loops with a fixed pre-reserved
footprint, hosts whose allocator belongs to another framework).  It must give the
same y = V x as the allocating bem_operator_matvec, on repeated calls that share
its static scratch, without changing the context's allocations.  This file is
collected last so that a failure here never hides the other tests.
"""
import ctypes

import numpy as np
import pytest

from paper_1901_08393_gb300 import bem, inputs

pytestmark = pytest.mark.gpu


def test_no_alloc_matvec_matches_allocating_matvec():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("needs a CUDA device")
    ctx = bem.Context()
    L = bem.lib()
    # 604 triangles, and 3888 = a ragged last 64-tile close to the 4096 limit
    for m in (inputs.workload_polycube_adaptive(), inputs.cube_mesh(18)):
        mesh = bem.Mesh.upload(ctx, m.verts, m.tris)
        op = bem.Operator.assemble(mesh, precision=bem.PREC_DF64)
        x = np.random.default_rng(m.N).standard_normal(m.N)
        y_ref = op.matvec(x)  # the existing, allocating entry point
        xd = torch.from_numpy(x).cuda()
        held = ctx.memory_in_use()
        for call in range(2):
            yd = torch.full((m.N,), float("nan"), dtype=torch.float64, device="cuda")
            st = L.bem_operator_matvec_noalloc(op.h, ctypes.c_void_p(xd.data_ptr()), ctypes.c_void_p(yd.data_ptr()))
            assert st == bem.BEM_OK, ctx.last_error()
            torch.cuda.synchronize()
            y = yd.cpu().numpy()
            assert np.max(np.abs(y - y_ref)) <= 1e-13 * np.max(np.abs(y_ref)), (m.name, call)
        assert ctx.memory_in_use() == held
        op.close()
        mesh.close()


def test_no_alloc_matvec_rejects_what_it_cannot_do():
    import torch

    ctx = bem.Context()
    L = bem.lib()
    big = inputs.cube_mesh(19)  # 4332 triangles > 4096
    mesh = bem.Mesh.upload(ctx, big.verts, big.tris)
    op = bem.Operator.assemble(mesh, precision=bem.PREC_DF64)
    xd = torch.zeros(big.N, dtype=torch.float64, device="cuda")
    yd = torch.zeros(big.N, dtype=torch.float64, device="cuda")
    st = L.bem_operator_matvec_noalloc(op.h, ctypes.c_void_p(xd.data_ptr()), ctypes.c_void_p(yd.data_ptr()))
    assert st == bem.BEM_ERR_INVALID and "4096" in ctx.last_error()
    small = inputs.cube_mesh(2)
    mesh2 = bem.Mesh.upload(ctx, small.verts, small.tris)
    op64 = bem.Operator.assemble(mesh2, precision=bem.PREC_F64)
    x2 = torch.zeros(small.N, dtype=torch.float64, device="cuda")
    y2 = torch.zeros(small.N, dtype=torch.float64, device="cuda")
    st = L.bem_operator_matvec_noalloc(op64.h, ctypes.c_void_p(x2.data_ptr()), ctypes.c_void_p(y2.data_ptr()))
    assert st == bem.BEM_ERR_INVALID and "DF64" in ctx.last_error()
    opdf = bem.Operator.assemble(mesh2, precision=bem.PREC_DF64)
    xh = np.zeros(small.N)
    st = L.bem_operator_matvec_noalloc(opdf.h, ctypes.c_void_p(xh.ctypes.data), ctypes.c_void_p(y2.data_ptr()))
    assert st == bem.BEM_ERR_INVALID and "device pointers" in ctx.last_error()


def test_no_alloc_matvec_inside_graph_capture():
    """The call recorded into a CUDA graph under global capture mode (which refuses
    device allocation from any thread while the capture runs), then replayed."""
    import torch

    s = torch.cuda.Stream()
    ctx = bem.Context(stream=s.cuda_stream)
    L = bem.lib()
    m = inputs.workload_polycube_adaptive()
    mesh = bem.Mesh.upload(ctx, m.verts, m.tris)
    op = bem.Operator.assemble(mesh, precision=bem.PREC_DF64)
    x = np.random.default_rng(7).standard_normal(m.N)
    y_ref = op.matvec(x)
    xd = torch.from_numpy(x).cuda()
    yd = torch.zeros(m.N, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    # the first call outside capture (its one-time set-up may query the runtime)
    st = L.bem_operator_matvec_noalloc(op.h, ctypes.c_void_p(xd.data_ptr()), ctypes.c_void_p(yd.data_ptr()))
    assert st == bem.BEM_OK, ctx.last_error()
    torch.cuda.synchronize()
    held = ctx.memory_in_use()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s, capture_error_mode="global"):
        st = L.bem_operator_matvec_noalloc(op.h, ctypes.c_void_p(xd.data_ptr()), ctypes.c_void_p(yd.data_ptr()))
    assert st == bem.BEM_OK, ctx.last_error()
    for _ in range(2):
        yd.fill_(float("nan"))
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        y = yd.cpu().numpy()
        assert np.max(np.abs(y - y_ref)) <= 1e-13 * np.max(np.abs(y_ref))
    assert ctx.memory_in_use() == held
    op.close()
    mesh.close()
