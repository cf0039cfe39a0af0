"""Continuous-batching server (bem_server_*): results in the mix equal results alone,
admission respects the HBM budget, and a bad request fails alone."""
import numpy as np
import pytest

from paper_1901_08393_gb300 import bem, inputs

pytestmark = pytest.mark.gpu


def _requests():
    rng = inputs.SplitMix64(11)
    reqs = [
        (inputs.polycube_mesh(4, 0.5, 3), 4, 2500),
        (inputs.transformed(inputs.cube_mesh(3), inputs.random_rotation(rng), 1.7), 3, 2000),
        (inputs.tetra_mesh(6), 4, 2500),
        (inputs.polycube_mesh(5, 0.4, 8), 3, 3000),
        (inputs.icosphere_mesh(3), 3, 1500),
        (inputs.fichera_mesh(2), 5, 2500),
    ]
    return reqs


@pytest.fixture(scope="module")
def cuda():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("needs a CUDA device")


@pytest.mark.parametrize("prec", [bem.PREC_F32, bem.PREC_DF64], ids=["f32", "df64"])
def test_mix_equals_alone(cuda, prec):
    reqs = _requests()
    srv = bem.Server(slots=4, hbm_budget_bytes=16 << 30, precision=prec)
    ids = [srv.submit(m.verts, m.tris, lv, mx) for m, lv, mx in reqs]
    mixed = [srv.wait(i) for i in ids]
    st = srv.stats()
    srv.close()
    assert st["peak_in_flight"] >= 2  # the requests really overlapped
    alone = []
    for m, lv, mx in reqs:
        s1 = bem.Server(slots=1, hbm_budget_bytes=16 << 30, precision=prec)
        alone.append(s1.wait(s1.submit(m.verts, m.tris, lv, mx)))
        s1.close()
    for a, b in zip(mixed, alone):
        assert a["status"] == 0 and b["status"] == 0, (a["message"], b["message"])
        assert a["Ns"] == b["Ns"]
        assert a["caps"] == b["caps"]  # bit-identical: every kernel reduces in a fixed order
        assert a["t_submit"] <= a["t_start"] <= a["t_done"]
    # the same requests through the single-request entry point
    ctx = bem.Context()
    m, lv, mx = reqs[0]
    recs, _ = bem.adaptive_run(bem.Mesh.upload(ctx, m.verts, m.tris), max_N=mx, max_levels=lv, precision=prec,
                               tol=1e-10)
    assert [r["cap"] for r in recs] == mixed[0]["caps"]


def test_admission_budget_and_bad_request(cuda):
    reqs = _requests()[:3]
    one = bem.Server(slots=1, hbm_budget_bytes=1 << 40)  # the admission estimate of each request
    est = max(one.wait(one.submit(m.verts, m.tris, lv, reqs[0][2]))["estimate_bytes"] for m, lv, mx in reqs)
    one.close()
    # budget for one of these requests at a time (four slots); the small bad request
    # may backfill beside one of them
    srv = bem.Server(slots=4, hbm_budget_bytes=int(est * 1.2))
    ids = [srv.submit(m.verts, m.tris, lv, reqs[0][2]) for m, lv, mx in reqs]
    bad = inputs.cube_mesh(2)
    bad_id = srv.submit(bad.verts, bad.tris[:-1], 3, 1000)  # open surface
    res = [srv.wait(i) for i in ids]
    rb = srv.wait(bad_id)
    st = srv.stats()
    srv.close()
    assert st["peak_bytes"] <= int(est * 1.2)
    assert all(r["status"] == 0 for r in res)
    assert rb["status"] == bem.BEM_ERR_MESH and "closed" in rb["message"]
    # served one after another, in arrival order of the fitting requests
    starts = sorted((r["t_start"], r["t_done"]) for r in res)
    assert all(b[0] >= a[1] - 1e-6 for a, b in zip(starts, starts[1:]))


def test_dual_basis_requests(cuda):
    """The paper's dual basis with its operator preconditioner through the server: each
    request's Cap history is the same alone, in the mix and through bem_adaptive_run."""
    reqs = [(inputs.cube_mesh(1), 8, 600), (inputs.fichera_mesh(1), 6, 600), (inputs.tetra_mesh(3), 6, 500)]
    kw = dict(precision=bem.PREC_DF64, precond=bem.PRECOND_CALDERON, basis=bem.BASIS_DUAL)
    srv = bem.Server(slots=3, hbm_budget_bytes=16 << 30, **kw)
    ids = [srv.submit(m.verts, m.tris, lv, mx) for m, lv, mx in reqs]
    mixed = [srv.wait(i) for i in ids]
    srv.close()
    ctx = bem.Context()
    for (m, lv, mx), r in zip(reqs, mixed):
        assert r["status"] == 0, r["message"]
        recs, _ = bem.adaptive_run(bem.Mesh.upload(ctx, m.verts, m.tris), max_N=mx, max_levels=lv, tol=1e-10, **kw)
        assert [x["cap"] for x in recs] == r["caps"] and [x["N"] for x in recs] == r["Ns"]


def test_server_profile_counts_the_slots_kernels(cuda):
    """Profiling through the server sums every slot's hot kernels; results do not change."""
    reqs = _requests()[:3]
    srv = bem.Server(slots=2, hbm_budget_bytes=16 << 30, precision=bem.PREC_F32)
    plain = [srv.wait(srv.submit(m.verts, m.tris, lv, mx)) for m, lv, mx in reqs]
    srv.profile(True)
    prof = [srv.wait(srv.submit(m.verts, m.tris, lv, mx)) for m, lv, mx in reqs]
    far = srv.profile_read(bem.KERNEL_FAR)
    mv = srv.profile_read(bem.KERNEL_MATVEC)
    srv.close()
    levels = sum(r["levels"] for r in prof)
    assert far[0] >= len(reqs) and far[1] > 0.0 and far[2] > 0.0
    assert mv[0] >= levels and mv[1] > 0.0 and mv[2] > 0.0  # a persistent solve per level at least
    assert [r["caps"] for r in prof] == [r["caps"] for r in plain]
