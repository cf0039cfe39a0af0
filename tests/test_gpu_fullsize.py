"""Parity at the full size of the benchmark workload, in the configuration bench.py
times: adaptive polycube (6^3, p=0.5, seed 1), ZZ + Doerfler theta=0.5 + NVB until
N >= 20,000, DF64 operator, PCG to 1e-10 with the block-Jacobi preconditioner (the
oracle runs Jacobi PCG: the solutions agree to the solver tolerance).

* the level sizes of the GPU run equal the oracle's own adaptive run, and every
  Cap_l agrees to 1e-8 (the bench's 1e-6 requirement, with margin);
* on the final mesh (N = 20,656): 6,000 sampled V entries (random, plus every
  touching pair of 64 random rows) within 1e-10 of the oracle; Cap of the GPU solve
  within 1e-8 of the oracle's FP64 PCG on the same mesh;
* the decisions at full size are bit-exact when both sides get the same bytes:
  ZZ indicators from the GPU solution, Doerfler marks, and the refined mesh.
"""
import numpy as np
import pytest

import oracle as O
from paper_1901_08393_gb300 import bem, inputs

pytestmark = pytest.mark.gpu

MAX_N, THETA, TOL = 20000, 0.5, 1e-10


@pytest.fixture(scope="module")
def run():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("needs a CUDA device")
    ctx = bem.Context()
    m = inputs.workload_polycube_adaptive()
    mesh = bem.Mesh.upload(ctx, m.verts, m.tris)
    recs, fin = bem.adaptive_run(mesh, theta=THETA, max_N=MAX_N, tol=TOL, precision=bem.PREC_DF64,
                                 precond=bem.PRECOND_BLOCK, want_final=True)
    hist = O.adaptive_run(m.verts, m.tris, theta=THETA, max_N=MAX_N, tol=1e-12)
    return ctx, recs, fin, hist


def test_level_history_matches_oracle(run):
    ctx, recs, fin, hist = run
    assert [r["N"] for r in recs] == [h["N"] for h in hist]
    assert recs[-1]["N"] >= MAX_N
    for r, h in zip(recs, hist):
        assert abs(r["cap"] / h["cap"] - 1) < 1e-8, (r["N"], r["cap"], h["cap"])
        assert r["relres"] <= TOL


def test_final_mesh_entries_and_cap(run):
    ctx, recs, fin, hist = run
    v, t, _, _ = fin.download()
    assert np.array_equal(v, hist[-1]["verts"]) and np.array_equal(t, hist[-1]["tris"])
    N = t.shape[0]
    op = bem.Operator.assemble(fin, precision=bem.PREC_DF64)
    rng = np.random.default_rng(20656)
    I = rng.integers(0, N, 4000)
    J = rng.integers(0, N, 4000)
    rows = rng.choice(N, 64, replace=False)
    near = []
    for i in rows:  # every triangle sharing a vertex with triangle i
        shared = np.sum(t[:, :, None] == t[i][None, None, :], axis=(1, 2))
        near += [(int(i), int(j)) for j in np.flatnonzero(shared > 0)]
    I = np.concatenate([I, [p[0] for p in near]])
    J = np.concatenate([J, [p[1] for p in near]])
    got = op.entries(I, J)
    ref = O.entries(v, t, I, J)
    assert np.max(np.abs(got / ref - 1)) < 1e-10
    cap, phi, info = bem.solve_capacity(op, tol=TOL, precond=bem.PRECOND_BLOCK)
    assert info["converged"]
    cap_ref = hist[-1]["cap"]  # the oracle's FP64 PCG (1e-12) on this mesh
    assert abs(cap / cap_ref - 1) < 1e-8
    assert abs(cap / recs[-1]["cap"] - 1) < 1e-9


def test_full_size_decisions_bitexact(run):
    ctx, recs, fin, hist = run
    v, t, _, _ = fin.download()
    op = bem.Operator.assemble(fin, precision=bem.PREC_DF64)
    _, phi, _ = bem.solve_capacity(op, tol=TOL, precond=bem.PRECOND_BLOCK)
    eta2, tot, scale = bem.zz_estimate(fin, phi)
    assert np.array_equal(eta2, O.zz(v, t, phi))
    marked, nm = bem.dorfler(ctx, eta2, THETA)
    assert np.array_equal(marked, O.dorfler(eta2, THETA))
    fine = bem.refine(fin, marked)
    v2, t2, p2, k2 = fine.download()
    vr, tr, pr, kr = O.refine(v, t, marked)
    assert np.array_equal(v2, vr) and np.array_equal(t2, tr)
    assert np.array_equal(p2, pr) and np.array_equal(k2, kr)
