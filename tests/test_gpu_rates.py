"""Convergence of Cap_l to the unit-cube capacity the paper quotes (Sec. 3.1): the
adaptive loop (theta = 1/2) converges at about O(N^-1), uniform refinement
(theta = 1 marks every element) at O(N^-2/3), and adaptivity is more accurate at a
comparable number of elements."""
import math

import numpy as np
import pytest

from paper_1901_08393_gb300 import bem, inputs

pytestmark = pytest.mark.gpu

CUBE_CAP = 0.66067815409957  # Sec. 3.1


def _run(theta, max_n):
    import torch

    if not torch.cuda.is_available():
        pytest.fail("needs a CUDA device")
    ctx = bem.Context()
    m = inputs.cube_mesh(1)
    mesh = bem.Mesh.upload(ctx, m.verts, m.tris)
    recs, _ = bem.adaptive_run(mesh, theta=theta, max_N=max_n, max_levels=100, tol=1e-10,
                               precision=bem.PREC_DF64, precond=bem.PRECOND_BLOCK)
    return [(r["N"], abs(r["cap"] - CUBE_CAP) / CUBE_CAP) for r in recs]


def _rate(rows, n_min):
    pts = [(math.log(n), math.log(e)) for n, e in rows if n >= n_min]
    return float(np.polyfit(*zip(*pts), 1)[0])


def test_adaptive_and_uniform_rates():
    ada = _run(0.5, 6000)
    uni = _run(1.0, 12000)
    ra, ru = _rate(ada, 500), _rate(uni, 700)
    assert -1.45 < ra < -0.9, (ra, ada)
    assert -0.8 < ru < -0.55, (ru, uni)
    assert all(e > 0 for _, e in ada + uni)
    # at N ~ 3,000 the adaptive mesh is several times more accurate than the uniform one
    ea = min(e for n, e in ada if n >= 2000)
    eu = min(e for n, e in uni if n <= 3100)
    assert ea < 0.6 * eu, (ada, uni)
