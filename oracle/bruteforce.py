"""Brute-force reference for pair integrals, independent of the oracle's
quadrature rules.  TEST INFRASTRUCTURE ONLY.

int_P int_Q 1/(4 pi |x-y|) dy dx is computed by nested adaptive quadrature:
  * innermost: the closed form of the line integral of 1/|x-s| along a segment,
    int_0^L ds / sqrt((s-t0)^2 + h^2) = asinh((L-t0)/h) + asinh(t0/h);
  * middle: scipy ``quad`` across Q (lines parallel to one edge) -> the potential
    of the uniform unit density on Q at x;
  * outer: scipy ``dblquad`` over P.
It shares nothing with bem_oracle.c (no Radon rule, no Gauss tables, no
Sauter-Schwab transforms) and is slow; it is used on a handful of pairs.
"""
from __future__ import annotations

import math

import numpy as np


def segment_potential(x, P, Q):
    d = Q - P
    L = float(np.linalg.norm(d))
    u = d / L
    w = x - P
    t0 = float(w @ u)
    h = math.sqrt(max(float(w @ w) - t0 * t0, 0.0))
    return math.asinh((L - t0) / h) + math.asinh(t0 / h)


def triangle_potential(x, A, B, C, eps=1e-13):
    """int_T 1/|x-y| dy for the triangle T = (A, B, C)."""
    from scipy import integrate

    area2 = float(np.linalg.norm(np.cross(B - A, C - A)))
    lc = float(np.linalg.norm(C - A))

    def f(s):
        if s >= 1.0:
            return 0.0
        P = A + s * (B - A)
        return segment_potential(x, P, P + (1.0 - s) * (C - A)) / lc

    v, _ = integrate.quad(f, 0.0, 1.0, epsabs=eps, epsrel=eps, limit=400)
    return area2 * v


def pair_integral(P, Q, epsabs=1e-12, epsrel=1e-11):
    """(1/4pi) int_P int_Q 1/|x-y|, P and Q given as 3x3 vertex arrays."""
    from scipy import integrate

    P = np.asarray(P, dtype=np.float64)
    Q = np.asarray(Q, dtype=np.float64)
    A, B, C = P
    area2 = float(np.linalg.norm(np.cross(B - A, C - A)))

    def g(t, s):
        return triangle_potential(A + s * (B - A) + t * (C - A), *Q)

    v, _ = integrate.dblquad(g, 0.0, 1.0, 0.0, lambda s: 1.0 - s, epsabs=epsabs, epsrel=epsrel)
    return area2 * v / (4.0 * math.pi)


def identical_closed_form(P):
    """(1/4pi) int_T int_T 1/|x-y| = (1/4pi)(4/3)|T|^2 sum_e (1/|e|) int_e ds/|s - v_e|,
    v_e the vertex opposite edge e (the difference-body identity for a triangle)."""
    P = np.asarray(P, dtype=np.float64)
    area = 0.5 * float(np.linalg.norm(np.cross(P[1] - P[0], P[2] - P[0])))
    s = 0.0
    for k in range(3):
        a, b, v = P[k], P[(k + 1) % 3], P[(k + 2) % 3]
        s += segment_potential(v, a, b) / float(np.linalg.norm(b - a))
    return (4.0 / 3.0) * area * area * s / (4.0 * math.pi)
