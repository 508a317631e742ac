"""Control parametrisation: per-wheel velocity targets as natural cubic splines.

The paper optimises K-knot wheel-velocity splines (Sec. IV-B); the servo targets of
step n are the spline evaluated at t_{n+1} = (n + 1) h.  Interpolation is linear in
the knot values, so the spline is a fixed basis matrix B [T, K]: controls = B @ knots,
and dL/dknots = B^T dL/dcontrols.
"""
from __future__ import annotations

import numpy as np


def basis(T: int, K: int, h: float) -> np.ndarray:
    """[T, K] evaluation matrix of the natural cubic spline through K knots spaced
    uniformly over [0, T h], sampled at t = (n + 1) h, n = 0..T-1."""
    tau = np.linspace(0.0, T * h, K)
    dt = np.diff(tau)
    t = (np.arange(T) + 1) * h
    B = np.zeros((T, K))
    for k in range(K):
        y = np.zeros(K)
        y[k] = 1.0
        # second derivatives with natural end conditions
        A = np.zeros((K, K))
        r = np.zeros(K)
        A[0, 0] = A[-1, -1] = 1.0
        for i in range(1, K - 1):
            A[i, i - 1] = dt[i - 1]
            A[i, i] = 2.0 * (dt[i - 1] + dt[i])
            A[i, i + 1] = dt[i]
            r[i] = 6.0 * ((y[i + 1] - y[i]) / dt[i] - (y[i] - y[i - 1]) / dt[i - 1])
        Mk = np.linalg.solve(A, r)
        seg = np.clip(np.searchsorted(tau, t, side="right") - 1, 0, K - 2)
        a, b = tau[seg], tau[seg + 1]
        hh = b - a
        u = (b - t) / hh
        v = (t - a) / hh
        B[:, k] = (u * y[seg] + v * y[seg + 1]
                   + ((u ** 3 - u) * Mk[seg] + (v ** 3 - v) * Mk[seg + 1]) * hh * hh / 6.0)
    return B
