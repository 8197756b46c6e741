"""FP64 reference of the FP32 calibration relaxation -- TEST INFRASTRUCTURE ONLY.

The relaxation drops the integer shift and clamp of the fit (the paper's
Sec. 2 linear form p = f.x + q) and evaluates, per track t of sector s,

    y_t = F[s] x_t + q[s]                      (6 rows: 3 parameters, 3 chi)
    L   = (1/N) sum_t sum_{k<3} w_k (y_tk - theta_tk)^2 + (1/N) sum_t sum_{k>=3} y_tk^2

with theta the true track parameters in output units and w_k their inverse
variances.  The gradients follow from the chain rule:

    g_tk = dL/dy_tk = (2/N) w_k (y_tk - theta_tk)   for k < 3
                    = (2/N) y_tk                      for k >= 3
    dL/dF[s][k][l] = sum_{t in s} g_tk x_tl,    dL/dq[s][k] = sum_{t in s} g_tk

Everything here is float64 numpy; ``fd_grad`` differentiates ``loss``
numerically and is independent of ``grad``.
"""
from __future__ import annotations

import numpy as np


def forward(x, sector, F, q):
    x = np.asarray(x, np.float64)
    F = np.asarray(F, np.float64)
    q = np.asarray(q, np.float64)
    return np.einsum("tkl,tl->tk", F[sector], x) + q[sector]


def loss(x, sector, theta, w, F, q):
    y = forward(x, sector, F, q)
    n = len(y)
    theta = np.asarray(theta, np.float64)
    w = np.asarray(w, np.float64)
    return float((np.sum(w[None, :] * (y[:, :3] - theta) ** 2) + np.sum(y[:, 3:] ** 2)) / n)


def grad(x, sector, theta, w, F, q):
    """Analytic (dL/dF, dL/dq) in float64."""
    x = np.asarray(x, np.float64)
    y = forward(x, sector, F, q)
    n = len(y)
    g = np.empty_like(y)
    g[:, :3] = 2.0 / n * np.asarray(w, np.float64)[None, :] * (y[:, :3] - np.asarray(theta, np.float64))
    g[:, 3:] = 2.0 / n * y[:, 3:]
    S = np.asarray(F).shape[0]
    dF = np.zeros((S, 6, 6))
    dq = np.zeros((S, 6))
    np.add.at(dF, sector, g[:, :, None] * x[:, None, :])
    np.add.at(dq, sector, g)
    return dF, dq


def fd_grad(x, sector, theta, w, F, q, entries, h_rel=1e-6):
    """Central finite differences of ``loss`` at the listed entries.

    ``entries`` holds tuples ("F", s, k, l) or ("q", s, k).
    """
    F = np.array(F, np.float64)
    q = np.array(q, np.float64)
    out = []
    for e in entries:
        arr = F if e[0] == "F" else q
        idx = tuple(e[1:])
        v = arr[idx]
        h = h_rel * max(abs(v), 1.0)
        arr[idx] = v + h
        lp = loss(x, sector, theta, w, F, q)
        arr[idx] = v - h
        lm = loss(x, sector, theta, w, F, q)
        arr[idx] = v
        out.append((lp - lm) / (2.0 * h))
    return np.array(out)
