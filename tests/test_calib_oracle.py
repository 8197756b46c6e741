"""Pins of the FP64 calibration reference (oracle/calib.py).

The analytic gradient is checked against central finite differences of the
loss (an independent numerical derivative) and against the normal equations:
at the per-sector least-squares solution of the parameter rows, with zero chi
rows, the gradient vanishes.
"""
import numpy as np

from oracle import calib
from paper_1311_0380_gb300 import synth


def small_set(n=1200, S=4, seed=1):
    consts = synth.make_constants(S)
    cs = synth.make_calib(n, consts, seed=seed)
    return cs


def test_gradient_matches_finite_differences():
    cs = small_set()
    rng = np.random.default_rng(2)
    F = cs.F0.astype(np.float64)
    q = cs.q0.astype(np.float64)
    dF, dq = calib.grad(cs.x, cs.sector, cs.theta, cs.weight, F, q)
    entries = []
    for _ in range(60):
        s, k, l = (int(v) for v in rng.integers(0, [4, 6, 6]))
        entries.append(("F", s, k, l))
    for _ in range(20):
        s, k = (int(v) for v in rng.integers(0, [4, 6]))
        entries.append(("q", s, k))
    fd = calib.fd_grad(cs.x, cs.sector, cs.theta, cs.weight, F, q, entries, h_rel=1e-6)
    an = np.array([dF[e[1:]] if e[0] == "F" else dq[e[1:]] for e in entries])
    scale = np.max(np.abs(an))
    assert np.max(np.abs(fd - an)) <= 1e-6 * scale + 1e-9


def test_gradient_vanishes_at_least_squares_solution():
    cs = small_set(n=2000, S=3, seed=7)
    x = cs.x.astype(np.float64)
    F = np.zeros((3, 6, 6))
    q = np.zeros((3, 6))
    for s in range(3):
        sel = cs.sector == s
        X = np.concatenate([x[sel], np.ones((sel.sum(), 1))], axis=1)
        sol, *_ = np.linalg.lstsq(X, cs.theta[sel].astype(np.float64), rcond=None)
        F[s, :3] = sol[:6].T
        q[s, :3] = sol[6]
    dF, dq = calib.grad(cs.x, cs.sector, cs.theta, cs.weight, F, q)
    # relative to the gradient at a perturbed point
    dF1, _ = calib.grad(cs.x, cs.sector, cs.theta, cs.weight, F * 1.001, q)
    assert np.max(np.abs(dF)) < 1e-6 * np.max(np.abs(dF1))
    assert np.max(np.abs(dq)) < 1e-6 * np.max(np.abs(dF1))


def test_loss_of_exact_relaxation_is_small():
    # the float relaxation of the integer constants reproduces the true
    # parameters of smeared tracks to about their resolution
    cs = small_set(n=3000, S=4, seed=3)
    consts = synth.make_constants(4)
    F = consts.F[:, 63].astype(np.float64) / 2 ** consts.oshift
    q = consts.q[:, 63].astype(np.float64) * 2.0 ** (consts.qshift - consts.oshift)
    y = calib.forward(cs.x, cs.sector, F, q)
    z = np.sum(y[:, 3:] ** 2, axis=1) * consts.unit_chi ** 2
    assert abs(z.mean() - 3.0) < 0.3
    pull = (y[:, :3] - cs.theta) * np.sqrt(cs.weight)[None, :]
    assert np.all(np.abs(pull.mean(axis=0)) < 0.1)
