"""Davidson eigensolver for the lowest eigenpair of H_eff (Sec. II).

Oracle module (test infrastructure only).  The paper names the Lanczos or
Davidson algorithm for the diagonalisation that takes 85-90 % of the run
time but gives no details; the reading used here: diagonal preconditioner
t = r / (H_ii - theta) with |H_ii - theta| clamped to >= 1e-12, classical
Gram-Schmidt applied twice, Rayleigh-Ritz with a dense symmetric
eigensolver, subspace of at most ``max_sub`` vectors restarted on the two
lowest Ritz vectors, converged when ||H x - theta x||_2 <= tol.

Parity: pinned against a dense eigensolver on explicitly assembled H_eff.
"""
from __future__ import annotations

import numpy as np


def fix_sign(x):
    i = int(np.argmax(np.abs(x)))
    return x if x[i] >= 0 else -x


def davidson(apply, diag, x0, tol=1e-8, max_sub=24, keep=2, max_iter=200):
    """Returns (theta, x, residual norm, iterations)."""
    x0 = np.asarray(x0, dtype=np.float64)
    V = [x0 / np.linalg.norm(x0)]
    AV = [apply(V[0])]
    theta, x, res = None, None, np.inf
    for it in range(1, max_iter + 1):
        Vm = np.array(V).T
        AVm = np.array(AV).T
        Hs = Vm.T @ AVm
        Hs = 0.5 * (Hs + Hs.T)
        w, Y = np.linalg.eigh(Hs)
        theta = w[0]
        y = Y[:, 0]
        x = Vm @ y
        r = AVm @ y - theta * x
        res = np.linalg.norm(r)
        if res <= tol:
            return theta, fix_sign(x), res, it
        den = diag - theta
        small = np.abs(den) < 1e-12
        den[small] = np.where(den[small] >= 0, 1e-12, -1e-12)
        t = r / den
        for _ in range(2):
            t = t - Vm @ (Vm.T @ t)
        nt = np.linalg.norm(t)
        if len(V) >= max_sub:
            nk = min(keep, Y.shape[1])
            Vn = Vm @ Y[:, :nk]
            AVn = AVm @ Y[:, :nk]
            V = [Vn[:, j] for j in range(nk)]
            AV = [AVn[:, j] for j in range(nk)]
            Vm = Vn
            for _ in range(2):
                t = t - Vm @ (Vm.T @ t)
            nt = np.linalg.norm(t)
        if nt < 1e-14:
            return theta, fix_sign(x), res, it
        t = t / nt
        V.append(t)
        AV.append(apply(t))
    return theta, fix_sign(x), res, max_iter
