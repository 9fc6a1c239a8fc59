"""Restarted GMRES (oracle), the iterative solver of Sec. V (Saad and Schultz 1986).

Textbook GMRES(m): x0 = 0, Arnoldi with modified Gram-Schmidt, complex
Givens rotations [[conj(c), conj(s)], [-s, c]], c = a/rho, s = b/rho, on the
Hessenberg matrix, stop when the residual estimate
|g_{k+1}| <= tol * ||b||; at each restart the true residual is recomputed.
"""
from __future__ import annotations

import numpy as np


def gmres(matvec, b: np.ndarray, tol: float = 1e-6, restart: int = 50, max_iter: int = 1000):
    """Solve A x = b.  Returns (x, iterations, relative residual history)."""
    n = len(b)
    x = np.zeros(n, dtype=np.complex128)
    bnorm = np.linalg.norm(b)
    hist = []
    if bnorm == 0:
        return x, 0, [0.0]
    it = 0
    while it < max_iter:
        r = b - matvec(x) if it > 0 else b.astype(np.complex128)
        beta = np.linalg.norm(r)
        hist.append(beta / bnorm)
        if beta <= tol * bnorm:
            break
        V = np.zeros((restart + 1, n), dtype=np.complex128)
        H = np.zeros((restart + 1, restart), dtype=np.complex128)
        cs = np.zeros(restart, dtype=np.complex128)
        sn = np.zeros(restart, dtype=np.complex128)
        g = np.zeros(restart + 1, dtype=np.complex128)
        g[0] = beta
        V[0] = r / beta
        j_done = 0
        for j in range(restart):
            w = matvec(V[j])
            for i in range(j + 1):
                H[i, j] = np.vdot(V[i], w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):
                t = np.conj(cs[i]) * H[i, j] + np.conj(sn[i]) * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            a, bb = H[j, j], H[j + 1, j]
            den = np.sqrt(abs(a) ** 2 + abs(bb) ** 2)
            cs[j] = a / den if den else 1.0
            sn[j] = bb / den if den else 0.0
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = np.conj(cs[j]) * g[j]
            it += 1
            j_done = j + 1
            hist.append(abs(g[j + 1]) / bnorm)
            if abs(g[j + 1]) <= tol * bnorm or it >= max_iter:
                break
        y = np.linalg.solve(np.triu(H[:j_done, :j_done]), g[:j_done])
        x = x + V[:j_done].T @ y
        if hist[-1] <= tol:
            r = b - matvec(x)
            hist.append(np.linalg.norm(r) / bnorm)
            if hist[-1] <= tol:
                break
    return x, it, hist
