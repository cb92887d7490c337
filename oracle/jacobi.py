"""Hand-written dense eigen-solver used to pin the oracle (test infrastructure only).

Cyclic Jacobi rotations (Jacobi 1846; textbook form, e.g. Golub & Van Loan,
"Matrix Computations", sec. 8.5) on the standard problem obtained from
H C = S C Lambda by a hand-written Cholesky factorisation S = L L^T and
forward substitution, H~ = L^-1 H L^-T.  Pure Python loops: for m <= 64 only.
No library eigen-solver, factorisation or triangular solve is used here, so
these functions are independent of the routines inside the oracle's CG.
"""
from __future__ import annotations

import math


def cholesky_lower(S):
    """L with S = L L^T (column-oriented textbook algorithm)."""
    m = len(S)
    L = [[0.0] * m for _ in range(m)]
    for j in range(m):
        d = S[j][j] - sum(L[j][k] * L[j][k] for k in range(j))
        if d <= 0.0:
            raise ValueError("matrix is not positive definite")
        L[j][j] = math.sqrt(d)
        for i in range(j + 1, m):
            L[i][j] = (S[i][j] - sum(L[i][k] * L[j][k] for k in range(j))) / L[j][j]
    return L


def forward_solve(L, B):
    """X with L X = B (L lower triangular), column by column."""
    m = len(L)
    ncol = len(B[0])
    X = [[0.0] * ncol for _ in range(m)]
    for c in range(ncol):
        for i in range(m):
            X[i][c] = (B[i][c] - sum(L[i][k] * X[k][c] for k in range(i))) / L[i][i]
    return X


def reduce_standard(H, S):
    """H~ = L^-1 H L^-T for S = L L^T."""
    L = cholesky_lower(S)
    Y = forward_solve(L, H)                       # L^-1 H
    Yt = [list(r) for r in zip(*Y)]               # (L^-1 H)^T = H L^-T
    Z = forward_solve(L, Yt)                      # L^-1 H L^-T
    m = len(Z)
    return [[0.5 * (Z[i][j] + Z[j][i]) for j in range(m)] for i in range(m)]


def jacobi_eigenvalues(A, sweeps: int = 100, tol: float = 1e-15):
    """Eigenvalues (ascending) of a symmetric matrix by cyclic Jacobi rotations."""
    m = len(A)
    a = [list(map(float, r)) for r in A]
    for _ in range(sweeps):
        off = sum(a[i][j] * a[i][j] for i in range(m) for j in range(m) if i != j)
        norm = sum(a[i][j] * a[i][j] for i in range(m) for j in range(m))
        if off <= tol * tol * norm:
            break
        for p in range(m - 1):
            for q in range(p + 1, m):
                apq = a[p][q]
                if apq == 0.0:
                    continue
                theta = (a[q][q] - a[p][p]) / (2.0 * apq)
                t = (1.0 if theta >= 0.0 else -1.0) / (abs(theta) + math.sqrt(theta * theta + 1.0))
                c = 1.0 / math.sqrt(t * t + 1.0)
                s = t * c
                for k in range(m):          # columns p, q
                    akp, akq = a[k][p], a[k][q]
                    a[k][p] = c * akp - s * akq
                    a[k][q] = s * akp + c * akq
                for k in range(m):          # rows p, q
                    apk, aqk = a[p][k], a[q][k]
                    a[p][k] = c * apk - s * aqk
                    a[q][k] = s * apk + c * aqk
    return sorted(a[i][i] for i in range(m))


def generalized_eigenvalues(H, S):
    return jacobi_eigenvalues(reduce_standard(H, S))
