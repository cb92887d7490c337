"""FP64 CPU oracle for orbital-minimization (OMM) conjugate-gradient solves.

TEST INFRASTRUCTURE ONLY.  Nothing in the product library imports, links or
calls this module; it exists so that tests, the smoke check and the CPU
baseline arm of the benchmark can compare the CUDA path with a plain,
slow, obviously correct implementation written from the paper
(arXiv 2209.05934, "Modular implementation of the linear and cubic-scaling
orbital minimization methods ...").

Notation follows the paper with the coefficient matrix C written as W (m x n,
one column per orbital):  H_W = W^T H W,  S_W = W^T S W.

Every function works on dense numpy arrays and, for the linear-scaling form,
on scipy.sparse matrices: the paper states that the sparse and dense forms
run the same equations, with sparse matrices instead of dense ones and the
gradient restricted to the sparsity pattern of W (section "Solver library").
Parity unpinned: CG iteration counts (they depend on the unnamed CG variant
and on rounding) and the converged energy of a truncated (localised) solve at
full size, which no closed form fixes; the pins in the tests cover the
localised form on small systems (full-pattern equivalence, variational
bound, stationarity by finite differences).

Library primitives used as single steps: matrix products (numpy / scipy.sparse),
polynomial roots (numpy.roots), Cholesky and triangular solves (scipy.linalg),
and one positive-definite linear solve for the kinetic-energy preconditioner.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

# status codes shared by name (not by code) with the library's C header
OK = 0
ERR_LINESEARCH = -5
ERR_MAXITER = -6


# ----------------------------------------------------------------------------
# small helpers: Frobenius inner product and trace for dense or sparse operands
# ----------------------------------------------------------------------------
def frob(A, B) -> float:
    """<A, B> = sum_ij A_ij B_ij."""
    if sp.issparse(A) or sp.issparse(B):
        A = sp.csr_matrix(A)
        return float(A.multiply(B).sum())
    return float(np.sum(np.asarray(A) * np.asarray(B)))


def trace(A) -> float:
    if sp.issparse(A):
        return float(A.diagonal().sum())
    return float(np.trace(A))


def _dense(A):
    return A.toarray() if sp.issparse(A) else np.asarray(A)


# ----------------------------------------------------------------------------
# Kim shift and its automatic choice
# ----------------------------------------------------------------------------
def shift(H, S, eta: float):
    """H' = H - eta S: the eigenspectrum shift of the Kim functional (section
    "Overview of OMM approaches", step (1) of the Kim construction)."""
    return H - eta * S


def gershgorin_eta(H, S) -> float:
    """An upper bound of the generalised eigenvalues of (H, S) from Gershgorin discs.

    lambda_max(H, S) = max_x x^T H x / x^T S x <= g_H / s_lo when g_H >= 0,
    where g_H = max_i (H_ii + sum_{j!=i} |H_ij|) bounds lambda_max(H) and
    s_lo = min_i (S_ii - sum_{j!=i} |S_ij|) bounds lambda_min(S) from below
    (must be > 0).  When g_H < 0 the bound is g_H / s_hi with
    s_hi = max_i (S_ii + sum_{j!=i} |S_ij|).  With eta >= lambda_max the shifted
    H' is negative semidefinite, so the line-search quartic has a non-negative
    leading coefficient.
    """
    if sp.issparse(H):
        dH, dS = H.diagonal(), S.diagonal()
        offH = np.asarray(abs(H).sum(axis=1)).ravel() - np.abs(dH)
        offS = np.asarray(abs(S).sum(axis=1)).ravel() - np.abs(dS)
    else:
        dH, dS = np.diag(H), np.diag(S)
        offH = np.abs(H).sum(axis=1) - np.abs(dH)
        offS = np.abs(S).sum(axis=1) - np.abs(dS)
    g_H = float(np.max(dH + offH))
    s_lo = float(np.min(dS - offS))
    s_hi = float(np.max(dS + offS))
    if s_lo <= 0.0:
        raise ValueError("S is not strictly diagonally dominant; no Gershgorin bound")
    return g_H / s_lo if g_H >= 0.0 else g_H / s_hi


# ----------------------------------------------------------------------------
# the functional, its gradient, the charge and the density matrix
# ----------------------------------------------------------------------------
def functional(W, H, S) -> float:
    """E~ = 2 Tr[(2 I - W^T S W) W^T H W]  (Eq. 4, the Ordejon-Mauri functional,
    spin factor 2 included)."""
    HW_ = W.T @ (H @ W)
    SW_ = W.T @ (S @ W)
    n = W.shape[1]
    two_I = 2.0 * (sp.identity(n, format="csr") if sp.issparse(SW_) else np.eye(n))
    return 2.0 * trace((two_I - SW_) @ HW_)


def gradient(W, H, S, mask=None):
    """G = dE~/dW* = 2 (2 H W - S W H_W - H W S_W), the libOMM gradient
    (section "Solver library"); for real W this is (1/2) dE~/dW.

    In the linear-scaling form the gradient is kept only on the sparsity
    pattern of the initial W (same section): `mask` is that pattern (a 0/1
    array or sparse matrix of W's shape), applied elementwise.
    """
    HW = H @ W
    SW = S @ W
    H_W = W.T @ HW
    S_W = W.T @ SW
    G = 2.0 * (2.0 * HW - SW @ H_W - HW @ S_W)
    return apply_mask(G, mask)


def apply_mask(A, mask):
    if mask is None:
        return A
    if sp.issparse(A) or sp.issparse(mask):
        return sp.csr_matrix(sp.csr_matrix(A).multiply(mask))
    return A * mask


def charge(W, S) -> float:
    """n_e = 2 Tr[(2 I - S_W) S_W]  (Listing 1, total charge)."""
    S_W = _dense(W.T @ (S @ W))
    n = S_W.shape[0]
    return 2.0 * float(np.trace((2.0 * np.eye(n) - S_W) @ S_W))


def density_matrix(W, S):
    """rho = 2 W (2 I - S_W) W^T  (Eq. 5)."""
    S_W = _dense(W.T @ (S @ W))
    n = S_W.shape[0]
    Wd = _dense(W)
    return 2.0 * Wd @ (2.0 * np.eye(n) - S_W) @ Wd.T


def energy_density_matrix(W, H, S, eta: float = 0.0):
    """rho_E = 2 W H_W W^T (defined with Eq. 6), plus eta*rho in the Kim construction
    (step (3)).  H is the Hamiltonian the functional was minimised for, i.e. the
    shifted H' = H - eta S when eta != 0, so that at S_W = I the result equals
    2 W H_W W^T of the unshifted H."""
    Wd = _dense(W)
    H_W = Wd.T @ (_dense(H) @ Wd)
    rho_E = 2.0 * Wd @ H_W @ Wd.T
    if eta != 0.0:
        rho_E = rho_E + eta * density_matrix(W, S)
    return rho_E


# ----------------------------------------------------------------------------
# exact line search: the quartic and its minimum
# ----------------------------------------------------------------------------
def quartic_coeffs(W, D, H, S) -> np.ndarray:
    """Coefficients c_0..c_4 of E~(W + x D) as a polynomial in x.

    The functional is quartic along a line (section "Introduction": the
    quartic's parameters are computed analytically).  Written out from the
    definition: H_W(x) = A0 + x A1 + x^2 A2 and S_W(x) = B0 + x B1 + x^2 B2 with
    A0 = W^T H W, A1 = W^T H D + D^T H W, A2 = D^T H D (same for S), and
    E~(x) = 2 (2 tr H_W(x) - <S_W(x), H_W(x)>), a product of two quadratics.
    """
    HW, HD = H @ W, H @ D
    SW, SD = S @ W, S @ D
    A = [W.T @ HW, W.T @ HD + D.T @ HW, D.T @ HD]
    B = [W.T @ SW, W.T @ SD + D.T @ SW, D.T @ SD]
    c = np.zeros(5)
    for k in range(3):
        c[k] += 2.0 * 2.0 * trace(A[k])
    for i in range(3):
        for j in range(3):
            c[i + j] -= 2.0 * frob(B[i], A[j])
    return c


def quartic(c, x):
    return c[0] + x * (c[1] + x * (c[2] + x * (c[3] + x * c[4])))


def line_min(c) -> tuple[float, int]:
    """Minimiser of the quartic c0 + c1 x + ... + c4 x^4.

    Candidates are the real roots of its derivative with a positive second
    derivative; the lowest quartic value wins, ties go to the smaller |x| and
    then to x > 0.  With c4 = c3 = 0 and c2 > 0 the parabola's vertex is taken.
    Returns (x, status); status is ERR_LINESEARCH when no minimum exists (the
    paper warns that the line minimisation can have none, section
    "Recommendations for OMM solver use").  With c4 < 0 (the Kim functional with
    eta inside the gap, where H' has positive eigenvalues) the quartic is
    unbounded below, and the lowest local minimum is taken when there is one.
    """
    c = np.asarray(c, dtype=np.float64)
    if c[4] == 0.0 and c[3] == 0.0:
        if c[2] > 0.0:
            return -c[1] / (2.0 * c[2]), OK
        return 0.0, ERR_LINESEARCH
    deriv = [4.0 * c[4], 3.0 * c[3], 2.0 * c[2], c[1]]
    while deriv and deriv[0] == 0.0:
        deriv = deriv[1:]
    roots = np.roots(deriv)
    scale = max(1.0, float(np.max(np.abs(roots)))) if roots.size else 1.0
    real = [float(r.real) for r in roots if abs(r.imag) <= 1e-10 * scale]
    cands = []
    for x in real:
        curv = 12.0 * c[4] * x * x + 6.0 * c[3] * x + 2.0 * c[2]
        if curv > 0.0:
            cands.append(x)
    if not cands:
        # a double root can have zero curvature; take the lowest real root value
        if real and c[4] > 0.0:
            cands = real
        else:
            return 0.0, ERR_LINESEARCH
    best = min(cands, key=lambda x: (quartic(c, x), abs(x), -x))
    return best, OK


# ----------------------------------------------------------------------------
# the CG minimisation
# ----------------------------------------------------------------------------
@dataclass
class Result:
    W: object
    E: float                 # E~_eta + 2 eta n at the final W (the minimised quantity)
    E_unshifted: float       # E~(W) with the unshifted H
    iters: int
    status: int
    eta: float
    history: list = field(default_factory=list)   # E_k per iteration
    orth: float = float("nan")                     # ||S_W - I||_F at the final W


def cg_direction(G, Z, G_prev, Z_prev, D):
    """Step 4 of omm_cg: the new search direction from the gradient G and the
    preconditioned gradient Z (Z = G without a preconditioner); D = None and
    G_prev = None at the first step."""
    if D is None:
        return -Z
    beta = max(0.0, frob(Z, G - G_prev) / frob(Z_prev, G_prev))
    D = -Z + beta * D
    if frob(G, D) >= 0.0:
        D = -Z
    return D


RY_EV = 13.605693122994      # one Rydberg in eV (CODATA 2018)
TAU_T_DEFAULT = 10.0 * RY_EV  # default kinetic-energy scale, 10 Ry (Table 1, OMM.TPreconScale)


def kinetic_preconditioner(S, T, tau: float = TAU_T_DEFAULT):
    """P = (S + T / tau)^-1 (Eq. 6), dense; T is the kinetic-energy matrix and
    tau the kinetic-energy scale in the energy unit of H.  One library solve
    against the identity."""
    M = _dense(S) + _dense(T) / tau
    return sla.solve(M, np.eye(M.shape[0]), assume_a="pos")


def omm_cg(H, S, W0, tol: float = 1e-10, eta: float | None = None, max_iter: int = 10000,
           orth_tol: float | None = None, mask=None, n_occ: int | None = None, P=None) -> Result:
    """Conjugate-gradient minimisation of the (shifted) Ordejon-Mauri functional.

    Steps, in the paper's order (sections "Overview of OMM approaches" and
    "Solver library", Table 1):
      0. H' = H - eta S (the Kim shift; eta=None picks the Gershgorin bound so
         the exact line search is always well posed).  The Kim functional
         proper (section "Overview of OMM approaches", steps (1)-(3)) takes
         n' = W0.shape[1] > n_occ columns and eta inside the gap.
      each iteration k:
      1. H_W = W^T H' W, S_W = W^T S W by definition; energy
         E_k = 2 (2 tr H_W - <S_W, H_W>) + 2 eta n_occ (n_occ = n' by default).
      2. stop at k >= 1 when |2 (E_k - E_{k-1}) / (E_k + E_{k-1})| < tol
         (OMM.RelTol) and, if orth_tol is given, ||S_W - I||_F < orth_tol.
      3. G = 2 (2 H'W - S W H_W - H'W S_W), restricted to W's pattern.
      4. D = -G at k = 0; otherwise Polak-Ribiere+ beta =
         max(0, <G, G - G_prev> / <G_prev, G_prev>), D = -G + beta D, and D = -G
         whenever <G, D> >= 0.  (The paper does not name its CG variant.)
         With a preconditioner P (dense only; Eq. 6, section "Overview of OMM
         approaches") the gradient is multiplied by P, Z = P G, and every G of
         step 4 that forms the direction or beta's numerator and denominator
         pairs with Z: beta = max(0, <Z, G - G_prev> / <Z_prev, G_prev>),
         D = -Z + beta D, and D = -Z whenever <G, D> >= 0.
      5. exact line search: coefficients of E~(W + x D), the quartic's minimum x.
      6. W <- W + x D.
    """
    if eta is None:
        eta = gershgorin_eta(H, S)
    Hs = shift(H, S, eta)
    n = W0.shape[1]
    n_occ = n if n_occ is None else n_occ
    W = apply_mask(W0.copy() if not sp.issparse(W0) else W0.copy(), mask)
    if sp.issparse(W):
        W = sp.csr_matrix(W)
    history = []
    E_prev = None
    G_prev = None
    Z_prev = None
    D = None
    k = 0
    if P is not None and (sp.issparse(W0) or mask is not None):
        raise ValueError("the kinetic-energy preconditioner is defined for the dense form only")
    status = OK
    while True:
        HW = Hs @ W
        SW = S @ W
        H_W = W.T @ HW
        S_W = W.T @ SW
        E = 2.0 * (2.0 * trace(H_W) - frob(S_W, H_W)) + 2.0 * eta * n_occ
        history.append(E)
        orth = float(np.linalg.norm(_dense(S_W) - np.eye(n)))
        if k >= 1:
            rel = abs(2.0 * (E - E_prev) / (E + E_prev))
            if rel < tol and (orth_tol is None or orth < orth_tol):
                break
        if k >= max_iter:
            status = ERR_MAXITER
            break
        G = apply_mask(2.0 * (2.0 * HW - SW @ H_W - HW @ S_W), mask)
        Z = G if P is None else P @ G
        D = cg_direction(G, Z, G_prev, Z_prev, D)
        c = quartic_coeffs(W, D, Hs, S)
        x, st = line_min(c)
        if st != OK:
            status = st
            break
        W = W + x * D
        E_prev = E
        G_prev = G
        Z_prev = Z
        k += 1
    E_unshifted = functional(W, H, S)
    return Result(W=W, E=E, E_unshifted=E_unshifted, iters=k, status=status, eta=eta,
                  history=history, orth=orth)


def omm_cg_cholesky(H, S, W0, tol: float = 1e-10, eta: float | None = None,
                    max_iter: int = 10000, orth_tol: float | None = None) -> Result:
    """Cholesky-reduced variant (dense only; section "Overview of OMM approaches").

    S = L L^T reduces H C = S C Lambda to the standard problem with
    H~ = L^-1 H' L^-T and overlap I; the CG runs on W~ = L^T W and the result
    is mapped back with W = L^-T W~.  Same eta as the plain form.
    """
    H = _dense(H)
    S = _dense(S)
    if eta is None:
        eta = gershgorin_eta(H, S)
    L = sla.cholesky(S, lower=True)
    Hs = shift(H, S, eta)
    Ht = sla.solve_triangular(L, sla.solve_triangular(L, Hs, lower=True).T, lower=True).T
    Ht = 0.5 * (Ht + Ht.T)
    m = H.shape[0]
    Wt0 = L.T @ np.asarray(W0)
    res = omm_cg(Ht, np.eye(m), Wt0, tol=tol, eta=0.0, max_iter=max_iter, orth_tol=orth_tol)
    W = sla.solve_triangular(L.T, res.W, lower=False)
    n = W.shape[1]
    return Result(W=W, E=res.E + 2.0 * eta * n, E_unshifted=functional(W, H, S),
                  iters=res.iters, status=res.status, eta=eta,
                  history=[e + 2.0 * eta * n for e in res.history], orth=res.orth)


# ----------------------------------------------------------------------------
# sparse-form helpers
# ----------------------------------------------------------------------------
def md_guess(W1, pat1, pat_new, W2=None, pat2=None):
    """Initial W of a new MD step (section "C† matrix initialization and update").

    The previous step's W blocks (W1 on pattern pat1) are carried onto the new
    localisation pattern pat_new: a block whose atoms moved farther apart than
    R_C is not in pat_new and is dropped; a block of pat_new that W1 does not
    hold (its atoms came within R_C) starts at zero.  With the step before
    (W2 on pat2) the guess is the linear extrapolation 2 W1 - W2 on the blocks
    W1 holds, a block that W2 lacks counting as zero there.  W1, W2: block
    values (nnz, bm, bn); patterns: (rowptr, col) over basis-atom rows.
    """
    def where(pat):
        rp, col = pat
        return {(I, int(col[b])): b for I in range(len(rp) - 1) for b in range(rp[I], rp[I + 1])}

    at1 = where(pat1)
    at2 = where(pat2) if W2 is not None else None
    rp, col = pat_new
    out = np.zeros((len(col),) + tuple(W1.shape[1:]))
    for I in range(len(rp) - 1):
        for b in range(rp[I], rp[I + 1]):
            key = (I, int(col[b]))
            if key not in at1:
                continue
            if W2 is None:
                out[b] = W1[at1[key]]
            else:
                out[b] = 2.0 * W1[at1[key]] - (W2[at2[key]] if key in at2 else 0.0)
    return out


def md_guess_dense(W1, W2=None):
    """Dense form of md_guess: W1, or the linear extrapolation 2 W1 - W2."""
    return np.array(W1, copy=True) if W2 is None else 2.0 * W1 - W2


def bsr_to_csr(rowptr, col, vals, nbrows: int, nbcols: int):
    """Assemble a scipy CSR matrix from block-CSR arrays (blocks row-major)."""
    bm, bn = vals.shape[1], vals.shape[2]
    A = sp.bsr_matrix((vals, np.asarray(col, dtype=np.int64), np.asarray(rowptr, dtype=np.int64)),
                      shape=(nbrows * bm, nbcols * bn))
    return A.tocsr()


def filter_blocks(vals, eps: float) -> np.ndarray:
    """Keep-mask of input blocks whose Frobenius norm is at least eps.

    The squared norm is summed in row-major element order, one rounded product
    and one rounded add per element, and compared strictly: ||B||^2 < eps^2
    drops the block (DBCSR-style block filtering).
    """
    flat = np.asarray(vals).reshape(vals.shape[0], -1)
    s = np.zeros(flat.shape[0])
    for t in range(flat.shape[1]):
        s = s + flat[:, t] * flat[:, t]
    return ~(s < eps * eps)


def filter_hs_blocks(H_vals, S_vals, eps: float) -> np.ndarray:
    """Keep-mask of the shared H/S pattern: a block is dropped only when both its
    H and its S block are below eps (H' = H - eta S is then negligible too)."""
    return filter_blocks(H_vals, eps) | filter_blocks(S_vals, eps)


def structural_pattern_product(rowptr_a, col_a, rowptr_b, col_b, nb_cols):
    """Boolean block pattern of A*B (block CSR in, block CSR out, sorted)."""
    na = rowptr_a.shape[0] - 1
    Pa = sp.csr_matrix((np.ones(col_a.shape[0]), col_a, rowptr_a), shape=(na, rowptr_b.shape[0] - 1))
    Pb = sp.csr_matrix((np.ones(col_b.shape[0]), col_b, rowptr_b), shape=(rowptr_b.shape[0] - 1, nb_cols))
    P = (Pa @ Pb).tocsr()
    P.sort_indices()
    return P.indptr.astype(np.int64), P.indices.astype(np.int32)


# ----------------------------------------------------------------------------
# norm-based screening of block products (linear-scaling form)
# ----------------------------------------------------------------------------
def _blocks(A, br: int, bc: int) -> np.ndarray:
    """Dense A of shape (NI*br, NJ*bc) viewed as blocks (NI, NJ, br, bc)."""
    A = _dense(A)
    NI, NJ = A.shape[0] // br, A.shape[1] // bc
    return A.reshape(NI, br, NJ, bc).transpose(0, 2, 1, 3)


def block_norms2(A, br: int, bc: int) -> np.ndarray:
    """Squared Frobenius norm of every br x bc block of A, shape (NI, NJ)."""
    Ab = _blocks(A, br, bc)
    return np.sum(Ab * Ab, axis=(2, 3))


def screened_product(A, B, br: int, bk: int, bc: int, eps: float):
    """C = A B computed block by block, skipping every block product A_ik B_kj
    with ||A_ik||_F ||B_kj||_F < eps (compared as ||A_ik||^2 ||B_kj||^2 < eps^2).

    A is cut into br x bk blocks, B into bk x bc blocks.  This is the
    norm-based filtering of the products of a DBCSR-style block-sparse
    multiply (section "Solver library": the sparse matrices and their algebra
    are DBCSR's): a skipped product changes C_ij by at most ||A_ik|| ||B_kj||
    < eps in Frobenius norm and never changes which blocks are stored.  A
    block that is not stored is a zero block, whose products are skipped for
    any eps > 0 and contribute nothing for eps = 0, so the result is the same
    on the structural pattern either way.  eps = 0 skips nothing: C = A B.
    """
    Ab, Bb = _blocks(A, br, bk), _blocks(B, bk, bc)
    nA = np.sum(Ab * Ab, axis=(2, 3))
    nB = np.sum(Bb * Bb, axis=(2, 3))
    NI, NK, NJ = Ab.shape[0], Ab.shape[1], Bb.shape[1]
    Cb = np.zeros((NI, NJ, br, bc))
    for k in range(NK):
        keep = ~(nA[:, k][:, None] * nB[k][None, :] < eps * eps)       # (NI, NJ)
        Cb += np.einsum("iab,jbc->ijac", Ab[:, k], Bb[k]) * keep[:, :, None, None]
    return Cb.transpose(0, 2, 1, 3).reshape(NI * br, NJ * bc)


def omm_cg_screened(H, S, W0, bm: int, bn: int, eps: float, tol: float = 1e-10,
                    eta: float | None = None, max_iter: int = 10000, mask=None) -> Result:
    """Linear-scaling CG with norm-based screening of every block product.

    The same minimisation as omm_cg (same shift, energy, RelTol test,
    gradient kept on W's pattern, PR+ direction, exact quartic line search),
    written with the products a block-sparse step forms (section "Solver
    library"), each one screened by screened_product with threshold eps:
      start:  H'W, SW; H_W = W^T (H'W), S_W = W^T (SW);
      step:   G = 2 (2 H'W - (SW) H_W - (H'W) S_W) on W's pattern; D;
              H'D, SD; X = W^T (H'D), Y = W^T (SD), h2 = D^T (H'D), s2 = D^T (SD);
              the line quartic's coefficients written out from
              H_W(x) = H_W + x (X + X^T) + x^2 h2, S_W(x) = S_W + x (Y + Y^T) + x^2 s2
              (H' and S symmetric) and E~(x) = 2 (2 tr H_W(x) - <S_W(x), H_W(x)>):
                c0 = 2 (2 tr H_W - <S_W, H_W>)
                c1 = 2 (4 tr X - 2 <S_W, X> - 2 <Y, H_W>)
                c2 = 2 (2 tr h2 - <S_W, h2> - 2 (<Y, X> + <Y, X^T>) - <s2, H_W>)
                c3 = 2 (-2 <Y, h2> - 2 <s2, X>)
                c4 = -2 <s2, h2>;
              W, H'W, SW carried to W + x D, and H_W, S_W by the expansions
              above with h2, s2 replaced by their symmetric parts.
    Screening makes X^T differ from D^T (H'W) and h2 from its transpose at
    the level of the skipped products; the forms above are the reading taken
    for a screened step (without screening they equal the definitions).
    Blocks: bm x bm for H and S, bm x bn for W (basis atom x orbitals of one
    atom), bn x bn for the n x n matrices.  Dense arrays in, zero blocks
    standing for blocks that are not stored.  With eps = 0 nothing is skipped
    and the iterates are omm_cg's up to rounding.
    """
    H, S = _dense(H), _dense(S)
    if eta is None:
        eta = gershgorin_eta(H, S)
    Hs = shift(H, S, eta)
    n = W0.shape[1]

    def P(A, B, br, bk, bc):
        return screened_product(A, B, br, bk, bc, eps)

    W = apply_mask(np.array(_dense(W0), dtype=np.float64), mask)
    HW, SW = P(Hs, W, bm, bm, bn), P(S, W, bm, bm, bn)
    h0, s0 = P(W.T, HW, bn, bm, bn), P(W.T, SW, bn, bm, bn)
    history, E_prev, G_prev, D = [], None, None, None
    k, status = 0, OK
    while True:
        E = 2.0 * (2.0 * np.trace(h0) - frob(s0, h0)) + 2.0 * eta * n
        history.append(E)
        orth = float(np.linalg.norm(s0 - np.eye(n)))
        if k >= 1 and abs(2.0 * (E - E_prev) / (E + E_prev)) < tol:
            break
        if k >= max_iter:
            status = ERR_MAXITER
            break
        G = apply_mask(2.0 * (2.0 * HW - P(SW, h0, bm, bn, bn) - P(HW, s0, bm, bn, bn)), mask)
        D = cg_direction(G, G, G_prev, G_prev, D)
        HD, SD = P(Hs, D, bm, bm, bn), P(S, D, bm, bm, bn)
        X, Y = P(W.T, HD, bn, bm, bn), P(W.T, SD, bn, bm, bn)
        h2, s2 = P(D.T, HD, bn, bm, bn), P(D.T, SD, bn, bm, bn)
        c = np.array([
            2.0 * (2.0 * np.trace(h0) - frob(s0, h0)),
            2.0 * (4.0 * np.trace(X) - 2.0 * frob(s0, X) - 2.0 * frob(Y, h0)),
            2.0 * (2.0 * np.trace(h2) - frob(s0, h2) - 2.0 * (frob(Y, X) + frob(Y, X.T)) - frob(s2, h0)),
            2.0 * (-2.0 * frob(Y, h2) - 2.0 * frob(s2, X)),
            -2.0 * frob(s2, h2)])
        x, st = line_min(c)
        if st != OK:
            status = st
            break
        W = W + x * D
        HW, SW = HW + x * HD, SW + x * SD
        h0 = h0 + x * (X + X.T) + x * x * (0.5 * (h2 + h2.T))
        s0 = s0 + x * (Y + Y.T) + x * x * (0.5 * (s2 + s2.T))
        E_prev, G_prev = E, G
        k += 1
    return Result(W=W, E=E, E_unshifted=functional(W, H, S), iters=k, status=status, eta=eta,
                  history=history, orth=orth)
