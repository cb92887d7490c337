"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

None of these checks re-calls the oracle routine it pins: each compares it with
a closed form, an independent library routine, a hand-written Jacobi solver,
finite differences, exact interpolation or brute force.
"""
import math

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

from oracle import jacobi
from oracle import omm as O

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def _sym(rng, m):
    A = rng.standard_normal((m, m))
    return 0.5 * (A + A.T)


# --------------------------------------------------------------- Jacobi solver
def test_jacobi_closed_form_2x2():
    a, b, c = 1.7, -0.4, -2.3
    ev = jacobi.jacobi_eigenvalues([[a, b], [b, c]])
    mid, rad = 0.5 * (a + c), math.sqrt(0.25 * (a - c) ** 2 + b * b)
    assert ev == pytest.approx([mid - rad, mid + rad], abs=1e-14)


def test_jacobi_known_spectrum_householder():
    rng = np.random.default_rng(11)
    m = 9
    v = rng.standard_normal(m)
    Q = np.eye(m) - 2.0 * np.outer(v, v) / (v @ v)          # exact reflector
    lam = np.sort(rng.uniform(-5, 5, m))
    A = Q @ np.diag(lam) @ Q.T
    ev = jacobi.jacobi_eigenvalues(A.tolist())
    np.testing.assert_allclose(ev, lam, atol=1e-12)


def test_jacobi_generalized_vs_library():
    rng = np.random.default_rng(5)
    m = 12
    H = _sym(rng, m)
    X = rng.standard_normal((m, m))
    S = X @ X.T / m + np.eye(m)
    ev = jacobi.generalized_eigenvalues(H.tolist(), S.tolist())
    ref = sla.eigh(H, S, eigvals_only=True)
    np.testing.assert_allclose(ev, ref, atol=1e-11)


# --------------------------------------------------------------- functional
def test_functional_on_scaled_eigenvectors(small_system):
    """W = a V with V the S-orthonormal lowest-n eigenvectors: S_W = a^2 I and
    H_W = a^2 Lambda, so E~ = 2 (2 a^2 - a^4) sum(lambda)."""
    H, S, n = small_system.dense_H(), small_system.dense_S(), small_system.n
    lam, V = sla.eigh(H, S)
    for a in (1.0, 0.7, 1.3):
        W = a * V[:, :n]
        expect = 2.0 * (2.0 * a * a - a ** 4) * lam[:n].sum()
        assert O.functional(W, H, S) == pytest.approx(expect, rel=1e-12)
        assert O.charge(W, S) == pytest.approx(2.0 * (2.0 * a * a - a ** 4) * n, rel=1e-12)


def test_gradient_finite_differences(small_system):
    H, S = small_system.dense_H(), small_system.dense_S()
    rng = np.random.default_rng(2)
    W = np.asfortranarray(small_system.W0_dense() * 3.0)
    G = O.gradient(W, H, S)
    h = 1e-5
    for _ in range(12):
        i, j = rng.integers(W.shape[0]), rng.integers(W.shape[1])
        Wp, Wm = W.copy(), W.copy()
        Wp[i, j] += h
        Wm[i, j] -= h
        fd = (O.functional(Wp, H, S) - O.functional(Wm, H, S)) / (2 * h)
        assert fd == pytest.approx(2.0 * G[i, j], rel=1e-6, abs=1e-8)
    # directional derivative along a random direction
    D = rng.standard_normal(W.shape)
    fd = (O.functional(W + h * D, H, S) - O.functional(W - h * D, H, S)) / (2 * h)
    assert fd == pytest.approx(2.0 * np.sum(G * D), rel=1e-7)


def test_gradient_mask_matches_pattern(small_system):
    H, S = small_system.dense_H(), small_system.dense_S()
    mask = small_system.w_mask(4.0)
    assert 0 < mask.sum() < mask.size
    W = small_system.W0_local(4.0)
    G = O.gradient(W, H, S, mask=mask)
    assert np.all(G[~mask] == 0.0)
    np.testing.assert_array_equal(G[mask], O.gradient(W, H, S)[mask])


# --------------------------------------------------------------- line search
def test_quartic_coeffs_exact_interpolation(small_system):
    """E~(W + x D) is a quartic: five samples determine it exactly."""
    H, S = small_system.dense_H(), small_system.dense_S()
    eta = O.gershgorin_eta(H, S)
    Hs = O.shift(H, S, eta)
    rng = np.random.default_rng(4)
    W = small_system.W0_dense() * 2.0
    D = rng.standard_normal(W.shape) * 0.05
    c = O.quartic_coeffs(W, D, Hs, S)
    xs = np.array([-2.0, -1.0, 0.0, 1.0, 2.0])
    vals = np.array([O.functional(W + x * D, Hs, S) for x in xs])
    V = np.vander(xs, 5, increasing=True)
    fit = np.linalg.solve(V, vals)
    np.testing.assert_allclose(c, fit, rtol=1e-9, atol=1e-9 * np.abs(vals).max())
    assert c[0] == pytest.approx(O.functional(W, Hs, S), rel=1e-13)
    G = O.gradient(W, Hs, S)
    assert c[1] == pytest.approx(2.0 * np.sum(G * D), rel=1e-12)
    assert c[4] >= 0.0          # shifted H' is negative semidefinite


def test_line_min_against_dense_sampling(small_system):
    H, S = small_system.dense_H(), small_system.dense_S()
    Hs = O.shift(H, S, O.gershgorin_eta(H, S))
    rng = np.random.default_rng(8)
    W = small_system.W0_dense()
    for trial in range(5):
        D = -O.gradient(W, Hs, S) + 0.1 * rng.standard_normal(W.shape) * trial
        c = O.quartic_coeffs(W, D, Hs, S)
        x, st = O.line_min(c)
        assert st == O.OK
        grid = np.linspace(x - 4 * abs(x) - 1, x + 4 * abs(x) + 1, 200001)
        qg = O.quartic(c, grid)
        assert O.quartic(c, x) <= qg.min() + 1e-9 * abs(qg.min())
        assert abs(grid[np.argmin(qg)] - x) <= 2 * (grid[1] - grid[0]) + 1e-6 * abs(x)
        # the quartic value at x equals the functional sampled at W + x D
        assert O.functional(W + x * D, Hs, S) == pytest.approx(O.quartic(c, x), rel=1e-10)


def test_line_min_closed_forms():
    # (x-1)^2 (x+2)^2 + 0.5 x: two wells, the left one is lower
    p = np.polynomial.polynomial.polymul([1, -2, 1], [4, 4, 1])
    c = np.array(p) + np.array([0, 0.5, 0, 0, 0])
    x, st = O.line_min(c)
    grid = np.linspace(-4, 3, 700001)
    assert st == O.OK and x == pytest.approx(grid[np.argmin(O.quartic(c, grid))], abs=1e-5)
    # parabola
    x, st = O.line_min([3.0, -4.0, 2.0, 0.0, 0.0])
    assert st == O.OK and x == pytest.approx(1.0)
    # unbounded below: no minimum
    assert O.line_min([0.0, -1.0, 1.0, 0.0, -1.0])[1] == O.ERR_LINESEARCH
    assert O.line_min([0.0, -1.0, -1.0, 0.0, 0.0])[1] == O.ERR_LINESEARCH
    # c4 < 0 with a local minimum between two maxima (Kim functional, eta in
    # the gap): -x^4 + 2x^2 - 0.5x has its wells' bottom near 0.127 and maxima
    # near -1.06 and 0.93; brute force between the maxima
    c = [0.0, -0.5, 2.0, 0.0, -1.0]
    x, st = O.line_min(c)
    grid = np.linspace(-1.0, 0.9, 1900001)
    assert st == O.OK and x == pytest.approx(grid[np.argmin(O.quartic(c, grid))], abs=2e-6)
    assert abs(-4 * x ** 3 + 4 * x - 0.5) < 1e-12


def test_gershgorin_bounds_spectrum(c1_system):
    H, S = c1_system.dense_H(), c1_system.dense_S()
    eta = O.gershgorin_eta(H, S)
    lam = sla.eigh(H, S, eigvals_only=True)
    assert eta >= lam[-1]
    assert np.linalg.eigvalsh(O.shift(H, S, eta)).max() <= 1e-12


# --------------------------------------------------------------- CG minimum
def test_cg_reaches_jacobi_ground_state(tiny_system):
    H, S, n = tiny_system.dense_H(), tiny_system.dense_S(), tiny_system.n
    res = O.omm_cg(H, S, tiny_system.W0_dense(), tol=1e-15, max_iter=5000)
    assert res.status in (O.OK, O.ERR_MAXITER)
    lam = jacobi.generalized_eigenvalues(H.tolist(), S.tolist())
    e_min = 2.0 * sum(lam[:n])
    assert res.E == pytest.approx(e_min, rel=1e-11)
    assert res.E_unshifted == pytest.approx(e_min, rel=1e-9)
    S_W = res.W.T @ S @ res.W
    assert np.linalg.norm(S_W - np.eye(n)) < 1e-6
    assert O.charge(res.W, S) == pytest.approx(2 * n, rel=1e-10)
    rho = O.density_matrix(res.W, S)
    # (rho/2) S (rho/2) = rho/2: projector onto the occupied subspace
    np.testing.assert_allclose(0.25 * rho @ S @ rho, 0.5 * rho, atol=1e-7)


def test_density_matrices_at_the_minimum(small_system):
    """At the exact minimum, rho = 2 V V^T and rho_E = 2 V Lambda V^T for the n
    lowest S-orthonormal generalised eigenvectors V (Eq. 5 and the energy
    density defined with Eq. 6), with the shifted Hamiltonian and its eta."""
    H, S, n = small_system.dense_H(), small_system.dense_S(), small_system.n
    lam, V = sla.eigh(H, S)
    res = O.omm_cg(H, S, small_system.W0_dense(), tol=1e-15, max_iter=5000)
    Vn = V[:, :n]
    np.testing.assert_allclose(O.density_matrix(res.W, S), 2 * Vn @ Vn.T, atol=1e-7)
    Hs = O.shift(H, S, res.eta)
    np.testing.assert_allclose(O.energy_density_matrix(res.W, Hs, S, res.eta),
                               2 * Vn @ np.diag(lam[:n]) @ Vn.T, atol=1e-6)


def test_kim_functional_reaches_jacobi_ground_state(tiny_system):
    """Kim construction (section "Overview of OMM approaches", steps (1)-(3)):
    n' = n + 4 columns, eta inside the gap, energy + 2 eta n.  The minimum is
    still 2 x the sum of the n lowest eigenvalues; the extra columns carry no
    charge (2 Tr[(2I - S_W) S_W] = 2n) and rho/2 is the occupied projector."""
    H, S, n = tiny_system.dense_H(), tiny_system.dense_S(), tiny_system.n
    lam = jacobi.generalized_eigenvalues(H.tolist(), S.tolist())
    eta = 0.5 * (lam[n - 1] + lam[n])
    rng = np.random.default_rng(5)
    # small start: along an unoccupied direction the functional 4 lam t^2 - 2 lam t^4
    # (lam > 0) has its barrier at t = 1, so the columns start well inside it
    W0 = 0.2 * np.hstack([tiny_system.W0_dense(), rng.standard_normal((tiny_system.m, 4)) / np.sqrt(tiny_system.m)])
    res = O.omm_cg(H, S, W0, tol=1e-15, eta=eta, n_occ=n, max_iter=20000)
    assert res.status in (O.OK, O.ERR_MAXITER)
    e_min = 2.0 * sum(lam[:n])
    assert res.E == pytest.approx(e_min, rel=1e-9)
    assert O.charge(res.W, S) == pytest.approx(2 * n, rel=1e-8)
    rho = O.density_matrix(res.W, S)
    np.testing.assert_allclose(0.25 * rho @ S @ rho, 0.5 * rho, atol=1e-6)


def test_cg_c1_energy_and_monotone(c1_system):
    H, S, n = c1_system.dense_H(), c1_system.dense_S(), c1_system.n
    res = O.omm_cg(H, S, c1_system.W0_dense(), tol=1e-12)
    assert res.status == O.OK
    e_min = 2.0 * sla.eigh(H, S, eigvals_only=True)[:n].sum()
    assert res.E == pytest.approx(e_min, rel=1e-10)
    hist = np.array(res.history)
    assert np.all(np.diff(hist) <= 1e-12 * np.abs(hist[1:]))


def test_cholesky_variant_same_minimum(small_system):
    H, S, n = small_system.dense_H(), small_system.dense_S(), small_system.n
    a = O.omm_cg(H, S, small_system.W0_dense(), tol=1e-14)
    b = O.omm_cg_cholesky(H, S, small_system.W0_dense(), tol=1e-14)
    assert b.E == pytest.approx(a.E, rel=1e-11)
    np.testing.assert_allclose(O.density_matrix(b.W, S), O.density_matrix(a.W, S), atol=1e-6)


# --------------------------------------------------------------- kinetic-energy preconditioning
def _transformed_problem(H, S, T, tau, W0):
    """M = S + T / tau = R R^T; in the variables V = R^T W the functional is the
    same with H_V = R^-1 H R^-T and S_V = R^-1 S R^-T, and its gradient is
    R^-1 G.  Plain CG there, mapped back with W = R^-T V, is CG preconditioned
    with P = M^-1 = R^-T R^-1 (Eq. 6)."""
    R = sla.cholesky(S + T / tau, lower=True)

    def sandwich(A):
        X = sla.solve_triangular(R, sla.solve_triangular(R, A, lower=True).T, lower=True).T
        return 0.5 * (X + X.T)
    return R, sandwich(H), sandwich(S), R.T @ W0


@pytest.mark.parametrize("tau", [2.0, O.TAU_T_DEFAULT])
def test_preconditioned_cg_is_cg_in_transformed_variables(small_system, tau):
    """Every iterate of the preconditioned CG equals R^-T times the iterate of
    plain CG run on the transformed problem, for the same eta: this fixes the
    product Z = P G, both dot products of beta and the restart test."""
    H, S, T = small_system.dense_H(), small_system.dense_S(), small_system.dense_T()
    W0 = small_system.W0_dense()
    eta = O.gershgorin_eta(H, S)
    R, Hv, Sv, V0 = _transformed_problem(H, S, T, tau, W0)
    P = O.kinetic_preconditioner(S, T, tau)
    for k in (1, 3, 8, 20):
        a = O.omm_cg(H, S, W0, tol=0.0, eta=eta, max_iter=k, P=P)
        b = O.omm_cg(Hv, Sv, V0, tol=0.0, eta=eta, max_iter=k)
        assert a.iters == b.iters == k
        np.testing.assert_allclose(a.history, b.history, rtol=1e-12)
        np.testing.assert_allclose(a.W, sla.solve_triangular(R.T, b.W, lower=False), rtol=1e-8, atol=1e-10)


def test_preconditioner_without_kinetic_term_is_the_cholesky_variant(small_system):
    """T = 0 gives P = S^-1, i.e. CG on the Cholesky-reduced problem (the
    oracle's reduction runs on W~ = L^T W with overlap I)."""
    H, S = small_system.dense_H(), small_system.dense_S()
    W0 = small_system.W0_dense()
    eta = O.gershgorin_eta(H, S)
    P = O.kinetic_preconditioner(S, np.zeros_like(S), 1.0)
    np.testing.assert_allclose(P @ S, np.eye(S.shape[0]), atol=1e-12)
    for k in (2, 6):
        a = O.omm_cg(H, S, W0, tol=0.0, eta=eta, max_iter=k, P=P)
        b = O.omm_cg_cholesky(H, S, W0, tol=0.0, eta=eta, max_iter=k)
        np.testing.assert_allclose(a.history, b.history, rtol=1e-12)
        np.testing.assert_allclose(a.W, b.W, rtol=1e-8, atol=1e-10)


def test_preconditioned_cg_reaches_jacobi_ground_state(tiny_system):
    """Preconditioning changes the path, not the minimum: 2 x the sum of the n
    lowest generalised eigenvalues, S_W = I, charge 2n."""
    H, S, T, n = tiny_system.dense_H_kinetic(), tiny_system.dense_S(), tiny_system.dense_T(), tiny_system.n
    P = O.kinetic_preconditioner(S, T)
    res = O.omm_cg(H, S, tiny_system.W0_dense(), tol=1e-15, max_iter=5000, P=P)
    assert res.status in (O.OK, O.ERR_MAXITER)
    lam = jacobi.generalized_eigenvalues(H.tolist(), S.tolist())
    assert res.E == pytest.approx(2.0 * sum(lam[:n]), rel=1e-11)
    assert np.linalg.norm(res.W.T @ S @ res.W - np.eye(n)) < 1e-6
    hist = np.array(res.history)
    assert np.all(np.diff(hist) <= 1e-12 * np.abs(hist[1:]))


# --------------------------------------------------------------- linear-scaling form
def _sparse_inputs(sysm, radius):
    rp, col, Hv, Sv = sysm.bsr()
    N = sysm.natoms
    H = O.bsr_to_csr(rp, col, Hv, N, N)
    S = O.bsr_to_csr(rp, col, Sv, N, N)
    mask = sp.csr_matrix(sysm.w_mask(radius).astype(np.float64))
    W0 = sp.csr_matrix(sysm.W0_local(radius))
    return H, S, W0, mask


def test_sparse_full_pattern_equals_dense(small_system):
    H, S, _, _ = _sparse_inputs(small_system, 100.0)
    W0 = small_system.W0_dense()
    mask = sp.csr_matrix(np.ones(W0.shape))
    a = O.omm_cg(H, S, sp.csr_matrix(W0), tol=1e-13, mask=mask)
    b = O.omm_cg(small_system.dense_H(), small_system.dense_S(), W0, tol=1e-13)
    assert a.iters == b.iters
    assert a.E == pytest.approx(b.E, rel=1e-12)


def test_sparse_types_match_dense_masked():
    """The scipy.sparse path and the dense-with-mask path give the same iterates."""
    import synth
    sysm = synth.make_system(3, 3, 2, seed=2)
    Hs, Ss, W0, mask = _sparse_inputs(sysm, 3.6)
    a = O.omm_cg(Hs, Ss, W0, tol=0.0, max_iter=40, mask=mask)
    b = O.omm_cg(sysm.dense_H(), sysm.dense_S(), sysm.W0_local(3.6), tol=0.0, max_iter=40,
                 mask=sysm.w_mask(3.6))
    assert a.iters == b.iters == 40
    np.testing.assert_allclose(a.history, b.history, rtol=1e-12)
    np.testing.assert_allclose(a.W.toarray(), b.W, atol=1e-12)


def test_truncated_minimum_is_variational():
    """The localised minimum lies above the dense one and drops as R_C grows
    (cf. the truncation-error study, Fig. 10)."""
    import synth
    sysm = synth.make_system(3, 3, 2, seed=2)
    H, S, n = sysm.dense_H(), sysm.dense_S(), sysm.n
    e_dense = 2.0 * sla.eigh(H, S, eigvals_only=True)[:n].sum()
    energies = []
    for radius in (2.8, 3.6, 4.5):
        mask = sysm.w_mask(radius)
        res = O.omm_cg(H, S, sysm.W0_local(radius), tol=1e-10, mask=mask, max_iter=4000)
        assert res.status == O.OK
        assert np.all(res.W[~mask] == 0.0)
        energies.append(res.E)
    assert energies[0] > energies[1] > energies[2] > e_dense


def test_truncated_minimum_stationary_brute_force():
    """At the localised minimum the functional is flat along every allowed
    entry (finite differences), and not along a forbidden one."""
    import synth
    sysm = synth.make_system(2, 2, 2, seed=1)
    H, S = sysm.dense_H(), sysm.dense_S()
    mask = sysm.w_mask(3.0)
    assert 0 < mask.sum() < mask.size
    res = O.omm_cg(H, S, sysm.W0_local(3.0), tol=1e-15, max_iter=6000, mask=mask)
    Hsh = O.shift(H, S, res.eta)
    W = res.W
    rng = np.random.default_rng(0)
    idx = np.argwhere(mask)
    h = 1e-5
    for i, j in idx[rng.choice(len(idx), 10, replace=False)]:
        Wp, Wm = W.copy(), W.copy()
        Wp[i, j] += h
        Wm[i, j] -= h
        fd = (O.functional(Wp, Hsh, S) - O.functional(Wm, Hsh, S)) / (2 * h)
        assert abs(fd) < 1e-5
    G_full = O.gradient(W, Hsh, S)
    assert np.abs(G_full[~mask]).max() > 1e-2


def test_block_filter_threshold():
    vals = np.zeros((3, 2, 2))
    vals[0, 0, 0] = 1e-9                     # ||B|| = 1e-9 < 1e-8: dropped
    vals[1, 1, 1] = 1e-8                     # exactly eps: kept (strict comparison)
    vals[2] = 0.3
    assert list(O.filter_blocks(vals, 1e-8)) == [False, True, True]


# --------------------------------------------------------------- MD-step guess
def _blocks_dense(vals, pat, nbr, nbc, bm, bn):
    """Expand block values on a block-CSR pattern into a dense array (test-side loop)."""
    rp, col = pat
    A = np.zeros((nbr * bm, nbc * bn))
    for I in range(nbr):
        for b in range(rp[I], rp[I + 1]):
            J = col[b]
            A[I * bm:(I + 1) * bm, J * bn:(J + 1) * bn] = vals[b]
    return A


def _pattern_mask(pat, nbr, nbc, bm, bn):
    rp, col = pat
    return _blocks_dense(np.ones((len(col), bm, bn)), pat, nbr, nbc, bm, bn)


def test_md_guess_same_pattern_is_identity(small_system):
    pat = small_system.w_pattern(4.5)
    W = np.random.default_rng(0).standard_normal((len(pat[1]), 8, 2))
    np.testing.assert_array_equal(O.md_guess(W, pat, pat), W)


def test_md_guess_extrapolation_is_exact_on_a_straight_line(small_system):
    """W(t) = A + t B on a fixed pattern: the guess from t = 1 and t = 0 is W(2)."""
    pat = small_system.w_pattern(4.5)
    rng = np.random.default_rng(1)
    A, B = rng.standard_normal((2, len(pat[1]), 8, 2))
    np.testing.assert_allclose(O.md_guess(A + B, pat, pat, A, pat), A + 2 * B, rtol=1e-14, atol=1e-14)
    Wd = rng.standard_normal((64, 16))
    np.testing.assert_allclose(O.md_guess_dense(Wd + 0.5, Wd), Wd + 1.0, rtol=1e-14, atol=1e-14)


def test_md_guess_pattern_rules():
    """Three snapshots of a trajectory whose W pattern changes: in dense terms the
    guess is mask_new * mask_1 * (2 W1 - W2) -- blocks that left the radius are
    gone, blocks that entered it are zero, W2's missing blocks count as zero."""
    import synth
    snaps = [synth.make_md_system(3, 3, 2, seed=4, t=t, step=0.25) for t in (0.0, 1.0, 2.0)]
    pats = [s.w_pattern(4.5) for s in snaps]
    nbr, nbc = snaps[0].natoms, snaps[0].natoms
    masks = [_pattern_mask(p, nbr, nbc, 8, 2) for p in pats]
    assert np.any(masks[0] != masks[1]) and np.any(masks[1] != masks[2])
    assert np.any(masks[1] * (1 - masks[2]) > 0) or np.any(masks[2] * (1 - masks[1]) > 0)
    rng = np.random.default_rng(2)
    W0 = rng.standard_normal((len(pats[0][1]), 8, 2))
    W1 = rng.standard_normal((len(pats[1][1]), 8, 2))
    d0 = _blocks_dense(W0, pats[0], nbr, nbc, 8, 2)
    d1 = _blocks_dense(W1, pats[1], nbr, nbc, 8, 2)
    carried = O.md_guess(W1, pats[1], pats[2])
    np.testing.assert_array_equal(_blocks_dense(carried, pats[2], nbr, nbc, 8, 2), masks[2] * masks[1] * d1)
    extra = O.md_guess(W1, pats[1], pats[2], W0, pats[0])
    np.testing.assert_allclose(_blocks_dense(extra, pats[2], nbr, nbc, 8, 2),
                               masks[2] * masks[1] * (2.0 * d1 - d0), rtol=0, atol=1e-15)


def test_md_system_is_smooth_in_time():
    """The MD snapshots share seeds per pair: a small time step moves H and S by
    a small amount (needed for a guess from earlier steps to help)."""
    import synth
    a = synth.make_md_system(3, 3, 2, seed=4, t=1.0, step=0.05)
    b = synth.make_md_system(3, 3, 2, seed=4, t=1.001, step=0.05)
    assert np.abs(a.dense_H() - b.dense_H()).max() < 1e-3
    assert np.abs(a.dense_S() - b.dense_S()).max() < 1e-3


# --------------------------------------------------------------- pattern, filter and shift helpers
def _pattern_product_by_hand(rp_a, col_a, rp_b, col_b):
    """Block pattern of A B by a plain loop over block triples (i, k, j)."""
    rows = []
    for i in range(len(rp_a) - 1):
        cols = set()
        for a in range(rp_a[i], rp_a[i + 1]):
            k = col_a[a]
            for b in range(rp_b[k], rp_b[k + 1]):
                cols.add(int(col_b[b]))
        rows.append(sorted(cols))
    rp = np.cumsum([0] + [len(r) for r in rows])
    return rp, np.array([c for r in rows for c in r], dtype=np.int64)


def test_structural_pattern_product_small_by_hand():
    """A 3 x 3 block pattern times a 3 x 2 one, worked out on paper:
    A = [[x . x], [. x .], [x . x]], B = [[x .], [. x], [. .]]  ->  A B = [[x .], [. x], [x .]]."""
    rp_a, col_a = np.array([0, 2, 3, 5]), np.array([0, 2, 1, 0, 2], dtype=np.int32)
    rp_b, col_b = np.array([0, 1, 2, 2]), np.array([0, 1], dtype=np.int32)
    rp, col = O.structural_pattern_product(rp_a, col_a, rp_b, col_b, 2)
    assert rp.tolist() == [0, 1, 2, 3]
    assert col.tolist() == [0, 1, 0]


def test_structural_pattern_product_against_triple_loop():
    """P_HW = P_H P_W and P_N = P_W^T P_HW of a 50-atom system (5 x 5 x 2 grid,
    W radius 2.8 A) against a triple loop over blocks."""
    import synth
    sysm = synth.make_system(5, 5, 2, seed=4)
    N = sysm.natoms
    rp_h, col_h, _, _ = sysm.bsr()
    rp_w, col_w = sysm.w_pattern(2.8)
    rp_hw, col_hw = O.structural_pattern_product(rp_h, col_h, rp_w, col_w, N)
    ref_rp, ref_col = _pattern_product_by_hand(rp_h, col_h, rp_w, col_w)
    assert rp_hw.tolist() == ref_rp.tolist() and col_hw.tolist() == ref_col.tolist()
    # W^T in block CSR by a loop, then P_N
    t_rows = [[] for _ in range(N)]
    for I in range(N):
        for b in range(rp_w[I], rp_w[I + 1]):
            t_rows[col_w[b]].append(I)
    rp_wt = np.cumsum([0] + [len(r) for r in t_rows])
    col_wt = np.array([c for r in t_rows for c in r], dtype=np.int32)
    rp_n, col_n = O.structural_pattern_product(rp_wt, col_wt, rp_hw, col_hw, N)
    ref_rp, ref_col = _pattern_product_by_hand(rp_wt, col_wt, rp_hw, col_hw)
    assert rp_n.tolist() == ref_rp.tolist() and col_n.tolist() == ref_col.tolist()
    assert 0 < len(col_n) < N * N                 # neither empty nor dense at this radius


def test_hs_block_filter_keeps_a_block_when_either_matrix_is_above_eps():
    """The shared H/S pattern keeps a block pair when H or S is at least eps."""
    H = np.zeros((4, 2, 2))
    S = np.zeros((4, 2, 2))
    H[0, 0, 1] = 3e-8                          # H above, S zero      -> kept
    S[1, 1, 0] = 2e-8                          # S above, H zero      -> kept
    H[2, 0, 0], S[2, 1, 1] = 5e-9, 6e-9        # both below           -> dropped
    H[3, 0, 0], S[3, 0, 0] = 1e-8, 0.0         # H exactly at eps     -> kept (strict)
    assert list(O.filter_hs_blocks(H, S, 1e-8)) == [True, True, False, True]


def test_gershgorin_eta_closed_form_both_branches():
    """eta from hand-computed Gershgorin discs: g_H / s_lo when g_H >= 0, g_H / s_hi
    when g_H < 0; each is an upper bound of the generalised spectrum, and in the
    g_H < 0 case the other quotient would not be."""
    S = np.array([[1.0, 0.1, 0.0], [0.1, 1.0, 0.2], [0.0, 0.2, 1.0]])
    s_lo, s_hi = 0.7, 1.3                      # rows: 1 -+ 0.1, 1 -+ 0.3, 1 -+ 0.2
    H_pos = np.array([[2.0, 1.0, -1.0], [1.0, -3.0, 0.5], [-1.0, 0.5, 1.0]])
    g_pos = 4.0                                # max(2 + 2, -3 + 1.5, 1 + 1.5)
    H_neg = np.array([[-10.0, 1.0, 0.0], [1.0, -12.0, 2.0], [0.0, 2.0, -9.0]])
    g_neg = -7.0                               # max(-10 + 1, -12 + 3, -9 + 2)
    for H, expect in ((H_pos, g_pos / s_lo), (H_neg, g_neg / s_hi)):
        eta = O.gershgorin_eta(H, S)
        assert eta == pytest.approx(expect, rel=1e-15)
        assert eta >= sla.eigh(H, S, eigvals_only=True)[-1]
        assert O.gershgorin_eta(sp.csr_matrix(H), sp.csr_matrix(S)) == pytest.approx(expect, rel=1e-15)
    assert g_neg / s_lo < sla.eigh(H_neg, S, eigvals_only=True)[-1]   # the wrong quotient fails


# --------------------------------------------------------------- screening of block products
def _screen_case(seed=0):
    """Block operands whose norms span decades, with a few tiny blocks in each."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((5 * 4, 6 * 3))
    B = rng.standard_normal((6 * 3, 4 * 2))
    tiny_a = [(0, 1), (3, 4), (4, 0)]
    tiny_b = [(2, 3), (5, 1)]
    for i, k in tiny_a:
        A[4 * i:4 * i + 4, 3 * k:3 * k + 3] *= 1e-10
    for k, j in tiny_b:
        B[3 * k:3 * k + 3, 2 * j:2 * j + 2] *= 1e-10
    A[8:12, 6:9] = 0.0                          # a block that is not stored
    return A, B, tiny_a, tiny_b


def test_screened_product_without_threshold_is_the_product():
    A, B, _, _ = _screen_case()
    np.testing.assert_allclose(O.screened_product(A, B, 4, 3, 2, 0.0), A @ B, rtol=0, atol=1e-13)


def test_screened_product_drops_exactly_the_tiny_blocks():
    """Every product with a 1e-10 block is below eps = 1e-6 and every other one
    is above it, so screening equals the plain product with those blocks zeroed."""
    A, B, tiny_a, tiny_b = _screen_case()
    nA, nB = np.sqrt(O.block_norms2(A, 4, 3)), np.sqrt(O.block_norms2(B, 3, 2))
    big = np.outer(nA[nA > 1e-5].min(keepdims=True), nB[nB > 1e-5].min(keepdims=True))
    assert big.min() > 1e-3 and nA.max() * 1e-10 * 10 < 1e-6
    A0, B0 = A.copy(), B.copy()
    for i, k in tiny_a:
        A0[4 * i:4 * i + 4, 3 * k:3 * k + 3] = 0.0
    for k, j in tiny_b:
        B0[3 * k:3 * k + 3, 2 * j:2 * j + 2] = 0.0
    C = O.screened_product(A, B, 4, 3, 2, 1e-6)
    np.testing.assert_allclose(C, A0 @ B0, rtol=0, atol=1e-13)
    assert np.abs(C - A @ B).max() > 1e-12     # the skipped products were not zero


def test_screened_product_error_bound():
    """||C_ij - (A B)_ij||_F <= sum of ||A_ik|| ||B_kj|| over the skipped k."""
    rng = np.random.default_rng(3)
    A = rng.standard_normal((24, 24)) * np.kron(10.0 ** rng.uniform(-4, 0, (6, 6)), np.ones((4, 4)))
    B = rng.standard_normal((24, 12)) * np.kron(10.0 ** rng.uniform(-4, 0, (6, 6)), np.ones((4, 2)))
    eps = 1e-4
    C = O.screened_product(A, B, 4, 4, 2, eps)
    nA = np.sqrt(np.sum(A.reshape(6, 4, 6, 4) ** 2, axis=(1, 3)))
    nB = np.sqrt(np.sum(B.reshape(6, 4, 6, 2) ** 2, axis=(1, 3)))
    err = np.sqrt(np.sum((C - A @ B).reshape(6, 4, 6, 2) ** 2, axis=(1, 3)))
    prod = nA[:, :, None] * nB[None, :, :]                   # (i, k, j)
    skipped = np.where(prod < eps, prod, 0.0).sum(axis=1)
    assert np.all(err <= skipped * (1 + 1e-12) + 1e-15)
    assert skipped.max() > 0                                  # some products were skipped


def test_screened_cg_without_threshold_is_the_cg():
    """The screened linear-scaling CG with eps = 0 takes omm_cg's steps."""
    import synth
    sysm = synth.make_system(3, 3, 2, seed=2)
    H, S, mask, W0 = sysm.dense_H(), sysm.dense_S(), sysm.w_mask(3.6), sysm.W0_local(3.6)
    a = O.omm_cg_screened(H, S, W0, 8, 2, 0.0, tol=0.0, max_iter=25, mask=mask)
    b = O.omm_cg(H, S, W0, tol=0.0, max_iter=25, mask=mask)
    np.testing.assert_allclose(a.history, b.history, rtol=1e-13)
    np.testing.assert_allclose(a.W, b.W, atol=1e-12)
    c = O.omm_cg_screened(H, S, W0, 8, 2, 0.0, tol=1e-12, mask=mask)
    d = O.omm_cg(H, S, W0, tol=1e-12, mask=mask)
    assert c.status == d.status == O.OK and c.E == pytest.approx(d.E, rel=1e-12)
