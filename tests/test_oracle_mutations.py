"""Planted mistakes in the oracle (on the CPU) must trip its pins.

Each case swaps one oracle routine for a plausibly wrong variant (a dropped
term, a flipped sign, a lost factor, a wrong root) and checks that the pin
guarding that routine rejects it.
"""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import omm as O


@pytest.fixture(scope="module")
def prob(small_system):
    H, S = small_system.dense_H(), small_system.dense_S()
    Hs = O.shift(H, S, O.gershgorin_eta(H, S))
    W = small_system.W0_dense() * 2.0
    D = np.random.default_rng(4).standard_normal(W.shape) * 0.05
    return H, S, Hs, W, D, small_system.n


def _fd_gradient_ok(grad, W, H, S):
    G = grad(W, H, S)
    h = 1e-5
    rng = np.random.default_rng(1)
    D = rng.standard_normal(W.shape)
    fd = (O.functional(W + h * D, H, S) - O.functional(W - h * D, H, S)) / (2 * h)
    return abs(fd - 2.0 * np.sum(G * D)) <= 1e-7 * abs(fd)


def _interp_ok(coeffs, W, D, H, S):
    c = coeffs(W, D, H, S)
    xs = np.array([-2.0, -1.0, 0.0, 1.0, 2.0])
    vals = np.array([O.functional(W + x * D, H, S) for x in xs])
    fit = np.linalg.solve(np.vander(xs, 5, increasing=True), vals)
    return np.allclose(c, fit, rtol=1e-9, atol=1e-9 * np.abs(vals).max())


def test_pins_accept_the_oracle(prob):
    H, S, Hs, W, D, n = prob
    assert _fd_gradient_ok(O.gradient, W, Hs, S)
    assert _interp_ok(O.quartic_coeffs, W, D, Hs, S)


def test_dropped_gradient_term_is_caught(prob):
    H, S, Hs, W, D, n = prob

    def bad(W, H, S):
        HW, SW = H @ W, S @ W
        return 2.0 * (2.0 * HW - SW @ (W.T @ HW))          # lost -H W S_W
    assert not _fd_gradient_ok(bad, W, Hs, S)


def test_gradient_sign_error_is_caught(prob):
    H, S, Hs, W, D, n = prob

    def bad(W, H, S):
        HW, SW = H @ W, S @ W
        return 2.0 * (2.0 * HW - SW @ (W.T @ HW) + HW @ (W.T @ SW))
    assert not _fd_gradient_ok(bad, W, Hs, S)


def test_quartic_cross_term_error_is_caught(prob):
    H, S, Hs, W, D, n = prob

    def bad(W, D, H, S):
        c = O.quartic_coeffs(W, D, H, S)
        # forget the transposed half of W^T H D + D^T H W in the linear term
        X = W.T @ H @ D
        c = c.copy()
        c[1] -= 2.0 * 2.0 * np.trace(X)
        return c
    assert not _interp_ok(bad, W, D, Hs, S)


def test_functional_missing_spin_factor_is_caught(small_system):
    H, S, n = small_system.dense_H(), small_system.dense_S(), small_system.n
    lam, V = sla.eigh(H, S)
    W = 0.7 * V[:, :n]

    def bad(W, H, S):
        return O.functional(W, H, S) / 2.0
    expect = 2.0 * (2.0 * 0.49 - 0.7 ** 4) * lam[:n].sum()
    assert bad(W, H, S) != pytest.approx(expect, rel=1e-6)


def test_wrong_root_choice_is_caught():
    p = np.polynomial.polynomial.polymul([1, -2, 1], [4, 4, 1])
    c = np.array(p) + np.array([0, 0.5, 0, 0, 0])
    roots = np.roots([4 * c[4], 3 * c[3], 2 * c[2], c[1]]).real
    bad_x = max(roots)               # right-hand well, the higher minimum
    grid = np.linspace(-4, 3, 700001)
    best = grid[np.argmin(O.quartic(c, grid))]
    assert abs(bad_x - best) > 1e-2
    assert abs(O.line_min(c)[0] - best) < 1e-5


# --------------------------------------------------------------- preconditioned direction
def _precon_pin_ok(system, monkeypatch=None, bad=None):
    """The transformed-variables pin of the preconditioned CG, at 6 steps."""
    H, S, T = system.dense_H(), system.dense_S(), system.dense_T()
    W0 = system.W0_dense()
    eta = O.gershgorin_eta(H, S)
    tau = 2.0
    R = sla.cholesky(S + T / tau, lower=True)
    sand = lambda A: sla.solve_triangular(R, sla.solve_triangular(R, A, lower=True).T, lower=True).T
    Hv, Sv = sand(H), sand(S)
    Hv, Sv = 0.5 * (Hv + Hv.T), 0.5 * (Sv + Sv.T)
    b = O.omm_cg(Hv, Sv, R.T @ W0, tol=0.0, eta=eta, max_iter=6)
    if bad is not None:
        monkeypatch.setattr(O, "cg_direction", bad)
    a = O.omm_cg(H, S, W0, tol=0.0, eta=eta, max_iter=6, P=O.kinetic_preconditioner(S, T, tau))
    return np.allclose(a.W, sla.solve_triangular(R.T, b.W, lower=False), rtol=1e-8, atol=1e-10)


def test_precon_pin_accepts_the_oracle(small_system):
    assert _precon_pin_ok(small_system)


def test_precon_beta_with_unpreconditioned_denominator_is_caught(small_system, monkeypatch):
    def bad(G, Z, G_prev, Z_prev, D):
        if D is None:
            return -Z
        beta = max(0.0, O.frob(Z, G - G_prev) / O.frob(G_prev, G_prev))   # <G_prev, G_prev>
        D = -Z + beta * D
        return -Z if O.frob(G, D) >= 0.0 else D
    assert not _precon_pin_ok(small_system, monkeypatch, bad)


def test_precon_unpreconditioned_direction_is_caught(small_system, monkeypatch):
    def bad(G, Z, G_prev, Z_prev, D):
        if D is None:
            return -Z
        beta = max(0.0, O.frob(Z, G - G_prev) / O.frob(Z_prev, G_prev))
        D = -G + beta * D                                                   # lost P
        return -Z if O.frob(G, D) >= 0.0 else D
    assert not _precon_pin_ok(small_system, monkeypatch, bad)


# --------------------------------------------------------------- MD-step guess
def _md_pin_ok(guess):
    """The pattern-rules pin of the MD-step guess with a given implementation:
    in dense terms the extrapolated guess is mask_new * mask_1 * (2 W1 - W2)."""
    import synth
    snaps = [synth.make_md_system(3, 3, 2, seed=4, t=t, step=0.25) for t in (0.0, 1.0, 2.0)]
    pats = [s.w_pattern(4.5) for s in snaps]
    N = snaps[0].natoms

    def dense(vals, pat):
        A = np.zeros((8 * N, 2 * N))
        rp, col = pat
        for I in range(N):
            for b in range(rp[I], rp[I + 1]):
                A[8 * I:8 * I + 8, 2 * col[b]:2 * col[b] + 2] = vals[b]
        return A

    mask = [dense(np.ones((len(p[1]), 8, 2)), p) for p in pats]
    rng = np.random.default_rng(2)
    W0 = rng.standard_normal((len(pats[0][1]), 8, 2))
    W1 = rng.standard_normal((len(pats[1][1]), 8, 2))
    ok = True
    # the next snapshot's pattern, and the older one's again (blocks that left the
    # radius at the middle step and came back: zero, whatever the older step held)
    for new in (2, 0):
        got = dense(guess(W1, pats[1], pats[new], W0, pats[0]), pats[new])
        want = mask[new] * mask[1] * (2.0 * dense(W1, pats[1]) - dense(W0, pats[0]))
        ok = ok and np.allclose(got, want, rtol=0, atol=1e-15)
    return ok


def test_md_pin_accepts_the_oracle():
    assert _md_pin_ok(O.md_guess)


def test_md_guess_new_blocks_from_the_older_step_are_caught():
    def bad(W1, pat1, pat_new, W2, pat2):
        # a block W1 lacks takes -W2 (the extrapolation run over the union of the patterns)
        out = O.md_guess(W1, pat1, pat_new, W2, pat2)
        at1 = {(I, int(pat1[1][b])) for I in range(len(pat1[0]) - 1) for b in range(pat1[0][I], pat1[0][I + 1])}
        at2 = {(I, int(pat2[1][b])): b for I in range(len(pat2[0]) - 1) for b in range(pat2[0][I], pat2[0][I + 1])}
        rp, col = pat_new
        for I in range(len(rp) - 1):
            for b in range(rp[I], rp[I + 1]):
                key = (I, int(col[b]))
                if key not in at1 and key in at2:
                    out[b] = -W2[at2[key]]
        return out
    assert not _md_pin_ok(bad)


def test_md_guess_lost_factor_two_is_caught():
    def bad(W1, pat1, pat_new, W2, pat2):
        return O.md_guess(W1, pat1, pat_new) - (O.md_guess(W2, pat2, pat_new) * (O.md_guess(W1, pat1, pat_new) != 0))
    assert not _md_pin_ok(bad)


# --------------------------------------------------------------- patterns, filter, shift, screening
# Each case plants a mistake in one oracle helper and runs that helper's pin
# from test_oracle_pins, which must then fail.
import test_oracle_pins as pins  # noqa: E402


def _pin_fails(pin, monkeypatch, name, bad, *args):
    monkeypatch.setattr(O, name, bad)
    with pytest.raises(AssertionError):
        pin(*args)


def test_hs_filter_and_instead_of_or_is_caught(monkeypatch):
    bad = lambda H, S, eps: O.filter_blocks(H, eps) & O.filter_blocks(S, eps)
    _pin_fails(pins.test_hs_block_filter_keeps_a_block_when_either_matrix_is_above_eps, monkeypatch,
               "filter_hs_blocks", bad)


def test_pattern_product_dropped_entry_is_caught(monkeypatch):
    good = O.structural_pattern_product

    def bad(rp_a, col_a, rp_b, col_b, nb):
        rp, col = good(rp_a, col_a, rp_b, col_b, nb)
        r = (len(rp) - 1) // 2
        while rp[r + 1] == rp[r]:
            r += 1
        col = np.delete(col, rp[r + 1] - 1)                # a middle row loses its last block
        rp = rp.copy()
        rp[r + 1:] -= 1
        return rp, col
    _pin_fails(pins.test_structural_pattern_product_against_triple_loop, monkeypatch,
               "structural_pattern_product", bad)


def test_gershgorin_wrong_branch_is_caught(monkeypatch):
    good = O.gershgorin_eta

    def bad(H, S):      # always divides by the lower overlap bound
        Hd, Sd = (H.toarray(), S.toarray()) if hasattr(H, "toarray") else (H, S)
        g = float(np.max(np.diag(Hd) + np.abs(Hd).sum(axis=1) - np.abs(np.diag(Hd))))
        return g / float(np.min(np.diag(Sd) - (np.abs(Sd).sum(axis=1) - np.abs(np.diag(Sd)))))
    assert bad(np.diag([1.0, 2.0]), np.eye(2)) == good(np.diag([1.0, 2.0]), np.eye(2))
    _pin_fails(pins.test_gershgorin_eta_closed_form_both_branches, monkeypatch, "gershgorin_eta", bad)


def test_screening_on_one_operand_norm_is_caught(monkeypatch):
    def bad(A, B, br, bk, bc, eps):     # skips on ||A_ik|| < eps alone
        Ab, Bb = O._blocks(A, br, bk), O._blocks(B, bk, bc)
        nA = np.sum(Ab * Ab, axis=(2, 3))
        Cb = np.zeros((Ab.shape[0], Bb.shape[1], br, bc))
        for k in range(Ab.shape[1]):
            keep = ~(nA[:, k] < eps * eps)
            Cb += np.einsum("iab,jbc->ijac", Ab[:, k], Bb[k]) * keep[:, None, None, None]
        return Cb.transpose(0, 2, 1, 3).reshape(Ab.shape[0] * br, Bb.shape[1] * bc)
    _pin_fails(pins.test_screened_product_drops_exactly_the_tiny_blocks, monkeypatch, "screened_product", bad)


def test_screening_on_norm_sum_is_caught(monkeypatch):
    def bad(A, B, br, bk, bc, eps):     # ||A_ik|| + ||B_kj|| < eps
        Ab, Bb = O._blocks(A, br, bk), O._blocks(B, bk, bc)
        nA, nB = np.sqrt(np.sum(Ab * Ab, axis=(2, 3))), np.sqrt(np.sum(Bb * Bb, axis=(2, 3)))
        Cb = np.zeros((Ab.shape[0], Bb.shape[1], br, bc))
        for k in range(Ab.shape[1]):
            keep = ~(nA[:, k][:, None] + nB[k][None, :] < eps)
            Cb += np.einsum("iab,jbc->ijac", Ab[:, k], Bb[k]) * keep[:, :, None, None]
        return Cb.transpose(0, 2, 1, 3).reshape(Ab.shape[0] * br, Bb.shape[1] * bc)
    _pin_fails(pins.test_screened_product_drops_exactly_the_tiny_blocks, monkeypatch, "screened_product", bad)


def test_screened_cg_lost_dsd_term_is_caught(monkeypatch):
    """A screened CG that loses D^T S D (s2) from its line quartic and its S_W
    update no longer takes omm_cg's steps at eps = 0."""
    good = O.omm_cg_screened

    def bad(H, S, W0, bm, bn, eps, tol=1e-10, eta=None, max_iter=10000, mask=None):
        calls = {"n": 0}
        real = O.screened_product

        def spy(A, B, br, bk, bc, e):
            C = real(A, B, br, bk, bc, e)
            calls["n"] += 1
            # products per step: G (2), H'D, SD, X, Y, h2, s2; the 8th is s2 -> zero it
            if calls["n"] > 4 and (calls["n"] - 4) % 8 == 0:
                return 0.0 * C
            return C
        monkeypatch.setattr(O, "screened_product", spy)
        try:
            return good(H, S, W0, bm, bn, eps, tol=tol, eta=eta, max_iter=max_iter, mask=mask)
        finally:
            monkeypatch.setattr(O, "screened_product", real)
    monkeypatch.setattr(O, "omm_cg_screened", bad)
    with pytest.raises(AssertionError):
        pins.test_screened_cg_without_threshold_is_the_cg()
