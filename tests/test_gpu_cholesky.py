"""Cholesky-reduced variant (S = L L^T, CG on W~ = L^T W with overlap I) on the
GPU, through the C ABI, against the oracle's reduction and the plain form."""
import numpy as np
import pytest

from oracle import omm as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def omm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_2209_05934_gb300 import omm as _omm
    _omm.lib()
    return _omm


def dev(a):
    return torch.from_numpy(np.asfortranarray(a)).to("cuda")


def empty_cm(rows, cols):
    return torch.zeros((cols, rows), dtype=torch.float64, device="cuda").T


# (3,3,3): m=216 spans several 64-wide panels plus a ragged one; (5,5,3): m=600, ragged tail 24
@pytest.mark.parametrize("dims", [(3, 3, 3), (4, 4, 4), (5, 5, 3)])
def test_cholesky_fp64_matches_oracle(omm, dims):
    import synth
    sysm = synth.make_system(*dims, seed=1)
    H, S = sysm.dense_H(), sysm.dense_S()
    W0 = np.asfortranarray(sysm.W0_dense())
    s = omm.Solver(sysm.m, sysm.n, 8, cholesky=1)
    s.set_HS(dev(H), dev(S))
    eta = s.diag().eta
    assert eta == pytest.approx(O.gershgorin_eta(H, S), rel=1e-14)
    W = empty_cm(sysm.m, sysm.n)
    E, iters, st = s.solve(dev(W0), tol=1e-12, W_out=W)
    ref = O.omm_cg_cholesky(H, S, W0, tol=1e-12, eta=eta)
    assert st == omm.OK and ref.status == O.OK
    assert abs(E - ref.E) / abs(ref.E) < 1e-10
    # H~ is rounded differently on the two sides (blocked triangular solves vs
    # LAPACK's), so the trajectories part slowly and the 1e-12 test fires a few
    # steps apart
    assert abs(iters - ref.iters) <= max(3, ref.iters // 10)
    Wn = W.cpu().numpy()
    # returned W lives in the original basis: S-orthonormal, same density matrix
    # (an energy converged to 1e-12 fixes W only to about its square root, so the
    # two runs' rounding paths leave differences of a few 1e-6 in rho)
    assert np.linalg.norm(Wn.T @ S @ Wn - np.eye(sysm.n)) < 1e-5
    np.testing.assert_allclose(O.density_matrix(Wn, S), O.density_matrix(ref.W, S), atol=2e-5)
    # energy of the returned W through the plain functional
    e_w = O.functional(Wn, O.shift(H, S, eta), S) + 2 * eta * sysm.n
    assert abs(e_w - E) / abs(E) < 1e-10
    # OMM_ARRAY_W reports the same original-basis W
    np.testing.assert_array_equal(s.get_array(omm.ARRAY_W), Wn)
    s.close()


def test_cholesky_fixed_iterations_track_oracle(omm):
    """k CG steps on the reduced problem: the back-transformed iterate equals the oracle's."""
    import synth
    sysm = synth.make_system(3, 4, 3, seed=3)
    H, S = sysm.dense_H(), sysm.dense_S()
    W0 = np.asfortranarray(sysm.W0_dense())
    for k in (1, 3, 8):
        s = omm.Solver(sysm.m, sysm.n, 8, cholesky=1, max_iter=k)
        s.set_HS(dev(H), dev(S))
        W = empty_cm(sysm.m, sysm.n)
        E, iters, st = s.solve(dev(W0), tol=0.0, W_out=W, raise_on_error=False)
        ref = O.omm_cg_cholesky(H, S, W0, tol=0.0, eta=s.diag().eta, max_iter=k)
        assert st == omm.ERR_MAXITER and iters == k == ref.iters
        assert E == pytest.approx(ref.E, rel=1e-12)
        np.testing.assert_allclose(W.cpu().numpy(), ref.W, rtol=1e-8, atol=1e-10)
        s.close()


def test_cholesky_and_plain_reach_the_same_minimum(omm):
    """Both forms minimise the same functional: equal E, equal density matrix, and
    the minimum is 2 x the sum of the n lowest generalised eigenvalues (eta-shift
    removed)."""
    import synth
    import scipy.linalg as sla
    sysm = synth.make_system(4, 4, 3, seed=6)
    H, S = sysm.dense_H(), sysm.dense_S()
    W0 = dev(sysm.W0_dense())
    out = {}
    for chol in (0, 1):
        s = omm.Solver(sysm.m, sysm.n, 8, cholesky=chol)
        s.set_HS(dev(H), dev(S))
        W = empty_cm(sysm.m, sysm.n)
        E, _, st = s.solve(W0, tol=1e-13, W_out=W)
        assert st == omm.OK
        out[chol] = (E, W.cpu().numpy())
        s.close()
    assert abs(out[0][0] - out[1][0]) / abs(out[0][0]) < 1e-11
    np.testing.assert_allclose(O.density_matrix(out[1][1], S), O.density_matrix(out[0][1], S), atol=2e-5)
    lam = sla.eigh(H, S, eigvals_only=True)
    assert abs(out[1][0] - 2 * lam[:sysm.n].sum()) / abs(out[1][0]) < 1e-10


@pytest.mark.parametrize("dims", [(4, 4, 4), (5, 5, 3)])
def test_cholesky_mixed_matches_oracle(omm, dims):
    """Split-precision CG on the reduced problem, then the exact-digit refinement."""
    import synth
    sysm = synth.make_system(*dims, seed=2)
    H, S = sysm.dense_H(), sysm.dense_S()
    W0 = np.asfortranarray(sysm.W0_dense())
    s = omm.Solver(sysm.m, sysm.n, 8, cholesky=1, precision=omm.PREC_MIXED, orth_tol=1e-6)
    s.set_HS(dev(H), dev(S))
    W = empty_cm(sysm.m, sysm.n)
    E, iters, st = s.solve(dev(W0), tol=1e-10, W_out=W)
    d = s.diag()
    ref = O.omm_cg_cholesky(H, S, W0, tol=1e-13, eta=d.eta)
    assert st == omm.OK
    assert abs(E - ref.E) / abs(ref.E) < 1e-8
    Wn = W.cpu().numpy()
    # orthonormality holds in the original metric (W~^T W~ = W^T S W)
    assert np.linalg.norm(Wn.T @ S @ Wn - np.eye(sysm.n)) < 2e-6 and d.orth < 1e-6
    np.testing.assert_allclose(O.density_matrix(Wn, S), O.density_matrix(ref.W, S), atol=1e-5)
    assert d.iters_mixed > 0 and d.iters_refine >= 1
    s.close()


def test_cholesky_warm_start_in_original_basis(omm):
    """Warm starts keep W in the original basis: a new S (new factor L) is honoured."""
    import synth
    sysm = synth.make_system(3, 3, 3, seed=4)
    H, S = sysm.dense_H(), sysm.dense_S()
    W0 = np.asfortranarray(sysm.W0_dense())
    s = omm.Solver(sysm.m, sysm.n, 8, cholesky=1)
    s.set_HS(np.asfortranarray(H), np.asfortranarray(S))
    W = np.zeros((sysm.m, sysm.n), order="F")
    E1, it1, _ = s.solve(W0, tol=1e-12, W_out=W)
    E2, it2, st2 = s.solve(None, tol=1e-12)
    assert st2 == omm.OK and it2 <= 3 and E2 == pytest.approx(E1, rel=1e-12)
    # perturbed H and a slightly scaled S: the warm start is W (original basis) under the new L
    Hp = synth.perturb_pairs(sysm, 7, 1).dense_H()
    Sp = S * 1.01 + 0.0
    s.set_HS(np.asfortranarray(Hp), np.asfortranarray(Sp))
    E3, it3, _ = s.solve(None, tol=1e-12)
    ref3 = O.omm_cg_cholesky(Hp, Sp, W, tol=1e-12, eta=s.diag().eta)
    assert abs(E3 - ref3.E) / abs(ref3.E) < 1e-10
    s.close()


@pytest.mark.parametrize("eta_auto", [1, 0])
def test_cholesky_not_spd_is_reported(omm, eta_auto):
    """An indefinite S stops set_HS with OMM_ERR_NOT_SPD (no solve runs).  With
    eta_auto the Gershgorin bound already rejects it; with a fixed eta the
    factorisation's pivot test does (pivot 70 of m=144 goes negative)."""
    import synth
    sysm = synth.make_system(3, 3, 2, seed=0)
    H, S = sysm.dense_H(), sysm.dense_S().copy()
    S[70, 70] = -1.0
    s = omm.Solver(sysm.m, sysm.n, 8, cholesky=1, eta_auto=eta_auto, eta=0.0)
    with pytest.raises(omm.OmmError) as ei:
        s.set_HS(dev(H), dev(S))
    assert ei.value.status == omm.ERR_NOT_SPD
    E, it, st = s.solve(dev(sysm.W0_dense()), tol=1e-10, raise_on_error=False)
    assert st == omm.ERR_STATE
    s.close()


@pytest.mark.parametrize("chol,prec", [(0, "fp64"), (1, "fp64"), (0, "mixed"), (1, "mixed")])
def test_set_H_equals_set_HS(omm, chol, prec):
    """omm_set_H keeps S (and the factor): the next solve is bit-identical to one
    after omm_set_HS with the same S."""
    import synth
    sysm = synth.make_system(4, 3, 3, seed=8)
    H, S = dev(sysm.dense_H()), dev(sysm.dense_S())
    Hp = dev(synth.perturb_pairs(sysm, 3, 1).dense_H())
    W0 = dev(sysm.W0_dense())
    p = omm.PREC_MIXED if prec == "mixed" else omm.PREC_FP64
    out = []
    for use_set_H in (False, True):
        s = omm.Solver(sysm.m, sysm.n, 8, cholesky=chol, precision=p, orth_tol=1e-6)
        s.set_HS(H, S)
        s.solve(W0, tol=1e-10)
        if use_set_H:
            s.set_H(Hp)
        else:
            s.set_HS(Hp, S)
        W = empty_cm(sysm.m, sysm.n)
        E, it, st = s.solve(None, tol=1e-10, W_out=W)
        assert st == omm.OK
        out.append((E, it, s.diag().eta, W.cpu().numpy()))
        s.close()
    assert out[0][0] == out[1][0] and out[0][1] == out[1][1] and out[0][2] == out[1][2]
    np.testing.assert_array_equal(out[0][3], out[1][3])
    # the minimum of the perturbed problem, by the oracle
    Hp_np = synth.perturb_pairs(sysm, 3, 1).dense_H()
    oracle = O.omm_cg_cholesky if chol else O.omm_cg
    ref = oracle(Hp_np, sysm.dense_S(), out[0][3], tol=1e-12, eta=out[0][2])
    assert abs(out[1][0] - ref.E) / abs(ref.E) < 1e-9


def test_set_H_requires_set_HS(omm):
    import synth
    sysm = synth.make_system(3, 3, 2, seed=1)
    s = omm.Solver(sysm.m, sysm.n, 8)
    with pytest.raises(omm.OmmError) as ei:
        s.set_H(dev(sysm.dense_H()))
    assert ei.value.status == omm.ERR_STATE
    s.close()
