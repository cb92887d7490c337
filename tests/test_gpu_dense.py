"""Dense FP64 CUDA path against the FP64 oracle, through the C ABI."""
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


# ------------------------------------------------------------------ GEMM
@pytest.mark.parametrize("tA,tB,M,N,K", [(0, 0, 128, 64, 96), (1, 0, 100, 70, 33), (0, 1, 65, 129, 17),
                                         (1, 1, 31, 7, 200), (0, 0, 5, 3, 0), (0, 0, 1, 1, 1)])
def test_dgemm_matches_numpy(omm, tA, tB, M, N, K):
    rng = np.random.default_rng(M * 7 + N)
    A = rng.standard_normal((K, M) if tA else (M, K))
    B = rng.standard_normal((N, K) if tB else (K, N))
    Cin = rng.standard_normal((M, N))
    out = empty_cm(M, N)
    lda, ldb = max(1, A.shape[0]), max(1, B.shape[0])
    st = omm.op_dgemm(tA, tB, M, N, K, 0.5, dev(A), lda, dev(B), ldb, -1.5, dev(Cin), M, out, M)
    assert st == omm.OK
    torch.cuda.synchronize()
    ref = 0.5 * (A.T if tA else A) @ (B.T if tB else B) - 1.5 * Cin
    np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=1e-13, atol=1e-13 * max(1, K))


# ------------------------------------------------------------------ line search pieces
def _blocks(sysm, seed):
    H, S = sysm.dense_H(), sysm.dense_S()
    Hs = O.shift(H, S, O.gershgorin_eta(H, S))
    W = np.asfortranarray(sysm.W0_dense())
    D = -O.gradient(W, Hs, S) + 0.01 * np.random.default_rng(seed).standard_normal(W.shape)
    blocks = dict(h0=W.T @ Hs @ W, s0=W.T @ S @ W, X=W.T @ Hs @ D, Y=W.T @ S @ D,
                  h2=D.T @ Hs @ D, s2=D.T @ S @ D)
    return W, D, Hs, S, blocks


@pytest.mark.parametrize("dims", [(4, 4, 4), (3, 4, 5)])
def test_quartic_coeffs_match_oracle(omm, dims):
    import synth
    sysm = synth.make_system(*dims, seed=1)
    W, D, Hs, S, b = _blocks(sysm, 0)
    n = sysm.n
    ref = O.quartic_coeffs(W, D, Hs, S)
    nb = omm.op_quartic_coeffs_scratch_bytes(n)
    scratch = torch.zeros(nb // 8 + 1, dtype=torch.float64, device="cuda")
    coeffs = torch.zeros(5, dtype=torch.float64, device="cuda")
    t = {k: dev(v) for k, v in b.items()}
    for rep in range(2):          # second call reuses the (self-resetting) counter
        st = omm.op_quartic_coeffs(n, t["h0"], t["s0"], n, t["X"], t["Y"], t["h2"], t["s2"], n,
                                   coeffs, scratch, nb)
        assert st == omm.OK
        torch.cuda.synchronize()
        c = coeffs.cpu().numpy()
        scale = np.abs(ref).max()
        np.testing.assert_allclose(c, ref, rtol=1e-11, atol=1e-12 * scale)


def test_line_min_matches_oracle(omm):
    rng = np.random.default_rng(3)
    cases = [np.array([1.0, -2.0, 0.5, 0.3, 0.8]), np.array([3.0, -4.0, 2.0, 0.0, 0.0]),
             np.array([0.0, -1.0, 1.0, 0.0, -1.0]), np.array([0.0, 0.5, -3.0, 0.0, 1.0])]
    for _ in range(40):
        c = rng.standard_normal(5)
        c[4] = abs(c[4]) + 1e-3
        cases.append(c)
    p = np.polynomial.polynomial.polymul([1, -2, 1], [4, 4, 1])
    cases.append(np.array(p) + np.array([0, 0.5, 0, 0, 0]))
    # c4 < 0 (Kim functional, eta in the gap): a local minimum, or none
    cases += [np.array([0.0, -0.5, 2.0, 0.0, -1.0]), np.array([1.0, 0.3, 1.5, -0.2, -0.4])]
    for _ in range(20):
        c = rng.standard_normal(5)
        c[4] = -abs(c[4]) - 1e-3
        cases.append(c)
    cin = torch.zeros(5, dtype=torch.float64, device="cuda")
    x = torch.zeros(1, dtype=torch.float64, device="cuda")
    stt = torch.zeros(1, dtype=torch.int32, device="cuda")
    for c in cases:
        cin.copy_(torch.from_numpy(c))
        assert omm.op_line_min(cin, x, stt) == omm.OK
        torch.cuda.synchronize()
        xr, sr = O.line_min(c)
        assert int(stt.item()) == sr
        if sr == O.OK:
            assert x.item() == pytest.approx(xr, rel=1e-9, abs=1e-12)


# ------------------------------------------------------------------ full solves
@pytest.mark.parametrize("dims,tol", [((4, 4, 4), 1e-12), ((3, 4, 5), 1e-12)])
def test_dense_solve_matches_oracle(omm, dims, tol):
    import synth
    sysm = synth.make_system(*dims, seed=0)
    H, S = sysm.dense_H(), sysm.dense_S()
    W0 = np.asfortranarray(sysm.W0_dense())
    s = omm.Solver(sysm.m, sysm.n, 8)
    s.set_HS(dev(H), dev(S))
    eta = s.diag().eta
    assert eta == pytest.approx(O.gershgorin_eta(H, S), rel=1e-14)
    W = empty_cm(sysm.m, sysm.n)
    E, iters, st = s.solve(dev(W0), tol=tol, W_out=W)
    ref = O.omm_cg(H, S, W0, tol=tol, eta=eta)
    assert st == omm.OK and ref.status == O.OK
    assert abs(E - ref.E) / abs(ref.E) < 1e-10
    assert abs(iters - ref.iters) <= 2
    Wn = W.cpu().numpy()
    np.testing.assert_allclose(O.density_matrix(Wn, S), O.density_matrix(ref.W, S), atol=1e-6)
    d = s.diag()
    assert d.orth == pytest.approx(np.linalg.norm(Wn.T @ S @ Wn - np.eye(sysm.n)), rel=1e-3, abs=1e-9)
    assert d.charge == pytest.approx(O.charge(Wn, S), rel=1e-12)
    s.close()


def test_fixed_iterations_track_oracle(omm):
    """Same number of CG steps from the same W0: the iterates coincide."""
    import synth
    sysm = synth.make_system(4, 4, 4, seed=2)
    H, S = sysm.dense_H(), sysm.dense_S()
    W0 = np.asfortranarray(sysm.W0_dense())
    for k in (1, 2, 7):
        s = omm.Solver(sysm.m, sysm.n, 8, max_iter=k)
        s.set_HS(dev(H), dev(S))
        W = empty_cm(sysm.m, sysm.n)
        E, iters, st = s.solve(dev(W0), tol=0.0, W_out=W, raise_on_error=False)
        ref = O.omm_cg(H, S, W0, tol=0.0, eta=s.diag().eta, max_iter=k)
        assert st == omm.ERR_MAXITER and iters == k == ref.iters
        assert E == pytest.approx(ref.E, rel=1e-13)
        np.testing.assert_allclose(W.cpu().numpy(), ref.W, rtol=1e-9, atol=1e-11)
        s.close()


def test_host_buffers_and_warm_start(omm):
    import synth
    sysm = synth.make_system(3, 3, 3, seed=4)
    H, S = sysm.dense_H(), sysm.dense_S()
    W0 = np.asfortranarray(sysm.W0_dense())
    s = omm.Solver(sysm.m, sysm.n, 8)
    s.set_HS(np.asfortranarray(H), np.asfortranarray(S))
    W = np.zeros((sysm.m, sysm.n), order="F")
    E1, it1, st = s.solve(W0, tol=1e-12, W_out=W)
    ref = O.omm_cg(H, S, W0, tol=1e-12, eta=s.diag().eta)
    assert abs(E1 - ref.E) / abs(ref.E) < 1e-10
    # warm start from the resident W: converges at once
    E2, it2, st2 = s.solve(None, tol=1e-12)
    assert st2 == omm.OK and it2 <= 3 and E2 == pytest.approx(E1, rel=1e-12)
    # a perturbed H (SCF-like) warm-started
    Hp = synth.perturb_pairs(sysm, 7, 1).dense_H()
    s.set_HS(np.asfortranarray(Hp), np.asfortranarray(S))
    E3, it3, _ = s.solve(None, tol=1e-12)
    ref3 = O.omm_cg(Hp, S, W, tol=1e-12, eta=s.diag().eta)
    assert abs(E3 - ref3.E) / abs(ref3.E) < 1e-10
    assert it3 < it1
    s.close()


def _kim_inputs(dims, seed, extra):
    import synth
    import scipy.linalg as sla
    sysm = synth.make_system(*dims, seed=seed)
    H, S = sysm.dense_H(), sysm.dense_S()
    lam = sla.eigh(H, S, eigvals_only=True)
    eta = 0.5 * (lam[sysm.n - 1] + lam[sysm.n])       # inside the gap
    rng = np.random.default_rng(seed + 7)
    # small start: inside the barrier the unoccupied directions have at unit norm
    W0 = 0.2 * np.hstack([sysm.W0_dense(), rng.standard_normal((sysm.m, extra)) / np.sqrt(sysm.m)])
    return sysm, H, S, np.asfortranarray(W0), eta, 2.0 * lam[:sysm.n].sum()


def test_kim_functional_matches_oracle(omm):
    """Kim construction: n' = n + 8 columns, eta in the gap, energy + 2 eta n."""
    sysm, H, S, W0, eta, e_min = _kim_inputs((4, 4, 3), 2, 8)
    n1 = W0.shape[1]
    s = omm.Solver(sysm.m, n1, 8, eta_auto=0, eta=eta, n_occupied=sysm.n)
    s.set_HS(dev(H), dev(S))
    W = empty_cm(sysm.m, n1)
    E, iters, st = s.solve(dev(W0), tol=1e-13, W_out=W)
    ref = O.omm_cg(H, S, W0, tol=1e-13, eta=eta, n_occ=sysm.n)
    assert st == omm.OK and ref.status == O.OK
    assert abs(E - ref.E) / abs(ref.E) < 1e-10
    assert abs(E - e_min) / abs(e_min) < 1e-10
    Wn = W.cpu().numpy()
    assert O.charge(Wn, S) == pytest.approx(2 * sysm.n, rel=1e-8)
    assert s.diag().charge == pytest.approx(2 * sysm.n, rel=1e-8)
    np.testing.assert_allclose(O.density_matrix(Wn, S), O.density_matrix(ref.W, S), atol=2e-5)
    s.close()
    # the Gershgorin bound is not in a gap: refused with extra columns
    with pytest.raises(omm.OmmError):
        omm.Solver(sysm.m, n1, 8, n_occupied=sysm.n)


def test_state_and_argument_errors(omm):
    s = omm.Solver(64, 16, 8)
    E, it, st = s.solve(np.zeros((64, 16), order="F"), tol=1e-10, raise_on_error=False)
    assert st == omm.ERR_STATE
    s.close()
    with pytest.raises(omm.OmmError):
        omm.Solver(64, 16, 8, precision=7)


def test_no_minimum_reports_linesearch_error(omm):
    """Unshifted functional (eta = 0) from a large start: the first line has no
    minimum, reported as OMM_ERR_LINESEARCH (cf. the paper's warning)."""
    import synth
    sysm = synth.make_system(4, 4, 4, seed=0)
    H, S = sysm.dense_H(), sysm.dense_S()
    W0 = np.asfortranarray(sysm.W0_dense() * 3.0)
    ref = O.omm_cg(H, S, W0, tol=1e-10, eta=0.0)
    s = omm.Solver(sysm.m, sysm.n, 8, eta_auto=0, eta=0.0)
    s.set_HS(dev(H), dev(S))
    E, it, st = s.solve(dev(W0), tol=1e-10, raise_on_error=False)
    assert ref.status == O.ERR_LINESEARCH
    assert st == omm.ERR_LINESEARCH and it == ref.iters
    s.close()
