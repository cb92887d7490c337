"""Mixed-precision dense solve (split-BF16 tensor-core bulk + FP64 refinement)
against the FP64 oracle: energy within 1e-8 relative, ||S_W - I||_F < 1e-6."""
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


@pytest.mark.parametrize("dims,refine,dir_digits", [((4, 4, 4), "exact", 1), ((3, 4, 5), "exact", 1),
                                                    ((5, 5, 5), "exact", 1), ((4, 4, 4), "fp64", 1),
                                                    ((3, 4, 5), "fp64", 1), ((4, 4, 4), "exact", 0),
                                                    ((3, 4, 5), "exact", 0)])
def test_mixed_solve_matches_oracle(omm, dims, refine, dir_digits):
    """dir_digits 1 (default): search directions rounded to one BF16 digit, the
    H'D, SD products on two digit pairs; 0: directions keep two digits."""
    import synth
    sysm = synth.make_system(*dims, seed=0)
    H, S = sysm.dense_H(), sysm.dense_S()
    W0 = np.asfortranarray(sysm.W0_dense())
    s = omm.Solver(sysm.m, sysm.n, 8, precision=omm.PREC_MIXED, orth_tol=1e-6, dir_digits=dir_digits,
                   refine=omm.REFINE_EXACT if refine == "exact" else omm.REFINE_FP64)
    s.set_HS(dev(H), dev(S))
    W = torch.zeros((sysm.n, sysm.m), dtype=torch.float64, device="cuda").T
    E, iters, st = s.solve(dev(W0), tol=1e-10, W_out=W)
    d = s.diag()
    ref = O.omm_cg(H, S, W0, tol=1e-13, eta=d.eta)
    assert st == omm.OK
    assert abs(E - ref.E) / abs(ref.E) < 1e-8
    Wn = W.cpu().numpy()
    orth = np.linalg.norm(Wn.T @ S @ Wn - np.eye(sysm.n))
    assert orth < 1e-6 and d.orth < 1e-6
    # energy of the returned W evaluated by the oracle agrees with the reported one
    e_w = O.functional(Wn, O.shift(H, S, d.eta), S) + 2 * d.eta * sysm.n
    assert abs(e_w - E) / abs(E) < 1e-9
    np.testing.assert_allclose(O.density_matrix(Wn, S), O.density_matrix(ref.W, S), atol=1e-5)
    assert d.iters_mixed > 0 and d.iters_refine >= 1
    s.close()


def test_kim_functional_mixed(omm):
    """Kim construction in the mixed form (orth_tol stays 0: S_W -> diag(I, 0)),
    with three-digit split products: the functional is unbounded beyond a barrier
    along unoccupied directions, and two-digit increments can cross it."""
    import synth
    import scipy.linalg as sla
    sysm = synth.make_system(4, 4, 3, seed=2)
    H, S = sysm.dense_H(), sysm.dense_S()
    lam = sla.eigh(H, S, eigvals_only=True)
    eta = 0.5 * (lam[sysm.n - 1] + lam[sysm.n])
    rng = np.random.default_rng(9)
    W0 = np.asfortranarray(0.2 * np.hstack([sysm.W0_dense(), rng.standard_normal((sysm.m, 8)) / np.sqrt(sysm.m)]))
    n1 = W0.shape[1]
    s = omm.Solver(sysm.m, n1, 8, precision=omm.PREC_MIXED, eta_auto=0, eta=eta, n_occupied=sysm.n,
                   split_digits=3)
    s.set_HS(dev(H), dev(S))
    W = torch.zeros((n1, sysm.m), dtype=torch.float64, device="cuda").T
    E, iters, st = s.solve(dev(W0), tol=1e-11, W_out=W)
    e_min = 2.0 * lam[:sysm.n].sum()
    assert st == omm.OK
    assert abs(E - e_min) / abs(e_min) < 1e-8
    assert O.charge(W.cpu().numpy(), S) == pytest.approx(2 * sysm.n, rel=1e-6)
    s.close()


def test_mixed_repeatable_bitwise(omm):
    """Fixed reduction orders: the same solve twice gives identical bits."""
    import synth
    sysm = synth.make_system(4, 4, 4, seed=5)
    H, S = dev(sysm.dense_H()), dev(sysm.dense_S())
    W0 = dev(sysm.W0_dense())
    out = []
    for _ in range(2):
        s = omm.Solver(sysm.m, sysm.n, 8, precision=omm.PREC_MIXED, orth_tol=1e-6)
        s.set_HS(H, S)
        W = torch.zeros((sysm.n, sysm.m), dtype=torch.float64, device="cuda").T
        E, it, st = s.solve(W0, tol=1e-10, W_out=W)
        out.append((E, it, W.cpu().numpy().copy()))
        s.close()
    assert out[0][0] == out[1][0] and out[0][1] == out[1][1]
    assert np.array_equal(out[0][2], out[1][2])
