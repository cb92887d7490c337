"""Density matrix (Eq. 5) and energy density (defined with Eq. 6) of a solve,
through the C ABI, against the oracle's definitions on the returned W."""
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


@pytest.mark.parametrize("prec,chol", [("fp64", 0), ("mixed", 0), ("mixed", 1)])
def test_density_matrices_match_oracle(omm, prec, chol):
    import synth
    sysm = synth.make_system(4, 3, 3, seed=3)            # m = 288: several tiles and a ragged tail
    H, S = sysm.dense_H(), sysm.dense_S()
    p = omm.PREC_MIXED if prec == "mixed" else omm.PREC_FP64
    s = omm.Solver(sysm.m, sysm.n, 8, precision=p, cholesky=chol, orth_tol=1e-6)
    with pytest.raises(omm.OmmError):
        s.get_density()                                   # no solve yet
    s.set_HS(dev(H), dev(S))
    W = np.zeros((sysm.m, sysm.n), order="F")
    s.solve(dev(sysm.W0_dense()), tol=1e-11, W_out=W)
    eta = s.diag().eta
    rho = s.get_density(omm.DENSITY_RHO)
    ref = O.density_matrix(W, S)
    scale = np.abs(ref).max()
    np.testing.assert_allclose(rho, ref, atol=1e-12 * scale)
    # device output, energy density with the shifted Hamiltonian and its eta
    rho_e = torch.zeros((sysm.m, sysm.m), dtype=torch.float64, device="cuda").T
    s.get_density(omm.DENSITY_RHO_E, rho_e)
    ref_e = O.energy_density_matrix(W, O.shift(H, S, eta), S, eta)
    np.testing.assert_allclose(rho_e.cpu().numpy(), ref_e, atol=1e-12 * np.abs(ref_e).max())
    # physical checks: Tr(rho S) = 2n (charge), Tr(rho_E S^-1 ...) through the energy
    assert np.trace(rho @ S) == pytest.approx(2 * sysm.n, rel=1e-8)
    assert np.sum(rho * H) == pytest.approx(O.functional(W, H, S), rel=1e-10)
    s.close()


def test_density_matrix_kim(omm):
    """Kim construction (n' = n + 8, eta in the gap): rho still holds 2n electrons."""
    import synth
    import scipy.linalg as sla
    sysm = synth.make_system(4, 3, 3, seed=4)
    H, S = sysm.dense_H(), sysm.dense_S()
    lam = sla.eigh(H, S, eigvals_only=True)
    eta = 0.5 * (lam[sysm.n - 1] + lam[sysm.n])
    rng = np.random.default_rng(2)
    W0 = np.asfortranarray(0.2 * np.hstack([sysm.W0_dense(), rng.standard_normal((sysm.m, 8)) / np.sqrt(sysm.m)]))
    n1 = W0.shape[1]
    s = omm.Solver(sysm.m, n1, 8, eta_auto=0, eta=eta, n_occupied=sysm.n)
    s.set_HS(dev(H), dev(S))
    W = np.zeros((sysm.m, n1), order="F")
    s.solve(dev(W0), tol=1e-13, W_out=W)
    rho = s.get_density(omm.DENSITY_RHO)
    np.testing.assert_allclose(rho, O.density_matrix(W, S), atol=1e-12 * np.abs(rho).max())
    assert np.trace(rho @ S) == pytest.approx(2 * sysm.n, rel=1e-8)
    s.close()
