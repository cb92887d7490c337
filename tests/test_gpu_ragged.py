"""Ragged sizes through the C ABI: m not a multiple of the 8-row blocks, of
the 128-row tiles or even of 4 or 2 (the vector paths' fallbacks), n odd;
generic gapped inputs (synth.make_dense_gapped).  Every dense form against
the oracle."""
import numpy as np
import pytest

from oracle import omm as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SIZES = [(151, 37), (150, 41), (97, 13)]


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


def problem(m, n):
    import synth
    return synth.make_dense_gapped(m, n, seed=m * 1000 + n)


@pytest.mark.parametrize("m,n", SIZES)
def test_ragged_fp64(omm, m, n):
    H, S, _, W0 = problem(m, n)
    s = omm.Solver(m, n, 1)
    s.set_HS(dev(H), dev(S))
    W = torch.zeros((n, m), dtype=torch.float64, device="cuda").T
    E, it, st = s.solve(dev(W0), tol=1e-12, W_out=W)
    ref = O.omm_cg(H, S, W0, tol=1e-12, eta=s.diag().eta)
    assert st == omm.OK and ref.status == O.OK
    assert abs(E - ref.E) / abs(ref.E) < 1e-10
    lam = np.linalg.eigvalsh(np.linalg.solve(np.linalg.cholesky(S), np.linalg.solve(np.linalg.cholesky(S), H).T))
    assert abs(E - 2 * lam[:n].sum()) / abs(E) < 1e-9
    s.close()


@pytest.mark.parametrize("m,n", SIZES)
def test_ragged_mixed(omm, m, n):
    H, S, _, W0 = problem(m, n)
    s = omm.Solver(m, n, 1, precision=omm.PREC_MIXED, orth_tol=1e-6)
    s.set_HS(dev(H), dev(S))
    E, it, st = s.solve(dev(W0), tol=1e-10)
    d = s.diag()
    ref = O.omm_cg(H, S, W0, tol=1e-13, eta=d.eta)
    assert st == omm.OK
    assert abs(E - ref.E) / abs(ref.E) < 1e-8 and d.orth < 1e-6
    rho = s.get_density(omm.DENSITY_RHO)
    np.testing.assert_allclose(rho, O.density_matrix(ref.W, S), atol=1e-5)
    s.close()


@pytest.mark.parametrize("form", ["cholesky", "precon"])
def test_ragged_variants(omm, form):
    m, n = SIZES[0]
    H, S, T, W0 = problem(m, n)
    opts = {"cholesky": 1} if form == "cholesky" else {"precon": -1, "tau_T": 2.0}
    for prec in (omm.PREC_FP64, omm.PREC_MIXED):
        s = omm.Solver(m, n, 1, precision=prec, orth_tol=1e-6, **opts)
        s.set_HS(dev(H), dev(S))
        if form == "precon":
            s.set_T(dev(T))
        E, it, st = s.solve(dev(W0), tol=1e-11)
        eta = s.diag().eta
        ref = O.omm_cg(H, S, W0, tol=1e-13, eta=eta)
        assert st == omm.OK
        assert abs(E - ref.E) / abs(ref.E) < (1e-10 if prec == omm.PREC_FP64 else 1e-8)
        s.close()
