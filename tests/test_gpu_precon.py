"""Kinetic-energy preconditioning (Eq. 6, section "Overview of OMM approaches")
on the GPU, through the C ABI, against the oracle's preconditioned CG.

Inputs: the kinetic workload of the synthetic generator, H + T with a
kinetic-dominated spectrum (~400 eV wide above a gap of a few eV), S, and T.
"""
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


def kinetic_system(dims, seed):
    import synth
    sysm = synth.make_system(*dims, seed=seed)
    return sysm, sysm.dense_H_kinetic(), sysm.dense_S(), sysm.dense_T(), np.asfortranarray(sysm.W0_dense())


# (3,3,3): m = 216, several 128-row tiles and a ragged one; (5,5,3): m = 600, n = 150
@pytest.mark.parametrize("dims", [(3, 3, 3), (5, 5, 3)])
@pytest.mark.parametrize("tau", [O.TAU_T_DEFAULT, 5.0])
def test_precon_fixed_iterations_track_oracle(omm, dims, tau):
    """k preconditioned CG steps in FP64: the iterate and energy equal the oracle's."""
    sysm, H, S, T, W0 = kinetic_system(dims, 1)
    P = O.kinetic_preconditioner(S, T, tau)
    for k in (1, 3, 8):
        s = omm.Solver(sysm.m, sysm.n, 8, precon=-1, tau_T=tau, max_iter=k)
        s.set_HS(dev(H), dev(S))
        s.set_T(dev(T))
        W = empty_cm(sysm.m, sysm.n)
        E, iters, st = s.solve(dev(W0), tol=0.0, W_out=W, raise_on_error=False)
        ref = O.omm_cg(H, S, W0, tol=0.0, eta=s.diag().eta, max_iter=k, P=P)
        assert st == omm.ERR_MAXITER and iters == k == ref.iters
        assert E == pytest.approx(ref.E, rel=1e-12)
        np.testing.assert_allclose(W.cpu().numpy(), ref.W, rtol=1e-8, atol=1e-10)
        s.close()


def test_precon_fp64_converged_matches_oracle(omm):
    sysm, H, S, T, W0 = kinetic_system((4, 4, 4), 2)
    s = omm.Solver(sysm.m, sysm.n, 8, precon=-1)
    s.set_HS(dev(H), dev(S))
    s.set_T(dev(T))
    W = empty_cm(sysm.m, sysm.n)
    E, iters, st = s.solve(dev(W0), tol=1e-12, W_out=W)
    eta = s.diag().eta
    ref = O.omm_cg(H, S, W0, tol=1e-12, eta=eta, P=O.kinetic_preconditioner(S, T))
    assert st == omm.OK and ref.status == O.OK
    assert abs(E - ref.E) / abs(ref.E) < 1e-10
    # the trajectories part at the rounding level over hundreds of steps
    assert abs(iters - ref.iters) <= max(3, ref.iters // 10)
    Wn = W.cpu().numpy()
    np.testing.assert_allclose(O.density_matrix(Wn, S), O.density_matrix(ref.W, S), atol=2e-5)
    s.close()


def test_precon_mixed_matches_oracle(omm):
    """Split-precision CG with the split product P G, then the exact-digit
    refinement (also preconditioned): the mixed-precision bar."""
    sysm, H, S, T, W0 = kinetic_system((4, 4, 4), 3)
    s = omm.Solver(sysm.m, sysm.n, 8, precon=-1, precision=omm.PREC_MIXED, orth_tol=1e-6)
    s.set_HS(dev(H), dev(S))
    s.set_T(dev(T))
    W = empty_cm(sysm.m, sysm.n)
    E, iters, st = s.solve(dev(W0), tol=1e-10, W_out=W)
    d = s.diag()
    ref = O.omm_cg(H, S, W0, tol=1e-13, eta=d.eta, P=O.kinetic_preconditioner(S, T))
    assert st == omm.OK
    assert abs(E - ref.E) / abs(ref.E) < 1e-8
    assert d.orth < 1e-6 and d.iters_mixed > 0 and d.iters_refine >= 1
    s.close()


def test_precon_without_kinetic_term_is_the_cholesky_variant(omm):
    """T = 0: P = S^-1, the same iterates as the Cholesky-reduced variant."""
    sysm, H, S, _, W0 = kinetic_system((3, 3, 3), 4)
    out = []
    for opts in ({"precon": -1}, {"cholesky": 1}):
        s = omm.Solver(sysm.m, sysm.n, 8, max_iter=6, **opts)
        s.set_HS(dev(H), dev(S))
        if "precon" in opts:
            s.set_T(dev(np.zeros_like(S)))
        W = empty_cm(sysm.m, sysm.n)
        E, it, st = s.solve(dev(W0), tol=0.0, W_out=W, raise_on_error=False)
        assert st == omm.ERR_MAXITER and it == 6
        out.append((E, W.cpu().numpy()))
        s.close()
    assert out[0][0] == pytest.approx(out[1][0], rel=1e-11)
    np.testing.assert_allclose(out[0][1], out[1][1], rtol=1e-7, atol=1e-9)


def test_precon_count_set_T_and_set_H(omm):
    """precon = 1: only the first solve after omm_set_T is preconditioned (the
    next equals a plain handle's solve bit for bit); omm_set_T re-arms it;
    omm_set_H keeps P (bit-identical to a rebuild from the same S and T)."""
    sysm, H, S, T, W0 = kinetic_system((3, 3, 3), 5)
    dH, dS, dT, dW0 = dev(H), dev(S), dev(T), dev(W0)
    plain = omm.Solver(sysm.m, sysm.n, 8)
    plain.set_HS(dH, dS)
    Ep, itp, _ = plain.solve(dW0, tol=1e-11)
    plain.close()
    s = omm.Solver(sysm.m, sysm.n, 8, precon=1)
    s.set_HS(dH, dS)
    s.set_T(dT)
    E1, it1, st1 = s.solve(dW0, tol=1e-11)
    E2, it2, st2 = s.solve(dW0, tol=1e-11)
    assert st1 == st2 == omm.OK
    assert (E2, it2) == (Ep, itp)
    assert (E1, it1) != (Ep, itp)
    s.set_T(dT)
    E3, it3, _ = s.solve(dW0, tol=1e-11)
    assert (E3, it3) == (E1, it1)
    s.close()
    # omm_set_H keeps P: equal to a handle that builds P for the same S and T
    import synth
    Hp = dev(synth.perturb_pairs(sysm, 3, 1).dense_H() + T)
    res = []
    for use_set_H in (True, False):
        s = omm.Solver(sysm.m, sysm.n, 8, precon=-1)
        s.set_HS(dH, dS)
        s.set_T(dT)
        if use_set_H:
            s.solve(dW0, tol=1e-10)
            s.set_H(Hp)
        else:
            s.set_HS(Hp, dS)
        W = empty_cm(sysm.m, sysm.n)
        E, it, st = s.solve(dW0, tol=1e-10, W_out=W)
        res.append((E, it, W.cpu().numpy()))
        s.close()
    assert res[0][:2] == res[1][:2]
    np.testing.assert_array_equal(res[0][2], res[1][2])


def test_precon_errors(omm):
    sysm, H, S, T, W0 = kinetic_system((3, 3, 2), 6)
    with pytest.raises(omm.OmmError) as e:
        omm.Solver(sysm.m, sysm.n, 8, precon=-1, cholesky=1)
    assert e.value.status == omm.ERR_UNSUPPORTED
    with pytest.raises(omm.OmmError) as e:
        omm.Solver(sysm.m, sysm.n, 8, precon=-1, tau_T=0.0)
    assert e.value.status == omm.ERR_ARG
    s = omm.Solver(sysm.m, sysm.n, 8)
    with pytest.raises(omm.OmmError) as e:
        s.set_T(dev(T))
    assert e.value.status == omm.ERR_UNSUPPORTED
    s.close()
    s = omm.Solver(sysm.m, sysm.n, 8, precon=-1, tau_T=1.0)
    s.set_HS(dev(H), dev(S))
    E, it, st = s.solve(dev(W0), tol=1e-10, raise_on_error=False)
    assert st == omm.ERR_STATE                      # no T yet
    # S + T / tau = S - 5 I is indefinite: the solve reports it and runs nothing
    s.set_T(dev(-5.0 * np.eye(sysm.m)))
    E, it, st = s.solve(dev(W0), tol=1e-10, raise_on_error=False)
    assert st == omm.ERR_NOT_SPD
    s.set_T(dev(T))
    E, it, st = s.solve(dev(W0), tol=1e-10)
    assert st == omm.OK
    s.close()


def test_sparse_precon_unsupported(omm):
    import synth
    sysm = synth.make_system(3, 3, 2, seed=0)
    rp, col, _, _ = sysm.bsr()
    wrp, wcol = sysm.w_pattern(4.5)
    with pytest.raises(omm.OmmError) as e:
        omm.SparseSolver(sysm.m, sysm.n, 8, 2, rp, col, wrp, wcol, precon=-1)
    assert e.value.status == omm.ERR_UNSUPPORTED
