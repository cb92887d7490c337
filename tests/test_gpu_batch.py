"""Batched and asynchronous solves: every result equals the same solve alone."""
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


def _systems(count, seed):
    import synth
    sizes = synth.batch_sizes(count, seed, lo=8, hi=64)
    return [synth.make_batch_system(int(N), seed=seed * 1000 + i) for i, N in enumerate(sizes)]


def test_batch_equals_alone_bitwise(omm):
    systems = _systems(6, 7)
    alone, solvers = [], []
    for sysm in systems:
        s = omm.Solver(sysm.m, sysm.n, 8, precision=omm.PREC_MIXED, orth_tol=1e-6)
        s.set_HS(dev(sysm.dense_H()), dev(sysm.dense_S()))
        W = torch.zeros((sysm.n, sysm.m), dtype=torch.float64, device="cuda").T
        E, it, st = s.solve(dev(sysm.W0_dense()), tol=1e-10, W_out=W)
        alone.append((E, it, W.cpu().numpy().copy()))
        solvers.append(s)
    E, it, st = omm.batch_solve(solvers, [dev(sysm.W0_dense()) for sysm in systems], tol=1e-10)
    assert (st == omm.OK).all()
    for i, sysm in enumerate(systems):
        assert E[i] == alone[i][0] and it[i] == alone[i][1]
        assert np.array_equal(solvers[i].get_array(omm.ARRAY_W), alone[i][2])
        ref = O.omm_cg(sysm.dense_H(), sysm.dense_S(), sysm.W0_dense(), tol=1e-13, eta=solvers[i].diag().eta)
        assert abs(E[i] - ref.E) / abs(ref.E) < 1e-8
    for s in solvers:
        s.close()


def test_mixed_forms_in_one_batch(omm):
    """Dense FP64, dense mixed and linear-scaling handles together."""
    import synth
    a = synth.make_system(3, 3, 3, seed=1)
    b = synth.make_system(4, 4, 4, seed=2)
    c = synth.make_system(3, 4, 5, seed=3)
    sa = omm.Solver(a.m, a.n, 8)
    sa.set_HS(dev(a.dense_H()), dev(a.dense_S()))
    sb = omm.Solver(b.m, b.n, 8, precision=omm.PREC_MIXED, orth_tol=1e-6)
    sb.set_HS(dev(b.dense_H()), dev(b.dense_S()))
    rp, col, Hv, Sv = c.bsr()
    wrp, wcol = c.w_pattern(4.5)
    sc = omm.SparseSolver(c.m, c.n, 8, 2, rp, col, wrp, wcol, max_iter=40)
    sc.set_HS(Hv, Sv)
    W0s = [dev(a.W0_dense()), dev(b.W0_dense()), torch.from_numpy(c.W0_bsr_values(4.5)).cuda()]
    E, it, st = omm.batch_solve([sa, sb, sc], W0s, tol=1e-10)
    assert st[0] == omm.OK and st[1] == omm.OK and st[2] in (omm.OK, omm.ERR_MAXITER)
    ea, _, _ = (lambda s: (s.solve(W0s[0], tol=1e-10)))(sa)
    assert ea == E[0]
    for s in (sa, sb, sc):
        s.close()


def test_async_driver_matches_blocking(omm):
    import synth
    sysm = synth.make_system(4, 4, 4, seed=9)
    s = omm.Solver(sysm.m, sysm.n, 8, precision=omm.PREC_MIXED, orth_tol=1e-6)
    s.set_HS(dev(sysm.dense_H()), dev(sysm.dense_S()))
    E1, it1, _ = s.solve(dev(sysm.W0_dense()), tol=1e-10)
    s.begin(dev(sysm.W0_dense()), tol=1e-10)
    polls = 0
    while not s.progress(blocking=False):
        polls += 1
    E2, it2, st = s.end()
    assert (E2, it2) == (E1, it1) and st == omm.OK
    with pytest.raises(omm.OmmError):
        s.end()                      # nothing to end any more
    s.close()


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_graph_replay_equals_eager(omm, prec):
    """Chunks replayed from captured CUDA graphs give the same bits as eager
    launches, over several solves of one handle (cold, warm, new H)."""
    import synth
    sysm = synth.make_system(4, 3, 3, seed=12)
    H, S = dev(sysm.dense_H()), dev(sysm.dense_S())
    Hp = dev(synth.perturb_pairs(sysm, 5, 1).dense_H())
    W0 = dev(sysm.W0_dense())
    p = omm.PREC_MIXED if prec == "mixed" else omm.PREC_FP64
    runs = []
    for graphs in (0, 1):
        s = omm.Solver(sysm.m, sysm.n, 8, precision=p, orth_tol=1e-6, graphs=graphs)   # own stream
        out = []
        s.set_HS(H, S)
        out.append(s.solve(W0, tol=1e-10))
        out.append(s.solve(None, tol=1e-10))
        s.set_H(Hp)
        out.append(s.solve(None, tol=1e-10))
        W = torch.zeros((sysm.n, sysm.m), dtype=torch.float64, device="cuda").T
        s.solve(W0, tol=1e-10, W_out=W)
        torch.cuda.synchronize()
        runs.append((out, W.cpu().numpy()))
        s.close()
    assert runs[0][0] == runs[1][0]
    np.testing.assert_array_equal(runs[0][1], runs[1][1])


def test_bounded_wait_gives_up_and_context_survives(omm):
    """A wait that nothing completes ends in OMM_ERR_TIMEOUT at its limit (the
    deadline mechanism of every tcgen05 pipeline wait); a solve runs afterwards."""
    import time
    t0 = time.perf_counter()
    st = omm.selftest_bounded_wait(50_000_000)          # 50 ms
    elapsed = time.perf_counter() - t0
    assert st == omm.ERR_TIMEOUT
    assert 0.045 <= elapsed < 5.0
    with pytest.raises(omm.OmmError):
        omm.selftest_bounded_wait(10)                   # limit out of range
    import synth
    sysm = synth.make_system(2, 2, 2, seed=0)
    s = omm.Solver(sysm.m, sysm.n, 8, precision=omm.PREC_MIXED)
    s.set_HS(np.asfortranarray(sysm.dense_H()), np.asfortranarray(sysm.dense_S()))
    E, it, status = s.solve(np.asfortranarray(sysm.W0_dense()), tol=1e-10)
    assert status == omm.OK
    s.close()
