"""Grouped batches (omm_batch_solve_grouped): the split products of every
system's first-phase CG step as one persistent grouped tensor-core launch, the
tile mode given or chosen by the autotuner.  Every result equals the same solve
alone bit for bit (energy, iterations, returned W), whatever the tile mode, and
the oracle within the mixed-precision bar; uneven sizes, ragged ones (m not a
multiple of the tiles) and a system that converges long before the others."""
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


def _inputs():
    import synth
    sizes = synth.batch_sizes(5, 21, lo=8, hi=96)
    out = [synth.make_batch_system(int(N), seed=21000 + i) for i, N in enumerate(sizes)]
    sysm = [(s.m, s.n, s.dense_H(), s.dense_S(), s.W0_dense()) for s in out]
    m, n = 300, 75                                      # ragged: no multiple of 128 or 256
    H, S, _, W0 = synth.make_dense_gapped(m, n, seed=4)
    sysm.append((m, n, H, S, W0))
    return sysm


def _alone(omm, systems):
    res = []
    for m, n, H, S, W0 in systems:
        s = omm.Solver(m, n, 8, precision=omm.PREC_MIXED, orth_tol=1e-6)
        s.set_HS(dev(H), dev(S))
        W = torch.zeros((n, m), dtype=torch.float64, device="cuda").T
        E, it, st = s.solve(dev(W0), tol=1e-10, W_out=W)
        torch.cuda.synchronize()
        res.append((E, it, st, W.cpu().numpy().copy(), s.diag().eta))
        s.close()
    return res


@pytest.mark.parametrize("tile_mode", [1, 0, -1])
def test_grouped_equals_alone_bitwise(omm, tile_mode):
    systems = _inputs()
    alone = _alone(omm, systems)
    solvers = []
    for m, n, H, S, W0 in systems:
        s = omm.Solver(m, n, 8, precision=omm.PREC_MIXED, orth_tol=1e-6)
        s.set_HS(dev(H), dev(S))
        solvers.append(s)
    E, it, st, rc = omm.batch_solve_grouped(solvers, [dev(sy[4]) for sy in systems], tol=1e-10,
                                           tile_mode=tile_mode)
    assert rc == omm.OK and (st == omm.OK).all()
    for i, (m, n, H, S, W0) in enumerate(systems):
        assert E[i] == alone[i][0] and it[i] == alone[i][1]
        assert np.array_equal(solvers[i].get_array(omm.ARRAY_W), alone[i][3])
        ref = O.omm_cg(H, S, W0, tol=1e-13, eta=alone[i][4])
        assert abs(E[i] - ref.E) / abs(ref.E) < 1e-8
    modes, ms = omm.batch_last_tuning()
    if tile_mode >= 0:
        assert (modes == tile_mode).all()
    else:
        assert set(modes.tolist()) <= {0, 1} and (ms > 0).all()
    # a second call of the same group reuses the stored tuning
    E2, it2, st2, rc2 = omm.batch_solve_grouped(solvers, [dev(sy[4]) for sy in systems], tol=1e-10,
                                               tile_mode=tile_mode)
    assert rc2 == omm.OK and np.array_equal(E2, E) and np.array_equal(it2, it)
    if tile_mode < 0:
        modes2, ms2 = omm.batch_last_tuning()
        assert np.array_equal(modes2, modes)
    for s in solvers:
        s.close()


def test_grouped_rejects_unsupported_handles(omm):
    import synth
    sysm = synth.make_system(2, 2, 2, seed=1)
    a = omm.Solver(sysm.m, sysm.n, 8, precision=omm.PREC_MIXED)
    b = omm.Solver(sysm.m, sysm.n, 8)                   # FP64 form
    for s in (a, b):
        s.set_HS(dev(sysm.dense_H()), dev(sysm.dense_S()))
    W0 = dev(sysm.W0_dense())
    E, it, st, rc = omm.batch_solve_grouped([a, b], [W0, W0], tol=1e-10)
    assert rc == omm.ERR_UNSUPPORTED
    # one grouped launch holds one operand layout: every handle's search directions
    # must carry the same number of digits
    c = omm.Solver(sysm.m, sysm.n, 8, precision=omm.PREC_MIXED, dir_digits=0)
    c.set_HS(dev(sysm.dense_H()), dev(sysm.dense_S()))
    E, it, st, rc = omm.batch_solve_grouped([a, c], [W0, W0], tol=1e-10)
    assert rc == omm.ERR_UNSUPPORTED
    a.close()
    b.close()
    c.close()
