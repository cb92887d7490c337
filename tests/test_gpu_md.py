"""MD-step guess of W (section "C† matrix initialization and update"; Table 1,
OMM.Extrapolate) through the C ABI: the pattern update of the localised W and
the linear extrapolation from two previous MD steps, against the oracle.

Inputs: snapshots t = 0, 1, 2 of a straight-line trajectory of the synthetic
geometry (make_md_system), far enough apart that the W pattern changes.
"""
import numpy as np
import pytest

from oracle import omm as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

R_C = 4.5


@pytest.fixture(scope="module")
def omm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_2209_05934_gb300 import omm as _omm
    _omm.lib()
    return _omm


def sparse_handle(omm, sysm, **opts):
    rp, col, Hv, Sv = sysm.bsr()
    wrp, wcol = sysm.w_pattern(R_C)
    s = omm.SparseSolver(sysm.m, sysm.n, 8, 2, rp, col, wrp, wcol, filter_eps=0.0, **opts)
    s.set_HS(Hv, Sv)
    return s, (wrp, wcol)


def resident_W(s):
    return s.get_array(0).reshape(-1, 8, 2)


def blocks_dense(sysm, pat, vals):
    W = np.zeros((sysm.m, sysm.n))
    rp, col = pat
    for I in range(sysm.natoms):
        for b in range(rp[I], rp[I + 1]):
            W[8 * I:8 * I + 8, 2 * col[b]:2 * col[b] + 2] = vals[b]
    return W


def oracle_steps_from(sysm, guess, pat, eta, k):
    """k oracle CG steps of the localised form from a block guess (dense masked arithmetic)."""
    return O.omm_cg(sysm.dense_H(), sysm.dense_S(), blocks_dense(sysm, pat, guess), tol=0.0, eta=eta,
                    max_iter=k, mask=sysm.w_mask(R_C))


def test_sparse_md_guess_matches_oracle(omm):
    """Three MD snapshots whose W patterns differ: the carried and the
    extrapolated guesses equal the oracle's bit for bit, and k CG steps from
    each equal the oracle's steps from the same guess."""
    import synth
    k = 10
    snaps = [synth.make_md_system(4, 4, 3, seed=2, t=t, step=0.25) for t in (0.0, 1.0, 2.0)]
    made = [sparse_handle(omm, s, max_iter=k if i else 30) for i, s in enumerate(snaps)]
    (h0, p0), (h1, p1), (h2, p2) = made
    assert not (np.array_equal(p0[0], p1[0]) and np.array_equal(p0[1], p1[1]))
    assert not (np.array_equal(p1[0], p2[0]) and np.array_equal(p1[1], p2[1]))
    _, _, st0 = h0.solve(snaps[0].W0_bsr_values(R_C), tol=0.0, raise_on_error=False)
    assert st0 == omm.ERR_MAXITER
    W0 = resident_W(h0)
    # carried onto the next pattern: bit-exact gather
    h1.md_guess(h0)
    g1 = resident_W(h1)
    np.testing.assert_array_equal(g1, O.md_guess(W0, p0, p1))
    E1, it1, st1 = h1.solve(None, tol=0.0, raise_on_error=False)
    ref1 = oracle_steps_from(snaps[1], g1, p1, h1.diag().eta, k)
    assert st1 == omm.ERR_MAXITER and it1 == k == ref1.iters
    assert E1 == pytest.approx(ref1.E, rel=1e-12)
    W1 = resident_W(h1)
    np.testing.assert_allclose(blocks_dense(snaps[1], p1, W1), ref1.W, rtol=1e-8, atol=1e-10)
    # linear extrapolation from the two previous steps: one rounding per element, bit-exact
    h2.md_guess(h1, h0)
    g2 = resident_W(h2)
    np.testing.assert_array_equal(g2, O.md_guess(W1, p1, p2, W0, p0))
    # onto the oldest snapshot's pattern again: blocks that left the radius at
    # the middle step and came back start at zero, whatever the older step held
    h3, p3 = sparse_handle(omm, snaps[0], max_iter=k)
    h3.md_guess(h1, h0)
    np.testing.assert_array_equal(resident_W(h3), O.md_guess(W1, p1, p3, W0, p0))
    h3.close()
    E2, it2, st2 = h2.solve(None, tol=0.0, raise_on_error=False)
    ref2 = oracle_steps_from(snaps[2], g2, p2, h2.diag().eta, k)
    assert it2 == k and E2 == pytest.approx(ref2.E, rel=1e-12)
    np.testing.assert_allclose(blocks_dense(snaps[2], p2, resident_W(h2)), ref2.W, rtol=1e-8, atol=1e-10)
    for h, _ in made:
        h.close()


def test_dense_md_guess_bit_exact(omm):
    import synth
    snaps = [synth.make_md_system(3, 3, 2, seed=1, t=t, step=0.05) for t in (0.0, 1.0)]
    m, n = snaps[0].m, snaps[0].n
    W0 = np.asfortranarray(snaps[0].W0_dense())
    hs, Ws = [], []
    for sysm in snaps:
        h = omm.Solver(m, n, 8)
        h.set_HS(np.asfortranarray(sysm.dense_H()), np.asfortranarray(sysm.dense_S()))
        W = np.zeros((m, n), order="F")
        h.solve(W0, tol=1e-11, W_out=W)
        hs.append(h)
        Ws.append(W)
    dst = omm.Solver(m, n, 8)
    dst.md_guess(hs[1])
    out = dst.get_array(0)
    np.testing.assert_array_equal(out, Ws[1])
    dst.md_guess(hs[1], hs[0])
    out = dst.get_array(0)
    np.testing.assert_array_equal(out, O.md_guess_dense(Ws[1], Ws[0]))
    # in place: the step-1 handle becomes the step-2 guess
    hs[1].md_guess(hs[1], hs[0])
    out = hs[1].get_array(0)
    np.testing.assert_array_equal(out, 2.0 * Ws[1] - Ws[0])
    # the Cholesky variant takes and keeps W in the original basis
    ch = omm.Solver(m, n, 8, cholesky=1)
    ch.set_HS(np.asfortranarray(snaps[1].dense_H()), np.asfortranarray(snaps[1].dense_S()))
    ch.md_guess(hs[0])
    out = ch.get_array(0)
    np.testing.assert_array_equal(out, Ws[0])
    E, it, st = ch.solve(None, tol=1e-11)
    assert st == omm.OK
    for h in hs + [dst, ch]:
        h.close()


def test_md_guess_errors(omm):
    import synth
    a = synth.make_system(3, 3, 2, seed=0)
    b = synth.make_system(3, 3, 3, seed=0)
    ha, hb = omm.Solver(a.m, a.n, 8), omm.Solver(b.m, b.n, 8)
    ha2 = omm.Solver(a.m, a.n, 8)
    with pytest.raises(omm.OmmError) as e:
        ha2.md_guess(ha)                       # ha has no solution yet
    assert e.value.status == omm.ERR_STATE
    ha.set_HS(np.asfortranarray(a.dense_H()), np.asfortranarray(a.dense_S()))
    ha.solve(np.asfortranarray(a.W0_dense()), tol=1e-8)
    with pytest.raises(omm.OmmError) as e:
        hb.md_guess(ha)                        # different sizes
    assert e.value.status == omm.ERR_ARG
    hs, _ = sparse_handle(omm, a)
    with pytest.raises(omm.OmmError) as e:
        hs.md_guess(ha)                        # dense into sparse
    assert e.value.status == omm.ERR_ARG
    for h in (ha, hb, ha2, hs):
        h.close()
