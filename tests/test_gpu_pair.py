"""The split products on CTA pairs (tcgen05.mma.cta_group::2, 256 x 256 tiles)
against the one-CTA tiles and the FP64 oracle: the same solves with
gemm_pair = 1 and 0 take the same steps to the same energy, on sizes that
fill the pair tiles and on ragged ones that leave the second CTA of a pair
partly or wholly outside the matrix.  With n = 150 and n = 256 the contraction
[W D]^T [H'D SD] has pair tiles wholly in the rows of D^T, whose one-digit A
operand those tiles load and multiply as one plane."""
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


def _solve(omm, H, S, W0, m, n, pair, max_iter=10000):
    s = omm.Solver(m, n, 8, precision=omm.PREC_MIXED, orth_tol=1e-6, gemm_pair=pair, max_iter=max_iter)
    s.set_HS(dev(H), dev(S))
    W = torch.zeros((n, m), dtype=torch.float64, device="cuda").T
    E, iters, st = s.solve(dev(W0), tol=1e-10, W_out=W, raise_on_error=False)
    d = s.diag()
    s.close()
    return E, iters, st, d, W.cpu().numpy()


@pytest.mark.parametrize("case", ["c1", "ragged_600_150", "ragged_136_34", "dense_1024_256"])
def test_pair_tiles_match_single_tiles_and_oracle(omm, case):
    import synth
    if case == "c1":
        sysm = synth.make_system(4, 4, 4, seed=0)
        H, S, W0, m, n = sysm.dense_H(), sysm.dense_S(), sysm.W0_dense(), sysm.m, sysm.n
    else:
        m, n = (int(v) for v in case.split("_")[1:])
        H, S, _, W0 = synth.make_dense_gapped(m, n, seed=3)
    W0 = np.asfortranarray(W0)
    # fixed steps: the two tilings give the same iterates up to the FP32 accumulation
    Ep, ip, sp_, dp, Wp = _solve(omm, H, S, W0, m, n, 1, max_iter=6)
    Es, is_, ss, ds, Ws = _solve(omm, H, S, W0, m, n, 0, max_iter=6)
    assert ip == is_ == 6
    assert abs(Ep - Es) / abs(Es) < 1e-9
    np.testing.assert_allclose(Wp, Ws, atol=1e-7)
    # converged: both within the mixed-precision bar of the oracle
    Ep, ip, stp, dp, Wp = _solve(omm, H, S, W0, m, n, 1)
    ref = O.omm_cg(H, S, W0, tol=1e-13, eta=dp.eta)
    assert stp == omm.OK and abs(Ep - ref.E) / abs(ref.E) < 1e-8 and dp.orth < 1e-6
