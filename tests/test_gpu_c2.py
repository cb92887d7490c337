"""The mixed-precision dense form at full benchmark size (512 atoms, m = 4096,
n = 1024) against the FP64 oracle's stored solve of the same input and the
exact minimum (tests/golden/oracle_reference.json, written by
make_oracle_reference.py from the oracle and scipy's eigensolver only):
energy within 1e-8 relative of the oracle (the mixed-precision bar) and 1e-10
of 2 x the sum of the n lowest eigenvalues, ||W^T S W - I||_F < 1e-6 on the
returned W, and the density matrix rho = 2 W (2I - S_W) W^T (Eq. 5) on 1600
sampled entries within 1e-5 of the oracle's and of the exact projector 2 V V^T."""
import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_reference.json")


@pytest.fixture(scope="module")
def omm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_2209_05934_gb300 import omm as _omm
    _omm.lib()
    return _omm


def test_c2_mixed_solve_against_stored_oracle_and_exact(omm):
    import synth
    g = json.load(open(GOLDEN))["c2"]
    sysm = synth.make_system(*g["dims"], seed=g["seed"])
    m, n = sysm.m, sysm.n
    dev = lambda a: torch.from_numpy(np.asfortranarray(a)).to("cuda")
    H, S, W0 = dev(sysm.dense_H()), dev(sysm.dense_S()), dev(sysm.W0_dense())
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    s = omm.Solver(m, n, 8, precision=omm.PREC_MIXED, orth_tol=1e-6, stream=stream.cuda_stream)
    s.set_HS(H, S)
    W = torch.zeros((n, m), dtype=torch.float64, device="cuda").T
    E, iters, st = s.solve(W0, tol=g["tol"], W_out=W)
    torch.cuda.synchronize()
    d = s.diag()
    assert st == omm.OK
    assert d.eta == pytest.approx(g["eta_gershgorin"], rel=1e-14)
    assert abs(E - g["oracle_E"]) / abs(g["oracle_E"]) < 1e-8
    assert abs(E - g["exact_E"]) / abs(g["exact_E"]) < 1e-10
    # orthonormality of the returned W, formed in FP64 here
    SW = W.T @ (S @ W)
    orth = torch.linalg.norm(SW - torch.eye(n, dtype=torch.float64, device="cuda")).item()
    assert orth < 1e-6 and d.orth < 1e-6
    # density matrix on the stored sampled entries
    rs = g["rho_samples"]
    idx = torch.tensor(rs["idx"], device="cuda")
    K = 2.0 * torch.eye(n, dtype=torch.float64, device="cuda") - SW
    Wi, Wj = W[idx[:, 0]], W[idx[:, 1]]
    rho = (2.0 * ((Wi @ K) * Wj).sum(dim=1)).cpu().numpy()
    np.testing.assert_allclose(rho, rs["exact"], rtol=0, atol=1e-5)
    np.testing.assert_allclose(rho, rs["oracle"], rtol=0, atol=1e-5)
    # the library's own rho (omm_get_density, exact-digit tensor-core products)
    R = torch.zeros((m, m), dtype=torch.float64, device="cuda").T
    s.get_density(omm.DENSITY_RHO, R)
    torch.cuda.synchronize()
    got = R[idx[:, 0], idx[:, 1]].cpu().numpy()
    np.testing.assert_allclose(got, rs["exact"], rtol=0, atol=1e-5)
    assert float(torch.sum(R * S).item()) == pytest.approx(2 * n, rel=1e-9)
    s.close()
