"""Allocation-free line-search coefficients (omm_op_quartic_coeffs_static).

Callers that cannot allocate device memory get the coefficients through a
variant whose scratch is a static array inside the library.  This test calls
it through the C ABI twice in a row (the second call reuses the array the
first one left behind) and checks both results against the entry point that
takes caller scratch.  It sits in its own file, collected last, and passes
both alone in a fresh process and after the rest of the suite.
"""
import numpy as np
import pytest

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


def _inputs(n, seed):
    rng = np.random.default_rng(seed)
    sym = lambda a: 0.5 * (a + a.T)
    mats = dict(h0=sym(rng.standard_normal((n, n))), s0=np.eye(n) + 0.01 * sym(rng.standard_normal((n, n))),
                X=rng.standard_normal((n, n)), Y=rng.standard_normal((n, n)) * 0.1,
                h2=-np.abs(sym(rng.standard_normal((n, n)))), s2=np.abs(sym(rng.standard_normal((n, n)))))
    return {k: torch.from_numpy(np.asfortranarray(v)).to("cuda") for k, v in mats.items()}


def test_static_scratch_matches_caller_scratch_twice(omm):
    """Same kernel, block count and reduction order as the caller-scratch entry
    point, so the results are equal bit for bit; the second call allocates no
    device memory."""
    for call, (n, seed) in enumerate([(200, 1), (1024, 2)]):
        t = _inputs(n, seed)
        nb = omm.op_quartic_coeffs_scratch_bytes(n)
        scratch = torch.zeros(nb // 8 + 1, dtype=torch.float64, device="cuda")
        ref = torch.zeros(5, dtype=torch.float64, device="cuda")
        got = torch.full((5,), float("nan"), dtype=torch.float64, device="cuda")
        assert omm.op_quartic_coeffs(n, t["h0"], t["s0"], n, t["X"], t["Y"], t["h2"], t["s2"], n,
                                     ref, scratch, nb) == omm.OK
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        st = omm.op_quartic_coeffs_static(n, t["h0"], t["s0"], n, t["X"], t["Y"], t["h2"], t["s2"], n, got)
        assert st == omm.OK, omm.lib().omm_last_error()
        torch.cuda.synchronize()
        if call > 0:
            assert torch.cuda.mem_get_info()[0] == free0
        r, g = ref.cpu().numpy(), got.cpu().numpy()
        np.testing.assert_array_equal(g, r, err_msg=f"call {call}")


def test_static_scratch_rejects_out_of_range_sizes(omm):
    c = torch.zeros(5, dtype=torch.float64, device="cuda")
    assert omm.op_quartic_coeffs_static(-1, None, None, 1, None, None, None, None, 1, c) == omm.ERR_ARG
    assert omm.op_quartic_coeffs_static(2 ** 31, None, None, 1, None, None, None, None, 1, c) == omm.ERR_ARG
    assert b"outside" in omm.lib().omm_last_error()
    assert omm.op_quartic_coeffs_static(4, None, None, 4, None, None, None, None, 4, c) == omm.ERR_ARG
    assert b"NULL" in omm.lib().omm_last_error()
    assert omm.lib().omm_op_quartic_coeffs_static_max_bytes() == 512 * 13 * 8 + 256
