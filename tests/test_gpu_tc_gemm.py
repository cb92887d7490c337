"""tcgen05 split-BF16 GEMM against an FP64 numpy product (through the C ABI)."""
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


def dev(a):
    return torch.from_numpy(np.asfortranarray(a)).to("cuda")


def run_split(omm, tA, tB, M, N, K, nd, A, B, alpha=1.0, beta=0.0, Cin=None):
    out = torch.zeros((N, M), dtype=torch.float64, device="cuda").T
    nb = omm.op_split_gemm_workspace_bytes(M, N, K, nd)
    ws = torch.zeros(nb // 8 + 64, dtype=torch.float64, device="cuda")
    st = omm.op_split_gemm(tA, tB, M, N, K, nd, alpha, dev(A), A.shape[0], dev(B), B.shape[0], beta,
                           dev(Cin) if Cin is not None else None, M, out, M, ws, nb)
    assert st == omm.OK, omm.lib().omm_last_error()
    torch.cuda.synchronize()
    return out.cpu().numpy()


# bound on the split error: the digit truncation and the tensor cores' FP32
# accumulation scale with sum_k |A_ik| |B_kj|.  With three digits the
# accumulation dominates (measured ~4e-7 of that sum at K = 4096); two digits
# keep ~16 bits, one digit 8 bits.
REL = {3: 1e-5, 2: 1e-4, 1: 2e-2}


@pytest.mark.parametrize("tA,tB,M,N,K", [(0, 0, 256, 128, 256), (1, 0, 100, 70, 33), (0, 1, 300, 200, 520),
                                         (1, 1, 129, 257, 64), (0, 0, 128, 128, 4096), (1, 0, 16, 8, 8),
                                         (0, 0, 640, 520, 1544)])
@pytest.mark.parametrize("nd", [3, 2, 1])
def test_split_gemm_matches_fp64(omm, tA, tB, M, N, K, nd):
    rng = np.random.default_rng(M + 3 * N + 7 * K + nd)
    A = rng.standard_normal((K, M) if tA else (M, K))
    B = rng.standard_normal((N, K) if tB else (K, N))
    opA = A.T if tA else A
    opB = B.T if tB else B
    C = run_split(omm, tA, tB, M, N, K, nd, A, B)
    ref = opA @ opB
    bound = REL[nd] * (np.abs(opA) @ np.abs(opB)) + 1e-300
    err = np.abs(C - ref)
    assert np.all(err <= bound), (err / bound).max()


def test_split_gemm_alpha_beta(omm):
    rng = np.random.default_rng(0)
    M, N, K = 200, 96, 160
    A, B, Cin = rng.standard_normal((M, K)), rng.standard_normal((K, N)), rng.standard_normal((M, N))
    C = run_split(omm, 0, 0, M, N, K, 3, A, B, alpha=-2.0, beta=4.0, Cin=Cin)
    ref = -2.0 * A @ B + 4.0 * Cin
    assert np.abs(C - ref).max() <= 4e-6 * (np.abs(A) @ np.abs(B)).max()


def test_split3_accuracy_beats_fp32_inputs(omm):
    """Three digits carry FP64 inputs to ~FP32 accumulation accuracy: far
    better than rounding the inputs to BF16 once."""
    rng = np.random.default_rng(1)
    M, N, K = 256, 256, 1024
    A, B = rng.standard_normal((M, K)), rng.standard_normal((K, N))
    ref = A @ B
    e3 = np.abs(run_split(omm, 0, 0, M, N, K, 3, A, B) - ref).max()
    e2 = np.abs(run_split(omm, 0, 0, M, N, K, 2, A, B) - ref).max()
    e1 = np.abs(run_split(omm, 0, 0, M, N, K, 1, A, B) - ref).max()
    print(f"max abs error: 3 digits {e3:.3e}, 2 digits {e2:.3e}, 1 digit {e1:.3e}")
    assert e3 < e2 < e1
    assert e3 < 1e-3 * e1


# ------------------------------------------------------------------ exact-digit GEMM
def run_exact(omm, tA, tB, M, N, K, nd, A, B, alpha=1.0, beta=0.0, Cin=None):
    out = torch.zeros((N, M), dtype=torch.float64, device="cuda").T
    nb = omm.op_exact_gemm_workspace_bytes(M, N, K, nd)
    ws = torch.zeros(nb // 8 + 64, dtype=torch.float64, device="cuda")
    st = omm.op_exact_gemm(tA, tB, M, N, K, nd, alpha, dev(A), A.shape[0], dev(B), B.shape[0], beta,
                           dev(Cin) if Cin is not None else None, M, out, M, ws, nb)
    assert st == omm.OK, omm.lib().omm_last_error()
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _exact_ref(opA, opB):
    """Product accurate beyond FP64: split both operands into hi + lo halves."""
    def split(X):
        hi = X.astype(np.float32).astype(np.float64)
        return hi, X - hi
    ah, al = split(opA)
    bh, bl = split(opB)
    return ((ah @ bh) + ((ah @ bl) + (al @ bh))) + al @ bl


@pytest.mark.parametrize("tA,tB,M,N,K", [(0, 0, 256, 128, 512), (1, 0, 100, 70, 33), (0, 1, 300, 200, 4100),
                                         (1, 1, 129, 257, 64), (0, 0, 128, 128, 4096)])
def test_exact_gemm_near_fp64(omm, tA, tB, M, N, K):
    rng = np.random.default_rng(M + N + K)
    # rows with very different scales stress the per-row exponents
    A = rng.standard_normal((K, M) if tA else (M, K)) * np.exp(rng.uniform(-4, 4, size=(1, M) if tA else (M, 1)))
    B = rng.standard_normal((N, K) if tB else (K, N)) * np.exp(rng.uniform(-4, 4, size=(N, 1) if tB else (1, N)))
    opA = A.T if tA else A
    opB = B.T if tB else B
    C = run_exact(omm, tA, tB, M, N, K, 7, A, B, alpha=0.5, beta=-1.0, Cin=np.ones((M, N)))
    ref = 0.5 * (opA @ opB) - 1.0
    scale = np.abs(opA).max(axis=1, keepdims=True) * np.abs(opB).max(axis=0, keepdims=True) * np.sqrt(K)
    err = np.abs(C - ref) / scale
    assert err.max() < 1e-12, err.max()


def test_exact_gemm_digits_control_accuracy(omm):
    rng = np.random.default_rng(7)
    M, N, K = 256, 256, 2048
    A, B = rng.standard_normal((M, K)), rng.standard_normal((K, N))
    ref = _exact_ref(A, B)
    scale = np.abs(A).max(axis=1, keepdims=True) * np.abs(B).max(axis=0, keepdims=True) * np.sqrt(K)
    errs = {nd: (np.abs(run_exact(omm, 0, 0, M, N, K, nd, A, B) - ref) / scale).max() for nd in (3, 5, 7)}
    print("exact-digit relative errors:", errs)
    assert errs[3] > errs[5] > errs[7]
    assert errs[7] < 1e-13
