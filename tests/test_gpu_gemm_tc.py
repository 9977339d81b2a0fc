"""The FP32 tensor-core GEMMs (tcgen05, three-term BF16 split) against a plain
FP64 product of the same FP32 inputs: FP32-level accuracy on ragged shapes,
both transposes, alpha/beta, K = 0, and the exact-BF16 B path used by the
sampling products; both kernels: the TMA pipeline over pre-split operands
(path 0) and the factorization's kernel that stages FP32 tiles with
asynchronous copies and splits them in its loop (path 2)."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _gemm(A, B, Cm, ta, tb, alpha, beta, b_exact=0, path=0):
    import paper_1502_07405_gb300 as P
    f = P.lib.hssmf_gemm_f32
    f.restype = C.c_int
    f.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_float, C.c_void_p, C.c_longlong,
                  C.c_void_p, C.c_longlong, C.c_float, C.c_void_p, C.c_longlong, C.c_int, C.c_void_p]
    m, n = Cm.shape
    k = A.shape[0] if ta else A.shape[1]
    # column-major device copies
    dA = torch.tensor(np.asfortranarray(A).T.copy(), dtype=torch.float32, device="cuda")
    dB = torch.tensor(np.asfortranarray(B).T.copy(), dtype=torch.float32, device="cuda")
    dC = torch.tensor(np.asfortranarray(Cm).T.copy(), dtype=torch.float32, device="cuda")
    st = f(ta, tb, m, n, k, alpha, dA.data_ptr(), A.shape[0], dB.data_ptr(), B.shape[0], beta,
           dC.data_ptr(), m, b_exact | path, None)
    assert st == 0
    return dC.cpu().numpy().T


def _bf16(x):
    return torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()


@pytest.mark.parametrize("shape", [(1, 1, 1), (128, 128, 64), (200, 70, 100), (300, 257, 513),
                                   (129, 16, 65), (1000, 300, 700)])
@pytest.mark.parametrize("ta,tb", [(0, 0), (1, 0), (0, 1), (1, 1)])
@pytest.mark.parametrize("path", [0, 2])
def test_fp32_accuracy(shape, ta, tb, path):
    m, n, k = shape
    rng = np.random.default_rng(m * 7 + n * 3 + k + 11 * ta + 5 * tb)
    A = rng.standard_normal((k, m) if ta else (m, k)).astype(np.float32)
    B = rng.standard_normal((n, k) if tb else (k, n)).astype(np.float32)
    C0 = rng.standard_normal((m, n)).astype(np.float32)
    alpha, beta = 1.5, -0.5
    got = _gemm(A, B, C0, ta, tb, alpha, beta, path=path)
    opA = (A.T if ta else A).astype(np.float64)
    opB = (B.T if tb else B).astype(np.float64)
    ref = alpha * opA @ opB + beta * C0.astype(np.float64)
    scale = abs(alpha) * np.abs(opA) @ np.abs(opB) + abs(beta) * np.abs(C0)
    err = np.abs(got - ref) / scale
    # FP32-level: a single BF16 product would give ~1e-3 here
    assert err.max() < 2e-6, err.max()


@pytest.mark.parametrize("ta", [0, 1])
@pytest.mark.parametrize("path", [0, 2])
def test_exact_bf16_b(ta, path):
    m, n, k = 777, 64, 1500
    rng = np.random.default_rng(3 + ta)
    A = rng.standard_normal((k, m) if ta else (m, k)).astype(np.float32)
    B = _bf16(rng.standard_normal((k, n))).astype(np.float32)
    C0 = rng.standard_normal((m, n)).astype(np.float32)
    got = _gemm(A, B, C0, ta, 0, 1.0, 1.0, b_exact=1, path=path)
    opA = (A.T if ta else A).astype(np.float64)
    ref = opA @ B.astype(np.float64) + C0
    scale = np.abs(opA) @ np.abs(B.astype(np.float64)) + np.abs(C0)
    assert (np.abs(got - ref) / scale).max() < 2e-6


@pytest.mark.parametrize("path", [0, 2])
def test_k_zero_and_beta_zero(path):
    rng = np.random.default_rng(0)
    C0 = rng.standard_normal((50, 30)).astype(np.float32)
    got = _gemm(np.zeros((50, 1), np.float32), np.zeros((1, 30), np.float32), C0, 0, 0, 2.0, 0.25, path=path)
    np.testing.assert_allclose(got, 0.25 * C0, rtol=1e-6)
    import paper_1502_07405_gb300 as P
    f = P.lib.hssmf_gemm_f32
    dC = torch.tensor(C0.T.copy(), device="cuda")
    st = f(0, 0, 50, 30, 0, 1.0, None, 50, None, 1, -1.0, dC.data_ptr(), 50, path, None)
    assert st == 0
    np.testing.assert_allclose(dC.cpu().numpy().T, -C0, rtol=0)
    # beta = 0 ignores NaN in C
    dC.fill_(float("nan"))
    Ad = torch.ones((7, 50), device="cuda")  # 50 x 7 column-major
    Bd = torch.ones((30, 7), device="cuda")  # 7 x 30 column-major
    st = f(0, 0, 50, 30, 7, 1.0, Ad.data_ptr(), 50, Bd.data_ptr(), 7, 0.0, dC.data_ptr(), 50, path, None)
    assert st == 0
    np.testing.assert_allclose(dC.cpu().numpy(), 7.0)
