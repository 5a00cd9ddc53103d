"""Gram products G = A^T diag(w) B (mor_gram, through the C ABI) on the FP32
CUDA cores and on the tcgen05 tensor cores (TF32, BF16 inputs, single pass or
split into head and remainder in three passes), against the FP64 product of
the same inputs."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1406_7042_gb300 import fdtdmor as F  # noqa: E402

# relative Frobenius error bounds of the three arithmetics on random inputs
TOL = {"native": 1e-5, "tf32": 2e-3, "bf16": 1.5e-2, "tf32x3": 2e-5, "bf16x3": 5e-4}


def _case(n, M, N, weighted, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((M, n)).astype(np.float32)
    B = rng.standard_normal((N, n)).astype(np.float32)
    w = rng.uniform(0.5, 2.0, n).astype(np.float32) if weighted else None
    Bw = B.astype(np.float64) * (w.astype(np.float64) if weighted else 1.0)
    G = A.astype(np.float64) @ Bw.T
    return A, B, w, G


@pytest.mark.parametrize("arith", ["native", "tf32", "bf16", "tf32x3", "bf16x3"])
@pytest.mark.parametrize("n,M,N,weighted", [(1000, 7, 1, False), (1000, 130, 16, True), (4096, 128, 200, True),
                                            (262181, 40, 300, False), (70001, 257, 33, True)])
def test_gram_matches_fp64(arith, n, M, N, weighted):
    A, B, w, G = _case(n, M, N, weighted, seed=n + M + N)
    Gg = F.gram(torch.tensor(A, device="cuda"), torch.tensor(B, device="cuda"),
                torch.tensor(w, device="cuda") if w is not None else None, arith).cpu().numpy()
    err = np.linalg.norm(Gg - G) / np.linalg.norm(G)
    assert err <= TOL[arith], err


def test_gram_symmetric_weighted_is_symmetric_and_exact_on_integers():
    """Small integers are exact in TF32 and BF16 (8 significant bits), and so
    are their products and the FP32 sums here: the tensor-core result must
    equal the exact product bit for bit."""
    rng = np.random.default_rng(3)
    n, M = 3000, 64
    A = rng.integers(-8, 9, (M, n)).astype(np.float32)
    G = A.astype(np.float64) @ A.astype(np.float64).T
    for arith in ("tf32", "bf16"):
        At = torch.tensor(A, device="cuda")
        Gg = F.gram(At, At, None, arith).cpu().numpy()
        assert np.array_equal(Gg, G), arith
