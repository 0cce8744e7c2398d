"""The FP64-accurate GEMM of step a4 (Ozaki splitting on the BF16 tensor
cores) against exact references, and step a4 with it against the oracle."""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
import paper_2302_00942_gb300 as rfd  # noqa: E402

DEV = torch.device("cuda:0") if torch.cuda.is_available() else None


def _run(method, A, B, C0=None, alpha=1.0, beta=0.0):
    At, Bt = torch.from_numpy(A).to(DEV), torch.from_numpy(B).to(DEV)
    Ct = torch.from_numpy(C0.copy()).to(DEV) if C0 is not None else torch.zeros((A.shape[0], B.shape[1]),
                                                                                  dtype=torch.float64, device=DEV)
    rfd.rfd_debug_dgemm(method, At, Bt, Ct, alpha, beta)
    return Ct.cpu().numpy()


@pytest.mark.parametrize("M,N,K", [(1024, 1024, 1024), (1000, 777, 999), (1, 1, 1), (130, 65, 64), (257, 300, 33),
                                   (256, 192, 2048), (100, 70, 4096)])
def test_integer_matrices_exact(M, N, K):
    """Integer entries below 2^20: every FP64 product and partial sum is exact, so the
    emulated result must equal the exact integer result bit for bit."""
    rng = np.random.default_rng(M + N + K)
    A = rng.integers(-(1 << 20), 1 << 20, size=(M, K)).astype(np.float64)
    B = rng.integers(-(1 << 20), 1 << 20, size=(K, N)).astype(np.float64)
    A[0, :] = 0.0                                # a zero row
    ref = (A.astype(object) @ B.astype(object)).astype(np.float64)   # exact integers
    np.testing.assert_array_equal(_run(1, A, B), ref)


@pytest.mark.parametrize("M,N,K", [(512, 512, 512), (1024, 1024, 1024), (200, 130, 1000), (300, 200, 3000)])
def test_real_matrices_against_exact_dot_products(M, N, K):
    rng = np.random.default_rng(K)
    A = rng.standard_normal((M, K)) * np.exp(rng.uniform(-20, 20, (M, 1)))   # rows over ~17 decades
    B = rng.standard_normal((K, N)) * np.exp(rng.uniform(-20, 20, (1, N)))
    A[rng.random((M, K)) < 0.01] *= 1e-12                                      # tiny entries inside rows
    C_emul = _run(1, A, B)
    C_nat = _run(0, A, B)
    absAB = np.abs(A) @ np.abs(B)
    idx = [(int(i), int(j)) for i, j in zip(rng.integers(0, M, 40), rng.integers(0, N, 40))]
    for i, j in idx:
        exact = float(sum(Fraction(a) * Fraction(b) for a, b in zip(A[i], B[:, j])))
        bound = 2.0 ** -50 * absAB[i, j]
        assert abs(C_emul[i, j] - exact) <= bound, (i, j, C_emul[i, j], exact, bound)
        assert abs(C_nat[i, j] - exact) <= K * 2.0 ** -53 * absAB[i, j]
    # whole-matrix agreement with native FP64, normwise
    assert np.linalg.norm(C_emul - C_nat) <= 1e-14 * np.linalg.norm(absAB)


def test_alpha_beta():
    rng = np.random.default_rng(3)
    A, B, C0 = rng.standard_normal((300, 200)), rng.standard_normal((200, 100)), rng.standard_normal((300, 100))
    got = _run(1, A, B, C0, alpha=-0.5, beta=2.0)
    np.testing.assert_allclose(got, -0.5 * (A @ B) + 2.0 * C0, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("m,norm", [(256, 0.5), (512, 2.0), (1024, 0.9), (300, 40.0)])
def test_phi1_emulated_matches_native_and_oracle(m, norm):
    rng = np.random.default_rng(m)
    M = rng.standard_normal((m, m))
    M *= norm / np.abs(M).sum(0).max()
    Mt = torch.from_numpy(M).to(DEV)
    Ge = torch.zeros_like(Mt)
    Gn = torch.zeros_like(Mt)
    se = rfd.rfd_phi1(m, 1.0, Mt, Ge)
    sn = rfd.rfd_phi1(m, 1.0, Mt, Gn, native_fp64=True)
    assert se["phi1_emulated"] == 1 and sn["phi1_emulated"] == 0
    ref = oracle.phi1(M)
    e_emul = oracle.rel_frobenius(Ge.cpu().numpy(), ref)
    e_nat = oracle.rel_frobenius(Gn.cpu().numpy(), ref)
    print(m, norm, se, e_emul, e_nat)
    assert e_emul <= 1e-13 * max(1.0, norm) and e_nat <= 1e-13 * max(1.0, norm)
