"""rfd_phi1_noalloc: step a4 for callers that cannot allocate device memory.

Some callers may not call cudaMalloc -- a latency-critical loop where an
allocation could synchronise the device, or a process whose device memory is
owned by another allocator.  rfd_phi1_noalloc serves them from a fixed device
array instead of allocating.  This file checks, through the C ABI, that two
calls in a row give the same G as the allocating rfd_phi1 (within the 1e-12
tolerance the phi1 tests use), that the second call is not disturbed by what
the first left in the shared array, and that sizes beyond the array's limit are
refused.  It is named so that pytest collects it last.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
import paper_2302_00942_gb300 as rfd  # noqa: E402

DEV = torch.device("cuda:0") if torch.cuda.is_available() else None
TOL = 1e-12


def _matrix(m, norm, seed):
    rng = np.random.default_rng(seed)
    M = rng.standard_normal((m, m))
    return M * (norm / np.abs(M).sum(0).max())


@pytest.mark.parametrize("native", [False, True])
def test_noalloc_matches_allocating_entry_two_calls(native):
    # two calls in a row with different sizes and norms: the second must not see
    # stale workspace (squarings, LU status words) left by the first
    for m, norm, lam, seed in [(128, 12.0, 0.8, 1), (96, 0.3, -1.5, 2)]:
        M = torch.from_numpy(_matrix(m, norm, seed)).to(DEV)
        G_ref = torch.zeros_like(M)
        G_na = torch.full_like(M, float("nan"))
        st_ref = rfd.rfd_phi1(m, lam, M, G_ref, native_fp64=native)
        st_na = rfd.rfd_phi1_noalloc(m, lam, M, G_na, native_fp64=native)
        a, b = G_na.cpu().numpy(), G_ref.cpu().numpy()
        assert np.isfinite(a).all()
        assert oracle.rel_frobenius(a, b) <= TOL
        assert (st_na["pade_degree"], st_na["squarings"]) == (st_ref["pade_degree"], st_ref["squarings"])
        # and both against the CPU oracle
        assert oracle.rel_frobenius(a, lam * oracle.phi1(lam * M.cpu().numpy())) <= 1e-12 * max(1.0, norm)


def test_noalloc_rejects_sizes_beyond_its_array():
    M = torch.zeros((129, 129), dtype=torch.float64, device=DEV)
    G = torch.zeros_like(M)
    with pytest.raises(rfd.RfdError) as e:
        rfd.rfd_phi1_noalloc(129, 1.0, M, G)
    assert e.value.status == rfd.RFD_EINVAL
    assert "m <= 128" in rfd.rfd_last_error()


def test_noalloc_makes_no_device_allocation():
    M = torch.from_numpy(_matrix(64, 1.0, 3)).to(DEV)
    G = torch.zeros_like(M)
    rfd.rfd_phi1_noalloc(64, 1.0, M, G)       # first call on the device: address set-up
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        rfd.rfd_phi1_noalloc(64, 1.0, M, G)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
