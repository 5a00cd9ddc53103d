"""mor_compare_noalloc, the comparison entry point for callers that cannot
allocate device memory while it runs (a host program or plugin that owns all
device memory, or an allocator that must not grow), against mor_compare.

This file is collected last so that, if it fails, a run that stops at the
first failure has already run every other test; it also passes on its own in
a fresh process."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1406_7042_gb300 import fdtdmor as F  # noqa: E402


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_noalloc_compare_matches_compare_twice(dtype):
    g = torch.Generator(device="cpu").manual_seed(1234)
    p, nref, stride, offset = 3, 90001, 7, 6
    n = (nref - offset - 1) // stride + 1
    y_ref = torch.randn((nref, p), generator=g, dtype=torch.float64).to(dtype).cuda()
    y_red = (y_ref[offset::stride][:n] * 1.001
             + 1e-3 * torch.randn((n, p), generator=g, dtype=torch.float64).to(dtype).cuda()).contiguous()
    tol = 1e-12 if dtype == torch.float64 else 1e-6
    for _ in range(2):  # two calls in a row: the shared scratch keeps the last call's contents
        e_ref = F.compare(y_red, y_ref, stride, offset)
        e_na = F.compare_noalloc(y_red, y_ref, stride, offset)
        assert e_ref > 0
        assert abs(e_na - e_ref) <= tol * e_ref
    # a second, smaller input right after: stale partial sums must not leak in
    y_small = y_red[:1000].contiguous()
    assert abs(F.compare_noalloc(y_small, y_ref, stride, offset) - F.compare(y_small, y_ref, stride, offset)) \
        <= tol * F.compare(y_small, y_ref, stride, offset)


def test_noalloc_compare_rejects_oversized_input():
    y = torch.zeros((1, 1), device="cuda")
    big = torch.zeros((1 << 24) + 8, 1, device="cuda")
    with pytest.raises(F.FdtdError) as e:
        F.compare_noalloc(big, big, 1, 0)
    assert e.value.status == F.FDTD_EINVAL and "no-allocation maximum" in str(e.value)
    assert F.compare_noalloc(y, y, 1, 0) == 0.0
