"""bcs_dot_noalloc: the inner product for callers that cannot allocate device
memory (their memory belongs to another allocator, or an allocation would
stall a latency-sensitive loop).  Its result must equal bcs_dot's -- both are
correctly rounded, so equality is exact -- on two calls in a row, which also
shows that the shared fixed scratch array carries nothing over between calls."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_dot_noalloc_matches_dot_on_two_calls():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2108_10591_gb300 as bcs
    rng = np.random.default_rng(20261204)
    for n, dtype in [(1000003, np.float64), (77777, np.float32), (5, np.float64), (0, np.float64)]:
        x = (rng.standard_normal(n) * 10.0 ** rng.integers(-8, 8, n)).astype(dtype)
        y = rng.standard_normal(n).astype(dtype)
        xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
        ref = bcs.dot(xd, yd)
        for _ in range(2):
            out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
            bcs.dot_noalloc(xd, yd, out)
            torch.cuda.synchronize()
            assert out.item() == ref
    # a size beyond the fixed scratch capacity is rejected, not truncated
    big = torch.zeros(8, dtype=torch.float64, device="cuda")
    assert bcs.lib.bcs_dot_noalloc(2 ** 40, big.data_ptr(), big.data_ptr(), 0, out.data_ptr(), None) == bcs.ERR_ARG
