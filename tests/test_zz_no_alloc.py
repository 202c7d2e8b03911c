"""bcs_dot_noalloc: the inner product for callers that cannot allocate device
memory (their memory belongs to another allocator, or an allocation would
stall a latency-sensitive loop).  Its result must equal bcs_dot's and the
oracle's correctly rounded inner product -- equality is exact -- on two calls
in a row, which also shows that the shared fixed scratch array carries nothing
over between calls.  Further checks: free device memory does not change across
calls, and a call made inside a torch side stream runs after the work already
queued there."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env(orc):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2108_10591_gb300 as bcs
    return bcs, torch, orc


def test_dot_noalloc_matches_dot_and_oracle_on_two_calls(env):
    bcs, torch, orc = env
    rng = np.random.default_rng(20261204)
    for n, dtype in [(1000003, np.float64), (77777, np.float32), (5, np.float64), (0, np.float64)]:
        x = (rng.standard_normal(n) * 10.0 ** rng.integers(-8, 8, n)).astype(dtype)
        y = rng.standard_normal(n).astype(dtype)
        xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
        ref = orc.dot(x.astype(np.float64), y.astype(np.float64))
        assert bcs.dot(xd, yd) == ref
        for _ in range(2):
            out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
            bcs.dot_noalloc(xd, yd, out)
            torch.cuda.synchronize()
            assert out.item() == ref
    # a size beyond the fixed scratch capacity is rejected, not truncated
    big = torch.zeros(8, dtype=torch.float64, device="cuda")
    assert bcs.lib.bcs_dot_noalloc(2 ** 40, big.data_ptr(), big.data_ptr(), 0, out.data_ptr(), None) == bcs.ERR_ARG


def test_dot_noalloc_allocates_nothing(env):
    bcs, torch, orc = env
    n = 1 << 22
    xd = torch.rand(n, dtype=torch.float64, device="cuda")
    yd = torch.rand(n, dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    bcs.dot_noalloc(xd, yd, out)   # the first call on the device looks up the scratch address
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(20):
        bcs.dot_noalloc(xd, yd, out)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_dot_noalloc_in_side_stream(env):
    """With no stream argument the call uses torch's current stream: inside a side stream it
    sees the vectors that the stream's earlier kernels write."""
    bcs, torch, orc = env
    n = 1 << 24
    rng = np.random.default_rng(7)
    x = rng.standard_normal(n)
    y = rng.standard_normal(n)
    ref = orc.dot(x, y)
    xs, ys = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        for _ in range(2):
            xd = torch.zeros_like(xs)
            yd = torch.zeros_like(ys)
            xd.copy_(xs)
            yd.add_(ys)
            out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
            bcs.dot_noalloc(xd, yd, out)
            assert bcs.dot(xd, yd) == ref
            host = out.to("cpu", non_blocking=False)
            assert host.item() == ref
    s.synchronize()
