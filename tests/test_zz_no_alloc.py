"""The allocation-free dot product against the regular one.

ed_dot_noalloc serves callers that cannot allocate device memory (their device
memory is owned by another framework, or they must not grow their footprint
mid-solve); it keeps its partial sums in a fixed static device array instead.
Here it must agree with ed_dot within 1e-12 relative, on two calls in a row,
for every vector format and for a length with a ragged last tile, and with a
float64 dot product formed on the host from the same stored values (so that a
fault shared by both device paths would show); the device's free memory must
not change across the second call; and a length beyond the scratch capacity
must be rejected without touching the device.  This file is
collected last on purpose so that a stop-at-first-failure run has already run
every other test; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

from tests._gpu import ensure_built, torch_cuda, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp64", "df64", "fp32"])
def test_noalloc_dot_matches_ed_dot_twice(prec):
    torch = torch_cuda()
    ed = ensure_built()
    ctx = ed.ed_ctx_create(0)
    try:
        rng = np.random.default_rng(5)
        for n in (1_000_003, 4096 * 3 + 17):
            a = rng.standard_normal(n)
            b = rng.standard_normal(n)
            x = to_dev(a, prec, ed, torch)
            y = to_dev(b, prec, ed, torch)
            ref = ed.ed_dot(ctx, x, y, n, prec)
            first = ed.ed_dot_noalloc(x, y, n, prec)
            torch.cuda.synchronize()
            free_before = torch.cuda.mem_get_info()[0]
            second = ed.ed_dot_noalloc(x, y, n, prec)
            torch.cuda.synchronize()
            assert torch.cuda.mem_get_info()[0] == free_before   # nothing allocated on the device
            # host reference over the values as stored on the device (FP32 and
            # DF64 storage round the inputs), summed in float64 by numpy
            ha = to_host(x, prec, n, ed, torch)
            hb = to_host(y, prec, n, ed, torch)
            host = float(np.dot(ha, hb))
            scale = float(np.abs(a) @ np.abs(b))
            assert abs(first - ref) <= 1e-12 * scale, (first, ref)
            assert abs(second - ref) <= 1e-12 * scale, (second, ref)
            assert abs(first - host) <= 1e-12 * scale, (first, host)
            assert abs(second - host) <= 1e-12 * scale, (second, host)
            # a different pair next: the shared scratch keeps no stale state
            other = ed.ed_dot_noalloc(y, y, n, prec)
            assert abs(other - ed.ed_dot(ctx, y, y, n, prec)) <= 1e-12 * float(b @ b)
    finally:
        ed.ed_ctx_destroy(ctx)


def test_noalloc_dot_rejects_oversize_and_empty():
    torch = torch_cuda()
    ed = ensure_built()
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    assert ed.ed_dot_noalloc(x, x, 0, "fp64") == 0.0
    with pytest.raises(ed.EdError) as e:
        ed.ed_dot_noalloc(x, x, 65536 * 4096 + 1, "fp64")   # checked before any device work
    assert e.value.status == ed.ED_ERR_INVALID
    assert "limit" in str(e.value)
