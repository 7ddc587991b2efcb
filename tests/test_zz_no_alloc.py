"""mpw_step_periodic_noalloc: the allocation-free entry point.

Some callers cannot allocate device memory when they advance a field (a
plugin whose host application owns every device allocation, a timing-critical
loop that must stay out of the driver's allocator).  This entry point steps a
single periodic patch with all work buffers in a fixed device array inside the
library.  Here it is called through the C ABI and compared with the ordinary
context path (mpw_step on the same periodic patch), on two calls in a row,
at the parity tolerance of the other GPU tests.  The file name makes pytest
collect it last.
"""
import numpy as np
import pytest

from paper_2002_00088_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n", [(40, 24, 20), (48, 48, 48), (6, 7, 8)],
                         ids=["ragged", "largest", "smallest"])
def test_noalloc_step_matches_context_step_twice(mpw_lib, n):
    """(48, 48, 48) fills the fixed work array exactly; (6, 7, 8) is the
    smallest patch the entry point accepts."""
    import torch
    M = mpw_lib
    lo, hi = (-0.5, -0.3, -0.2), (0.5, 0.4, 0.3)
    ps, pi = wl.random_fields((n[2], n[1], n[0]), 7)
    h = min((hi[a] - lo[a]) / n[a] for a in range(3))
    dt = 0.1 * h
    ctx = M.Multipatch(6, 0.005)
    ctx.create_patch(M.PATCH_GLOBAL, n, lo, hi, M.BC_PERIODIC)
    ctx.set_fields(0, ps, pi)
    d_ps = torch.tensor(ps, dtype=torch.float64, device="cuda")
    d_pi = torch.tensor(pi, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    for call in range(2):
        ctx.step(dt, 3)
        M.step_periodic_noalloc(n, lo, hi, 0.005, dt, 3, d_ps, d_pi, stream)
        torch.cuda.synchronize()
        want = ctx.get_fields(0)
        got = (d_ps.cpu().numpy(), d_pi.cpu().numpy())
        for a, b in zip(got, want):
            assert np.isfinite(a).all()
            assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max(), f"call {call}"


def test_noalloc_rejects_oversize_patch(mpw_lib):
    import torch
    M = mpw_lib
    n = (M.NOALLOC_MAX_N + 1, 8, 8)
    d = torch.zeros((8, 8, n[0]), dtype=torch.float64, device="cuda")
    with pytest.raises(M.MpwError) as e:
        M.step_periodic_noalloc(n, (0, 0, 0), (1, 1, 1), 0.005, 1e-3, 1, d, d.clone())
    assert e.value.status == 1 and "48" in str(e.value)
