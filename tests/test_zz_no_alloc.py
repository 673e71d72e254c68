"""vlbm_totals_static: the conservation totals for callers that cannot
allocate device memory (an application that reserves its GPU memory up front
and forbids later allocations, or one that only holds raw device pointers to
its populations).  Checked against vlbm_audit on the same state, on two calls
in a row; this file is collected last so that a failure here comes after
every other test has run."""
import ctypes

import numpy as np
import pytest

from paper_2609_35529_b300 import inputs as I

pytestmark = pytest.mark.gpu


def test_totals_static_matches_audit_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_35529_b300 import build, vlbm as V
    build.build()
    # a single-level periodic grid: every cell is active, area weight 1
    nx, ny = 200, 136
    cs = I.smooth_random(nx, ny, 1, [], seed=77, amp=0.2, beta=0.9, steps=5)
    h = V.Hierarchy.from_case(cs)
    h.advance(cs.steps)
    ref_tot, ref_abs = h.audit()
    ld = 208
    f = torch.zeros((16, ny, ld), dtype=torch.float64, device="cuda")
    st = V.lib().vlbm_get_populations(h.handle, 0, ctypes.c_void_p(f.data_ptr()), ld, 1)
    assert st == 0
    stream = torch.cuda.current_stream()
    bufs = [torch.full((8,), float("nan"), dtype=torch.float64, device="cuda") for _ in range(2)]
    outs, free = [], []
    for out in bufs:
        V.totals_static(f.data_ptr(), ld, nx, ny, 1.0, out.data_ptr(), stream)
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        outs.append(out.cpu().numpy())
    # the first call loads the module (code and scratch array); the second
    # takes no device memory at all
    assert free[1] == free[0]
    for o in outs:
        np.testing.assert_allclose(o[:4], ref_tot, rtol=1e-14, atol=1e-14 * np.max(ref_abs))
        np.testing.assert_allclose(o[4:], ref_abs, rtol=1e-14)
    assert np.array_equal(outs[0], outs[1])
    h.close()


def test_totals_static_rejects_oversized_grid():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_35529_b300 import vlbm as V
    dummy = torch.zeros(8, dtype=torch.float64, device="cuda")
    # 16384 slots x 4096 cells is the limit; one more row of 8192 cells is over it
    with pytest.raises(V.VlbmError) as ei:
        V.totals_static(dummy.data_ptr(), 8192, 8192, 8193, 1.0, dummy.data_ptr())
    assert ei.value.name == "ERR_ARG"
