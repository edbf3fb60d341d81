"""The allocation-free reduction entry point against the allocating one.

mlbm_reduce_fields_device_noalloc serves callers that cannot allocate device
memory (fixed memory budgets, foreign memory pools, allocation-free hot
loops): its partial sums live in the library's static device array.  Calls in
a row on different data must each match mlbm_reduce_fields_device, called
through the C ABI with a caller-provided scratch buffer: with and without a
mask, above the 1024-block cap of the first pass (so its grid-stride loop
runs), and for n = 0 (all sums zero).  A later call must leave the device's
free memory unchanged.  This file is collected last so that a failure here
does not hide any other test.
"""
import numpy as np
import pytest

from paper_2312_14789_gb300 import mlbm

pytestmark = pytest.mark.gpu


def _call_both(torch, n, seed, with_mask):
    rng = np.random.default_rng(seed)
    h = {k: rng.uniform(0.5, 1.5, n).astype(np.float32) for k in ("rho", "ux", "uy", "area")}
    d = {k: torch.from_numpy(v).cuda() for k, v in h.items()}
    dm = torch.from_numpy((rng.uniform(size=n) > 0.2).astype(np.uint8)).cuda() if with_mask else None
    ns = mlbm.reduce_scratch_doubles(n)
    scratch = torch.empty(max(ns, 1), dtype=torch.float64, device="cuda")
    out_ref = torch.empty(6, dtype=torch.float64, device="cuda")
    out_new = torch.full((6,), float("nan"), dtype=torch.float64, device="cuda")
    ptrs = [d[k].data_ptr() for k in ("rho", "ux", "uy", "area")]
    mp = dm.data_ptr() if dm is not None else None
    mlbm.reduce_fields_device(*ptrs, mp, n, scratch.data_ptr(), ns, out_ref.data_ptr(), 0)
    mlbm.reduce_fields_device_noalloc(*ptrs, mp, n, out_new.data_ptr(), 0)
    torch.cuda.synchronize()
    return out_ref.cpu().numpy(), out_new.cpu().numpy(), (ptrs, mp, out_new)


def test_noalloc_reduction_matches_scratch_reduction_on_calls_in_a_row():
    torch = pytest.importorskip("torch")
    assert mlbm.lib().mlbm_reduce_noalloc_max_nodes() == 2 ** 31 - 1
    cases = [(1_000_003, True), (4097, True), (3_000_017, True), (2_500_000, False), (0, True), (0, False),
             (1, False)]
    for call, (n, with_mask) in enumerate(cases):
        a, b, _ = _call_both(torch, n, call, with_mask)
        assert np.all(np.isfinite(b)), (n, b)
        assert np.allclose(b, a, rtol=1e-12, atol=0), (call, n, a, b)
        if n == 0:
            assert np.all(b == 0.0)
    # n above the 1024-block cap of the first pass: the grid-stride loop runs
    assert mlbm.reduce_scratch_doubles(3_000_017) == 6 * 1024
    # a later call allocates nothing on the device
    _, _, (ptrs, mp, out_new) = _call_both(torch, 200_003, 99, True)
    torch.cuda.synchronize()
    free0, total0 = torch.cuda.mem_get_info()
    for _ in range(3):
        mlbm.reduce_fields_device_noalloc(*ptrs, mp, 200_003, out_new.data_ptr(), 0)
    torch.cuda.synchronize()
    free1, total1 = torch.cuda.mem_get_info()
    assert (free1, total1) == (free0, total0)
    with pytest.raises(mlbm.MlbmError) as e:
        mlbm.reduce_fields_device_noalloc(*ptrs, 0, 2 ** 31, out_new.data_ptr(), 0)
    assert e.value.status == 1
