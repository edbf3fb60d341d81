"""The allocation-free reduction entry point against the allocating one.

mlbm_reduce_fields_device_noalloc serves callers that cannot allocate device
memory (fixed memory budgets, foreign memory pools, allocation-free hot
loops): its partial sums live in the library's static device array.  Two
calls in a row on different data must each match mlbm_reduce_fields_device,
called through the C ABI with a caller-provided scratch buffer.  This file is
collected last so that a failure here does not hide any other test.
"""
import numpy as np
import pytest

from paper_2312_14789_gb300 import mlbm

pytestmark = pytest.mark.gpu


def test_noalloc_reduction_matches_scratch_reduction_on_two_calls():
    torch = pytest.importorskip("torch")
    assert mlbm.lib().mlbm_reduce_noalloc_max_nodes() == 2 ** 31 - 1
    for call, n in enumerate((1_000_003, 4097)):
        rng = np.random.default_rng(call)
        h = {k: rng.uniform(0.5, 1.5, n).astype(np.float32) for k in ("rho", "ux", "uy", "area")}
        mask = (rng.uniform(size=n) > 0.2).astype(np.uint8)
        d = {k: torch.from_numpy(v).cuda() for k, v in h.items()}
        dm = torch.from_numpy(mask).cuda()
        ns = mlbm.reduce_scratch_doubles(n)
        scratch = torch.empty(ns, dtype=torch.float64, device="cuda")
        out_ref = torch.empty(6, dtype=torch.float64, device="cuda")
        out_new = torch.full((6,), float("nan"), dtype=torch.float64, device="cuda")
        ptrs = [d[k].data_ptr() for k in ("rho", "ux", "uy", "area")]
        mlbm.reduce_fields_device(*ptrs, dm.data_ptr(), n, scratch.data_ptr(), ns, out_ref.data_ptr(), 0)
        mlbm.reduce_fields_device_noalloc(*ptrs, dm.data_ptr(), n, out_new.data_ptr(), 0)
        torch.cuda.synchronize()
        a, b = out_ref.cpu().numpy(), out_new.cpu().numpy()
        assert np.all(np.isfinite(b))
        assert np.allclose(b, a, rtol=1e-12, atol=0), (call, a, b)
    with pytest.raises(mlbm.MlbmError) as e:
        mlbm.reduce_fields_device_noalloc(*ptrs, 0, 2 ** 31, out_new.data_ptr(), 0)
    assert e.value.status == 1
