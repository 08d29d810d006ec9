"""rts_bin_noalloc, the binning entry point for callers that cannot allocate device
memory (its working memory is a fixed array inside the library), must give exactly what
rts_bin + rts_get_bins give, call after call: the array is shared and reused, so a
second call on other positions must not see the first call's counters.

This file sorts last so that a run stopping at the first failure has already run every
other test."""
import numpy as np
import pytest

from paper_2009_14514_gb300 import rts, scenes

pytestmark = pytest.mark.gpu


def _reference_bins(sc, x):
    ctx = rts.rts_init(sc.params, x, np.zeros_like(x), sc.xb)
    rts.rts_bin(ctx)
    out = rts.rts_get_bins(ctx)
    ctx.close()
    return out


def test_noalloc_binning_equals_rts_bin_on_two_calls_in_a_row():
    import torch
    sc = scenes.wcsph_dam_break_8k()
    P = rts.make_params(sc.params)
    nblocks = int(np.prod(sc.params["grid_dim"]))
    rng = np.random.default_rng(31)
    shifted = (sc.x + rng.uniform(-0.01, 0.01, sc.x.shape)).astype(np.float32)
    inputs = [sc.x, shifted[: sc.n - 77]]            # second call: other positions, fewer particles
    for x in inputs:
        n = x.shape[0]
        key_ref, perm_ref, cs_ref = _reference_bins(sc, x)
        xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
        key = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        perm = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        cstart = torch.full((nblocks + 1,), -1, dtype=torch.int32, device="cuda")
        rts.rts_bin_noalloc(P, xd, key, perm, cstart)
        torch.cuda.synchronize()
        assert np.array_equal(key.cpu().numpy(), key_ref)
        assert np.array_equal(perm.cpu().numpy(), perm_ref)
        assert np.array_equal(cstart.cpu().numpy(), cs_ref)


def test_noalloc_binning_rejects_sizes_beyond_its_fixed_memory():
    import torch
    sc = scenes.wcsph_dam_break_8k()
    d = dict(sc.params)
    d["grid_dim"] = [1000, 1000, 1]                    # 1M blocks: more than the fixed memory
    x = torch.zeros((8, 3), dtype=torch.float32, device="cuda")
    key = torch.zeros(8, dtype=torch.int32, device="cuda")
    with pytest.raises(rts.RtsError) as e:
        rts.rts_bin_noalloc(d, x, key, key.clone(), torch.zeros(16, dtype=torch.int32, device="cuda"))
    assert e.value.status == 1
    assert "RTS_NOALLOC_MAX" in str(e.value)
