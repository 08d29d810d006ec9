"""rts_bin_noalloc, the binning entry point for callers that cannot allocate device
memory (its working memory is a fixed array inside the library), must give exactly what
the oracle's binning gives, call after call: the array is shared and reused, so a second
call on other positions must not see the first call's counters, and a call that failed
(a particle outside the grid) must leave nothing behind for the next one.

This file sorts last so that a run stopping at the first failure has already run every
other test."""
import numpy as np
import pytest

import oracle as O
from paper_2009_14514_gb300 import rts, scenes

pytestmark = pytest.mark.gpu


def _reference_bins(sc, x):
    ctx = rts.rts_init(sc.params, x, np.zeros_like(x), sc.xb)
    rts.rts_bin(ctx)
    out = rts.rts_get_bins(ctx)
    ctx.close()
    return out


def _noalloc(sc, x):
    import torch
    P = rts.make_params(sc.params)
    nblocks = int(np.prod(sc.params["grid_dim"]))
    n = x.shape[0]
    xd = torch.from_numpy(np.ascontiguousarray(x, np.float32)).cuda()
    key = torch.full((max(n, 1),), -1, dtype=torch.int32, device="cuda")
    perm = torch.full((max(n, 1),), -1, dtype=torch.int32, device="cuda")
    cstart = torch.full((nblocks + 1,), -1, dtype=torch.int32, device="cuda")
    rts.rts_bin_noalloc(P, xd, key, perm, cstart)
    torch.cuda.synchronize()
    return key.cpu().numpy()[:n], perm.cpu().numpy()[:n], cstart.cpu().numpy()


def _dyadic_on_faces():
    # spacing 1/64, edge 1/32: half the particles sit exactly on block faces
    sc = scenes.dam_break((12, 10, 9), 1.0 / 64, (0.5, 0.25, 0.25), 1e-4)
    return sc, (sc.x - np.float32(0.5 / 64)).astype(np.float32)


def test_noalloc_binning_equals_rts_bin_on_two_calls_in_a_row():
    sc = scenes.wcsph_dam_break_8k()
    rng = np.random.default_rng(31)
    shifted = (sc.x + rng.uniform(-0.01, 0.01, sc.x.shape)).astype(np.float32)
    for x in (sc.x, shifted[: sc.n - 77]):      # second call: other positions, fewer particles
        key_ref, perm_ref, cs_ref = _reference_bins(sc, x)
        key, perm, cstart = _noalloc(sc, x)
        assert np.array_equal(key, key_ref)
        assert np.array_equal(perm, perm_ref)
        assert np.array_equal(cstart, cs_ref)


@pytest.mark.parametrize("case", ["jittered_8k", "dyadic_on_block_faces"])
def test_noalloc_binning_equals_the_oracle(case):
    if case == "jittered_8k":
        sc = scenes.wcsph_dam_break_8k()
        x = sc.x
    else:
        sc, x = _dyadic_on_faces()
    okey, operm, ocs = O.bin_particles(O.make_params(sc.params), x)
    for _ in range(2):                          # the second call reuses the working memory
        key, perm, cstart = _noalloc(sc, x)
        assert np.array_equal(key, okey)
        assert np.array_equal(perm, operm)
        assert np.array_equal(cstart, ocs)


def test_noalloc_binning_reports_a_particle_outside_the_grid_then_recovers():
    sc = scenes.wcsph_dam_break_8k()
    bad = sc.x.copy()
    bad[123, 0] = -1.0                          # left of the grid's origin
    with pytest.raises(rts.RtsError) as e:
        _noalloc(sc, bad)
    assert e.value.status == rts.RTS_ERR_DOMAIN
    okey, operm, ocs = O.bin_particles(O.make_params(sc.params), sc.x)
    key, perm, cstart = _noalloc(sc, sc.x)      # clean status and counters
    assert np.array_equal(key, okey)
    assert np.array_equal(perm, operm)
    assert np.array_equal(cstart, ocs)


def test_noalloc_binning_of_no_particles_gives_empty_blocks():
    sc = scenes.wcsph_dam_break_8k()
    _noalloc(sc, sc.x)                          # leave counts behind in the working memory
    key, perm, cstart = _noalloc(sc, np.zeros((0, 3), np.float32))
    assert len(key) == 0 and np.all(cstart == 0)


def test_noalloc_binning_rejects_an_overfull_block():
    # 5,000 particles in one block: more than RTS_NOALLOC_MAX_PER_BLOCK (the in-block
    # ordering scans the block, so its cost is bounded by refusing such blocks)
    sc = scenes.wcsph_dam_break_8k()
    rng = np.random.default_rng(5)
    edge = sc.params["block_edge"]
    lo = np.asarray(sc.params["domain_min"]) + 3 * edge      # the corner of block (3, 3, 3)
    x = (lo + rng.uniform(0.1 * edge, 0.9 * edge, (5000, 3))).astype(np.float32)
    with pytest.raises(rts.RtsError) as e:
        _noalloc(sc, x)
    assert e.value.status == rts.RTS_ERR_CAPACITY
    key, perm, cstart = _noalloc(sc, sc.x)
    assert np.array_equal(perm, O.bin_particles(O.make_params(sc.params), sc.x)[1])


def test_noalloc_binning_rejects_sizes_beyond_its_fixed_memory():
    import torch
    sc = scenes.wcsph_dam_break_8k()
    d = dict(sc.params)
    d["grid_dim"] = [1000, 1000, 1]                    # 1M blocks: more than the fixed memory
    x = torch.zeros((8, 3), dtype=torch.float32, device="cuda")
    key = torch.zeros(8, dtype=torch.int32, device="cuda")
    with pytest.raises(rts.RtsError) as e:
        rts.rts_bin_noalloc(d, x, key, key.clone(),
                            torch.zeros(1000 * 1000 + 1, dtype=torch.int32, device="cuda"))
    assert e.value.status == rts.RTS_ERR_ARG
    assert "RTS_NOALLOC_MAX" in str(e.value)
