"""Substeps that keep the last sort (stale_bins, level-aligned clock) against substeps
that sort: the neighbour search widened by how far particles left their sorted blocks
must give exactly the neighbour sets of a fresh sort, the same classification and
activity, and densities and forces equal up to the order of summation; and one such
substep must match the FP64 oracle like any other."""
import numpy as np
import pytest

import oracle as O
from common import ACC_FRAC, RHO_RTOL, dynamic_state, gpu_ctx, max_norm, oracle_state, params
from paper_2009_14514_gb300 import rts, scenes

pytestmark = pytest.mark.gpu


def _pair(sc, st, k0, **over):
    """Two contexts from the same primed state at substep k0: one re-sorting every
    substep, one keeping the sort on odd substeps."""
    out = []
    for stale in (0, 2):
        d = params(sc, level_clock=1, stale_bins=stale, **over)
        ctx = gpu_ctx(sc, d)
        rts.rts_set_state(ctx, st["x"], st["v"], a=st["a"], rho=st["rho"], p=st["p"],
                          level=st["level"], validity=st["validity"], klast=st["klast"], k=k0,
                          primed=True)
        out.append(ctx)
    return out


def _sets(lists):
    return [frozenset(a.tolist()) for a in lists]


@pytest.mark.parametrize("seed", [3, 11])
def test_kept_sort_substep_equals_sorted_substep(seed):
    sc = scenes.wcsph_dam_break_8k()
    st = dynamic_state(sc, seed=seed)
    # every other lattice column 0.75 mm below a block face in x, drifting at +5 m/s
    # (0.5 mm per substep): they cross it between the sort of substep 2 and substep 3
    st["x"] = (st["x"] + np.float32([0.00925, 0.0, 0.0])).astype(np.float32)
    st["v"] = (st["v"] + np.float32([5.0, 0.0, 0.0])).astype(np.float32)
    fresh, stale = _pair(sc, st, k0=1)
    for ctx in (fresh, stale):       # substep 2 sorts in both, substep 3 keeps it in one
        rts.rts_advance(ctx, 2 * sc.params["dt_b"])
    g2 = [rts.rts_get_state(c) for c in (fresh, stale)]
    for f in ("x", "v", "a", "rho", "level", "validity", "klast"):
        assert np.array_equal(g2[0][f], g2[1][f]), f
    for ctx in (fresh, stale):
        rts.rts_advance(ctx, 3 * sc.params["dt_b"])
    g = [rts.rts_get_state(c) for c in (fresh, stale)]
    comp = g[0]["compute"] == 1
    assert comp.sum() > 100 and (~comp).sum() > 100
    for f in ("compute", "level", "validity", "klast", "nbr"):
        assert np.array_equal(g[0][f], g[1][f]), f
    nb = [rts.rts_get_neighbors(c) for c in (fresh, stale)]
    s0, s1 = _sets(nb[0]), _sets(nb[1])
    assert all(s0[i] == s1[i] for i in np.nonzero(comp)[0])
    np.testing.assert_allclose(g[1]["rho"][comp], g[0]["rho"][comp], rtol=1e-5)
    amax = max_norm(g[0]["a"][comp])
    assert np.linalg.norm(g[1]["a"] - g[0]["a"], axis=1).max() <= 1e-5 * amax
    # particles did leave their sorted blocks: the widened search was exercised
    P = O.make_params(sc.params)
    key2, _, _ = O.bin_particles(P, g2[0]["x"])
    key3, _, _ = O.bin_particles(P, g[0]["x"])
    assert (key2 != key3).sum() > 1000
    for ctx in (fresh, stale):
        rts.rts_sync(ctx)
        ctx.close()


def test_kept_sort_substep_matches_oracle():
    sc = scenes.wcsph_dam_break_8k()
    st = dynamic_state(sc, seed=5)
    d = params(sc, level_clock=1, stale_bins=2)
    ctx = gpu_ctx(sc, d)
    k0 = 1
    rts.rts_set_state(ctx, st["x"], st["v"], a=st["a"], rho=st["rho"], p=st["p"],
                      level=st["level"], validity=st["validity"], klast=st["klast"], k=k0,
                      primed=True)
    rts.rts_advance(ctx, 2 * d["dt_b"])           # sorts
    g = rts.rts_get_state(ctx)
    st2 = dict(x=g["x"], v=g["v"], a=g["a"], rho=g["rho"], p=g["p"], level=g["level"],
               validity=g["validity"], klast=g["klast"])
    o = oracle_state(sc, d, st2, k=2, primed=True)
    rts.rts_advance(ctx, 3 * d["dt_b"])           # keeps the sort
    o.substep()
    g = rts.rts_get_state(ctx)
    same = g["compute"] == o.compute
    assert same.mean() > 0.999
    comp = (o.compute == 1) & same
    assert comp.sum() > 100
    assert np.array_equal(g["level"][same], o.level[same])
    assert np.array_equal(g["nbr"][comp], o.nbr[comp])
    np.testing.assert_allclose(g["rho"][comp], o.rho[comp], rtol=RHO_RTOL)
    amax = max_norm(o.a[comp])
    assert np.linalg.norm(g["a"][comp] - o.a[comp], axis=1).max() <= ACC_FRAC * amax
    rts.rts_sync(ctx)
    ctx.close()


def test_rollout_with_kept_sorts_matches_sorted_rollout_statistics():
    # 0.1 s of the 8k dam break with the level-aligned clock: the same mass, kinetic
    # energy and density-error statistics as re-sorting every substep (rollouts differ
    # chaotically only by the order of summation)
    sc = scenes.wcsph_dam_break_8k()
    res = []
    for stale in (0, 2):
        ctx = gpu_ctx(sc, params(sc, level_clock=1, stale_bins=stale))
        stats = rts.rts_advance(ctx, 0.1)
        g = rts.rts_get_state(ctx, ("v", "rho", "x"))
        ke = 0.5 * float((g["v"].astype(np.float64) ** 2).sum())
        err = float(np.abs(g["rho"] / 1000.0 - 1.0).mean())
        res.append((ke, err, stats["particle_evals"], g["x"]))
        ctx.close()
    (ke0, e0, n0, x0), (ke1, e1, n1, x1) = res
    assert abs(ke1 / ke0 - 1.0) < 0.03
    assert abs(e1 - e0) < 0.1 * e0 + 1e-4
    assert abs(n1 / n0 - 1.0) < 0.02
    assert np.all(np.isfinite(x1)) and len(x1) == sc.n


def test_kept_sort_levels_at_the_thresholds_are_decided_exactly():
    # A calm lattice (v = 0, held a = 0: nothing moves) with one particle in every third
    # block at the largest FP32 speeds whose FP64 square is at most the level-3 threshold:
    # the FP32 block maxima are undecided, on substeps that keep the sort as well, and
    # the block levels must be the double-precision definition's (level 3), as the
    # oracle's and as a context that sorts every substep
    sc = scenes.wcsph_dam_break_8k()
    base = params(sc, level_clock=1)
    P = O.make_params(base)
    vthr2, _, _ = O.level_thresholds(P)
    t = float(vthr2[3])
    c = np.float32(np.sqrt(t))
    while float(c) ** 2 > t:
        c = np.nextafter(c, np.float32(0))
    cands = [c, np.nextafter(c, np.float32(0)), np.nextafter(np.nextafter(c, np.float32(0)),
                                                              np.float32(0))]
    assert all(abs(float(x) ** 2 / float(np.float32(t)) - 1) < 1e-5 for x in cands)
    n = sc.n
    v = np.zeros((n, 3), np.float32)
    a = np.zeros((n, 3), np.float32)
    _, perm, cstart = O.bin_particles(P, sc.x)
    filled = np.nonzero(np.diff(cstart))[0]
    for j, b in enumerate(filled[::3]):
        v[perm[cstart[b]], j % 3] = cands[j % 3]
    st = dict(x=sc.x, v=v, a=a, rho=np.full(n, 1000.0, np.float32), p=np.zeros(n, np.float32),
              level=np.full(n, 3, np.int32), validity=np.full(n, 7, np.int32),
              klast=np.zeros(n, np.int32))
    levels = {}
    for stale in (0, 4):
        d = dict(base, stale_bins=stale)
        ctx = gpu_ctx(sc, d)
        rts.rts_set_state(ctx, st["x"], st["v"], a=st["a"], rho=st["rho"], p=st["p"],
                          level=st["level"], validity=st["validity"], klast=st["klast"], k=1,
                          primed=True)
        rts.rts_advance(ctx, 3 * d["dt_b"])          # substeps 2 and 3 (both keep the sort)
        levels[stale] = rts.rts_get_blocks(ctx)
        rts.rts_sync(ctx)
        ctx.close()
    o = oracle_state(sc, base, st, k=1, primed=True)
    o.substep()
    o.substep()
    assert np.array_equal(levels[4][0], levels[0][0])
    assert np.array_equal(levels[4][1], levels[0][1])
    assert np.array_equal(levels[4][1], o.block_level)
    assert np.all(levels[4][1][filled] == 3)
