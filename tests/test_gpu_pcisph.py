"""GPU parity of RTS-PCISPH (Algorithms 2 and 3) against the FP64 oracle.

Same seeded input state on both sides.  Regions and neighbour sets at a major-step start:
bit-exact.  Iteration counts and the local / global decisions: equal (the inputs keep
every decision away from its threshold).  Predicted density 1e-4 relative; pressure
accelerations 1e-3 of the max-norm; positions and velocities within what those bounds
allow after one minor step.
"""
import numpy as np
import pytest

import oracle as O
from common import ACC_FRAC, RHO_RTOL, max_norm
from paper_2009_14514_gb300 import rts, scenes

pytestmark = pytest.mark.gpu


def _pair(sc, x=None, v=None, a=None, **over):
    d = dict(sc.params)
    d.update(over)
    x = sc.x if x is None else x
    v = sc.v if v is None else v
    ctx = rts.rts_init(d, x, v, sc.xb)
    if a is not None:
        rts.rts_set_state(ctx, x, v, a=a)
    P = O.make_params(d)
    S = O.PCISPH(P, x, v, sc.xb)
    if a is not None:
        S.anp[:] = a
    return ctx, S, P


def _dynamic(sc, seed=11, vscale=1.0, ascale=1.0):
    st = scenes.perturbed_state(sc, seed, vmax=3.0 * vscale, amax=2.0e3 * ascale)
    return st["v"], st["a"]


def test_regions_and_neighbourhoods_at_a_major_step_start():
    sc = scenes.pcisph_drop_small()
    v, a = _dynamic(sc, vscale=5.0, ascale=10.0)     # spans all four regions
    # one minor step per major step (no pre-emption yet); no expansion, which would cover
    # this small domain with region 1 (the expansion is pinned on the oracle)
    ctx, S, P = _pair(sc, v=v, a=a, n_minor=1, expand_layers=0)
    x0 = S.x.copy()
    rts.rts_pcisph_step(ctx)
    S.step()
    raw, lev = rts.rts_get_blocks(ctx)
    assert np.array_equal(lev, S.block_level)
    assert len(set(S.block_level[S.block_level >= 0].tolist())) == 4
    g = rts.rts_get_state(ctx, ("level",))
    assert np.array_equal(g["level"], S.level)
    lists = rts.rts_get_neighbors(ctx)
    for i in range(sc.n):
        assert set(lists[i].tolist()) == set(S.neighbors(i).tolist()), i
    # the region-1 particles searched two rings: their lists are still exact sets
    off, idx = O.neighbors_brute(x0, sc.xb, P.r)
    r1 = np.nonzero(S.level == 0)[0]
    assert len(r1) > 0
    for i in r1[:50]:
        assert set(lists[i].tolist()) == set(idx[off[i]:off[i + 1]].tolist())


def _compare_step(ctx, S, P, comp_rtol=RHO_RTOL):
    info = rts.rts_pcisph_last(ctx)
    assert info["iterations"] == S.stats["iters"]
    assert info["local_iterations"] == S.stats["local_iters"]
    assert info["reverts"] == S.stats["reverts"]
    assert info["global_iterations"] == S.stats["global_iters"]
    g = rts.rts_get_state(ctx, ("x", "v", "rho", "p", "level", "validity"))
    ps = rts.rts_get_pcisph_state(ctx)
    np.testing.assert_allclose(g["rho"], S.rho, rtol=comp_rtol)
    tol_a = ACC_FRAC * max(max_norm(S.ap), 1e-6)
    assert np.linalg.norm(ps["ap"] - S.ap, axis=1).max() <= tol_a
    dt = P.dt_b
    assert np.abs(g["v"] - S.v).max() <= tol_a * dt + 1e-5 * max(1.0, np.abs(S.v).max())
    assert np.abs(g["x"] - S.x).max() <= tol_a * dt * dt + 2e-6
    assert np.array_equal(g["validity"], S.validity)
    return info


def test_one_minor_step_matches_oracle():
    sc = scenes.pcisph_drop_small()
    v, a = _dynamic(sc, seed=3)
    ctx, S, P = _pair(sc, v=v, a=a)
    for _ in range(3):
        rts.rts_pcisph_step(ctx)
        S.step()
        _compare_step(ctx, S, P)


def test_rest_lattice_stays_at_rest_on_gpu():
    s = 1.0 / 64
    sc = scenes.pool_drop((8, 7, 6), 0, 0.0, s, (8 * s, 7 * s, 6 * s), 3.5e-4)
    d = dict(sc.params)
    d["gravity"] = [0.0, 0.0, 0.0]
    ctx = rts.rts_init(d, sc.x, sc.v, sc.xb)
    for _ in range(6):
        rts.rts_pcisph_step(ctx)
        assert rts.rts_pcisph_last(ctx)["iterations"] == 3
    g = rts.rts_get_state(ctx, ("x", "v", "p"))
    assert np.array_equal(g["x"], sc.x) and np.all(g["v"] == 0) and np.all(g["p"] == 0)


def _compressed(sc):
    x = sc.x.copy()
    rng = np.random.default_rng(3)
    pick = rng.choice(sc.n, 40, replace=False)
    x[pick] += rng.uniform(-0.004, 0.004, (40, 3)).astype(np.float32)
    return x


@pytest.mark.parametrize("over", [
    dict(eta=0.002, eta_T=0.5),                                  # extra local iterations
    dict(eta=0.002, eta_T=0.0),                                  # extra global iterations
    dict(eta=1e-9, eta_T=0.5, max_local_iters=2, max_iters=12),  # local failure and revert
])
def test_iteration_control_decisions_match_oracle(over):
    sc = scenes.pcisph_drop_small()
    x = _compressed(sc)
    ctx, S, P = _pair(sc, x=x, **over)
    rts.rts_pcisph_step(ctx, allow_not_converged=True)
    S.step()
    info = rts.rts_pcisph_last(ctx)
    assert info["iterations"] == S.stats["iters"] > 3
    assert info["local_iterations"] == S.stats["local_iters"]
    assert info["reverts"] == S.stats["reverts"]
    assert info["not_converged"] == S.stats["not_converged"]


def test_state_after_local_iterations_matches_oracle():
    # local iterations take S_e and R_ob only (R_ob formed just before each of them): the
    # state after the minor step, not only the counts, follows the oracle
    sc = scenes.pcisph_drop_small()
    x = _compressed(sc)
    ctx, S, P = _pair(sc, x=x, eta=0.002, eta_T=0.5)
    rts.rts_pcisph_step(ctx, allow_not_converged=True)
    S.step()
    info = _compare_step(ctx, S, P)
    assert info["local_iterations"] > 0


def test_major_step_shortening_matches_oracle():
    sc = scenes.pcisph_drop_small()
    ctx, S, P = _pair(sc, max_global_iters=1, clean_majors=2)
    for _ in range(3):
        rts.rts_pcisph_step(ctx)
        S.step()
        info = rts.rts_pcisph_last(ctx)
        assert info["minor"] == S.S.minor and info["n_minor_current"] == S.S.n_minor_cur


def test_rollout_statistics_match_oracle():
    # the cube falls into the pool: 120 minor steps, compare mass, kinetic energy,
    # density-error statistics and the iteration budget
    sc = scenes.pcisph_drop_small()
    ctx, S, P = _pair(sc)
    stats = rts.rts_advance(ctx, 120 * P.dt_b)
    its = 0
    for _ in range(120):
        S.step()
        its += S.stats["iters"]
    g = rts.rts_get_state(ctx, ("v", "rho", "level"))
    assert stats["substeps"] == 120
    ke_g, ke_o = (g["v"].astype(np.float64) ** 2).sum(), (S.v ** 2).sum()
    assert abs(ke_g / ke_o - 1) < 0.05
    assert abs(stats["pcisph_iterations"] / its - 1) < 0.1
    ps = rts.rts_get_pcisph_state(ctx)
    assert ps["err"].max() <= P.eta * 1.5 and S.err.max() <= P.eta * 1.5
    assert abs(np.bincount(g["level"], minlength=4) - np.bincount(S.level, minlength=4)).sum() < 0.05 * sc.n


def test_full_size_pool_drop_runs_one_major_step():
    sc = scenes.pcisph_drop_1m()
    ctx = rts.rts_init(sc.params, sc.x, sc.v, sc.xb)
    s = rts.rts_advance(ctx, 4 * sc.params["dt_b"])
    assert s["substeps"] == 4 and s["pcisph_iterations"] >= 12
    info = rts.rts_pcisph_last(ctx)
    assert info["err_max"] <= sc.params["eta"]
    g = rts.rts_get_state(ctx, ("x",))
    assert np.isfinite(g["x"]).all()
    # sampled neighbourhoods of the last refresh against brute force in the oracle
    lists = rts.rts_get_neighbors(ctx)
    rng = np.random.default_rng(2)
    P = O.make_params(sc.params)
    assert max(len(l) for l in lists) <= P.max_neighbors
    assert np.mean([len(lists[i]) for i in rng.choice(sc.n, 1000, replace=False)]) > 15


@pytest.mark.parametrize("mode", [1, 2])
def test_global_comparators_match_oracle(mode):
    sc = scenes.pcisph_drop_small()
    ctx, S, P = _pair(sc, mode=mode)
    for _ in range(3):
        k0 = ctx.substep_index
        rts.rts_pcisph_step(ctx)
        m = S.global_step()
        assert ctx.substep_index - k0 == m == (1 if mode == 2 else m)
        assert rts.rts_pcisph_last(ctx)["iterations"] == S.S.iters
    g = rts.rts_get_state(ctx, ("x", "v", "rho"))
    np.testing.assert_allclose(g["rho"], S.rho, rtol=RHO_RTOL)
    assert np.abs(g["x"] - S.x).max() < 2e-5


def test_region_expansion_matches_oracle():
    # a resting pool with two fast spots: one needs region 1, the other region 2; the
    # regions grow by expand_layers = 4 blocks around them (Section 5.5) on a domain large
    # enough that a quarter of the blocks stay in region 4
    sc = scenes.pool_drop((48, 48, 6), 4, 0.03, 0.01, (0.48, 0.48, 0.16), 3.5e-4)
    v = np.zeros_like(sc.x)
    for c, speed, rad in (((0.10, 0.12, 0.03), 15.0, 0.012), ((0.36, 0.30, 0.03), 3.0, 0.02)):
        m = np.linalg.norm(sc.x - np.asarray(c, np.float32), axis=1) < rad
        v[m] = (speed, 0.0, 0.0)
    a = np.zeros_like(sc.x)
    ctx, S, P = _pair(sc, v=v, a=a, n_minor=1)
    rts.rts_pcisph_step(ctx)
    S.step()
    _, lev = rts.rts_get_blocks(ctx)
    assert np.array_equal(lev, S.block_level)
    filled = S.block_level[S.block_level >= 0]
    assert set(np.unique(filled).tolist()) == {0, 1, 3}
    assert (filled == 3).sum() > 100 and (filled == 0).sum() > 100
    g = rts.rts_get_state(ctx, ("level",))
    assert np.array_equal(g["level"], S.level)


def test_region2_two_ring_ablation_matches_oracle():
    # r2_search_rings = 2: region-2 particles search two rings (the paper: region 1 only);
    # over a major step of 4 minor steps the refreshed lists, iterations and states match
    sc = scenes.pcisph_drop_small()
    v, a = _dynamic(sc, seed=21, vscale=2.0, ascale=2.0)
    ctx, S, P = _pair(sc, v=v, a=a, r2_search_rings=2)
    for _ in range(4):
        rts.rts_pcisph_step(ctx)
        S.step()
        _compare_step(ctx, S, P)
        lists = rts.rts_get_neighbors(ctx)
        r2 = np.nonzero(S.level == 1)[0]
        for i in r2[:300]:
            assert set(lists[i].tolist()) == set(S.neighbors(i).tolist()), i
    assert (S.level == 1).sum() > 0
