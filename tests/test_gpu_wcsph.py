"""GPU parity of the WCSPH regional-time-stepping path against the FP64 oracle.

Every test drives the CUDA library through its C ABI and the oracle with the same seeded
input state.  Bins, neighbour counts, block levels, activity flags: bit-exact.  Density:
1e-4 relative.  Accelerations: 1e-3 of the max-norm.  Positions and velocities after a
substep: the consequences of those bounds (plus FP32 rounding of the predictor).
"""
import math

import numpy as np
import pytest

import oracle as O
from common import ACC_FRAC, RHO_RTOL, dynamic_state, gpu_ctx, max_norm, oracle_state, params, ulp32
from paper_2009_14514_gb300 import rts, scenes

pytestmark = pytest.mark.gpu


def _levels_by_particle(P, x, block_levels):
    key, _, _ = O.bin_particles(P, x)
    return block_levels[key]


# ------------------------------------------------------------------- binning ---

@pytest.mark.parametrize("which", ["jittered", "dyadic_on_block_faces", "ragged_37"])
def test_bins_are_bit_exact(which):
    if which == "jittered":
        sc = scenes.wcsph_dam_break_8k()
        x = sc.x
    elif which == "dyadic_on_block_faces":
        # spacing 1/64, edge 1/32: half the particles sit exactly on block faces
        sc = scenes.dam_break((12, 10, 9), 1.0 / 64, (0.5, 0.25, 0.25), 1e-4)
        x = (sc.x - np.float32(0.5 / 64)).astype(np.float32)
    else:
        sc = scenes.dam_break((37, 1, 1), 0.02, (0.8, 0.4, 0.4), 1e-4, jitter=3e-3, seed=4)
        x = sc.x
    P = O.make_params(sc.params)
    ctx = gpu_ctx(sc, x=x)
    rts.rts_bin(ctx)
    key, perm, cstart = rts.rts_get_bins(ctx)
    okey, operm, ocstart = O.bin_particles(P, x)
    assert np.array_equal(key, okey)
    assert np.array_equal(perm, operm)
    assert np.array_equal(cstart, ocstart)


# ------------------------------------------------------------ classification ---

# the third case: speed thresholds that rise from level 1 to level 2 (beta_3 / 4 >
# beta_2 / 2), so the levels a block passes are not a prefix and R_min cannot be taken
# from the union's maxima: every block is decided on its own
@pytest.mark.parametrize("force_level,beta", [(-1, None), (2, None),
                                              (-1, [math.inf, 0.4, 1.6, 0.016])])
def test_block_levels_are_bit_exact(force_level, beta):
    sc = scenes.wcsph_dam_break_8k()
    st = dynamic_state(sc, seed=21)
    d = params(sc, force_level=force_level)
    if beta is not None:
        d["beta"] = beta
    P = O.make_params(d)
    ctx = gpu_ctx(sc, d)
    rts.rts_set_state(ctx, st["x"], st["v"], a=st["a"])
    rts.rts_classify_blocks(ctx)
    raw, lev = rts.rts_get_blocks(ctx)
    oraw, olev = O.classify_wcsph(P, st["x"], st["v"], st["a"])
    assert np.array_equal(raw, oraw)
    assert np.array_equal(lev, olev)
    if force_level < 0 and beta is None:
        assert len(set(oraw[oraw >= 0].tolist())) == 4        # every level occurs


def test_block_levels_at_the_thresholds_are_decided_exactly():
    # one particle per block set to the two FP32 neighbours of an FP64 threshold (|v|^2
    # just below and just above it, the FP32 maximum undecided), the rest at rest: the
    # level must be the double-precision definition's, as the oracle's
    sc = scenes.wcsph_dam_break_8k()
    d = params(sc)
    P = O.make_params(d)
    vthr2, athr2, _ = O.level_thresholds(P)
    key, perm, cstart = O.bin_particles(P, sc.x)
    v = np.zeros((sc.n, 3), np.float32)
    a = np.zeros((sc.n, 3), np.float32)
    a[:, 2] = -9.81
    filled = np.nonzero(np.diff(cstart))[0]
    rng = np.random.default_rng(8)
    for j, b in enumerate(filled):
        i = perm[cstart[b]]
        L = 1 + j % (len(vthr2) - 1)
        if j % 3 == 2:                          # an acceleration threshold instead
            t = np.sqrt(athr2[L])
            c = np.float32(t)
            c = np.nextafter(c, np.float32(np.inf)) if j % 2 else np.nextafter(c, np.float32(0))
            a[i] = [0.0, 0.0, c]
        else:
            t = np.sqrt(vthr2[L])
            c = np.float32(t)
            c = np.nextafter(c, np.float32(np.inf)) if j % 2 else c
            v[i] = [c, 0.0, 0.0]
        assert rng is not None
    ctx = gpu_ctx(sc, d)
    rts.rts_set_state(ctx, sc.x, v, a=a)
    rts.rts_classify_blocks(ctx)
    raw, _ = rts.rts_get_blocks(ctx)
    oraw, _ = O.classify_wcsph(P, sc.x, v, a)
    assert np.array_equal(raw, oraw)
    assert len(set(oraw[filled].tolist())) >= 3


# ----------------------------------------------------------------- evaluation ---

def _near_tie(i, xp, xb, r, rel=1e-5):
    """Particle i has a pair within rel of the support radius in the FP64 state xp."""
    d2 = np.concatenate([((xp - xp[i]) ** 2).sum(1), ((xb - xp[i]) ** 2).sum(1)])
    return bool(np.any(np.abs(d2 / (r * r) - 1.0) < rel))


def _check_eval(g, o, mask=None, xpred=None):
    m = np.ones(len(o.rho), bool) if mask is None else mask
    if xpred is None:
        assert np.array_equal(g["nbr"][m], o.nbr[m])
    else:
        # counts on predicted positions: FP32 and FP64 predictors round differently, so a
        # pair within rounding of r may flip; every other count must agree exactly
        bad = np.nonzero(m & (g["nbr"] != o.nbr))[0]
        xb = o.xb
        assert all(_near_tie(i, xpred, xb, o.P.r) for i in bad), f"{len(bad)} count mismatches"
        assert len(bad) <= 1e-3 * m.sum() + 2
    np.testing.assert_allclose(g["rho"][m], o.rho[m], rtol=RHO_RTOL, atol=0)
    tol = ACC_FRAC * max_norm(o.a[m])
    err = np.linalg.norm(g["a"][m].astype(np.float64) - o.a[m], axis=1)
    assert err.max() <= tol, (err.max(), tol)


@pytest.mark.parametrize("wide", [False, True])
def test_evaluate_density_neighbours_forces_match_oracle(wide):
    # wide: the literal reading h = 2 s, r = 4 s with four boundary layers
    sc = scenes.wcsph_dam_break_8k_wide_kernel() if wide else scenes.wcsph_dam_break_8k()
    st = dynamic_state(sc, seed=5)
    ctx = gpu_ctx(sc)
    rts.rts_set_state(ctx, st["x"], st["v"], a=st["a"], rho=st["rho"], p=st["p"])
    rts.rts_evaluate(ctx)
    g = rts.rts_get_state(ctx)
    o = oracle_state(sc, sc.params, st)
    o.evaluate()
    _check_eval(g, o)
    assert np.array_equal(g["level"], o.level)
    assert np.array_equal(g["validity"], o.validity)
    assert np.all(g["compute"] == 1) and np.all(g["klast"] == 0)
    # positions and velocities are untouched by the priming evaluation
    assert np.array_equal(g["x"], st["x"]) and np.array_equal(g["v"], st["v"])


def _dam_break_64k():
    # 40^3 = 64,000 particles: more evaluated particles than eight warps of lanes per SM
    # of a GB300 (38,912), so a pass that evaluates most of them runs one lane per
    # particle (k_density_dense); the 8k scenes of the other tests run the warp-per-block
    # pass
    return scenes.dam_break((40, 40, 40), 0.01, (1.6, 0.8, 0.8), 5e-5, jitter=2e-4, seed=99,
                            name="wcsph_dam_break_64k")


def test_lane_per_particle_density_pass_matches_oracle():
    sc = _dam_break_64k()
    st = dynamic_state(sc, seed=13)
    ctx = gpu_ctx(sc)
    rts.rts_set_state(ctx, st["x"], st["v"], a=st["a"], rho=st["rho"], p=st["p"])
    rts.rts_evaluate(ctx)
    g = rts.rts_get_state(ctx)
    o = oracle_state(sc, sc.params, st)
    o.evaluate()
    _check_eval(g, o)
    lists = rts.rts_get_neighbors(ctx)
    off, idx = O.neighbors_grid(O.make_params(sc.params), st["x"], sc.xb)
    for i in range(sc.n):
        assert sorted(lists[i].tolist()) == sorted(idx[off[i]:off[i + 1]].tolist()), i


def test_lane_per_particle_density_pass_in_global_steps_matches_oracle():
    sc = _dam_break_64k()
    d = params(sc, mode=1)
    ctx = gpu_ctx(sc, d)
    o = oracle_state(sc, d, {"x": sc.x, "v": sc.v})
    for _ in range(3):
        o.global_step()                            # every particle evaluated each step
    st = rts.rts_advance(ctx, o.k * d["dt_b"])     # the same steps (the level is exact)
    assert ctx.substep_index == o.k and st["steps"] == 3
    assert st["candidate_tests"] == st["tests_performed"]   # no cull: the lane-per-particle pass
    g = rts.rts_get_state(ctx)
    np.testing.assert_allclose(g["x"], o.x, atol=2e-5)
    np.testing.assert_allclose(g["rho"], o.rho, rtol=RHO_RTOL)


def test_rest_lattice_density_on_gpu():
    # fluid filling the tank: every particle has a complete lattice (dyadic spacing)
    s = 1.0 / 64
    sc = scenes.dam_break((8, 6, 5), s, (8 * s, 6 * s, 5 * s), 1e-4)
    ctx = gpu_ctx(sc)
    rts.rts_evaluate(ctx)
    g = rts.rts_get_state(ctx, ("rho", "nbr"))
    o = oracle_state(sc, sc.params, {"x": sc.x, "v": sc.v})
    o.evaluate()
    assert np.all(g["nbr"] == 26)
    np.testing.assert_allclose(g["rho"], o.rho, rtol=RHO_RTOL)


# -------------------------------------------------------------------- substep ---

def _predicted(st, dt):
    x = st["x"].astype(np.float64)
    v = st["v"].astype(np.float64)
    a = st["a"].astype(np.float64)
    return x + v * dt + a * dt * dt / 2, v + a * dt


def _near_threshold(P, xt, vt, a, blocks, rel=1e-5):
    """Blocks whose FP64 maxima lie within rel of a level threshold (don't-care band)."""
    key, _, _ = O.bin_particles(P, xt)
    v2 = (vt ** 2).sum(1)
    a2 = (a ** 2).sum(1)
    vthr2, athr2, _ = O.level_thresholds(P)
    near = set()
    for b in blocks:
        sel = key == b
        for val, thr in ((v2[sel].max(), vthr2), (a2[sel].max(), athr2)):
            if np.any(np.abs(val / thr - 1.0) < rel):
                near.add(int(b))
    return near


@pytest.mark.parametrize("seed,clock,serna_off", [(1, 0, 0), (2, 0, 0), (3, 1, 0), (4, 1, 0),
                                                  (5, 0, 1)])
def test_one_regional_substep_matches_oracle(seed, clock, serna_off):
    # serna_off = 1: the ablation without the Section 4.1 correction
    sc = scenes.wcsph_dam_break_8k()
    st = dynamic_state(sc, seed=seed)
    k0 = 8 + clock      # the aligned clock: an odd substep follows
    d = params(sc, level_clock=clock, serna_off=serna_off)
    ctx = gpu_ctx(sc, d)
    rts.rts_set_state(ctx, st["x"], st["v"], a=st["a"], rho=st["rho"], p=st["p"],
                      level=st["level"], validity=st["validity"], klast=st["klast"], k=k0,
                      primed=True)
    rts.rts_wcsph_substep(ctx)
    g = rts.rts_get_state(ctx)
    o = oracle_state(sc, d, st, k=k0, primed=True)
    o.substep()
    P = o.P
    mism = np.nonzero(g["compute"] != o.compute)[0]
    if len(mism):
        xt, vt = _predicted(st, P.dt_b)
        key, _, _ = O.bin_particles(P, xt)
        near = _near_threshold(P, xt, vt, st["a"].astype(np.float64), np.unique(key[mism]))
        assert all(int(key[i]) in near for i in mism), f"{len(mism)} activity mismatches"
    same = g["compute"] == o.compute
    assert same.mean() > 0.999
    comp = (o.compute == 1) & same
    assert comp.sum() > 100 and (~comp).sum() > 100   # both kinds present
    assert np.array_equal(g["level"][same], o.level[same])
    assert np.array_equal(g["validity"][same], o.validity[same])
    assert np.array_equal(g["klast"][same], o.klast[same])
    xt, _ = _predicted(st, P.dt_b)
    _check_eval(g, o, comp, xpred=xt)
    # positions / velocities: FP32 predictor rounding plus the force tolerance
    tol_a = ACC_FRAC * max_norm(o.a[comp])
    dt = (k0 + 1 - st["klast"].astype(np.float64)) * P.dt_b
    dx = np.abs(g["x"] - o.x).max(axis=1)
    dv = np.abs(g["v"] - o.v).max(axis=1)
    x_tol = 8 * ulp32(o.x).max(axis=1) + np.where(comp, tol_a * dt * dt / 6, 0)
    v_tol = 8 * ulp32(o.v).max(axis=1) + 1e-6 * np.abs(st["a"]).max() * P.dt_b + np.where(comp, tol_a * dt / 2, 0)
    assert np.all(dx[same] <= x_tol[same])
    assert np.all(dv[same] <= v_tol[same])


def test_forced_finest_level_reproduces_global_stepping_bit_for_bit():
    sc = scenes.wcsph_dam_break_8k()
    a = gpu_ctx(sc, params(sc, force_level=0))
    b = gpu_ctx(sc, params(sc, mode=2))
    for _ in range(10):
        rts.rts_wcsph_substep(a)
        rts.rts_wcsph_substep(b)
    ga, gb = rts.rts_get_state(a), rts.rts_get_state(b)
    for f in ("x", "v", "a", "rho", "p", "klast", "nbr"):
        assert np.array_equal(ga[f], gb[f]), f
    assert np.all(ga["compute"] == 1)


def test_global_adaptive_step_size_matches_oracle():
    sc = scenes.wcsph_dam_break_8k()
    d = params(sc, mode=1)
    ctx = gpu_ctx(sc, d)
    o = oracle_state(sc, d, {"x": sc.x, "v": sc.v})
    for _ in range(4):
        rts.rts_wcsph_substep(ctx)                 # one global step of the finest level
        o.global_step()
        assert ctx.substep_index == o.k
    g = rts.rts_get_state(ctx)
    np.testing.assert_allclose(g["x"], o.x, atol=2e-5)


# ------------------------------------------------------------------ rollouts ---

def test_rollout_statistics_match_oracle():
    # 0.05 s of the 8k dam break with regional stepping: trajectories diverge, so compare
    # mass (particle count), kinetic energy and density-error statistics.
    sc = scenes.wcsph_dam_break_8k()
    T = 0.05
    ctx = gpu_ctx(sc)
    stats = rts.rts_advance(ctx, T)
    g = rts.rts_get_state(ctx)
    o = oracle_state(sc, sc.params, {"x": sc.x, "v": sc.v})
    evals = 0
    while o.k < stats["substeps"]:
        o.substep()
        evals += int(o.compute.sum())
    assert stats["substeps"] == round(T / sc.params["dt_b"])
    ke_g = 0.5 * (g["v"].astype(np.float64) ** 2).sum()
    ke_o = 0.5 * (o.v ** 2).sum()
    assert abs(ke_g / ke_o - 1) < 0.05
    err_g = np.abs(g["rho"] / 1000.0 - 1)
    err_o = np.abs(o.rho / 1000.0 - 1)
    assert abs(err_g.mean() - err_o.mean()) < 0.1 * err_o.mean() + 1e-4
    assert abs(np.percentile(err_g, 99) - np.percentile(err_o, 99)) < 0.1 * np.percentile(err_o, 99) + 1e-3
    assert abs(stats["particle_evals"] / evals - 1) < 0.05
    assert sum(stats["level_count"]) == sc.n


# ------------------------------------------------------------- full size ---

def test_full_size_evaluation_sampled():
    # 1M-particle dam break, evaluated in the launch configuration of the benchmark;
    # the oracle computes a seeded sample of particles one by one.
    sc = scenes.wcsph_dam_break_1m()
    ctx = gpu_ctx(sc)
    rts.rts_evaluate(ctx)
    g = rts.rts_get_state(ctx, ("rho", "nbr", "a", "level"))
    rng = np.random.default_rng(9)
    sample = rng.choice(sc.n, 3000, replace=False)
    P = O.make_params(sc.params)
    mask = np.zeros(sc.n, np.uint8)
    mask[sample] = 1
    rho, prs, nbr = O.density(P, sc.x, sc.xb)          # all: forces need every neighbour's rho
    a = O.accel(P, sc.x, sc.v, rho, prs, sc.xb, mask)
    assert np.array_equal(g["nbr"][sample], nbr[sample])
    np.testing.assert_allclose(g["rho"][sample], rho[sample], rtol=RHO_RTOL)
    tol = ACC_FRAC * max_norm(a[sample])
    assert np.linalg.norm(g["a"][sample] - a[sample], axis=1).max() <= tol
    raw, lev = O.classify_wcsph(P, sc.x, sc.v, np.zeros_like(sc.x))
    assert np.array_equal(g["level"], _levels_by_particle(P, sc.x, lev))


def test_full_size_substeps_run_and_conserve_particles():
    sc = scenes.wcsph_dam_break_1m()
    ctx = gpu_ctx(sc)
    s = rts.rts_advance(ctx, 40 * sc.params["dt_b"])
    assert s["substeps"] == 40
    assert sum(s["level_count"]) == sc.n
    g = rts.rts_get_state(ctx, ("x", "rho"))
    assert np.isfinite(g["x"]).all()
    assert np.all(g["x"].min(0) > -0.02) and np.all(g["x"].max(0) < np.array([4.02, 2.02, 2.02]))


# ---------------------------------------------------------------- edge cases ---

def test_empty_fluid_and_no_boundary():
    sc = scenes.wcsph_dam_break_8k()
    ctx = rts.rts_init(sc.params, np.zeros((0, 3), np.float32), np.zeros((0, 3), np.float32), sc.xb)
    s = rts.rts_advance(ctx, 5 * sc.params["dt_b"])
    assert s["substeps"] == 5 and s["particle_evals"] == 0
    ctx2 = rts.rts_init(sc.params, sc.x, sc.v, np.zeros((0, 3), np.float32))
    rts.rts_advance(ctx2, 3 * sc.params["dt_b"])
    g = rts.rts_get_state(ctx2, ("nbr",))
    assert g["nbr"].max() <= 40


def test_out_of_domain_particle_is_a_sticky_error_until_set_state():
    sc = scenes.wcsph_dam_break_8k()
    x = sc.x.copy()
    x[123] = [50.0, 0.1, 0.1]
    ctx = gpu_ctx(sc, x=x)
    with pytest.raises(rts.RtsError) as e:
        rts.rts_advance(ctx, 2 * sc.params["dt_b"])
    assert e.value.status == 2
    with pytest.raises(rts.RtsError) as e:
        rts.rts_wcsph_substep(ctx)
    assert e.value.status == 8
    rts.rts_set_state(ctx, sc.x, sc.v)
    rts.rts_advance(ctx, 2 * sc.params["dt_b"])


def test_block_over_capacity_is_reported():
    sc = scenes.wcsph_dam_break_8k()
    x = sc.x.copy()
    x[:100] = x[0] + np.linspace(0, 1e-3, 100, dtype=np.float32)[:, None]   # 100 in one block
    ctx = gpu_ctx(sc, params(sc, max_per_block=64), x=x)
    with pytest.raises(rts.RtsError) as e:
        rts.rts_sync(ctx)
        rts.rts_advance(ctx, sc.params["dt_b"])
    assert e.value.status == 5


def test_neighbour_lists_of_evaluated_particles_equal_brute_force():
    sc = scenes.wcsph_dam_break_8k()
    st = dynamic_state(sc, seed=8)
    ctx = gpu_ctx(sc)
    rts.rts_set_state(ctx, st["x"], st["v"], a=st["a"], rho=st["rho"], p=st["p"])
    rts.rts_evaluate(ctx)
    lists = rts.rts_get_neighbors(ctx)
    off, idx = O.neighbors_brute(st["x"], sc.xb, O.make_params(sc.params).r)
    for i in range(sc.n):
        assert sorted(lists[i].tolist()) == sorted(idx[off[i]:off[i + 1]].tolist()), i


def test_deferred_corrections_and_reruns_are_bit_identical():
    # rts_advance defers each substep's Serna correction into the next key pass; single
    # substeps apply it at once: same function, same bits.  A rerun gives the same bits.
    sc = scenes.wcsph_dam_break_8k()
    dt = sc.params["dt_b"]
    a, b, c = gpu_ctx(sc), gpu_ctx(sc), gpu_ctx(sc)
    rts.rts_advance(a, 24 * dt)
    rts.rts_advance(c, 24 * dt)
    for _ in range(24):
        rts.rts_wcsph_substep(b)
    ga, gb, gc = rts.rts_get_state(a), rts.rts_get_state(b), rts.rts_get_state(c)
    for f in ("x", "v", "a", "rho", "p", "klast", "validity", "level", "nbr"):
        assert np.array_equal(ga[f], gb[f]), f
        assert np.array_equal(ga[f], gc[f]), f


def test_bins_and_lists_on_a_grid_of_more_than_a_thousand_scan_tiles():
    # The 1M dam-break grid has 202 x 102 x 102 = 2.1M blocks, 1027 scan tiles of 2048
    # blocks: the scan of the tile sums then spans all 32 warps of its CTA.  Bins over the
    # whole grid (the top layers included) and the neighbour lists of particles under the
    # ceiling, boundary neighbours included, against the oracle.
    sc = scenes.wcsph_dam_break_1m()
    P = O.make_params(sc.params)
    rng = np.random.default_rng(21)
    cloud = rng.uniform([0.0, 0.0, 0.0], [4.0, 2.0, 2.0], (100000, 3))
    slab = scenes.lattice((50, 50, 10), 0.01, offset=(0.0, 0.0, 1.9))
    x = np.concatenate([cloud, slab]).astype(np.float32)
    ctx = rts.rts_init(sc.params, x, np.zeros_like(x), sc.xb)
    rts.rts_bin(ctx)
    key, perm, cstart = rts.rts_get_bins(ctx)
    okey, operm, ocstart = O.bin_particles(P, x)
    assert np.array_equal(key, okey)
    assert np.array_equal(perm, operm)
    assert np.array_equal(cstart, ocstart)
    rts.rts_evaluate(ctx)
    lists = rts.rts_get_neighbors(ctx)
    off, idx = O.neighbors_grid(P, x, sc.xb)
    top = np.nonzero(x[:, 2] > 1.95)[0]
    assert len(top) > 10000
    for i in top[::17]:
        assert sorted(lists[i].tolist()) == sorted(idx[off[i]:off[i + 1]].tolist()), i
    assert max(off[i + 1] - off[i] for i in top) > 20


def test_container_projection_matches_oracle():
    # the bottom layer is thrown into the floor at 200 m/s: one constant global step
    # predicts it 1 cm below the floor face; both sides put it back on the face, drop the
    # downward velocity and then evaluate and correct it against the same walls
    sc = scenes.wcsph_dam_break_8k()
    d = params(sc, mode=2)
    v = sc.v.copy()
    bottom = sc.x[:, 2] < 0.015
    v[bottom, 2] = -200.0
    ctx = gpu_ctx(sc, d, v=v)
    o = oracle_state(sc, d, {"x": sc.x, "v": v})
    rts.rts_wcsph_substep(ctx)
    o.global_step()
    g = rts.rts_get_state(ctx, ("x", "v", "a"))
    assert bottom.sum() == 400
    # corrected heights: within the correction's reach of the face, far above -1 cm
    assert np.abs(o.x[bottom, 2]).max() < 2e-3 and np.abs(g["x"][bottom, 2]).max() < 2e-3
    tol_a = ACC_FRAC * max_norm(o.a)
    dt = d["dt_b"]
    assert np.abs(g["x"] - o.x).max() <= tol_a * dt * dt + 2e-6
    assert np.abs(g["v"] - o.v).max() <= tol_a * dt + 1e-4


def test_level_aligned_clock_rollout_matches_oracle_schedule():
    # 16 substeps of the level-aligned variant from a dynamic state: the evaluated sets
    # agree substep by substep (up to threshold ties), and the blocks hold more
    # evaluated particles each than with Algorithm 1's drifting phases
    sc = scenes.wcsph_dam_break_8k()
    st = dynamic_state(sc, seed=6)
    out = {}
    for clock in (0, 1):
        d = params(sc, level_clock=clock)
        ctx = gpu_ctx(sc, d)
        rts.rts_set_state(ctx, st["x"], st["v"], a=st["a"], rho=st["rho"], p=st["p"])
        o = oracle_state(sc, d, st)
        rts.rts_evaluate(ctx)
        o.evaluate()
        evals = blocks = 0
        for _ in range(16):
            s = rts.rts_advance(ctx, (ctx.substep_index + 1) * d["dt_b"])
            o.substep()
            g = rts.rts_get_state(ctx, ("compute",))
            assert (g["compute"] != o.compute).sum() <= 1e-3 * sc.n + 2
            evals += s["particle_evals"]
            blocks += s["active_blocks"]
        out[clock] = evals / blocks
    assert out[1] > out[0]
