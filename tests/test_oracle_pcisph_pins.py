"""Pins of the FP64 oracle's PCISPH part (Algorithms 2 and 3, Sections 5.2-5.6).

The density-correction schedule (Figure 5) is missing from the paper; the table used is
a reconstruction, so its iteration counts are "parity unpinned" beyond the properties
Section 5.3 states, which the first test checks.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2009_14514_gb300 import scenes


def _params(scene, **over):
    d = dict(scene.params)
    d.update(over)
    return O.make_params(d)


def test_schedule_has_the_properties_section_5_3_states():
    d = scenes.pcisph_drop_small().params
    sched = np.array(d["sched"])                      # region x minor step
    N = d["n_minor"]
    mult = d["level_mult"]
    assert np.all(sched[:, :N] >= 1)                 # every region at least once per step
    assert np.all(sched[:, 0] >= 2)                  # first minor step: two for everyone
    assert np.all(sched[0, :N] == 3)                 # R_1: 3 per step (classic PCISPH)
    for j in range(0, N, 2):                         # R_2: 3 per two minor steps
        assert sched[1, j] + sched[1, j + 1] == 3
    for n in range(4):                               # >= 3 within a region's true step
        true_step = mult[n]
        for j0 in range(0, N - true_step + 1, true_step):
            assert sched[n, j0:j0 + true_step].sum() >= 3
    per_major = sched[:, :N].sum(axis=1)             # slower regions fewer (non-strictly)
    assert np.all(np.diff(per_major) <= 0)
    assert sched[:, :N].max() == 3                    # rows 1..3: the standard schedule


def test_delta_closed_form_on_cubic_lattice():
    sc = scenes.pcisph_drop_small()
    P = _params(sc)
    s, h = P.s, 0.5 * P.r
    sigma = 1.0 / (math.pi * h ** 3)
    # |dW/dd| at q = 1, sqrt 2, sqrt 3 (h = s): 0.75 sigma / h * (2 - q)^2 for q >= 1
    g1 = 0.75 * sigma / h
    g2 = 0.75 * sigma / h * (2 - math.sqrt(2)) ** 2
    g3 = 0.75 * sigma / h * (2 - math.sqrt(3)) ** 2
    sum_gg = 6 * g1 ** 2 + 12 * g2 ** 2 + 8 * g3 ** 2
    m = P.rho0 * s ** 3
    beta = 2 * (P.dt_b * m / P.rho0) ** 2
    assert O.pcisph_delta(P) == pytest.approx(1.0 / (beta * sum_gg), rel=1e-12)


def _rest_box(**over):
    s = 1.0 / 64
    box = (8 * s, 7 * s, 6 * s)
    sc = scenes.pool_drop((8, 7, 6), 0, 0.0, s, box, 3.5e-4)
    sc.x = sc.x[: 8 * 7 * 6].copy()                  # drop the empty cube
    sc.v = sc.v[: 8 * 7 * 6].copy()
    return sc, _params(sc, gravity=[0.0, 0.0, 0.0], **over)


def test_rest_lattice_stays_at_rest_with_the_minimum_iterations():
    sc, P = _rest_box()
    S = O.PCISPH(P, sc.x, sc.v, sc.xb)
    for _ in range(6):
        S.step()
        assert S.stats["iters"] == 3
        assert S.err.max() == 0.0 and np.all(S.p == 0.0)
    np.testing.assert_array_equal(S.x, sc.x.astype(np.float64))
    assert np.all(S.v == 0.0)


def test_first_minor_step_neighbourhoods_equal_brute_force():
    sc = scenes.pcisph_drop_small()
    P = _params(sc)
    S = O.PCISPH(P, sc.x, sc.v, sc.xb)
    x0 = S.x.copy()
    S.step()
    off, idx = O.neighbors_brute(x0, sc.xb, P.r)
    for i in range(0, sc.n, 37):
        assert set(S.neighbors(i).tolist()) == set(idx[off[i]:off[i + 1]].tolist())


def _block_field(P, lev_of_centre, nb=11):
    """A filled nb^3 block region (one particle per block centre) in the grid."""
    idx = np.stack(np.meshgrid(*[np.arange(nb) for _ in range(3)], indexing="ij"), -1).reshape(-1, 3)
    x = (idx + 0.5) * P.edge
    key, _, _ = O.bin_particles(P, x)
    lev = np.full(O.n_blocks(P), -1, np.int32)
    lev[key] = [lev_of_centre(c) for c in idx]
    return idx, key, lev


def test_region_expansion_dilates_r1_then_r2_by_four_blocks():
    s = 0.01
    sc = scenes.pool_drop((50, 50, 50), 0, 0.0, s, (0.5, 0.5, 0.5), 3.5e-4)
    P = _params(sc)
    idx, key, raw = _block_field(P, lambda c: 3, nb=21)
    centre = np.array([5, 5, 5])
    n = len(idx)
    v = np.zeros((n, 3))
    a = np.zeros((n, 3))
    c = int(np.argmin(np.abs(idx - centre).sum(1)))
    c2 = int(np.argmin(np.abs(idx - np.array([20, 20, 20])).sum(1)))
    x = (idx + 0.5) * P.edge
    vt = np.sqrt(O.level_thresholds(P)[0])
    v[c, 0] = vt[1] * 2                    # needs region 1
    v[c2, 0] = (vt[1] + vt[2]) / 2         # needs region 2
    raw, lev = O.classify_pcisph(P, x, v, a)
    per = lev[key]
    cheb = np.abs(idx - centre).max(1)
    cheb2 = np.abs(idx - 20).max(1)
    # R_min first widens each by one layer, then the 4-layer expansions; region 2 grows
    # from every block of region <= 2, so it also forms a 4-block shell around region 1
    expect = np.where(cheb <= 5, 0, np.where((cheb <= 9) | (cheb2 <= 5), 1, 3))
    assert np.array_equal(per, expect)


def test_observed_blocks_border_smaller_regions_and_re():
    s = 0.01
    sc = scenes.pool_drop((50, 50, 50), 0, 0.0, s, (0.5, 0.5, 0.5), 3.5e-4)
    P = _params(sc)
    idx, key, lev = _block_field(P, lambda c: 0 if c[0] <= 4 else 2)
    ob = O.observed_blocks(P, lev)[key]
    assert np.all(ob[idx[:, 0] == 5] == 1)             # larger-dt side of the border
    assert np.all(ob[idx[:, 0] != 5] == 0)
    in_re = np.zeros(O.n_blocks(P), np.uint8)
    re_block = key[np.argmin(np.abs(idx - np.array([8, 5, 5])).sum(1))]
    in_re[re_block] = 1
    ob = O.observed_blocks(P, lev, in_re)
    blocks = key
    around = (np.abs(idx - np.array([8, 5, 5])).max(1) == 1)
    assert np.all(ob[blocks[around]] == 1) and ob[re_block] == 0


def test_forced_region_one_equals_plain_pcisph():
    # every block in R_1, one minor step per major step, no local iterations (eta_T = 0):
    # the regional machinery reduces to plain PCISPH (summation order aside)
    sc = scenes.pcisph_drop_small()
    P = _params(sc, force_level=0, n_minor=1, eta_T=0.0)
    A = O.PCISPH(P, sc.x, sc.v, sc.xb)
    B = O.PCISPH(P, sc.x, sc.v, sc.xb)
    for _ in range(8):
        A.step()
        B.plain_step()
        assert A.stats["iters"] == B.S.iters
    np.testing.assert_allclose(A.x, B.x, rtol=0, atol=1e-12)
    np.testing.assert_allclose(A.v, B.v, rtol=0, atol=1e-10)
    np.testing.assert_allclose(A.p, B.p, rtol=1e-9, atol=1e-9)


def _compressed_pool(**over):
    sc = scenes.pcisph_drop_small()
    x = sc.x.copy()
    rng = np.random.default_rng(3)
    # squeeze a handful of particles towards their neighbours: local density errors
    pick = rng.choice(sc.n, 40, replace=False)
    x[pick] += rng.uniform(-0.004, 0.004, (40, 3)).astype(np.float32)
    return sc, x, _params(sc, **over)


def test_infinite_tolerance_gives_exactly_the_schedule_minimum():
    sc, x, P = _compressed_pool(eta=1e9)
    S = O.PCISPH(P, x, sc.v, sc.xb)
    for _ in range(5):
        S.step()
        assert S.stats["iters"] == 3 and S.stats["local_iters"] == 0


def test_impossible_tolerance_hits_the_cap_and_reports_it():
    sc, x, P = _compressed_pool(eta=1e-12, max_iters=7)
    S = O.PCISPH(P, x, sc.v, sc.xb)
    st = S.step()
    assert st == 6 and S.stats["iters"] == 7 and S.stats["not_converged"] == 1


def test_local_iterations_when_the_average_error_is_small():
    sc, x, P = _compressed_pool(eta=0.002, eta_T=0.5)
    S = O.PCISPH(P, x, sc.v, sc.xb)
    S.step()
    st = S.stats
    assert st["iters"] > 3 and st["local_iters"] > 0
    sc, x, P = _compressed_pool(eta=0.002, eta_T=0.0)   # always global
    S = O.PCISPH(P, x, sc.v, sc.xb)
    S.step()
    assert S.stats["local_iters"] == 0 and S.stats["iters"] > 3


def test_local_failure_reverts_pressures_and_goes_global():
    sc, x, P = _compressed_pool(eta=1e-9, eta_T=0.5, max_local_iters=2, max_iters=12)
    S = O.PCISPH(P, x, sc.v, sc.xb)
    S.step()
    st = S.stats
    assert st["local_iters"] == 2 and st["reverts"] == 1   # after 2 local iterations: revert
    assert st["iters"] == 12


def test_major_step_shortening_and_restoration():
    sc = scenes.pcisph_drop_small()
    # minor step 1 of the schedule has two global iterations: a limit of 1 is exceeded
    P = _params(sc, max_global_iters=1, clean_majors=2)
    S = O.PCISPH(P, sc.x, sc.v, sc.xb)
    S.step()
    assert S.S.minor == 0 and S.S.n_minor_cur == 2           # major step ended early
    # a limit of 2 is not exceeded: shortened majors run clean and are restored after 2
    P2 = _params(sc, max_global_iters=2, clean_majors=2)
    S.P = P2
    S.step()
    S.step()
    assert S.S.minor == 0 and S.S.n_minor_cur == 2 and S.S.clean == 1
    S.step()
    S.step()
    assert S.S.n_minor_cur == 4 and S.S.clean == 0


def test_region2_two_ring_search_equals_brute_force_at_the_major_start():
    # the r2_rings ablation: region-2 particles search two rings; at the major-step start
    # their lists are still exactly the particles within r (brute force), and a region-2
    # particle in a block far from its neighbours' blocks finds them only with 2 rings
    sc = scenes.pcisph_drop_small()
    st = scenes.perturbed_state(sc, 11, vmax=15.0, amax=2.0e4)
    d = dict(sc.params, n_minor=1, expand_layers=0, r2_search_rings=2)
    P = O.make_params(d)
    S = O.PCISPH(P, sc.x, st["v"], sc.xb)
    S.anp[:] = st["a"]
    S.step()
    off, idx = O.neighbors_brute(sc.x, sc.xb, P.r)
    r2 = np.nonzero(S.level == 1)[0]
    assert len(r2) > 0
    for i in r2[:200]:
        assert set(S.neighbors(i).tolist()) == set(idx[off[i]:off[i + 1]].tolist())
