"""Neighbour sets at the cutoff: the FP32-piece exact predicate decides pairs in the guard
band as the double-precision definition does.

A perfect lattice of spacing s with support r = 2 s puts every axis-aligned pair two
spacings apart at |x_i - x_j| = r up to the FP32 rounding of the positions (exact ties
for small coordinates); nudging coordinates by a few units in the last place moves
pairs to either side of r by 1e-7 relative, far inside the FP32 guard band.  The
neighbour lists of the WCSPH evaluation and of the PCISPH refresh must equal the FP64
brute-force sets of the oracle."""
import numpy as np
import pytest

import oracle as O
from paper_2009_14514_gb300 import rts, scenes

pytestmark = pytest.mark.gpu


def _nudged(x, seed, frac=0.3, max_ulps=3):
    rng = np.random.default_rng(seed)
    x = x.copy()
    pick = rng.random(x.shape) < frac
    steps = rng.integers(-max_ulps, max_ulps + 1, size=x.shape)
    for k in range(1, max_ulps + 1):
        for sgn in (1, -1):
            m = pick & (steps * sgn >= k)
            x[m] = np.nextafter(x[m], np.float32(sgn * np.inf))
    return x


def _check(lists, x, xb, r):
    off, idx = O.neighbors_brute(x, xb, r)
    for i in range(len(x)):
        assert sorted(lists[i].tolist()) == sorted(idx[off[i]:off[i + 1]].tolist()), i


@pytest.mark.parametrize("nudge", [False, True])
def test_wcsph_lists_at_the_cutoff_equal_fp64_brute_force(nudge):
    sc = scenes.dam_break((12, 10, 9), 0.02, (0.48, 0.24, 0.24), 1e-4, jitter=0.0)
    x = _nudged(sc.x, 5) if nudge else sc.x
    ctx = rts.rts_init(sc.params, x, sc.v, sc.xb)
    rts.rts_evaluate(ctx)
    _check(rts.rts_get_neighbors(ctx), x, sc.xb, O.make_params(sc.params).r)


@pytest.mark.parametrize("nudge", [False, True])
def test_pcisph_lists_at_the_cutoff_equal_fp64_brute_force(nudge):
    sc = scenes.pool_drop((14, 12, 6), 4, 0.03, 0.01, (0.14, 0.12, 0.16), 3.5e-4)
    x = _nudged(sc.x, 6) if nudge else sc.x
    # one minor step per major step, no expansion: every particle refreshes with one ring
    d = dict(sc.params, n_minor=1, expand_layers=0, r1_search_rings=1)
    ctx = rts.rts_init(d, x, sc.v, sc.xb)
    rts.rts_pcisph_step(ctx)
    _check(rts.rts_get_neighbors(ctx), x, sc.xb, O.make_params(sc.params).r)
