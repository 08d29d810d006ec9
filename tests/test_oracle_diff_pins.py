"""Pins of the FP64 reference gradient (oracle/diff_oracle.py): the reverse-mode gradient
of a global-stepping WCSPH rollout equals central finite differences of the same FP64
forward (the C oracle), for the stiffness B, the viscosity coefficient alpha and initial
velocities; with the container correction active and inactive."""
import numpy as np
import pytest

from oracle.diff_oracle import DiffRollout, centroid_density_loss
from paper_2009_14514_gb300 import scenes

B0 = 57344.0        # exact in FP32, as are B0 +- 8 (the parameters pass through FP32)
A0 = 0.0625         # exact in FP32, as are A0 +- 2^-14
TARGET = [0.1, 0.12, 0.05]


def _case(wall_shift=0.0):
    sc = scenes.dam_break((6, 6, 6), 0.02, (0.24, 0.24, 0.3), 1e-4, jitter=2e-3, seed=3)
    x = sc.x.astype(np.float64)
    x[:, 2] += wall_shift
    rng = np.random.default_rng(4)
    v0 = rng.normal(0.0, 0.3, (sc.n, 3))
    return sc, x, v0


def _loss(R, v0, B, a, steps):
    xT, rhoT, _ = R.forward(v0, B, a, steps, record=False)
    return centroid_density_loss(xT, rhoT, TARGET, 1000.0)[0]


@pytest.mark.parametrize("wall_shift,vz,no_clamp", [(0.0, 0.0, 0), (-0.0098, -0.6, 0), (0.0, 0.0, 1)])
def test_reference_gradient_matches_central_differences(wall_shift, vz, no_clamp):
    # second case: the bottom layer starts 0.2 mm above the floor moving down, so the
    # container clamps it during the rollout; third: negative Tait pressure kept
    sc, x, v0 = _case(wall_shift)
    v0[:, 2] += vz
    steps = 20
    R = DiffRollout(dict(sc.params, tait_no_clamp=no_clamp), x, sc.xb)
    xT, rhoT, recs = R.forward(v0, B0, A0, steps)
    if vz:
        assert any(r["mx"].any() for r in recs[1:])
    L, xbar, rhobar = centroid_density_loss(xT, rhoT, TARGET, 1000.0)
    gv, gB, ga = R.backward(recs, B0, A0, xT, xbar, rhobar)
    fdB = (_loss(R, v0, B0 + 8.0, A0, steps) - _loss(R, v0, B0 - 8.0, A0, steps)) / 16.0
    ha = 2.0 ** -14
    fda = (_loss(R, v0, B0, A0 + ha, steps) - _loss(R, v0, B0, A0 - ha, steps)) / (2 * ha)
    assert abs(gB - fdB) <= 1e-4 * abs(fdB) and abs(fdB) > 0
    assert abs(ga - fda) <= 1e-4 * abs(fda) and abs(fda) > 0
    rng = np.random.default_rng(5)
    scale = np.abs(gv).max()
    for i, k in zip(rng.choice(sc.n, 6, replace=False), rng.integers(0, 3, 6)):
        hv = 1e-6
        vp, vm = v0.copy(), v0.copy()
        vp[i, k] += hv
        vm[i, k] -= hv
        fd = (_loss(R, vp, B0, A0, steps) - _loss(R, vm, B0, A0, steps)) / (2 * hv)
        assert abs(gv[i, k] - fd) <= 1e-4 * scale, (i, k, gv[i, k], fd)
