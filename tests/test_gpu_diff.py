"""GPU parity of the differentiable WCSPH rollout (rts_diff_*) against the FP64 oracle.

4,096 particles, 100 steps of global constant stepping, checkpoints every 10 steps.
Loss |mean(x_T) - target|^2 + mean |rho_T - rho0| / rho0; gradients with respect to every
initial velocity, the Tait stiffness B and the viscosity coefficient alpha.

With negative Tait pressure kept the rollout is smooth (apart from the viscosity's
approach test), and the GPU gradients match the FP64 reference gradient (pinned on
finite differences on a small case) element by element, and the two scalar gradients
match central differences of the oracle's forward.  With the pressure clamped at zero the loss is
only piecewise smooth: FP32 and FP64 trajectories cross the clamp at slightly different
times for the free-surface particles, so single entries of dL/dv0 may differ by up to
~15 % of the largest one; the comparison is then on the whole gradient (relative L2), on
the two scalar gradients, and on central finite differences of the oracle's forward,
and entry by entry on the entries that the FP64 reference shows to be insensitive to
small perturbations of the initial velocities (where the branch is stable).
"""
import numpy as np
import pytest
import torch

from oracle.diff_oracle import DiffRollout, centroid_density_loss
from paper_2009_14514_gb300 import diff, scenes

pytestmark = pytest.mark.gpu

B0 = 57344.0      # exact in FP32 (the oracle rounds parameters through FP32)
A0 = 0.0625
STEPS = 100
TARGET = [0.2, 0.1, 0.05]


def _make(no_clamp):
    sc = scenes.diff_dam_break_4k()
    d = dict(sc.params, tait_no_clamp=no_clamp)
    v0 = scenes.seeded_velocities(sc.n, seed=777, scale=0.3)
    R = DiffRollout(d, sc.x, sc.xb)
    xT, rhoT, recs = R.forward(v0, B0, A0, STEPS)
    L, xbar, rhobar = centroid_density_loss(xT, rhoT, TARGET, 1000.0)
    gv, gB, ga = R.backward(recs, B0, A0, xT, xbar, rhobar)
    eng = diff.DiffEngine(d, sc.x, sc.xb, STEPS, ckpt_every=10)
    return dict(sc=sc, d=d, v0=v0, R=R, xT=xT, rhoT=rhoT, L=L, gv=gv, gB=gB, ga=ga, eng=eng)


@pytest.fixture(scope="module")
def smooth():
    return _make(1)


@pytest.fixture(scope="module")
def clamped():
    return _make(0)


def _gpu_grads(case):
    v0 = torch.tensor(case["v0"], device="cuda", requires_grad=True)
    B = torch.tensor(B0, dtype=torch.float64, device="cuda", requires_grad=True)
    a = torch.tensor(A0, dtype=torch.float64, device="cuda", requires_grad=True)
    x, rho = diff.rollout(case["eng"], v0, B, a)
    L = diff.centroid_density_loss(x, rho, TARGET)
    L.backward()
    return (float(L.detach()), x.detach().cpu().numpy().astype(np.float64),
            rho.detach().cpu().numpy().astype(np.float64),
            v0.grad.cpu().numpy().astype(np.float64), float(B.grad), float(a.grad))


@pytest.mark.parametrize("which", ["smooth", "clamped"])
def test_forward_matches_the_fp64_rollout(which, request):
    case = request.getfixturevalue(which)
    L, x, rho, _, _, _ = _gpu_grads(case)
    assert np.abs(x - case["xT"]).max() < 2e-6                 # 100 FP32 steps of ~1e-5 m
    np.testing.assert_allclose(rho, case["rhoT"], rtol=2e-4)
    assert abs(L - case["L"]) <= 1e-4 * abs(case["L"])


def test_smooth_rollout_gradients_match_the_reference_entry_by_entry(smooth):
    _, _, _, gv, gB, ga = _gpu_grads(smooth)
    ref = smooth["gv"]
    assert np.abs(gv - ref).max() <= 2e-3 * np.abs(ref).max()
    assert abs(gB - smooth["gB"]) <= 2e-3 * abs(smooth["gB"])
    assert abs(ga - smooth["ga"]) <= 2e-3 * abs(smooth["ga"])


def test_clamped_rollout_gradients_match_the_reference_in_aggregate(clamped):
    _, _, _, gv, gB, ga = _gpu_grads(clamped)
    ref = clamped["gv"]
    assert np.linalg.norm(gv - ref) <= 0.05 * np.linalg.norm(ref)
    assert np.median(np.abs(gv - ref)) <= 1e-3 * np.abs(ref).max()
    assert abs(gB - clamped["gB"]) <= 0.02 * abs(clamped["gB"])
    assert abs(ga - clamped["ga"]) <= 0.02 * abs(clamped["ga"])


def test_clamped_rollout_gradients_match_entry_by_entry_where_the_branch_is_stable(clamped):
    # The clamp makes some entries of dL/dv0 depend on exactly when a particle's density
    # crosses rho0, which FP32 and FP64 trajectories decide at different steps.  The FP64
    # reference itself tells which entries are insensitive: rerun it from initial
    # velocities perturbed by 1e-4 relative (three seeds); the entries that move by at most
    # 1e-3 of the largest in every rerun are stable, and there the GPU gradient must match
    # the reference entry by entry: 99 % of them within 2e-3 of the largest entry, every
    # one within 1e-2 (the FP32 trajectory departs from the FP64 one by more than the
    # perturbation, so a few stable entries still see a different crossing).
    R, v0 = clamped["R"], clamped["v0"].astype(np.float64)
    ref = clamped["gv"]
    mx = np.abs(ref).max()
    rng = np.random.default_rng(2024)
    dev = np.zeros(len(ref))
    for _ in range(3):
        vp = v0 * (1.0 + 1e-4 * rng.standard_normal(v0.shape))
        xT, rhoT, recs = R.forward(vp, B0, A0, STEPS)
        _, xbar, rhobar = centroid_density_loss(xT, rhoT, TARGET, 1000.0)
        gp = R.backward(recs, B0, A0, xT, xbar, rhobar)[0]
        dev = np.maximum(dev, np.abs(gp - ref).max(axis=1))
    stable = dev <= 1e-3 * mx
    assert stable.mean() > 0.8
    _, _, _, gv, _, _ = _gpu_grads(clamped)
    err = np.abs(gv[stable] - ref[stable]).max(axis=1)
    assert np.mean(err <= 2e-3 * mx) >= 0.99, np.quantile(err / mx, [0.5, 0.99, 1.0])
    assert err.max() <= 1e-2 * mx


@pytest.mark.parametrize("which", ["smooth", "clamped"])
def test_scalar_gradients_match_central_differences(which, request):
    case = request.getfixturevalue(which)
    R, v0 = case["R"], case["v0"]

    def loss(B, a):
        xT, rhoT, _ = R.forward(v0, B, a, STEPS, record=False)
        return centroid_density_loss(xT, rhoT, TARGET, 1000.0)[0]

    # the loss has kinks in the parameters even without the pressure clamp (the viscosity
    # acts on approaching pairs only and 4k particles x 100 steps hold many pairs near
    # v_ij . x_ij = 0): steps of 0.25 in B (exact in FP32) and 2^-16 in alpha stay clear
    # of them (larger steps in B drift by several per cent)
    fdB = (loss(B0 + 0.25, A0) - loss(B0 - 0.25, A0)) / 0.5
    ha = 2.0 ** -16
    fda = (loss(B0, A0 + ha) - loss(B0, A0 - ha)) / (2 * ha)
    _, _, _, _, gB, ga = _gpu_grads(case)
    tol = 2e-3 if which == "smooth" else 0.02
    assert abs(gB - fdB) <= tol * abs(fdB)
    assert abs(ga - fda) <= tol * abs(fda)


def test_backward_needs_a_forward_and_checkpoint_intervals_agree(smooth):
    sc, d, v0 = smooth["sc"], smooth["d"], torch.tensor(smooth["v0"], device="cuda")
    eng25 = diff.DiffEngine(d, sc.x, sc.xb, STEPS, ckpt_every=25)
    x, rho = eng25.forward(v0, B0, A0)
    gx = torch.full_like(x, 1e-3)
    g1 = eng25.backward(gx, None)
    with pytest.raises(Exception):
        eng25.backward(gx, None)
    x2, _ = smooth["eng"].forward(v0, B0, A0)
    assert torch.equal(x, x2)                                   # deterministic passes
    g2 = smooth["eng"].backward(gx, None)
    # per-particle gradients are bit-identical; the scalar ones are sums of CTA totals
    # added by atomics in arrival order, equal to rounding
    assert torch.equal(g1[0], g2[0])
    assert abs(g1[1] - g2[1]) <= 1e-12 * abs(g1[1]) and abs(g1[2] - g2[2]) <= 1e-12 * abs(g1[2])
