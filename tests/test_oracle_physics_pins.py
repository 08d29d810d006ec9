"""Magnitude pins of the oracle's SPH physics (WCSPH and PCISPH), fixed by the mathematics.

The paper cites its physics (Becker & Teschner WCSPH, Solenthaler & Pajarola PCISPH)
without restating it, so these pins come from identities of the textbook definitions,
not from the oracle's own expressions:

* the Tait equation of state vanishes at rest density and its slope there is the
  squared sound speed (dp/drho = B gamma / rho0 = c^2), its curvature (gamma - 1) c^2 / rho0;
* on a full cubic lattice a linear pressure field p = p0 + G.x gives, by cubic symmetry,
  the pressure acceleration -(G / rho0) * C with C a closed-form shell sum (1.02004 at
  h = s) that tends to the continuum value 1 as h / s grows;
* artificial viscosity vanishes for rigid translation and rotation, and for a uniform
  compression v = -k x it has a closed form at a free surface (a half-space stencil);
* a particle above a floor of static boundary particles feels -m (p_i / rho_i^2) grad W
  from them (the energy-consistent reading), half of what fluid neighbours of equal
  pressure exert, and viscosity with rho_b = rho_i, v_b = 0.

The half-space closed forms: with h = s, a particle on a plane with a full lattice
layer below it has 1 neighbour below at s, 4 at sqrt2 s and 4 at sqrt3 s (the one at 2 s
is a tie the predicate excludes, and W' vanishes there); in-plane neighbours cancel.
With W'(q s) = -0.75 (2 - q)^2 / (pi s^4) for 1 <= q < 2 the sums below are exact.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2009_14514_gb300 import scenes

S_DYADIC = 1.0 / 64          # every lattice coordinate exact in FP32 and FP64
BELOW = ((1.0, 1), (math.sqrt(2.0), 4), (math.sqrt(3.0), 4))   # (q, count) below a surface


def _box_params(counts, s=S_DYADIC, **over):
    sc = scenes.dam_break(counts, s, tuple(c * s for c in counts), 1e-4)
    d = dict(sc.params)
    d.update(over)
    return sc, O.make_params(d)


def _lattice_index(x, s=S_DYADIC):
    return np.round(np.asarray(x, np.float64) / s - 0.5).astype(int)


def _shell_coefficient(hs):
    """(1/3) sum over lattice offsets d (units of s) with 0 < |d| < 2 hs of -|d| W'(|d|) s^3
    for the M4 spline with h = hs s; written here from the spline's definition."""
    R = 2 * hs
    o = np.arange(-R, R + 1)
    X, Y, Z = np.meshgrid(o, o, o, indexing="ij")
    d = np.sqrt(X ** 2 + Y ** 2 + Z ** 2).ravel()
    d = d[(d > 0) & (d < 2 * hs)]
    q = d / hs
    g = np.where(q < 1, -3 * q + 2.25 * q * q, -0.75 * (2 - q) ** 2) / math.pi   # h^4 W'
    return float(-np.sum(d * g) / hs ** 4 / 3.0)


# ------------------------------------------------------------------- Tait EOS ---

def test_tait_vanishes_at_rest_and_its_slope_is_the_squared_sound_speed():
    sc = scenes.wcsph_dam_break_8k()
    P = O.make_params(dict(sc.params, tait_no_clamp=1))
    rho0, c, gamma = P.rho0, P.c_s, P.gamma
    assert O.tait(P, rho0) == 0.0
    e = 0.1
    slope = (O.tait(P, rho0 + e) - O.tait(P, rho0 - e)) / (2 * e)
    assert slope == pytest.approx(c * c, rel=1e-6)
    e = 1.0
    curv = (O.tait(P, rho0 + e) - 2 * O.tait(P, rho0) + O.tait(P, rho0 - e)) / (e * e)
    assert curv == pytest.approx((gamma - 1.0) * c * c / rho0, rel=1e-5)
    # the default clamps negative pressure (free surface) and keeps compression
    Pc = O.make_params(sc.params)
    assert O.tait(Pc, rho0 - 1.0) == 0.0
    assert O.tait(Pc, rho0 + 1.0) == O.tait(P, rho0 + 1.0) > 0.0
    # a given stiffness B replaces c^2 rho0 / gamma: slope B gamma / rho0
    Pb = O.make_params(dict(sc.params, tait_no_clamp=1, tait_B=80000.0))
    slope = (O.tait(Pb, rho0 + 0.1) - O.tait(Pb, rho0 - 0.1)) / 0.2
    assert slope == pytest.approx(80000.0 * gamma / rho0, rel=1e-6)


# --------------------------------------------------- pressure-force magnitude ---

def _linear_field_case(counts, hs=1):
    s = S_DYADIC
    sc, P = _box_params(counts, gravity=[0.0, 0.0, 0.0],
                        support_r=2.0 * hs * s, block_edge=2.0 * hs * s)
    x = sc.x.astype(np.float64)
    G = np.array([3000.0, -2000.0, 5000.0])
    prs = 1.0e4 + x @ G
    rho = np.full(sc.n, P.rho0)
    idx = _lattice_index(x)
    m = 2 * hs
    inner = np.all((idx >= m) & (idx < np.asarray(counts) - m), axis=1)
    return sc, P, G, prs, rho, inner


@pytest.mark.parametrize("scheme", ["wcsph", "pcisph"])
def test_pressure_force_of_a_linear_field_on_the_lattice(scheme):
    sc, P, G, prs, rho, inner = _linear_field_case((10, 10, 10))
    if scheme == "wcsph":
        a = O.accel(P, sc.x, np.zeros((sc.n, 3)), rho, prs, np.zeros((0, 3)))
    else:
        a = O.pcisph_pressure_accel(P, sc.x, prs, rho, np.zeros((0, 3)))
    C = 0.25 / math.pi * (6.0 + 12.0 * math.sqrt(2.0) * (2.0 - math.sqrt(2.0)) ** 2
                          + 8.0 * math.sqrt(3.0) * (2.0 - math.sqrt(3.0)) ** 2)
    assert C == pytest.approx(_shell_coefficient(1), rel=1e-14)
    expect = -(G / P.rho0) * C
    assert inner.sum() == 216
    err = np.abs(a[inner] - expect).max() / np.abs(expect).max()
    assert err < 1e-12


def test_pressure_force_approaches_minus_grad_p_over_rho_as_the_kernel_widens():
    # h = 2 s (support 4 s, about 250 neighbours): the lattice sum is within 1e-4 of the
    # continuum -grad p / rho0, against 2 % at h = s
    sc, P, G, prs, rho, inner = _linear_field_case((14, 14, 14), hs=2)
    a = O.accel(P, sc.x, np.zeros((sc.n, 3)), rho, prs, np.zeros((0, 3)))
    C = _shell_coefficient(2)
    assert abs(C - 1.0) < 1e-4 < abs(_shell_coefficient(1) - 1.0)
    expect = -(G / P.rho0) * C
    assert inner.sum() == 6 ** 3
    assert np.abs(a[inner] - expect).max() / np.abs(expect).max() < 1e-12


# ------------------------------------------------------------------ viscosity ---

def _surface_case():
    # a 12 x 12 x 6 lattice block; the probe particles are the top layer's interior ones
    sc, P = _box_params((12, 12, 6), gravity=[0.0, 0.0, 0.0])
    x = sc.x.astype(np.float64)
    idx = _lattice_index(x)
    top = (idx[:, 2] == 5) & np.all((idx[:, :2] >= 2) & (idx[:, :2] <= 9), axis=1)
    return sc, P, x, top


@pytest.mark.parametrize("scheme", ["wcsph", "pcisph"])
def test_viscosity_vanishes_for_rigid_motion(scheme):
    sc, P, x, top = _surface_case()
    zero = np.zeros(sc.n)
    rho = np.full(sc.n, P.rho0)

    def acc(v):
        if scheme == "wcsph":
            return O.accel(P, sc.x, v, rho, zero, np.zeros((0, 3)))
        return O.pcisph_nonpressure_accel(P, sc.x, v, np.zeros((0, 3)))

    v_tr = np.tile([0.7, -1.1, 0.4], (sc.n, 1))
    assert np.all(acc(v_tr) == 0.0)
    w = np.array([0.3, -0.8, 1.7])
    c = x.mean(axis=0)
    v_rot = np.cross(w, x - c)
    a_rot = acc(v_rot)
    # exact in exact arithmetic; rounding of v_ij . x_ij leaves at most ~1e-14 of the
    # compression case's magnitude
    assert np.abs(a_rot).max() < 1e-9


@pytest.mark.parametrize("scheme", ["wcsph", "pcisph"])
def test_viscosity_of_a_uniform_compression_at_a_free_surface(scheme):
    # v = -k x: v_ij . x_ij = -k d^2 < 0 for every pair, Pi = nu k d^2 / (d^2 + 0.01 h^2),
    # nu = alpha h c / rho0.  In the top layer only the neighbours below survive the x, y
    # symmetry: a_z = alpha c k (0.75 / pi) sum_below q (2 - q)^2 / (q^2 + 0.01)
    # (independent of s; m nu = alpha c s^4), a_x = a_y = 0.
    sc, P, x, top = _surface_case()
    k = 2.5
    v = -k * x
    rho = np.full(sc.n, P.rho0)
    if scheme == "wcsph":
        a = O.accel(P, sc.x, v, rho, np.zeros(sc.n), np.zeros((0, 3)))
    else:
        a = O.pcisph_nonpressure_accel(P, sc.x, v, np.zeros((0, 3)))
    az = P.visc_alpha * P.c_s * k * 0.75 / math.pi * sum(
        cnt * q * (2 - q) ** 2 / (q * q + 0.01) for q, cnt in BELOW)
    assert top.sum() == 64
    np.testing.assert_allclose(a[top, 2], az, rtol=1e-12)
    assert np.abs(a[top, :2]).max() < 1e-12 * az
    # the bulk of a uniform compression cancels: interior particles feel no viscosity
    idx = _lattice_index(x)
    inner = np.all((idx >= 2) & (idx <= np.array([9, 9, 3])), axis=1)
    assert np.abs(a[inner]).max() < 1e-12 * az


# ------------------------------------------------------------ static boundary ---

def _particle_on_floor(rho_i):
    # one fluid particle at height s/2 above the tank floor of a 16 x 16 x 8 s tank, its
    # x, y in the middle: the 2-layer boundary shell below it is a full lattice floor
    s = S_DYADIC
    box = (16 * s, 16 * s, 8 * s)
    sc = scenes.dam_break((1, 1, 1), s, box, 1e-4)
    P = O.make_params(dict(sc.params, gravity=[0.0, 0.0, 0.0]))
    x = np.array([[7.5 * s, 7.5 * s, 0.5 * s]])
    return sc, P, x


def test_boundary_floor_pushes_with_the_fluid_pressure_once():
    # a_z = m (p_i / rho_i^2) (0.75 / (pi s^4)) sum_below (2 - q)^2 / q, m = rho0 s^3
    s = S_DYADIC
    rho_i, p_i = 1020.0, 3000.0
    sc, P, x = _particle_on_floor(rho_i)
    a = O.accel(P, x, np.zeros((1, 3)), [rho_i], [p_i], sc.xb)
    shell = sum(cnt * (2 - q) ** 2 / q for q, cnt in BELOW)
    az = P.rho0 * p_i / rho_i ** 2 * 0.75 / (math.pi * s) * shell
    assert a[0, 2] == pytest.approx(az, rel=1e-12)
    assert abs(a[0, 0]) < 1e-12 * az and abs(a[0, 1]) < 1e-12 * az
    # the same floor made of fluid particles of equal pressure and density pushes twice
    # as hard (symmetric p_i / rho_i^2 + p_j / rho_j^2)
    xb = sc.xb.astype(np.float64)
    floor = xb[np.abs(xb[:, 2] + 0.5 * s) < 1e-12]
    xf = np.vstack([x, floor])
    nf = len(xf)
    af = O.accel(P, xf, np.zeros((nf, 3)), np.full(nf, rho_i), np.full(nf, p_i), np.zeros((0, 3)))
    assert af[0, 2] == pytest.approx(2.0 * az, rel=1e-12)


def test_boundary_floor_viscosity_uses_the_fluid_density_and_zero_velocity():
    # approaching the floor at speed u: Pi = nu u s / (d^2 + 0.01 h^2), nu = alpha h c / rho_i
    # (rho_b = rho_i), so a_z = (rho0 / rho_i) alpha c u (0.75 / (pi s))
    # sum_below (2 - q)^2 / (q (q^2 + 0.01)); moving away: no viscosity
    s = S_DYADIC
    rho_i, u = 1020.0, 0.8
    sc, P, x = _particle_on_floor(rho_i)
    a = O.accel(P, x, np.array([[0.0, 0.0, -u]]), [rho_i], [0.0], sc.xb)
    shell = sum(cnt * (2 - q) ** 2 / (q * (q * q + 0.01)) for q, cnt in BELOW)
    az = P.rho0 / rho_i * P.visc_alpha * P.c_s * u * 0.75 / (math.pi * s) * shell
    assert a[0, 2] == pytest.approx(az, rel=1e-12)
    a = O.accel(P, x, np.array([[0.0, 0.0, u]]), [rho_i], [0.0], sc.xb)
    assert np.all(a == 0.0)
