"""Seeded synthetic scenes and parameter sets for regional time stepping (RTS).

This module only lays particles out and lists parameter values.  It holds none of
the method's arithmetic (no kernel, no level thresholds, no integrator): both the
CUDA library and the CPU oracle receive exactly the arrays and numbers made here.

The paper's own scenes (dam breaks, a block dropped into a pool, stairs, a turbine;
Section 6, Figures 1, 4, 8-10) exist only as pictures, so the scenes below stand in
for them at the paper's scales (about 1M particles, spacing s = 0.01 m):

* ``wcsph_dam_break_8k``  - 20^3 column, s = 0.02 m, 0.8 x 0.4 x 0.4 m box
* ``wcsph_dam_break_1m``  - 100^3 column, s = 0.01 m, 4 x 2 x 2 m box
* ``pcisph_drop_1m``      - 200 x 200 x 25 pool + 30^3 cube 0.2 m above it,
                            s = 0.01 m, 2 x 2 x 1 m box

Fluid particles sit on the lattice points (i + 1/2) s of the box.  Static boundary
particles continue that lattice through every wall, face, edge and corner, in
``layers`` layers outside the box (Section 6 uses static boundary particles; the
paper does not give their layout).  The box is also passed as the container
(``wall_project``): a fluid particle that crosses a face is put back on it.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

WCSPH = 0
PCISPH = 1

MODE_REGIONAL = 0
MODE_GLOBAL_ADAPTIVE = 1
MODE_GLOBAL_CONSTANT = 2


@dataclasses.dataclass
class Scene:
    name: str
    x: np.ndarray          # (N, 3) float32 fluid positions
    v: np.ndarray          # (N, 3) float32 fluid velocities
    xb: np.ndarray         # (Nb, 3) float32 static boundary positions
    params: dict           # parameter values (see ``wcsph_params``/``pcisph_params``)
    box: tuple

    @property
    def n(self) -> int:
        return int(self.x.shape[0])

    @property
    def nb(self) -> int:
        return int(self.xb.shape[0])


def lattice(counts, s, offset=(0.0, 0.0, 0.0)):
    """Points offset + (i + 1/2) s for i in [0, counts) per axis, x fastest."""
    nx, ny, nz = counts
    iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    pts = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], axis=1).astype(np.float64)
    pts = (pts + 0.5) * s + np.asarray(offset, np.float64)
    return pts


def boundary_shell(box, s, layers=2):
    """Lattice points (i + 1/2) s, i in [-layers, n + layers), that lie outside the box."""
    n = [int(round(L / s)) for L in box]
    ax = [np.arange(-layers, k + layers) for k in n]
    iz, iy, ix = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    ix, iy, iz = ix.ravel(), iy.ravel(), iz.ravel()
    inside = (ix >= 0) & (ix < n[0]) & (iy >= 0) & (iy < n[1]) & (iz >= 0) & (iz < n[2])
    pts = np.stack([ix[~inside], iy[~inside], iz[~inside]], axis=1).astype(np.float64)
    return (pts + 0.5) * s


def grid_for_box(box, edge):
    """Block grid covering [-edge, L + edge] per axis (room for the boundary shell)."""
    dims = [int(math.ceil(L / edge - 1e-6)) + 2 for L in box]
    origin = [-edge, -edge, -edge]
    return origin, dims


def _f32(v):
    return float(np.float32(v))


def wcsph_params(s, box, dt_b, *, support_factor=2.0):
    """Parameter values for WCSPH (Becker & Teschner physics, Section 3.1 criteria).

    Kernel support r = 2 s (block edge = r, Section 3), cubic spline with h = r / 2.
    Level ladder dt_b * {1, 2, 4, 8}; beta_1 = inf, beta_n = 0.4 * 0.2^(n - 2).
    """
    r = support_factor * s
    origin, dims = grid_for_box(box, r)
    return dict(
        scheme=WCSPH, mode=MODE_REGIONAL, force_level=-1,
        spacing=s, support_r=r, block_edge=r,
        domain_min=origin, grid_dim=dims,
        rho0=1000.0, c_s=20.0, gamma=7.0, visc_alpha=0.05,
        gravity=[0.0, 0.0, -9.81],
        lambda_v=0.4, lambda_f=0.25, alpha=0.4,
        n_levels=4, level_mult=[1, 2, 4, 8],
        beta=[math.inf, 0.4, 0.08, 0.016],
        dt_b=dt_b, max_per_block=64,
        n_minor=4, eta=0.01, eta_T=0.0025, max_iters=20,
        max_global_iters=6, max_local_iters=3, expand_layers=4, r1_search_rings=2,
        clean_majors=10, short_minor=2,
        sched=[[3, 3, 3, 3], [2, 1, 2, 1], [2, 1, 1, 1], [2, 1, 1, 1]],
        refresh=[1, 2, 4, 4], max_neighbors=96,
        wall_project=1, wall_lo=[0.0, 0.0, 0.0], wall_hi=[float(L) for L in box],
        stale_bins=4,
    )


def pcisph_params(s, box, dt_b):
    """Parameter values for RTS-PCISPH (Sections 5.2-5.6, 6).

    r = 2 s, block edge 2.2 s (Section 5.6), regions n in {1,2,3,4} with
    dt_n = n dt_b, alpha = 1 and no sound-speed criterion (Section 3.1), N = 4 minor
    steps per major step (Section 5.2), density-error tolerance 1 %, eta_T = 0.25 %.
    """
    r = 2.0 * s
    edge = 2.2 * s
    origin, dims = grid_for_box(box, edge)
    return dict(
        scheme=PCISPH, mode=MODE_REGIONAL, force_level=-1,
        spacing=s, support_r=r, block_edge=edge,
        domain_min=origin, grid_dim=dims,
        rho0=1000.0, c_s=20.0, gamma=7.0, visc_alpha=0.05,
        gravity=[0.0, 0.0, -9.81],
        lambda_v=0.4, lambda_f=0.25, alpha=1.0,
        n_levels=4, level_mult=[1, 2, 3, 4],
        beta=[math.inf, 0.4, 0.08, 0.016],
        dt_b=dt_b, max_per_block=64,
        n_minor=4, eta=0.01, eta_T=0.0025, max_iters=20,
        max_global_iters=6, max_local_iters=3, expand_layers=4, r1_search_rings=2,
        clean_majors=10, short_minor=2,
        sched=[[3, 3, 3, 3], [2, 1, 2, 1], [2, 1, 1, 1], [2, 1, 1, 1]],
        refresh=[1, 2, 4, 4], max_neighbors=96,
        wall_project=1, wall_lo=[0.0, 0.0, 0.0], wall_hi=[float(L) for L in box],
    )


def _finish(name, fluid, box, s, params, seed, jitter, layers=2):
    rng = np.random.Generator(np.random.PCG64(seed))
    if jitter > 0:
        fluid = fluid + rng.uniform(-jitter, jitter, size=fluid.shape)
    xb = boundary_shell(box, s, layers)
    return Scene(
        name=name,
        x=np.ascontiguousarray(fluid, np.float32),
        v=np.zeros((fluid.shape[0], 3), np.float32),
        xb=np.ascontiguousarray(xb, np.float32),
        params=params, box=tuple(box),
    )


def dam_break(counts, s, box, dt_b, *, jitter=0.0, seed=1234, name="dam_break"):
    """A column of counts[0] x counts[1] x counts[2] fluid particles in the box corner."""
    fluid = lattice(counts, s)
    return _finish(name, fluid, box, s, wcsph_params(s, box, dt_b), seed, jitter)


def wcsph_dam_break_8k(seed=1234):
    """20^3 = 8,000 particles, s = 0.02 m, 0.8 x 0.4 x 0.4 m box, jitter +-1e-4 m."""
    return dam_break((20, 20, 20), 0.02, (0.8, 0.4, 0.4), 1e-4, jitter=1e-4, seed=seed,
                     name="wcsph_dam_break_8k")


def wcsph_dam_break_8k_wide_kernel(seed=1234):
    """The 8k dam break under the literal reading of the kernel size: h = 2 s, support
    r = 4 s (block edge r), boundary of 4 layers; blocks hold 64 particles at rest and a
    particle about 270 neighbours (max_per_block 160, max_neighbors 512)."""
    s, box = 0.02, (0.8, 0.4, 0.4)
    p = wcsph_params(s, box, 1e-4, support_factor=4.0)
    p.update(max_per_block=160, max_neighbors=512)
    fluid = lattice((20, 20, 20), s)
    return _finish("wcsph_dam_break_8k_wide_kernel", fluid, box, s, p, seed, 1e-4, layers=4)


def wcsph_dam_break_1m(seed=1234):
    """100^3 = 1,000,000 particles, s = 0.01 m, 4 x 2 x 2 m box, dt_b = 5e-5 s."""
    return dam_break((100, 100, 100), 0.01, (4.0, 2.0, 2.0), 5e-5, jitter=0.0, seed=seed,
                     name="wcsph_dam_break_1m")


def diff_dam_break_250k(seed=1234):
    """Differentiable rollout: 100 x 50 x 50 = 250,000 particles, s = 0.01 m, in the corner
    of a 2 x 1 x 1 m tank, dt_b = 5e-5 s."""
    return dam_break((100, 50, 50), 0.01, (2.0, 1.0, 1.0), 5e-5, jitter=0.0, seed=seed,
                     name="diff_dam_break_250k")


def diff_dam_break_4k(seed=1234):
    """The same setup at 16^3 = 4,096 particles (gradient checks), 0.32 x 0.16 x 0.32 m,
    jittered +-1e-4 m."""
    return dam_break((16, 16, 16), 0.01, (0.32, 0.16, 0.32), 5e-5, jitter=1e-4, seed=seed,
                     name="diff_dam_break_4k")


def seeded_velocities(n, seed=777, scale=0.5):
    """A smooth-ish seeded initial velocity field (normal components, m/s)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return (scale * rng.standard_normal((n, 3))).astype(np.float32)


def pool_drop(pool_counts, cube_side, gap, s, box, dt_b, *, jitter=0.0, seed=1234, name="pool_drop"):
    """A resting pool filling the box floor plus a cube of fluid centred above it."""
    pool = lattice(pool_counts, s)
    surface = pool_counts[2] * s
    c0 = [0.5 * box[0] - 0.5 * cube_side * s, 0.5 * box[1] - 0.5 * cube_side * s, surface + gap]
    cube = lattice((cube_side, cube_side, cube_side), s, offset=c0)
    fluid = np.concatenate([pool, cube], axis=0)
    return _finish(name, fluid, box, s, pcisph_params(s, box, dt_b), seed, jitter)


def pcisph_drop_1m(seed=1234):
    """200 x 200 x 25 pool + 30^3 cube 0.2 m above, s = 0.01 m, 2 x 2 x 1 m box."""
    return pool_drop((200, 200, 25), 30, 0.2, 0.01, (2.0, 2.0, 1.0), 3.5e-4, seed=seed,
                     name="pcisph_drop_1m")


def pcisph_drop_small(seed=1234):
    """32 x 32 x 8 pool + 8^3 cube 0.06 m above, s = 0.01 m, 0.32 x 0.32 x 0.3 m box."""
    return pool_drop((32, 32, 8), 8, 0.06, 0.01, (0.32, 0.32, 0.3), 3.5e-4, jitter=2e-5,
                     seed=seed, name="pcisph_drop_small")


def perturbed_state(scene, seed=777, *, vmax=40.0, amax=6e5, frac_levels=None):
    """Seeded dynamic state for same-input-state parity tests.

    Velocities and held accelerations get log-uniform magnitudes spanning the
    level thresholds of the scene's parameters, random directions, and a
    spatially smooth component so that whole blocks share a scale; validity
    counters and particle levels are random within the ladder.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    n = scene.n
    x = scene.x.astype(np.float64)
    lo = x.min(axis=0)
    hi = x.max(axis=0) + 1e-9
    u = (x - lo) / (hi - lo)
    # smooth field in [0, 1] so neighbouring particles have similar magnitudes
    smooth = 0.5 + 0.5 * np.sin(6.1 * u[:, 0] + 2.3) * np.cos(4.7 * u[:, 1] - 0.4) * np.sin(3.3 * u[:, 2] + 1.1)
    lv = np.log(1e-3) + (np.log(vmax) - np.log(1e-3)) * np.clip(smooth + 0.08 * rng.standard_normal(n), 0, 1)
    la = np.log(1.0) + (np.log(amax) - np.log(1.0)) * np.clip(smooth + 0.08 * rng.standard_normal(n), 0, 1) ** 2
    dv = rng.standard_normal((n, 3))
    dv /= np.linalg.norm(dv, axis=1, keepdims=True)
    da = rng.standard_normal((n, 3))
    da /= np.linalg.norm(da, axis=1, keepdims=True)
    v = (np.exp(lv)[:, None] * dv).astype(np.float32)
    a = (np.exp(la)[:, None] * da).astype(np.float32)
    nl = scene.params["n_levels"]
    level = rng.integers(0, nl, size=n).astype(np.int32)
    mult = np.asarray(scene.params["level_mult"], np.int32)
    validity = (rng.integers(0, 8, size=n) % np.maximum(mult[level], 1) + 1).astype(np.int32)
    klast = rng.integers(0, 8, size=n).astype(np.int32)
    rho = (scene.params["rho0"] * (1.0 + 0.01 * rng.uniform(-1, 1, size=n))).astype(np.float32)
    prs = np.maximum(0.0, 2000.0 * rng.uniform(-0.2, 1.0, size=n)).astype(np.float32)
    return dict(v=v, a=a, level=level, validity=validity, klast=klast, rho=rho, p=prs)


# ------------------------------------------------------------ batched scenes ---

@dataclasses.dataclass
class Batch:
    """Independent scenes advanced together: shared parameters, per-scene grids and
    containers, particles concatenated scene after scene."""
    name: str
    scenes: list
    params: dict
    desc: list             # per scene: n_fluid, n_boundary, domain_min, grid_dim, wall_lo, wall_hi
    x: np.ndarray
    v: np.ndarray
    xb: np.ndarray

    @property
    def n(self) -> int:
        return int(self.x.shape[0])

    @property
    def nb(self) -> int:
        return int(self.xb.shape[0])


def make_batch(scenes_list, name="batch") -> Batch:
    """Concatenate scenes that share every parameter but their grid and container."""
    p0 = dict(scenes_list[0].params)
    desc = []
    for sc in scenes_list:
        p = sc.params
        for k, val in p.items():
            if k not in ("domain_min", "grid_dim", "wall_lo", "wall_hi") and val != p0[k]:
                raise ValueError(f"scene {sc.name} differs from the batch in {k}")
        desc.append(dict(n_fluid=sc.n, n_boundary=sc.nb, domain_min=list(p["domain_min"]),
                         grid_dim=list(p["grid_dim"]), wall_lo=list(p["wall_lo"]),
                         wall_hi=list(p["wall_hi"])))
    x = np.ascontiguousarray(np.concatenate([sc.x for sc in scenes_list]), np.float32)
    v = np.ascontiguousarray(np.concatenate([sc.v for sc in scenes_list]), np.float32)
    xb = np.ascontiguousarray(np.concatenate([sc.xb for sc in scenes_list]), np.float32)
    return Batch(name=name, scenes=list(scenes_list), params=p0, desc=desc, x=x, v=v, xb=xb)


def batch_counts(n_scenes=64, seed=4321, lo=1.0e4, hi=2.0e5):
    """Target particle counts drawn log-uniformly in [lo, hi] (seeded)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.round(np.exp(rng.uniform(np.log(lo), np.log(hi), n_scenes))).astype(np.int64)


def batch_member(i, n_target, s=0.01, dt_b=3.5e-4):
    """Scene i of a batch: even i a dam break, a column of ceil(N^(1/3))^3 particles in the
    corner of a (4, 2, 2) x column-side tank; odd i the 1M pool drop scaled to about N
    particles (pool a x a x a/8, cube 0.15 a on a side, dropped from 0.1 a s above the
    pool, tank a x a x a/2 spacings).  PCISPH parameters of the 1M pool drop."""
    if i % 2 == 0:
        c = int(math.ceil(n_target ** (1.0 / 3.0) - 1e-9))
        box = (4 * c * s, 2 * c * s, 2 * c * s)
        fluid = lattice((c, c, c), s)
        name = f"dam_break_{c}^3"
    else:
        a = max(8, int(round((8.0 * n_target / (1.0 + 8 * 0.15 ** 3)) ** (1.0 / 3.0))))
        hz = max(2, int(round(a / 8)))
        k = max(2, int(round(0.15 * a)))
        box = (a * s, a * s, int(round(a / 2)) * s)
        pool = lattice((a, a, hz), s)
        c0 = [0.5 * box[0] - 0.5 * k * s, 0.5 * box[1] - 0.5 * k * s, hz * s + 0.1 * a * s]
        cube = lattice((k, k, k), s, offset=c0)
        fluid = np.concatenate([pool, cube], axis=0)
        name = f"pool_{a}x{a}x{hz}_drop_{k}^3"
    return _finish(f"batch{i}_{name}", fluid, box, s, pcisph_params(s, box, dt_b), 1234, 0.0)


def pcisph_batch(n_scenes=64, seed=4321, lo=1.0e4, hi=2.0e5, s=0.01, dt_b=3.5e-4) -> Batch:
    """The batched workload: n_scenes dam breaks and pool drops with particle counts
    drawn log-uniformly in [lo, hi] (seed 4321)."""
    counts = batch_counts(n_scenes, seed, lo, hi)
    members = [batch_member(i, int(n), s, dt_b) for i, n in enumerate(counts)]
    return make_batch(members, name=f"pcisph_batch_{n_scenes}")


def pcisph_batch_small() -> Batch:
    """Three small scenes for parity tests: the small pool drop, a 12^3 dam break and a
    16 x 16 x 2 pool with a 3^3 drop (about 12k particles in all)."""
    return make_batch([pcisph_drop_small(), batch_member(0, 1728), batch_member(1, 600)],
                      name="pcisph_batch_small")
