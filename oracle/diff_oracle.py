"""FP64 reference gradient of a WCSPH rollout (TEST INFRASTRUCTURE ONLY).

Only the tests and bench.py's baseline leg use this module; the product path never does.

The rollout is global constant stepping at dt_b (every particle active every step) with
the Serna predictor-corrector of Section 4.1 and the WCSPH physics of the oracle: priming
evaluation a_0 = A(x_0, v_0); per step x~ = x + v dt + a dt^2 / 2, v~ = v + a dt, the
container correction, a' = A(x~, v~), x <- x~ + (a' - a) dt^2 / 6, v <- v~ + (a' - a) dt / 2,
a <- a'.  The forward is the C oracle itself (orc_wcsph_global_step); every step's
evaluation point is recorded.  The final density rho_T = rho(x_T) is a summation at x_T.

The backward is reverse-mode differentiation written out from those definitions (no
automatic differentiation): A(x, v) = g + sum over neighbour pairs of
-m (p_i/rho_i^2 + p_j/rho_j^2 + Pi_ij) grad W_ij, with rho a kernel sum, p the Tait
equation (stiffness B, clamped at 0) and Pi the artificial viscosity (coefficient alpha).
For an ordered pair (i, j) of i's list the scalar S = P_i + P_j + Pi_ij and G = W'(r)/r x_ij
enter a_i with -m S G and a_j with +m S G, so with w = abar_i - abar_j:
    Sbar = -m G . w,   Gbar = -m S w.
Pass A gathers Pbar_i = sum Sbar and the viscosity's density terms, giving rhobar_i,
Bbar and alphabar; pass B gathers the position and velocity adjoints of every pair
(kernel gradient, density sums of both particles, viscosity).  Boundary particles are
fixed, have no pressure and lend the fluid particle its density in the viscosity.

Gradients are pinned against central finite differences of the same forward in FP64.
"""
from __future__ import annotations

import math

import numpy as np

from . import make_params, WCSPH, neighbors_grid, density as _density


def spline(r, h):
    """Cubic spline W(r), W'(r), W''(r) for support 2h (sigma = 1 / (pi h^3))."""
    sigma = 1.0 / (math.pi * h ** 3)
    q = r / h
    t = np.clip(2.0 - q, 0.0, None)
    inner = q < 1.0
    outer = (q >= 1.0) & (q < 2.0)
    W = np.where(inner, sigma * (1.0 - 1.5 * q * q + 0.75 * q ** 3),
                 np.where(outer, 0.25 * sigma * t ** 3, 0.0))
    dW = np.where(inner, sigma / h * (-3.0 * q + 2.25 * q * q),
                  np.where(outer, -0.75 * sigma / h * t * t, 0.0))
    d2W = np.where(inner, sigma / h ** 2 * (-3.0 + 4.5 * q),
                   np.where(outer, 1.5 * sigma / h ** 2 * t, 0.0))
    return W, dW, d2W


def _pairs(P, x, xb):
    off, idx = neighbors_grid(P, x, xb)
    n = x.shape[0]
    I = np.repeat(np.arange(n), np.diff(off))
    J = idx.astype(np.int64)
    return I, J


def _add3(n, I, vec):
    out = np.zeros((n, 3))
    for k in range(3):
        out[:, k] = np.bincount(I, vec[:, k], minlength=n)
    return out


class DiffRollout:
    """Loss gradient of a global-stepping WCSPH rollout with respect to the initial
    velocities, the Tait stiffness B and the viscosity coefficient alpha."""

    def __init__(self, params: dict, x0, xb):
        self.d = dict(params)
        self.x0 = np.asarray(x0, np.float64)
        self.xb = np.asarray(xb, np.float64)

    def P(self, B, alpha):
        d = dict(self.d, mode=2, tait_B=float(B), visc_alpha=float(alpha))
        return make_params(d)

    # ------------------------------------------------------------------ forward ---
    def forward(self, v0, B, alpha, n_steps, record=True):
        P = self.P(B, alpha)
        S = WCSPH(P, self.x0, np.asarray(v0, np.float64), self.xb)
        S.evaluate()
        recs = [dict(x=S.x.copy(), v=S.v.copy(), rho=S.rho.copy(), p=S.p.copy())] if record else None
        dt = P.dt_b
        lo = np.array([P.wall_lo[k] for k in range(3)])
        hi = np.array([P.wall_hi[k] for k in range(3)])
        for _ in range(n_steps):
            if record:
                xk, vk, ak = S.x.copy(), S.v.copy(), S.a.copy()
            if S.global_step() != 1:
                raise RuntimeError("global constant stepping advanced more than one substep")
            if record:
                xt = xk + vk * dt + ak * dt * dt / 2.0
                vt = vk + ak * dt
                mx = np.zeros_like(xt, bool)
                mv = np.zeros_like(vt, bool)
                if P.wall_project:
                    below, above = xt < lo, xt > hi
                    mx = below | above
                    mv = (below & (vt < 0.0)) | (above & (vt > 0.0))
                    xt = np.where(below, lo, np.where(above, hi, xt))
                    vt = np.where(mv, 0.0, vt)
                recs.append(dict(xt=xt, vt=vt, mx=mx, mv=mv, rho=S.rho.copy(), p=S.p.copy()))
        xT = S.x.copy()
        rhoT = _density(P, xT, self.xb)[0]
        return xT, rhoT, recs

    # -------------------------------------------------------------- evaluation ---
    def eval_adjoint(self, P, x, v, rho, p, abar):
        """Adjoints of A(x, v; B, alpha) for the output adjoint abar."""
        n = x.shape[0]
        h = 0.5 * P.r
        m = P.rho0 * P.s ** 3
        B = P.tait_B if P.tait_B > 0 else P.c_s ** 2 * P.rho0 / P.gamma
        K = 2.0 * P.visc_alpha * h * P.c_s
        I, J = _pairs(P, x, self.xb)
        fl = J < n
        Jf = np.where(fl, J, 0)
        Jb = np.where(fl, 0, J - n)
        xj = np.where(fl[:, None], x[Jf], self.xb[Jb])
        vj = np.where(fl[:, None], v[Jf], 0.0)
        rj = np.where(fl, rho[Jf], rho[I])
        Pj = np.where(fl, p[Jf] / rho[Jf] ** 2, 0.0)
        xij = x[I] - xj
        d2 = (xij * xij).sum(1)
        r = np.sqrt(d2)
        pos = r > 0.0
        rs = np.where(pos, r, 1.0)
        _, dW, d2W = spline(r, h)
        f = np.where(pos, dW / rs, 0.0)
        G = f[:, None] * xij
        Pi = p[I] / rho[I] ** 2
        vij = v[I] - vj
        u = (vij * xij).sum(1)
        D = d2 + 0.01 * h * h
        nu = K / (rho[I] + rj)
        visc = u < 0.0
        Pv = np.where(visc, -nu * u / D, 0.0)
        S = Pi + Pj + Pv
        w = abar[I] - np.where(fl[:, None], abar[Jf], 0.0)
        Sbar = -m * (G * w).sum(1)
        # pass A: rhobar, Bbar, alphabar
        Pbar = np.bincount(I, Sbar, minlength=n)
        g = P.gamma
        ratio = rho / P.rho0
        posp = (p > 0.0) | bool(P.tait_no_clamp)
        dPdrho = np.where(posp, g * B * ratio ** (g - 1.0) / P.rho0 / rho ** 2 - 2.0 * p / rho ** 3, 0.0)
        dPdB = np.where(posp, (ratio ** g - 1.0) / rho ** 2, 0.0)
        # d Pi / d rho_i: -Pi / (rho_i + rho_j); a boundary neighbour lends rho_i itself
        dPv = np.where(fl, -Pv / (rho[I] + rj), -Pv / rho[I])
        rhobar = Pbar * dPdrho + np.bincount(I, Sbar * dPv, minlength=n)
        Bbar = float((Pbar * dPdB).sum())
        alpha_terms = np.where(fl, 0.5, 1.0) * Sbar * Pv
        alphabar = float(alpha_terms.sum() / P.visc_alpha) if P.visc_alpha > 0 else 0.0
        # pass B: position and velocity adjoints of every pair
        Gbar = (-m * S)[:, None] * w
        xg = (xij * Gbar).sum(1)
        coef = np.where(pos, (d2W - f) / np.where(pos, d2, 1.0), 0.0)
        X = f[:, None] * Gbar + (coef * xg)[:, None] * xij
        rb = rhobar[I] + np.where(fl, rhobar[Jf], 0.0)
        X += (rb * m * f)[:, None] * xij
        ubar = np.where(visc, Sbar * (-nu / D), 0.0)
        r2bar = np.where(visc, Sbar * nu * u / (D * D), 0.0)
        X += ubar[:, None] * vij + (2.0 * r2bar)[:, None] * xij
        xbar = _add3(n, I, X)
        vbar = _add3(n, I, ubar[:, None] * xij)
        return xbar, vbar, Bbar, alphabar

    def density_adjoint(self, P, x, rhobar):
        """Adjoint of the summation density rho(x) for the output adjoint rhobar."""
        n = x.shape[0]
        h = 0.5 * P.r
        m = P.rho0 * P.s ** 3
        I, J = _pairs(P, x, self.xb)
        fl = J < n
        Jf = np.where(fl, J, 0)
        xj = np.where(fl[:, None], x[Jf], self.xb[np.where(fl, 0, J - n)])
        xij = x[I] - xj
        r = np.sqrt((xij * xij).sum(1))
        pos = r > 0.0
        _, dW, _ = spline(r, h)
        f = np.where(pos, dW / np.where(pos, r, 1.0), 0.0)
        rb = rhobar[I] + np.where(fl, rhobar[Jf], 0.0)
        return _add3(n, I, (rb * m * f)[:, None] * xij)

    # ----------------------------------------------------------------- backward ---
    def backward(self, recs, B, alpha, xT, xbar_T, rhobar_T):
        """d loss / d (v0, B, alpha) from the recorded forward and the adjoints of x_T
        and rho_T."""
        P = self.P(B, alpha)
        dt = P.dt_b
        c1, c2 = dt * dt / 6.0, dt / 2.0
        xbar = xbar_T + self.density_adjoint(P, xT, rhobar_T)
        vbar = np.zeros_like(xbar)
        abar = np.zeros_like(xbar)
        Bbar = alphabar = 0.0
        for rec in reversed(recs[1:]):
            anew_bar = abar + c1 * xbar + c2 * vbar
            ak_bar = -c1 * xbar - c2 * vbar
            xt_bar, vt_bar = xbar.copy(), vbar.copy()
            ex, ev, eB, ea = self.eval_adjoint(P, rec["xt"], rec["vt"], rec["rho"], rec["p"], anew_bar)
            xt_bar += ex
            vt_bar += ev
            Bbar += eB
            alphabar += ea
            xt_bar[rec["mx"]] = 0.0
            vt_bar[rec["mv"]] = 0.0
            xbar = xt_bar
            vbar = xt_bar * dt + vt_bar
            abar = ak_bar + xt_bar * dt * dt / 2.0 + vt_bar * dt
        r0 = recs[0]
        ex, ev, eB, ea = self.eval_adjoint(P, r0["x"], r0["v"], r0["rho"], r0["p"], abar)
        return vbar + ev, Bbar + eB, alphabar + ea


def centroid_density_loss(xT, rhoT, target, rho0):
    """|mean(x_T) - target|^2 + mean |rho_T - rho0| / rho0 and its adjoints."""
    n = xT.shape[0]
    c = xT.mean(0) - np.asarray(target, np.float64)
    L = float((c * c).sum() + np.abs(rhoT - rho0).mean() / rho0)
    xbar = np.broadcast_to(2.0 * c / n, xT.shape).copy()
    rhobar = np.sign(rhoT - rho0) / (n * rho0)
    return L, xbar, rhobar
