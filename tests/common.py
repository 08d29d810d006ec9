"""Shared helpers of the GPU parity tests: the same seeded input state goes to the CUDA
library (through the C ABI) and to the oracle."""
import numpy as np

import oracle as O
from paper_2009_14514_gb300 import rts, scenes

# Tolerances (the benchmark spec): density 1e-4 relative, forces 1e-3 of the max-norm.
RHO_RTOL = 1e-4
ACC_FRAC = 1e-3


def params(scene, **over):
    d = dict(scene.params)
    d.update(over)
    return d


def gpu_ctx(scene, d=None, x=None, v=None):
    d = d or scene.params
    return rts.rts_init(d, scene.x if x is None else x, scene.v if v is None else v, scene.xb)


def oracle_state(scene, d, st, k=0, primed=False):
    P = O.make_params(d)
    return O.WCSPH(P, st["x"], st["v"], scene.xb, a=st.get("a"), rho=st.get("rho"),
                   p=st.get("p"), klast=st.get("klast"), validity=st.get("validity"),
                   level=st.get("level"), k=k, primed=primed)


def dynamic_state(scene, seed=777, vmax=None, amax=None):
    """Positions of the scene plus a seeded dynamic state spanning the level thresholds."""
    P = O.make_params(scene.params)
    vthr2, athr2, _ = O.level_thresholds(P)
    vt = np.sqrt(vthr2[1:])
    at = np.sqrt(athr2)
    vmax = vmax or float(vt[0] * 1.3)
    amax = amax or float(at[0] * 1.3)
    st = scenes.perturbed_state(scene, seed, vmax=vmax, amax=amax)
    st["x"] = scene.x.copy()
    return st


def ulp32(a):
    return np.spacing(np.abs(a).astype(np.float32)).astype(np.float64)


def max_norm(a):
    return float(np.max(np.linalg.norm(np.asarray(a, np.float64), axis=1)))
