"""Small helpers shared by the tests (no SPH arithmetic here)."""
import numpy as np


def oracle_params(orc, w, **kw):
    """oracle.Params from a workload's parameter dict, with overrides."""
    p = dict(w.params)
    p.update(kw)
    keys = set(orc.Params.__dataclass_fields__)
    return orc.Params(**{k: v for k, v in p.items() if k in keys})


def oracle_state(orc, w):
    return orc.State(w.x.copy(), w.y.copy(), w.z.copy(), w.vx.copy(), w.vy.copy(), w.vz.copy(),
                     w.m.copy(), w.h.copy(), w.u.copy())


def rel_err(a, b, scale):
    return np.max(np.abs(np.asarray(a) - np.asarray(b)) / np.maximum(scale, 1e-300))
