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


def fig1_quadtree():
    """The ten particles of Fig. 1 (Sec. 2.1) from ``golden/fig1_quadtree.txt``.

    Returns (labels, x, y, refined, path): each particle's cell label, its
    position in the unit square, the labels of the subdivided cells and the
    Z-order path of the figure.  The figure draws child 2 below child 0, so
    its vertical axis runs against the key's y bit: y = 1 - (y_cm + 2.5) / 5."""
    import os
    path_ = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "fig1_quadtree.txt")
    labels, xs, ys, refined, path = [], [], [], [], []
    with open(path_) as f:
        for line in f:
            t = line.split()
            if not t or t[0].startswith("#"):
                continue
            if t[0] == "particle":
                labels.append(t[1])
                xs.append((float(t[2]) + 2.5) / 5.0)
                ys.append(1.0 - (float(t[3]) + 2.5) / 5.0)
            elif t[0] == "refined":
                refined = t[1:]
            elif t[0] == "path":
                path = t[1:]
    return labels, np.array(xs), np.array(ys), refined, path
