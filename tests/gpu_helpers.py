"""Helpers for the GPU parity tests: run the CUDA path through the binding
and the oracle on the same seeded inputs (no SPH arithmetic here)."""
import numpy as np
import pytest


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2007_03097_gb300 import build
    build.build()
    from paper_2007_03097_gb300 import binding
    return binding


def to_oracle_params(orc, params, **kw):
    p = dict(params)
    p.update(kw)
    keys = set(orc.Params.__dataclass_fields__)
    return orc.Params(**{k: v for k, v in p.items() if k in keys})


def gpu_state(p):
    """GPU particle arrays in the current (Morton) order, as float64 numpy."""
    return p.numpy()


def rel(a, b):
    return np.max(np.abs(np.asarray(a) / np.asarray(b) - 1.0))
