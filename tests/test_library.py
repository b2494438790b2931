"""Host-side checks of the C ABI (no GPU needed): the library builds for
sm_103a, exports every function include/sph.h declares, the ctypes mirrors
of the C structs have the C layout, and parameter validation rejects bad
input before any CUDA call."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sph.h")


@pytest.fixture(scope="module")
def libpath():
    from paper_2007_03097_gb300 import build
    return build.build()


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|const char \*)\s*\*?\s*(sph_\w+)\s*\(", text, re.M)))


def test_header_functions_are_exported(libpath):
    from paper_2007_03097_gb300 import binding
    names = declared_functions()
    assert len(names) >= 20
    lib = ctypes.CDLL(libpath)
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(binding.EXPORTED)


def test_struct_layout_matches_c():
    from paper_2007_03097_gb300 import binding as B
    structs = {"sph_params": B.sph_params, "sph_particles": B.sph_particles,
               "sph_density_stats": B.sph_density_stats, "sph_force_stats": B.sph_force_stats,
               "sph_step_stats": B.sph_step_stats}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "sph.h"', "int main(void){"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{name}.{f} %zu\\n", offsetof({name}, {f}));')
    lines.append("return 0;}")
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "l.c"), os.path.join(d, "l")
        open(src, "w").write("\n".join(lines))
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), src, "-o", exe])
        out = subprocess.check_output([exe], text=True).split("\n")
    got = dict(line.split() for line in out if line)
    for name, cls in structs.items():
        assert int(got[name]) == ctypes.sizeof(cls), name
        for f, _ in cls._fields_:
            assert int(got[f"{name}.{f}"]) == getattr(cls, f).offset, f"{name}.{f}"


def test_invalid_params_rejected_without_gpu(libpath):
    from paper_2007_03097_gb300 import binding as B
    lib = B.load(libpath)
    bad = [dict(kernel=7), dict(leaf_size=0), dict(leaf_size=33), dict(h_min=1.0, h_max=0.5),
           dict(periodic=True, box_hi=(1.0, 2.0, 1.0)), dict(max_sweeps=0), dict(gamma=1.0),
           dict(periodic=True, h_max=0.3), dict(dim=2), dict(dim=0), dict(curve=2), dict(energy=3)]
    for kw in bad:
        q = B.make_params(kw)
        h = ctypes.c_void_p()
        assert lib.sph_create(ctypes.byref(q), 100, ctypes.byref(h)) == B.SPH_ERR_ARG, kw
    q = B.make_params({})
    assert lib.sph_create(ctypes.byref(q), 0, ctypes.byref(ctypes.c_void_p())) == B.SPH_ERR_ARG


def test_version_string(libpath):
    from paper_2007_03097_gb300 import binding as B
    assert "sm_103a" in B.load(libpath).sph_version().decode()
