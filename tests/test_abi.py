"""CPU checks of the C ABI: the library builds for sm_103a, loads, exports every
function that include/ddlpb.h declares, and its structs have the layout the
Python binding assumes.  No compute call is made (no GPU here)."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

from paper_2203_00552_gb300 import _binding
from paper_2203_00552_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ddlpb.h")


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(_binding.LIB_PATH):
        B.build()
    return _binding.library()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ddlpb_\w+)\s*\(", text)))


def test_header_declares_the_api():
    names = declared_functions()
    for n in ("ddlpb_setup", "ddlpb_solve", "ddlpb_adjoint", "ddlpb_energy", "ddlpb_forces", "ddlpb_free"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", _binding.LIB_PATH], capture_output=True, text=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    for n in declared_functions():
        assert n in exported, n
        assert hasattr(lib, n)
    # nothing else leaks out of the shared object
    assert exported == set(declared_functions())
    assert set(_binding.EXPORTS) == set(declared_functions())


def test_struct_layout_matches_header(tmp_path):
    src = tmp_path / "sz.c"
    src.write_text('#include "ddlpb.h"\n#include <stdio.h>\n#include <stddef.h>\n'
                   'int main(){printf("%zu %zu %zu %zu\\n", sizeof(ddlpb_options), sizeof(ddlpb_info),'
                   ' offsetof(ddlpb_options, cuda_stream), offsetof(ddlpb_info, refinement_steps));return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    a, b, c, d = map(int, subprocess.run([str(exe)], capture_output=True, text=True).stdout.split())
    assert a == ctypes.sizeof(_binding.Options)
    assert b == ctypes.sizeof(_binding.Info)
    assert c == _binding.Options.cuda_stream.offset
    assert d == _binding.Info.refinement_steps.offset


def test_default_options(lib):
    o = _binding.default_options()
    assert o.eta == 0.1 and o.tol == 1e-8 and o.gmres_restart == 150 and o.fmm_order == 0
    assert o.precond_fp16 == 1 and o.precond_coupling == 0


def test_setup_rejects_bad_input_before_touching_the_gpu(lib):
    import numpy as np
    c = np.zeros((2, 3))
    c[1, 0] = 3.0
    r = np.array([2.0, 2.0])
    q = np.array([0.1, -0.1])
    bad = [dict(n_lebedev=111), dict(lmax=17), dict(lmax=9, n_lebedev=110), dict(kappa=-1.0),
           dict(eps_solvent=0.5)]
    for kw in bad:
        args = dict(eps_solvent=78.54, kappa=0.05, lmax=4, n_lebedev=110)
        args.update(kw)
        with pytest.raises(_binding.DDLPBError) as e:
            _binding.Context(c, r, q, args["eps_solvent"], args["kappa"], args["lmax"], args["n_lebedev"])
        assert e.value.status == 1


def test_setup_rejects_bad_solver_and_fmm_options(lib):
    """Options outside their documented ranges (include/ddlpb.h) are refused with EINVAL before
    any device work: FMM order below lmax + 1 or above 21, admissibility ratio outside (0, 1),
    restart length outside [1, 2000], preconditioner tolerance outside (0, 1]."""
    import numpy as np
    c = np.zeros((2, 3))
    c[1, 0] = 3.0
    r = np.array([2.0, 2.0])
    q = np.array([0.1, -0.1])
    bad = [dict(fmm_order=4), dict(fmm_order=22), dict(fmm_order=8, fmm_theta=1.0), dict(fmm_order=8, fmm_theta=0.0),
           dict(gmres_restart=2001), dict(gmres_restart=0), dict(precond_tol=1.5), dict(eta=0.0)]
    for kw in bad:
        with pytest.raises(_binding.DDLPBError) as e:
            _binding.Context(c, r, q, 78.54, 0.05, 4, 110, **kw)
        assert e.value.status == 1, kw
        assert str(e.value), kw


def test_binding_fails_loudly_without_library(monkeypatch):
    monkeypatch.setattr(_binding, "_lib", None)
    monkeypatch.setattr(_binding, "LIB_PATH", "/nonexistent/libddlpb.so")
    with pytest.raises(RuntimeError):
        _binding.library()
