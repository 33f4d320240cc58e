"""The C-ABI library loads and exports every symbol include/bpshear.h declares;
host-side argument validation answers without any CUDA call (CPU only)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2604_22048_gb300 import _ffi, build
    build.build()
    return _ffi.lib()


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "bpshear.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bs_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(L):
    from paper_2604_22048_gb300 import _ffi
    syms = declared_symbols()
    assert len(syms) >= 10
    for s in syms:
        assert hasattr(L, s), s
    assert sorted(_ffi.EXPORTED) == syms


def test_version_and_prior_default(L):
    from paper_2604_22048_gb300 import _ffi
    assert b"sm_103a" in L.bs_version()
    p = _ffi.Prior()
    L.bs_prior_default(C.byref(p))
    assert (p.lf_lo, p.lf_hi, p.ls_lo, p.ls_hi, p.sigma_xy) == (-1.0, 9.0, -2.0, 1.0, 0.5)
    assert abs(p.sigma_e - 0.3) < 1e-7


def test_host_validation(L):
    from paper_2604_22048_gb300 import _ffi
    assert L.bs_render(-1, None, None, None, None, 25, None, 1, 0.2, None, None) == -1
    assert b"n < 0" in L.bs_last_error()
    assert L.bs_render(3, None, None, None, None, 25, None, 1, 0.2, None, None) == -1
    assert L.bs_fit_galaxies(None, None, None, 0, None) == -1
    a = _ffi.FitArgs()
    a.n_gal = 4
    assert L.bs_fit_galaxies(C.byref(a), None, None, 0, None) == -1
    assert L.bs_shear_loglike(None, 0.0, 0.0, 0.2, None, 1, None, 0, None) == -1
    d = _ffi.ShearData()
    d.n_gal, d.K, d.family, d.sigma_e0 = 5, 10, 0, 0.3
    assert L.bs_shear_loglike(C.byref(d), 0.0, 0.0, 0.2, None, 1, None, 0, None) == -1   # NULL e1/e2
    assert L.bs_chain_ess(None, 1, 4, 100, None, None, None) == -1
    assert L.bs_logpost_points(None, 1, None, None, None, None, None) == -1


def test_struct_layouts_match_header(tmp_path):
    """sizeof/offsetof of every struct, as gcc sees include/bpshear.h, equal the
    ctypes declarations the binding marshals with."""
    import subprocess
    from paper_2604_22048_gb300 import _ffi
    structs = {"bs_fit_args": _ffi.FitArgs, "bs_fit_out": _ffi.FitOut, "bs_shear_data": _ffi.ShearData,
               "bs_estimate_cfg": _ffi.EstimateCfg, "bs_serve_cfg": _ffi.ServeCfg,
               "bs_serve_request": _ffi.ServeRequest, "bs_serve_completion": _ffi.ServeCompletion,
               "bs_serve_stats": _ffi.ServeStats, "bs_psf": _ffi.Psf, "bs_prior": _ffi.Prior,
               "bs_fit_plan_launch_info": _ffi.PlanLaunchInfo, "bs_shear_sample_cfg": _ffi.ShearSampleCfg}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "bpshear.h"', "int main(void) {"]
    for cn, py in structs.items():
        lines.append(f'printf("{cn} size %zu\\n", sizeof({cn}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cn} {f} %zu\\n", offsetof({cn}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    for line in filter(None, out):
        cn, f, v = line.split()
        py = structs[cn]
        got = C.sizeof(py) if f == "size" else getattr(py, f).offset
        assert got == int(v), (cn, f, got, v)
