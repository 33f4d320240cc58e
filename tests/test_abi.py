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


def test_launch_counter_without_a_gpu(L):
    # nothing has been launched in a process without a GPU; reading never fails
    assert L.bs_kernel_launches() == 0


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
    # exposures, profile (host checks before any device access)
    one = C.c_float(1.0)
    a = _ffi.FitArgs()
    a.n_gal, a.data_dtype, a.max_side, a.n_psf, a.pixel_scale = 2, 0, 25, 1, 0.2
    a.data = a.offsets = a.side = a.psf = a.noise_sigma = C.addressof(one)
    a.prior = _ffi.Prior(-1.0, 9.0, -2.0, 1.0, 0.5, 0.3)
    for field, value, msg in (("n_exposures", 65, b"n_exposures"), ("profile", 3, b"profile"),
                              ("spergel_nu", -0.95, b"spergel_nu")):
        b = _ffi.FitArgs.from_buffer_copy(a)
        setattr(b, field, value)
        if field == "spergel_nu":
            b.profile = 1
        assert L.bs_logpost_points(C.byref(b), 1, None, None, None, None, None) == -1
        assert msg in L.bs_last_error(), L.bs_last_error()
    b = _ffi.FitArgs.from_buffer_copy(a)
    b.pixel_weight, b.profile = C.addressof(one), 1      # per-pixel weights: exponential only
    assert L.bs_logpost_points(C.byref(b), 1, None, None, None, None, None) == -1
    assert b"pixel_weight" in L.bs_last_error()
    b.profile, b.max_side = 0, 65                         # and stamps of at most 63 px
    assert L.bs_logpost_points(C.byref(b), 1, None, None, None, None, None) == -1
    assert b"63" in L.bs_last_error()
    b = _ffi.FitArgs.from_buffer_copy(a)
    b.n_exposures, b.n_psf = 2, 3          # n_psf must be 1 or n_gal x n_exposures
    assert L.bs_logpost_points(C.byref(b), 1, None, None, None, None, None) == -1
    assert b"n_psf" in L.bs_last_error()


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


def test_host_validation_of_plan_serve_and_sampler(L):
    """Argument errors of the batching, serving and shear-sampling calls are
    caught on the host, before any CUDA call."""
    from paper_2604_22048_gb300 import _ffi
    assert L.bs_fit_resident_galaxies(0, 53, 0) == 0          # n_chains < 1
    assert L.bs_fit_resident_galaxies(4, 54, 0) == 0          # even side
    assert L.bs_fit_resident_galaxies(4, 53, 100) == 0        # register cap not offered
    # serving: NULL / undersized arena, bad stream count, bad register cap
    cfg = _ffi.ServeCfg()
    h = C.c_void_p()
    assert L.bs_serve_create(None, None, 0, C.byref(h)) == -1
    assert L.bs_serve_create(C.byref(cfg), C.c_void_p(1), 1 << 10, C.byref(h)) == -1
    assert b"arena" in L.bs_last_error()
    cfg.n_streams = 2
    assert L.bs_serve_create(C.byref(cfg), C.c_void_p(1), 1 << 20, C.byref(h)) == -1
    assert b"n_streams" in L.bs_last_error()
    cfg.n_streams = 0
    cfg.registers[1] = 100
    assert L.bs_serve_create(C.byref(cfg), C.c_void_p(1), 1 << 20, C.byref(h)) == -1
    assert b"registers" in L.bs_last_error()
    # shear sampler: g must be free, flux/size parameters need lf/ls
    d = _ffi.ShearData()
    d.n_gal, d.K, d.family, d.sigma_e0 = 2, 4, 0, 0.3
    sc = _ffi.ShearSampleCfg()
    out = (C.c_double * 16)()
    sc.free_mask = 0b100
    assert L.bs_shear_sample(C.byref(d), C.byref(sc), out, None, None, None, None, 0, None) == -1
    assert b"free_mask" in L.bs_last_error()
    sc.free_mask = 0b1011
    assert L.bs_shear_sample(C.byref(d), C.byref(sc), out, None, None, None, None, 0, None) == -1
    assert b"lf and ls" in L.bs_last_error()
    sc.free_mask = 0b11
    sc.n_samples = 0
    assert L.bs_shear_sample(C.byref(d), C.byref(sc), out, None, None, None, None, 0, None) == -1
    # weighted galaxies: the weight sum must be finite and >= 0
    wd = _ffi.ShearData()
    wd.n_gal, wd.K, wd.family, wd.sigma_e0 = 2, 4, 0, 0.3
    wd.e1 = wd.e2 = wd.gal_weight = 16
    for bad in (-1.0, float("nan"), float("inf")):
        wd.gal_weight_sum = bad
        assert L.bs_shear_loglike(C.byref(wd), 0.0, 0.0, 0.2, out, 1, None, 0, None) == -1
        assert b"gal_weight_sum" in L.bs_last_error()
    # several points per pass: b must be NULL, n_points >= 0
    pts = (C.c_double * 3)(0.0, 0.0, 0.2)
    md = _ffi.ShearData()
    md.n_gal, md.K, md.family, md.sigma_e0 = 2, 4, 0, 0.3
    md.e1 = md.e2 = md.b = 16
    assert L.bs_shear_loglike_multi(C.byref(md), 1, pts, out, 1, None, 0, None) == -1
    assert b"b must be NULL" in L.bs_last_error()
    md.b = None
    assert L.bs_shear_loglike_multi(C.byref(md), -1, pts, out, 1, None, 0, None) == -1
    assert L.bs_shear_loglike_multi(C.byref(md), 0, None, None, 1, None, 0, None) == 0
    # all-free likelihood: b must be NULL, sigma_f > 0
    th = (C.c_double * 8)(0.0, 0.0, 0.2, 2.4, -0.1, 1.0, -0.4, 0.05)
    im = (C.c_double * 4)(-1.0, 9.0, -2.0, 1.0)
    assert L.bs_shear_loglike_full(None, None, None, im, th, out, 1, None, 0, None) == -1
    # plan: unknown flags
    a = _ffi.FitArgs()
    o = _ffi.FitOut()
    p = C.c_void_p()
    assert L.bs_fit_plan_create(C.byref(a), C.byref(o), None, 8, None, 0, None, C.byref(p)) == -1
    assert b"flags" in L.bs_last_error()
