"""ctypes declarations of the bpshear C ABI (include/bpshear.h).

Argument marshalling only: every computation runs in libbpshear.so.  Loading
fails loudly when the library has not been built; there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIBPATH = os.path.join(_HERE, "csrc", "libbpshear.so")

BS_OK = 0
BS_F32, BS_F64 = 0, 1
BS_PSF_GAUSSIAN, BS_PSF_MOFFAT = 1, 2
BS_EPRIOR_BA14, BS_EPRIOR_TRUNC_GAUSS = 0, 1
BS_MAX_SIDE = 127

STATUS_NAMES = {0: "BS_OK", -1: "BS_ERR_INVALID_ARG", -2: "BS_ERR_CUDA", -3: "BS_ERR_OUT_OF_MEMORY",
                -4: "BS_ERR_TIMEOUT", -5: "BS_ERR_UNSUPPORTED"}

# every symbol the header declares
EXPORTED = ["bs_prior_default", "bs_last_error", "bs_version", "bs_render", "bs_fit_workspace_bytes",
            "bs_fit_galaxies", "bs_logpost_points", "bs_chain_ess", "bs_shear_workspace_bytes",
            "bs_shear_loglike", "bs_shear_estimate", "bs_shear_loglike_noalloc", "bs_shear_loglike_full",
            "bs_fit_plan_workspace_bytes", "bs_fit_plan_create", "bs_fit_plan_launch", "bs_fit_plan_destroy",
            "bs_fit_resident_galaxies", "bs_fit_plan_num_launches", "bs_fit_plan_info", "bs_serve_request_bytes", "bs_serve_create", "bs_serve_submit",
            "bs_serve_poll", "bs_serve_get_stats", "bs_serve_now_ns", "bs_serve_destroy",
            "bs_shear_hyperprior_default", "bs_shear_sample", "bs_fp32_peak", "bs_fp64_peak", "bs_shear_loglike_multi",
            "bs_kernel_launches", "bs_shear_bias", "bs_shear_bias_custom", "bs_shear_estimate_custom",
            "bs_dense_precision", "bs_dense_precision_workspace_bytes"]


class BsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Psf(C.Structure):
    _fields_ = [("kind", C.c_int32), ("fwhm", C.c_float), ("beta", C.c_float)]


class Prior(C.Structure):
    _fields_ = [("lf_lo", C.c_float), ("lf_hi", C.c_float), ("ls_lo", C.c_float), ("ls_hi", C.c_float),
                ("sigma_xy", C.c_float), ("sigma_e", C.c_float)]


class FitArgs(C.Structure):
    _fields_ = [("n_gal", C.c_int32), ("data_dtype", C.c_int32), ("data", C.c_void_p),
                ("offsets", C.c_void_p), ("side", C.c_void_p), ("max_side", C.c_int32),
                ("psf", C.c_void_p), ("n_psf", C.c_int32), ("noise_sigma", C.c_void_p),
                ("gal_id", C.c_void_p), ("init", C.c_void_p), ("pixel_scale", C.c_float),
                ("prior", Prior), ("n_chains", C.c_int32), ("n_warmup", C.c_int32),
                ("n_samples", C.c_int32), ("n_leapfrog", C.c_int32), ("target_accept", C.c_float),
                ("jitter", C.c_float), ("adapt_mass", C.c_int32), ("random_steps", C.c_int32),
                ("seed", C.c_uint64), ("init_step_size", C.c_void_p), ("init_inv_mass", C.c_void_p),
                ("registers", C.c_int32), ("n_exposures", C.c_int32), ("noise_corr", C.c_void_p),
                ("profile", C.c_int32), ("spergel_nu", C.c_float), ("pixel_weight", C.c_void_p),
                ("pixel_prec", C.c_void_p), ("prec_offsets", C.c_void_p), ("chains_per_cta", C.c_int32)]


class FitOut(C.Structure):
    _fields_ = [("samples", C.c_void_p), ("logp", C.c_void_p), ("accepted", C.c_void_p),
                ("accept_rate", C.c_void_p), ("step_size", C.c_void_p), ("inv_mass", C.c_void_p),
                ("n_divergent", C.c_void_p), ("status", C.c_void_p), ("n_grad", C.c_void_p),
                ("warmup_accepted", C.c_void_p), ("warmup_accept_stat", C.c_void_p),
                ("warmup_step_size", C.c_void_p)]


class ShearData(C.Structure):
    _fields_ = [("e1", C.c_void_p), ("e2", C.c_void_p), ("b", C.c_void_p), ("n_gal", C.c_int64),
                ("K", C.c_int32), ("family", C.c_int32), ("trunc_r", C.c_float), ("sigma_e0", C.c_float),
                ("gal_weight", C.c_void_p), ("gal_weight_sum", C.c_double)]


ALLREDUCE_FN = C.CFUNCTYPE(None, C.POINTER(C.c_double), C.c_void_p)


class EstimateCfg(C.Structure):
    _fields_ = [("free_alpha", C.c_int32), ("alpha", C.c_double), ("alpha_lo", C.c_double),
                ("alpha_hi", C.c_double), ("n_gh", C.c_int32), ("allreduce", ALLREDUCE_FN),
                ("allreduce_user", C.c_void_p)]


G_ESTIMATOR_FN = C.CFUNCTYPE(C.c_int32, C.POINTER(C.c_float), C.c_double, C.POINTER(C.c_double), C.c_void_p)
BS_BIAS_QUADRATURE, BS_BIAS_HMC = 0, 1


class BiasCfg(C.Structure):
    _fields_ = [("g_abs", C.c_double), ("n_boot", C.c_int32), ("seed", C.c_uint64), ("base_weight", C.c_void_p),
                ("m_boot", C.c_void_p), ("c_boot", C.c_void_p)]


LOGLIKE_POINTS_FN = C.CFUNCTYPE(C.c_int32, C.POINTER(C.c_double), C.c_int32, C.POINTER(C.c_double), C.c_void_p)

BS_PLAN_CAPTURE, BS_PLAN_AUTOTUNE = 1, 2


class PlanLaunchInfo(C.Structure):
    _fields_ = [("slot_class", C.c_int32), ("max_side", C.c_int32), ("n_gal", C.c_int32), ("grid", C.c_int32),
                ("registers", C.c_int32), ("trial_ms_128", C.c_float), ("trial_ms_96", C.c_float),
                ("trial_ms_80", C.c_float), ("chains_per_cta", C.c_int32), ("trial_ms_128_half", C.c_float),
                ("trial_ms_96_half", C.c_float), ("trial_ms_80_half", C.c_float)]


class ServeCfg(C.Structure):
    _fields_ = [("max_side", C.c_int32), ("pixel_scale", C.c_float), ("prior", Prior), ("n_chains", C.c_int32),
                ("n_warmup", C.c_int32), ("n_samples", C.c_int32), ("n_leapfrog", C.c_int32),
                ("target_accept", C.c_float), ("jitter", C.c_float), ("adapt_mass", C.c_int32),
                ("random_steps", C.c_int32), ("seed", C.c_uint64), ("max_inflight", C.c_int32),
                ("batch_us", C.c_int32), ("n_streams", C.c_int32), ("registers", C.c_int32 * 4)]


class ServeRequest(C.Structure):
    _fields_ = [("tag", C.c_uint64), ("gal_id", C.c_uint64), ("side", C.c_int32), ("psf", Psf),
                ("noise_sigma", C.c_float), ("stamp", C.c_void_p), ("init", C.c_void_p),
                ("t_arrival_ns", C.c_int64)]


class ServeCompletion(C.Structure):
    _fields_ = [("tag", C.c_uint64), ("status", C.c_int32), ("side", C.c_int32), ("t_arrival_ns", C.c_int64),
                ("t_submit_ns", C.c_int64), ("t_admit_ns", C.c_int64), ("t_done_ns", C.c_int64),
                ("samples", C.c_void_p), ("plane_stride", C.c_int64), ("logp", C.c_void_p),
                ("accepted", C.c_void_p), ("accept_rate", C.c_void_p), ("step_size", C.c_void_p),
                ("inv_mass", C.c_void_p), ("n_divergent", C.c_void_p), ("n_grad", C.c_void_p)]


class ShearSampleCfg(C.Structure):
    _fields_ = [("free_mask", C.c_uint32), ("theta0", C.c_double * 8), ("lo", C.c_double * 8),
                ("hi", C.c_double * 8), ("lf", C.c_void_p), ("ls", C.c_void_p), ("interim", C.c_double * 4),
                ("n_warmup", C.c_int32), ("n_samples", C.c_int32), ("n_leapfrog", C.c_int32),
                ("target_accept", C.c_float), ("random_steps", C.c_int32), ("seed", C.c_uint64),
                ("allreduce", ALLREDUCE_FN), ("allreduce_user", C.c_void_p)]


class ServeStats(C.Structure):
    _fields_ = [(n, C.c_int64) for n in ("submitted", "admitted", "completed", "launches", "ticks", "waits_memory",
                                         "waits_inflight", "waits_streams", "arena_bytes", "arena_used",
                                         "arena_high_water")] + [("pending", C.c_int32), ("inflight", C.c_int32)]


def struct_dtype(S):
    """numpy dtype with the byte layout of ctypes structure S (flat fields;
    a nested bs_psf is spelled out as psf_kind, psf_fwhm, psf_beta)."""
    import numpy as np
    names, formats, offsets = [], [], []
    conv = {C.c_uint64: "<u8", C.c_int64: "<i8", C.c_int32: "<i4", C.c_float: "<f4", C.c_void_p: "<u8"}
    for name, t in S._fields_:
        off = getattr(S, name).offset
        if t is Psf:
            for sub, st in Psf._fields_:
                names.append(f"{name}_{sub}")
                formats.append(conv[st])
                offsets.append(off + getattr(Psf, sub).offset)
        else:
            names.append(name)
            formats.append(conv[t])
            offsets.append(off)
    return np.dtype({"names": names, "formats": formats, "offsets": offsets, "itemsize": C.sizeof(S)})


_lib = None


def lib():
    """Load libbpshear.so (built by paper_2604_22048_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIBPATH):
        raise ImportError(f"{LIBPATH} is missing: build it with `python -m paper_2604_22048_gb300.build`"
                          " (the CUDA path has no fallback)")
    L = C.CDLL(LIBPATH)
    vp, i32, i64, f32, f64, sz = C.c_void_p, C.c_int32, C.c_int64, C.c_float, C.c_double, C.c_size_t
    L.bs_prior_default.argtypes = [C.POINTER(Prior)]
    L.bs_prior_default.restype = None
    L.bs_last_error.restype = C.c_char_p
    L.bs_version.restype = C.c_char_p
    L.bs_kernel_launches.argtypes = []
    L.bs_kernel_launches.restype = C.c_uint64
    L.bs_render.argtypes = [i32, vp, vp, vp, vp, i32, vp, i32, f32, vp, vp]
    L.bs_fit_workspace_bytes.argtypes = [C.POINTER(FitArgs)]
    L.bs_fit_workspace_bytes.restype = sz
    L.bs_fit_galaxies.argtypes = [C.POINTER(FitArgs), C.POINTER(FitOut), vp, sz, vp]
    L.bs_logpost_points.argtypes = [C.POINTER(FitArgs), i32, vp, vp, vp, vp, vp]
    L.bs_chain_ess.argtypes = [vp, i32, i32, i32, vp, vp, vp]
    L.bs_shear_workspace_bytes.argtypes = [i64, i32]
    L.bs_shear_workspace_bytes.restype = sz
    L.bs_shear_loglike.argtypes = [C.POINTER(ShearData), f64, f64, f64, vp, i32, vp, sz, vp]
    L.bs_shear_estimate.argtypes = [C.POINTER(ShearData), C.POINTER(EstimateCfg), vp, vp, vp, vp, sz, vp]
    L.bs_shear_loglike_noalloc.argtypes = [C.POINTER(ShearData), f64, f64, f64, vp, vp]
    L.bs_shear_loglike_multi.argtypes = [C.POINTER(ShearData), i32, vp, vp, i32, vp, sz, vp]
    L.bs_shear_loglike_full.argtypes = [C.POINTER(ShearData), vp, vp, vp, vp, vp, i32, vp, sz, vp]
    L.bs_fit_plan_workspace_bytes.argtypes = [C.POINTER(FitArgs)]
    L.bs_fit_plan_workspace_bytes.restype = sz
    L.bs_fit_plan_create.argtypes = [C.POINTER(FitArgs), C.POINTER(FitOut), vp, i32, vp, sz, vp,
                                     C.POINTER(C.c_void_p)]
    L.bs_fit_plan_launch.argtypes = [vp, vp]
    L.bs_fit_plan_destroy.argtypes = [vp]
    L.bs_fp32_peak.argtypes = [i32, vp, vp]
    L.bs_fp64_peak.argtypes = [vp, vp]
    L.bs_shear_hyperprior_default.argtypes = [vp, vp]
    L.bs_shear_hyperprior_default.restype = None
    L.bs_shear_sample.argtypes = [C.POINTER(ShearData), C.POINTER(ShearSampleCfg), vp, vp, vp, vp, vp, sz, vp]
    L.bs_shear_bias_custom.argtypes = [i64, G_ESTIMATOR_FN, vp, G_ESTIMATOR_FN, vp, C.POINTER(BiasCfg), vp]
    L.bs_dense_precision_workspace_bytes.argtypes = [i32]
    L.bs_dense_precision_workspace_bytes.restype = sz
    L.bs_dense_precision.argtypes = [i32, vp, i32, vp, vp, vp, vp, vp, sz, vp]
    L.bs_shear_estimate_custom.argtypes = [LOGLIKE_POINTS_FN, vp, C.POINTER(EstimateCfg), vp, vp, vp]
    L.bs_shear_bias.argtypes = [C.POINTER(ShearData), C.POINTER(ShearData), i32, C.POINTER(EstimateCfg),
                                C.POINTER(ShearSampleCfg), C.POINTER(BiasCfg), vp, vp, vp, sz, vp]
    L.bs_fit_plan_num_launches.argtypes = [vp]
    L.bs_fit_plan_num_launches.restype = i32
    L.bs_fit_plan_info.argtypes = [vp, i32, C.POINTER(PlanLaunchInfo)]
    L.bs_fit_resident_galaxies.argtypes = [i32, i32, i32]
    L.bs_fit_resident_galaxies.restype = i32
    L.bs_serve_request_bytes.argtypes = [C.POINTER(ServeCfg), i32]
    L.bs_serve_request_bytes.restype = sz
    L.bs_serve_create.argtypes = [C.POINTER(ServeCfg), vp, sz, C.POINTER(C.c_void_p)]
    L.bs_serve_submit.argtypes = [vp, vp, i32]
    L.bs_serve_poll.argtypes = [vp, vp, i32, i32, C.POINTER(C.c_int32)]
    L.bs_serve_get_stats.argtypes = [vp, C.POINTER(ServeStats)]
    L.bs_serve_now_ns.argtypes = [vp]
    L.bs_serve_now_ns.restype = i64
    L.bs_serve_destroy.argtypes = [vp]
    for nm in ("bs_render", "bs_fit_galaxies", "bs_logpost_points", "bs_chain_ess", "bs_shear_loglike",
               "bs_shear_loglike_full", "bs_shear_sample", "bs_fp32_peak", "bs_fp64_peak", "bs_shear_loglike_multi",
               "bs_shear_estimate", "bs_shear_loglike_noalloc", "bs_fit_plan_create", "bs_fit_plan_launch",
               "bs_fit_plan_destroy", "bs_fit_plan_info", "bs_serve_create", "bs_serve_submit", "bs_serve_poll", "bs_serve_get_stats",
               "bs_serve_destroy"):
        getattr(L, nm).restype = C.c_int
    _lib = L
    return L


def check(status):
    if status != BS_OK:
        raise BsError(status, lib().bs_last_error().decode(errors="replace"))
