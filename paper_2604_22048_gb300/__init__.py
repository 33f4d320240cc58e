"""GB300 (sm_103a) hot path of Bayesian shear inference with a known PSF and
sky background (Mendoza et al., "Differentiable Forward Modeling for Efficient
and Accurate Shear Inference").

  fit_galaxies(stamps, psf, noise_sigma, init, cfg) -> interim samples
      image sampling phase (Sec. 3.3), one persistent CUDA launch;
  ShearPlan(e1, e2).loglike(g1, g2, alpha) -> value, gradient
      MC shear likelihood of Eq. likelihood-shear (Sec. 3.2);
  ShearPlan.estimate(...) -> posterior mean of g (and alpha) (Sec. 3.4);
  Server(cfg).submit(requests) / .poll() -> the same fits for stamps that
      arrive one by one (continuous batching, admission by memory).

The C ABI lives in include/bpshear.h; this package only marshals torch
tensors into it (see ``api``), and ``synth`` draws seeded synthetic inputs.
"""
from . import _ffi
from .api import (DEFAULT_PRIOR, PIXEL_SCALE, FitConfig, FitPlan, RaggedFitPlan, RenderLogPost, Server,
                  ShearLogLike, ShearPlan, chain_ess, fit_galaxies, logpost_points, pack_stamps, psf_table,
                  render, resident_galaxies, shear_loglike)

__all__ = ["DEFAULT_PRIOR", "PIXEL_SCALE", "FitConfig", "FitPlan", "RaggedFitPlan", "RenderLogPost", "Server",
           "ShearLogLike", "ShearPlan", "chain_ess", "fit_galaxies", "logpost_points", "pack_stamps", "psf_table",
           "render", "resident_galaxies", "shear_loglike", "lib"]


def lib():
    """The loaded libbpshear.so (raises ImportError if it was not built)."""
    return _ffi.lib()
