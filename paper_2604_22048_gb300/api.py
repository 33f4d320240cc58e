"""Torch-facing binding of the bpshear C ABI.

PyTorch provides device memory and streams only; every step of the path runs
in libbpshear.so.  Functions take CUDA tensors, enqueue on the current torch
stream and return CUDA tensors unless stated otherwise.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np
import torch

from . import _ffi as F

PIXEL_SCALE = 0.2
DEFAULT_PRIOR = (-1.0, 9.0, -2.0, 1.0, 0.5, 0.3)   # Eq. interim-prior


def _p(t):
    return None if t is None else t.data_ptr()


def _stream(dev=None):
    return C.c_void_p(torch.cuda.current_stream(dev).cuda_stream)


def _need_cuda(*ts):
    for t in ts:
        if t is not None and not t.is_cuda:
            raise ValueError("expected CUDA tensors (the bpshear path has no CPU fallback)")


def psf_table(kind, fwhm, beta=3.0, device="cuda"):
    """Pack per-galaxy (or one shared) PSFs into a device array of bs_psf.

    kind: "gaussian" | "moffat" (or BS_PSF_* ints); fwhm: scalar or array."""
    fwhm = np.atleast_1d(np.asarray(fwhm, dtype=np.float32))
    n = len(fwhm)
    if isinstance(kind, str):
        kind = {"gaussian": F.BS_PSF_GAUSSIAN, "moffat": F.BS_PSF_MOFFAT}[kind]
    rec = np.zeros(n, dtype=[("kind", "<i4"), ("fwhm", "<f4"), ("beta", "<f4")])
    rec["kind"] = kind
    rec["fwhm"] = fwhm
    rec["beta"] = beta
    return torch.from_numpy(rec.view(np.uint8).copy()).to(device), n


def pack_stamps(sides, align=4):
    """Offsets of stamps packed back to back, each start rounded up to `align`
    elements.  Returns (offsets int64 array, total elements)."""
    sides = np.asarray(sides, dtype=np.int64)
    sizes = sides * sides
    sizes = (sizes + align - 1) // align * align
    offs = np.zeros(len(sides), dtype=np.int64)
    if len(sides) > 1:
        offs[1:] = np.cumsum(sizes)[:-1]
    return offs, int(sizes.sum())


def render(theta, side, psf, *, shear=None, offsets=None, total=None, pixel_scale=PIXEL_SCALE,
           max_side=None):
    """Noiseless model stamps (bs_render).  theta: [n, 6] float32 CUDA;
    side: [n] int32 CUDA; psf: (table, n_psf) from psf_table.  Returns
    (flat stamps, offsets)."""
    _need_cuda(theta, side, shear)
    n = theta.shape[0]
    sides_h = side.cpu().numpy()
    if offsets is None:
        offs_h, total = pack_stamps(sides_h)
        offsets = torch.from_numpy(offs_h).to(theta.device)
    out = torch.zeros(total, dtype=torch.float32, device=theta.device)
    ms = int(max_side or sides_h.max())
    table, n_psf = psf
    F.check(F.lib().bs_render(n, _p(theta.contiguous()), _p(shear), _p(offsets), _p(side), ms,
                              _p(table), n_psf, pixel_scale, _p(out), _stream()))
    return out, offsets


@dataclass
class FitConfig:
    n_chains: int = 4
    n_warmup: int = 100
    n_samples: int = 100
    n_leapfrog: int = 16
    target_accept: float = 0.8
    jitter: float = 0.1
    adapt_mass: bool = True
    random_steps: bool = True
    seed: int = 22048
    pixel_scale: float = PIXEL_SCALE
    prior: tuple = DEFAULT_PRIOR
    profile: int = 0            # 0 exponential, 1 Spergel (spergel_nu), 2 Gaussian (Appendix B)
    spergel_nu: float = 0.5


class FitPlan:
    """Preallocated arguments, outputs and workspace of one bs_fit_galaxies
    launch, so that repeated fits (benchmark steps) allocate nothing."""

    def __init__(self, data, offsets, side, psf, noise_sigma, init, cfg: FitConfig, *, gal_id=None,
                 max_side=None, init_step_size=None, init_inv_mass=None, registers=0, n_exposures=1,
                 noise_corr=None, pixel_weight=None, pixel_prec=None, prec_offsets=None, chains_per_cta=0,
                 want=("logp", "accept_rate", "step_size", "inv_mass", "n_div", "status", "n_grad")):
        """init_step_size [n_gal, C] / init_inv_mass [n_gal, C, 6] (optional):
        resume adapted chains (no initial step-size search).  registers: the
        fit kernel's register cap (128, 96, 80; 0 = 128): all three give the
        same chains bit for bit (the cap changes only the speed).
        n_exposures J: each galaxy's J stamps lie one after another from its
        offset, psf has n_gal * J entries (or one), noise_sigma n_gal * J;
        noise_corr (float32, layout of data): per-exposure noise correlation
        at pixel lag, centred; pixel_weight (float32, layout of data):
        per-pixel inverse-variance factors, 0 masks a pixel (Appendix C);
        pixel_prec, prec_offsets: a general pixel covariance as its precision
        matrices (dense_precision), Appendix C."""
        _need_cuda(data, offsets, side, noise_sigma, init, gal_id, init_step_size, init_inv_mass, noise_corr,
                   pixel_weight, pixel_prec, prec_offsets)
        dev = data.device
        n_gal, n_chains = init.shape[0], init.shape[1]
        assert n_chains == cfg.n_chains, "init must be [n_gal, n_chains, 6]"
        self.cfg = cfg
        self.keep = (data, offsets, side, psf, noise_sigma, init, gal_id, init_step_size, init_inv_mass, noise_corr,
                     pixel_weight, pixel_prec, prec_offsets)
        table, n_psf = psf
        a = F.FitArgs()
        a.n_gal = n_gal
        a.data_dtype = F.BS_F64 if data.dtype == torch.float64 else F.BS_F32
        a.data = _p(data)
        a.offsets = _p(offsets)
        a.side = _p(side)
        a.max_side = int(max_side or int(side.max().item()))
        a.psf = _p(table)
        a.n_psf = n_psf
        a.noise_sigma = _p(noise_sigma)
        a.gal_id = _p(gal_id)
        a.init = _p(init)
        a.pixel_scale = cfg.pixel_scale
        a.prior = F.Prior(*cfg.prior)
        a.n_chains = cfg.n_chains
        a.n_warmup = cfg.n_warmup
        a.n_samples = cfg.n_samples
        a.n_leapfrog = cfg.n_leapfrog
        a.target_accept = cfg.target_accept
        a.jitter = cfg.jitter
        a.adapt_mass = int(cfg.adapt_mass)
        a.random_steps = int(cfg.random_steps)
        a.seed = cfg.seed
        a.init_step_size = _p(init_step_size)
        a.init_inv_mass = _p(init_inv_mass)
        a.registers = int(registers)
        a.n_exposures = int(n_exposures)
        a.noise_corr = _p(noise_corr)
        a.profile = int(cfg.profile)
        a.spergel_nu = float(cfg.spergel_nu)
        a.pixel_weight = _p(pixel_weight)
        a.pixel_prec = _p(pixel_prec)
        a.prec_offsets = _p(prec_offsets)
        a.chains_per_cta = int(chains_per_cta)
        self.args = a
        S, Cn = cfg.n_samples, cfg.n_chains
        f32 = dict(dtype=torch.float32, device=dev)
        self.samples = torch.empty((6, n_gal, Cn, S), **f32)
        self.logp = torch.empty((n_gal, Cn, S), **f32) if "logp" in want else None
        self.accepted = torch.empty((n_gal, Cn, S), dtype=torch.uint8, device=dev) if "accepted" in want else None
        self.accept_rate = torch.empty((n_gal, Cn), **f32) if "accept_rate" in want else None
        self.step_size = torch.empty((n_gal, Cn), **f32) if "step_size" in want else None
        self.inv_mass = torch.empty((n_gal, Cn, 6), **f32) if "inv_mass" in want else None
        self.n_div = torch.empty((n_gal, Cn), dtype=torch.int32, device=dev) if "n_div" in want else None
        self.status = torch.empty((n_gal,), dtype=torch.int32, device=dev) if "status" in want else None
        self.n_grad = torch.empty((n_gal, Cn), dtype=torch.int32, device=dev) if "n_grad" in want else None
        self.warm_accepted = (torch.empty((n_gal, Cn, cfg.n_warmup), dtype=torch.uint8, device=dev)
                              if "warm_accepted" in want else None)
        self.warm_stat = torch.empty((n_gal, Cn, cfg.n_warmup), **f32) if "warm_stat" in want else None
        self.warm_step = torch.empty((n_gal, Cn, cfg.n_warmup), **f32) if "warm_step" in want else None
        o = F.FitOut()
        o.samples = _p(self.samples)
        o.logp = _p(self.logp)
        o.accepted = _p(self.accepted)
        o.accept_rate = _p(self.accept_rate)
        o.step_size = _p(self.step_size)
        o.inv_mass = _p(self.inv_mass)
        o.n_divergent = _p(self.n_div)
        o.status = _p(self.status)
        o.n_grad = _p(self.n_grad)
        o.warmup_accepted = _p(self.warm_accepted)
        o.warmup_accept_stat = _p(self.warm_stat)
        o.warmup_step_size = _p(self.warm_step)
        self.out = o
        self.ws_bytes = F.lib().bs_fit_workspace_bytes(C.byref(a))
        self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=dev)

    def run(self, stream=None):
        st = C.c_void_p(stream.cuda_stream) if stream is not None else _stream()
        F.check(F.lib().bs_fit_galaxies(C.byref(self.args), C.byref(self.out), _p(self.ws),
                                        self.ws_bytes, st))
        return self

    def result(self):
        return dict(samples=self.samples, logp=self.logp, accepted=self.accepted,
                    accept_rate=self.accept_rate, step_size=self.step_size, inv_mass=self.inv_mass,
                    n_div=self.n_div, status=self.status, n_grad=self.n_grad,
                    warm_accepted=self.warm_accepted, warm_stat=self.warm_stat, warm_step=self.warm_step)


class RaggedFitPlan(FitPlan):
    """A FitPlan over stamps of mixed sizes: galaxies are grouped by column-slot
    class, each class runs its own persistent launch sized for it, and (with
    capture) the launches replay as one CUDA graph (bs_fit_plan_*)."""

    def __init__(self, data, offsets, side, psf, noise_sigma, init, cfg: FitConfig, *, capture=True,
                 autotune=False, **kw):
        super().__init__(data, offsets, side, psf, noise_sigma, init, cfg, **kw)
        side_h = np.ascontiguousarray(side.cpu().numpy(), dtype=np.int32)
        self.plan_ws_bytes = F.lib().bs_fit_plan_workspace_bytes(C.byref(self.args))
        self.plan_ws = torch.empty(self.plan_ws_bytes, dtype=torch.uint8, device=data.device)
        h = C.c_void_p()
        F.check(F.lib().bs_fit_plan_create(C.byref(self.args), C.byref(self.out), side_h.ctypes.data_as(C.c_void_p),
                                           (F.BS_PLAN_CAPTURE if capture else 0) |
                                           (F.BS_PLAN_AUTOTUNE if autotune else 0), _p(self.plan_ws),
                                           self.plan_ws_bytes, _stream(), C.byref(h)))
        self.handle = h

    def info(self):
        """Per class launch: slot class, largest side, galaxies, grid, register
        budget and the autotune trial times (ms)."""
        out = []
        for i in range(F.lib().bs_fit_plan_num_launches(self.handle)):
            r = F.PlanLaunchInfo()
            F.check(F.lib().bs_fit_plan_info(self.handle, i, C.byref(r)))
            out.append({n: getattr(r, n) for n, _ in F.PlanLaunchInfo._fields_})
        return out

    def run(self, stream=None):
        st = C.c_void_p(stream.cuda_stream) if stream is not None else _stream()
        F.check(F.lib().bs_fit_plan_launch(self.handle, st))
        return self

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            F.lib().bs_fit_plan_destroy(h)
            self.handle = None


REQUEST_DTYPE = F.struct_dtype(F.ServeRequest)
COMPLETION_DTYPE = F.struct_dtype(F.ServeCompletion)


class Server:
    """Fit requests admitted while others run (bs_serve_*): FIFO admission by
    arena memory and an in-flight cap, one CTA per galaxy, results delivered
    to pinned host memory.  The arena is a torch uint8 tensor owned here."""

    def __init__(self, cfg: FitConfig, *, max_side=101, arena_bytes=256 << 20, max_inflight=0, batch_us=0,
                 n_streams=0, registers=(0, 0, 0, 0), device="cuda"):
        """registers: fit-kernel register cap per slot class (e.g. from a
        RaggedFitPlan(autotune=True).info()); 0 = 128."""
        self.cfg = cfg
        self.arena = torch.empty(int(arena_bytes), dtype=torch.uint8, device=device)
        c = F.ServeCfg()
        c.max_side = max_side
        c.pixel_scale = cfg.pixel_scale
        c.prior = F.Prior(*cfg.prior)
        c.n_chains, c.n_warmup, c.n_samples, c.n_leapfrog = cfg.n_chains, cfg.n_warmup, cfg.n_samples, cfg.n_leapfrog
        c.target_accept, c.jitter = cfg.target_accept, cfg.jitter
        c.adapt_mass, c.random_steps, c.seed = int(cfg.adapt_mass), int(cfg.random_steps), cfg.seed
        c.max_inflight, c.batch_us, c.n_streams = max_inflight, batch_us, n_streams
        for i, r in enumerate(registers):
            c.registers[i] = int(r)
        self.scfg = c
        torch.cuda.synchronize(self.arena.device)
        h = C.c_void_p()
        with torch.cuda.device(self.arena.device):
            F.check(F.lib().bs_serve_create(C.byref(c), _p(self.arena), int(arena_bytes), C.byref(h)))
        self.handle = h
        self._cbuf = (F.ServeCompletion * 8192)()
        self._keep = []

    @staticmethod
    def requests(stamps, offsets, sides, psf_kind, fwhm, beta, noise_sigma, init, gal_id, tags=None,
                 t_arrival_ns=None, init_index=None):
        """Structured array of bs_serve_request pointing into host arrays:
        stamps float32 (flat, stamp i at offsets[i]), init float32 [m, C, 6]
        (request i starts from init[init_index[i]], default init[i]).
        The caller keeps `stamps` and `init` alive until the completions."""
        assert stamps.dtype == np.float32 and stamps.flags.c_contiguous
        assert init.dtype == np.float32 and init.flags.c_contiguous
        n = len(sides)
        r = np.zeros(n, dtype=REQUEST_DTYPE)
        r["tag"] = np.arange(n) if tags is None else tags
        r["gal_id"] = gal_id
        r["side"] = sides
        r["psf_kind"] = {"gaussian": F.BS_PSF_GAUSSIAN, "moffat": F.BS_PSF_MOFFAT}.get(psf_kind, psf_kind)
        r["psf_fwhm"] = fwhm
        r["psf_beta"] = beta
        r["noise_sigma"] = noise_sigma
        r["stamp"] = stamps.ctypes.data + 4 * np.asarray(offsets, dtype=np.int64)
        per = init[0].nbytes if len(init) else 0
        ii = np.arange(n, dtype=np.int64) if init_index is None else np.asarray(init_index, dtype=np.int64)
        r["init"] = init.ctypes.data + per * ii
        r["t_arrival_ns"] = -1 if t_arrival_ns is None else t_arrival_ns
        return r

    def submit(self, reqs):
        reqs = np.ascontiguousarray(reqs, dtype=REQUEST_DTYPE)
        F.check(F.lib().bs_serve_submit(self.handle, reqs.ctypes.data, len(reqs)))

    def poll(self, max_n=8192, timeout_us=0):
        """Completions as a structured array (COMPLETION_DTYPE); their result
        pointers stay valid until the next poll."""
        n = C.c_int32(0)
        F.check(F.lib().bs_serve_poll(self.handle, self._cbuf, min(max_n, len(self._cbuf)), int(timeout_us),
                                      C.byref(n)))
        raw = np.frombuffer(self._cbuf, dtype=COMPLETION_DTYPE, count=n.value)
        return raw.copy()

    def result(self, comp):
        """Copy one completion's results (valid until the next poll) into numpy."""
        Cn, S = self.cfg.n_chains, self.cfg.n_samples
        cs = Cn * S

        def arr(ptr, ctype, count, dtype):
            return np.frombuffer((ctype * count).from_address(int(ptr)), dtype=dtype).copy()
        stride = int(comp["plane_stride"])
        samples = np.stack([arr(int(comp["samples"]) + 4 * k * stride, C.c_float, cs, np.float32)
                            for k in range(6)]).reshape(6, Cn, S)
        return dict(samples=samples, logp=arr(comp["logp"], C.c_float, cs, np.float32).reshape(Cn, S),
                    accepted=arr(comp["accepted"], C.c_uint8, cs, np.uint8).reshape(Cn, S),
                    accept_rate=arr(comp["accept_rate"], C.c_float, Cn, np.float32),
                    step_size=arr(comp["step_size"], C.c_float, Cn, np.float32),
                    inv_mass=arr(comp["inv_mass"], C.c_float, 6 * Cn, np.float32).reshape(Cn, 6),
                    n_div=arr(comp["n_divergent"], C.c_int32, Cn, np.int32),
                    n_grad=arr(comp["n_grad"], C.c_int32, Cn, np.int32), status=int(comp["status"]))

    def stats(self):
        s = F.ServeStats()
        F.check(F.lib().bs_serve_get_stats(self.handle, C.byref(s)))
        return {n: getattr(s, n) for n, _ in F.ServeStats._fields_}

    def now_ns(self):
        return F.lib().bs_serve_now_ns(self.handle)

    def close(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            self.handle = None
            F.check(F.lib().bs_serve_destroy(h))

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fp32_peak_tflops(packed=False):
    """Measured FP32 FMA throughput of the current GPU (TFLOP/s, FMA = 2)."""
    t = C.c_double(0)
    F.check(F.lib().bs_fp32_peak(int(packed), C.cast(C.byref(t), C.c_void_p), _stream()))
    return t.value


def kernel_launches():
    """Kernels the library has launched in this process so far (graph replays
    count the kernels they hold); the difference over a region counts its
    launches."""
    return int(F.lib().bs_kernel_launches())


def fp64_peak_tflops():
    """Measured FP64 FMA throughput of the current GPU (TFLOP/s, FMA = 2)."""
    t = C.c_double(0)
    F.check(F.lib().bs_fp64_peak(C.cast(C.byref(t), C.c_void_p), _stream()))
    return t.value


def resident_galaxies(n_chains, max_side, registers=0):
    """Galaxies of side max_side one fit launch holds at once on the current GPU
    with the given register cap (0 = 128)."""
    return int(F.lib().bs_fit_resident_galaxies(n_chains, max_side, int(registers)))


def fit_galaxies(data, offsets, side, psf, noise_sigma, init, cfg: FitConfig | None = None, **kw):
    """fit_galaxies(stamps, psf, noise_sigma, prior, n_samples) -> interim samples
    (Sec. 3.3 image sampling phase).  Returns a dict of CUDA tensors; samples
    are [6, n_gal, n_chains, n_samples]."""
    cfg = cfg or FitConfig(n_chains=init.shape[1])
    want = kw.pop("want", ("logp", "accepted", "accept_rate", "step_size", "inv_mass", "n_div", "status",
                           "n_grad"))
    return FitPlan(data, offsets, side, psf, noise_sigma, init, cfg, want=want, **kw).run().result()


def logpost_points(data, offsets, side, psf, noise_sigma, gal_index, theta, *, max_side=None,
                   pixel_scale=PIXEL_SCALE, prior=DEFAULT_PRIOR, n_exposures=1, noise_corr=None, profile=0,
                   spergel_nu=0.5, pixel_weight=None, pixel_prec=None, prec_offsets=None):
    """Log posterior (float64) and gradient (float32) at points theta [n, 6]
    (n_exposures, noise_corr, pixel_weight, pixel_prec, prec_offsets as in
    FitPlan; profile, spergel_nu as in FitConfig)."""
    _need_cuda(data, offsets, side, noise_sigma, gal_index, theta, noise_corr, pixel_weight, pixel_prec,
               prec_offsets)
    table, n_psf = psf
    a = F.FitArgs()
    a.n_gal = int(side.shape[0])
    a.data_dtype = F.BS_F64 if data.dtype == torch.float64 else F.BS_F32
    a.data = _p(data)
    a.offsets = _p(offsets)
    a.side = _p(side)
    a.max_side = int(max_side or int(side.max().item()))
    a.psf = _p(table)
    a.n_psf = n_psf
    a.noise_sigma = _p(noise_sigma)
    a.pixel_scale = pixel_scale
    a.prior = F.Prior(*prior)
    a.n_exposures = int(n_exposures)
    a.noise_corr = _p(noise_corr)
    a.profile = int(profile)
    a.spergel_nu = float(spergel_nu)
    a.pixel_weight = _p(pixel_weight)
    a.pixel_prec = _p(pixel_prec)
    a.prec_offsets = _p(prec_offsets)
    n = theta.shape[0]
    lp = torch.empty(n, dtype=torch.float64, device=theta.device)
    g = torch.empty((n, 6), dtype=torch.float32, device=theta.device)
    F.check(F.lib().bs_logpost_points(C.byref(a), n, _p(gal_index), _p(theta.contiguous()), _p(lp),
                                      _p(g), _stream()))
    return lp, g


def dense_precision(cov, cov_offsets, side, max_side=None):
    """Precision matrices Sigma^-1 of general pixel covariances
    (bs_dense_precision; Appendix C): cov float32 CUDA, galaxy n's
    [N^2, N^2] block at cov_offsets[n] (int64 CUDA), side int32 CUDA.
    Returns (prec in the same layout, status int32 [n_gal]: 3 where Sigma is
    not positive definite)."""
    _need_cuda(cov, cov_offsets, side)
    n_gal = int(side.shape[0])
    ms = int(max_side or int(side.max().item()))
    prec = torch.empty_like(cov)
    status = torch.zeros(n_gal, dtype=torch.int32, device=cov.device)
    wsb = F.lib().bs_dense_precision_workspace_bytes(ms)
    ws = torch.empty(max(int(wsb), 1), dtype=torch.uint8, device=cov.device)
    F.check(F.lib().bs_dense_precision(n_gal, _p(side), ms, _p(cov.contiguous()), _p(cov_offsets), _p(prec),
                                       _p(status), _p(ws), wsb, _stream()))
    return prec, status


def chain_ess(samples):
    """ESS and R-hat per galaxy and parameter from samples [6, n_gal, C, S]."""
    _need_cuda(samples)
    _, n_gal, Cn, S = samples.shape
    ess = torch.empty((n_gal, 6), dtype=torch.float32, device=samples.device)
    rh = torch.empty((n_gal, 6), dtype=torch.float32, device=samples.device)
    F.check(F.lib().bs_chain_ess(_p(samples.contiguous()), n_gal, Cn, S, _p(ess), _p(rh), _stream()))
    return ess, rh


class ShearPlan:
    """Interim ellipticity samples plus the workspace of bs_shear_loglike."""

    def __init__(self, e1, e2, b=None, *, family=F.BS_EPRIOR_BA14, trunc_r=0.7, sigma_e0=0.3, weights=None):
        _need_cuda(e1, e2, b)
        if e1.dim() != 2 or e1.shape != e2.shape:
            raise ValueError("e1, e2 must be [n_gal, K]")
        self.keep = (e1.contiguous(), e2.contiguous(), None if b is None else b.contiguous())
        e1c, e2c, bc = self.keep
        d = F.ShearData()
        d.e1, d.e2, d.b = _p(e1c), _p(e2c), _p(bc)
        d.n_gal, d.K = e1.shape
        d.family = family
        d.trunc_r = trunc_r
        d.sigma_e0 = sigma_e0
        self.data = d
        self.ws_bytes = F.lib().bs_shear_workspace_bytes(d.n_gal, d.K)
        self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=e1.device)
        self.out = torch.empty(4, dtype=torch.float64, device=e1.device)
        self._host = np.zeros(4)
        self.set_weights(weights)

    def set_weights(self, weights, weight_sum=None):
        """Per-galaxy weights w_n >= 0 of the galaxies' log-likelihood terms
        (None: all 1).  Integer weights are a bootstrap resample: w_n copies of
        galaxy n.  numpy or CUDA [n_gal]; weight_sum (sum of w) is computed when
        not given (a device sync for a CUDA tensor)."""
        d = self.data
        if weights is None:
            self._w = None
            d.gal_weight, d.gal_weight_sum = None, 0.0
            return
        dev = self.keep[0].device
        if isinstance(weights, torch.Tensor):
            w = weights.to(device=dev, dtype=torch.float32).contiguous()
        else:
            wn = np.ascontiguousarray(weights, dtype=np.float32)
            if weight_sum is None:
                if not (np.isfinite(wn).all() and (wn >= 0).all()):
                    raise ValueError("weights must be finite and >= 0")
                weight_sum = float(wn.astype(np.float64).sum())
            w = torch.from_numpy(wn).to(dev)
        if w.shape != (d.n_gal,):
            raise ValueError("weights must be [n_gal]")
        if weight_sum is None:
            if not bool(torch.isfinite(w).all() and (w >= 0).all()):
                raise ValueError("weights must be finite and >= 0")
            weight_sum = float(w.double().sum())
        self._w = w
        d.gal_weight, d.gal_weight_sum = _p(w), float(weight_sum)

    def loglike(self, g1, g2, alpha, *, host=False):
        """(value, d/dg1, d/dg2, d/dalpha): a float64 CUDA tensor (async) or,
        with host=True, a numpy array (synchronises)."""
        if host:
            buf = self._host
            F.check(F.lib().bs_shear_loglike(C.byref(self.data), g1, g2, alpha,
                                             buf.ctypes.data_as(C.c_void_p), 1, _p(self.ws),
                                             self.ws_bytes, _stream()))
            return buf.copy()
        F.check(F.lib().bs_shear_loglike(C.byref(self.data), g1, g2, alpha, _p(self.out), 0, _p(self.ws),
                                         self.ws_bytes, _stream()))
        return self.out

    def loglike_multi(self, points, *, host=True):
        """(value, d/dg1, d/dg2, d/dalpha) at points [n, 3] = (g1, g2, alpha),
        several points per pass over the samples (bs_shear_loglike_multi).
        Returns a numpy [n, 4] array (host=True, synchronises) or a float64
        CUDA tensor [n, 4]."""
        pts = np.ascontiguousarray(points, dtype=np.float64).reshape(-1, 3)
        n = pts.shape[0]
        if host:
            out = np.zeros((n, 4))
            F.check(F.lib().bs_shear_loglike_multi(C.byref(self.data), n, pts.ctypes.data_as(C.c_void_p),
                                                   out.ctypes.data_as(C.c_void_p), 1, _p(self.ws), self.ws_bytes,
                                                   _stream()))
            return out
        out = torch.empty((n, 4), dtype=torch.float64, device=self.keep[0].device)
        F.check(F.lib().bs_shear_loglike_multi(C.byref(self.data), n, pts.ctypes.data_as(C.c_void_p), _p(out), 0,
                                               _p(self.ws), self.ws_bytes, _stream()))
        return out

    def loglike_full(self, lf, ls, theta, *, interim=(-1.0, 9.0, -2.0, 1.0)):
        """All properties free: lf, ls [n_gal, K] float32 CUDA (log10 flux and
        log10 hlr samples); theta = (g1, g2, sigma_e, mu_f, sigma_f, a_f, mu_s,
        sigma_s).  Returns numpy (value, gradient[8]) (synchronises)."""
        _need_cuda(lf, ls)
        if self.keep[2] is not None:
            raise ValueError("the all-free likelihood takes no b offsets")
        self._full_keep = (lf.contiguous(), ls.contiguous())
        th = np.ascontiguousarray(theta, dtype=np.float64)
        im = np.ascontiguousarray(interim, dtype=np.float64)
        buf = np.zeros(9)
        F.check(F.lib().bs_shear_loglike_full(C.byref(self.data), _p(self._full_keep[0]), _p(self._full_keep[1]),
                                              im.ctypes.data_as(C.c_void_p), th.ctypes.data_as(C.c_void_p),
                                              buf.ctypes.data_as(C.c_void_p), 1, _p(self.ws), self.ws_bytes,
                                              _stream()))
        return buf[0], buf[1:].copy()

    def _sample_cfg(self, theta0, *, free=("g1", "g2"), lf=None, ls=None, lo=None, hi=None, n_warmup=500,
                    n_samples=1000, n_leapfrog=8, target_accept=0.8, random_steps=True, seed=2604,
                    interim=(-1.0, 9.0, -2.0, 1.0), allreduce=None):
        """bs_shear_sample_cfg and the objects it points to (kept alive by the caller)."""
        names = ("g1", "g2", "sigma_e", "mu_f", "sigma_f", "a_f", "mu_s", "sigma_s")
        c = F.ShearSampleCfg()
        c.free_mask = sum(1 << names.index(n) for n in free)
        dlo, dhi = (C.c_double * 8)(), (C.c_double * 8)()
        F.lib().bs_shear_hyperprior_default(dlo, dhi)
        for i in range(8):
            c.theta0[i] = float(theta0[i])
            c.lo[i] = float(lo[i]) if lo is not None else dlo[i]
            c.hi[i] = float(hi[i]) if hi is not None else dhi[i]
        keep = None
        if lf is not None or ls is not None:
            _need_cuda(lf, ls)
            keep = (lf.contiguous(), ls.contiguous())
            c.lf, c.ls = _p(keep[0]), _p(keep[1])
        for i in range(4):
            c.interim[i] = float(interim[i])
        c.n_warmup, c.n_samples, c.n_leapfrog = n_warmup, n_samples, n_leapfrog
        c.target_accept, c.random_steps, c.seed = target_accept, int(random_steps), seed
        cb = _allreduce_cb(allreduce)
        if cb is not None:
            c.allreduce = cb
        return c, (keep, cb)

    def sample(self, theta0, **kw):
        """HMC over g and the named hyperparameters (bs_shear_sample).
        theta0: (g1, g2, sigma_e, mu_f, sigma_f, a_f, mu_s, sigma_s) start and
        fixed values; keywords free, lf, ls (log-flux / log-size samples, CUDA
        [n_gal, K], for the all-free likelihood), lo, hi, n_warmup, n_samples,
        n_leapfrog, target_accept, random_steps, seed, interim, allreduce.
        Returns (samples [n_samples, 8], info)."""
        c, keep = self._sample_cfg(theta0, **kw)
        out = np.zeros((c.n_samples, 8))
        acc, eps, nev = C.c_double(0), C.c_double(0), C.c_int32(0)
        F.check(F.lib().bs_shear_sample(C.byref(self.data), C.byref(c), out.ctypes.data_as(C.c_void_p),
                                        C.cast(C.byref(acc), C.c_void_p), C.cast(C.byref(eps), C.c_void_p),
                                        C.cast(C.byref(nev), C.c_void_p), _p(self.ws), self.ws_bytes, _stream()))
        del keep
        return out, {"accept_rate": acc.value, "step_size": eps.value, "n_evals": nev.value}

    @staticmethod
    def _estimate_cfg(*, free_alpha=False, alpha=0.2, alpha_lo=1e-4, alpha_hi=1.0, n_gh=7, allreduce=None):
        cfg = F.EstimateCfg()
        cfg.free_alpha = int(free_alpha)
        cfg.alpha = alpha
        cfg.alpha_lo = alpha_lo
        cfg.alpha_hi = alpha_hi
        cfg.n_gh = n_gh
        cb = _allreduce_cb(allreduce)
        if cb is not None:
            cfg.allreduce = cb
        return cfg, cb

    def estimate(self, **kw):
        """Posterior mean and covariance of (g1, g2[, alpha]) (numpy);
        keywords free_alpha, alpha, alpha_lo, alpha_hi, n_gh, allreduce."""
        cfg, cb = self._estimate_cfg(**kw)
        mean = np.zeros(3)
        cov = np.zeros(9)
        nev = C.c_int32(0)
        F.check(F.lib().bs_shear_estimate(C.byref(self.data), C.byref(cfg), mean.ctypes.data_as(C.c_void_p),
                                          cov.ctypes.data_as(C.c_void_p), C.cast(C.byref(nev), C.c_void_p),
                                          _p(self.ws), self.ws_bytes, _stream()))
        del cb
        self.last_n_evals = nev.value
        n = 3 if cfg.free_alpha else 2
        return mean[:n], cov.reshape(3, 3)[:n, :n]


def shear_estimate_custom(loglike, **kw):
    """bs_shear_estimate_custom: the library's posterior-mean estimate of g
    (and alpha) over the caller's likelihood loglike(points [m, 3]) ->
    [m, 4] (value, d/dg1, d/dg2, d/dalpha; numpy), on the host.  Keywords as
    ShearPlan.estimate (allreduce included).  Returns (mean, cov, n_evals)."""
    cfg, cb = ShearPlan._estimate_cfg(**kw)
    errors = []

    def f(xp, m, outp, user):
        try:
            x = np.ctypeslib.as_array(xp, shape=(m, 3)).copy()
            o = np.asarray(loglike(x), dtype=np.float64).reshape(m, 4)
            np.ctypeslib.as_array(outp, shape=(m, 4))[:] = o
            return 0
        except Exception as e:          # reported after the call returns
            errors.append(e)
            return 1

    fn = F.LOGLIKE_POINTS_FN(f)
    mean, cov, nev = np.zeros(3), np.zeros(9), C.c_int32(0)
    st = F.lib().bs_shear_estimate_custom(fn, None, C.byref(cfg), mean.ctypes.data_as(C.c_void_p),
                                          cov.ctypes.data_as(C.c_void_p), C.cast(C.byref(nev), C.c_void_p))
    if errors:
        raise errors[0]
    F.check(st)
    del fn, cb
    n = 3 if cfg.free_alpha else 2
    return mean[:n], cov.reshape(3, 3)[:n, :n], nev.value


def _allreduce_cb(allreduce):
    """The C callback summing the 4 doubles of an evaluation over ranks."""
    if allreduce is None:
        return None

    def _cb(buf, user):
        arr = np.ctypeslib.as_array(buf, shape=(4,))
        arr[:] = allreduce(arr.copy())
    return F.ALLREDUCE_FN(_cb)


def _bias_cfg(n_gal, g_abs, n_boot, seed, base_weights):
    cfg = F.BiasCfg()
    cfg.g_abs, cfg.n_boot, cfg.seed = float(g_abs), int(n_boot), int(seed)
    base = None
    if base_weights is not None:
        base = np.ascontiguousarray(base_weights, dtype=np.float32)
        if base.shape != (n_gal,):
            raise ValueError("base_weights must be [n_gal]")
        cfg.base_weight = base.ctypes.data_as(C.c_void_p)
    boot = np.full((2, max(int(n_boot), 0)), np.nan)
    cfg.m_boot = boot[0].ctypes.data_as(C.c_void_p)
    cfg.c_boot = boot[1].ctypes.data_as(C.c_void_p)
    return cfg, base, boot


def _bias_result(out, boot):
    return {"m": float(out[0]), "c": float(out[1]), "m_sd": float(out[2]), "c_sd": float(out[3]),
            "m_boot": boot[0].copy(), "c_boot": boot[1].copy()}


def shear_bias(estimate_plus, estimate_minus, n_gal, *, g_abs=0.02, n_boot=500, seed=0, base_weights=None):
    """Multiplicative and additive bias by shape-noise cancellation (Sec. 3.4)
    with bootstrap errors, through bs_shear_bias_custom: estimate_plus /
    estimate_minus map per-galaxy weights (numpy float32 [n_gal], or None for
    the original sample) to the estimate (g1, g2) of the datasets sheared by
    +g and -g, g = (g_abs, 0).  Returns m, c, their bootstrap standard
    deviations m_sd, c_sd and the per-resample m_boot, c_boot."""
    cfg, base, boot = _bias_cfg(n_gal, g_abs, n_boot, seed, base_weights)
    errors = []

    def wrap(f):
        def cb(wp, wsum, gout, user):
            try:
                w = np.ctypeslib.as_array(wp, shape=(n_gal,)).copy() if wp else None
                g = f(w)
                gout[0], gout[1] = float(g[0]), float(g[1])
                return 0
            except Exception as e:          # reported after the call returns
                errors.append(e)
                return 1
        return F.G_ESTIMATOR_FN(cb)

    cbp, cbm = wrap(estimate_plus), wrap(estimate_minus)
    out = np.zeros(4)
    st = F.lib().bs_shear_bias_custom(int(n_gal), cbp, None, cbm, None, C.byref(cfg), out.ctypes.data_as(C.c_void_p))
    if errors:
        raise errors[0]
    F.check(st)
    del cbp, cbm, base
    return _bias_result(out, boot)


def shear_bias_plans(plan_plus, plan_minus, *, g_abs=0.02, n_boot=500, seed=0, method="quadrature",
                     base_weights=None, **kw):
    """shear_bias on the GPU (bs_shear_bias) with the posterior mean of g from
    two ShearPlans as the estimator: method "quadrature" (bs_shear_estimate,
    keywords as ShearPlan.estimate) or "hmc" (the mean of bs_shear_sample's g
    draws, keywords as ShearPlan.sample, theta0 included).  base_weights
    (numpy [n_gal], optional) multiply every resample's counts, e.g. 0 for
    galaxies left out of both datasets.  The plans' own weights are not used
    and not changed."""
    n = plan_plus.data.n_gal
    if plan_minus.data.n_gal != n:
        raise ValueError("the +g and -g datasets must hold the same galaxies")
    cfg, base, boot = _bias_cfg(n, g_abs, n_boot, seed, base_weights)
    est = smp = keep = None
    if method == "quadrature":
        est, keep = ShearPlan._estimate_cfg(**kw)
        mcode = F.BS_BIAS_QUADRATURE
    elif method == "hmc":
        smp, keep = plan_plus._sample_cfg(**kw)
        mcode = F.BS_BIAS_HMC
    else:
        raise ValueError("method: quadrature or hmc")
    big = plan_plus if plan_plus.ws_bytes >= plan_minus.ws_bytes else plan_minus
    wdev = torch.empty(n, dtype=torch.float32, device=plan_plus.keep[0].device)
    out = np.zeros(4)
    F.check(F.lib().bs_shear_bias(C.byref(plan_plus.data), C.byref(plan_minus.data), mcode,
                                  C.byref(est) if est is not None else None,
                                  C.byref(smp) if smp is not None else None, C.byref(cfg), _p(wdev),
                                  out.ctypes.data_as(C.c_void_p), _p(big.ws), big.ws_bytes, _stream()))
    del keep, base
    return _bias_result(out, boot)


def shear_loglike(e1, e2, g1, g2, alpha, *, b=None, family=F.BS_EPRIOR_BA14, trunc_r=0.7, sigma_e0=0.3):
    """shear_loglike(samples, g, alpha) -> (value, grad[3]) as numpy."""
    v = ShearPlan(e1, e2, b, family=family, trunc_r=trunc_r, sigma_e0=sigma_e0).loglike(g1, g2, alpha, host=True)
    return v[0], v[1:]


class ShearLogLike(torch.autograd.Function):
    """Eq. likelihood-shear as a differentiable function of (g1, g2, alpha);
    the backward uses the gradient from the same kernel pass (the adjoint of
    the streaming log-sum-exp), nothing is recomputed on the host."""

    @staticmethod
    def forward(ctx, params, plan: ShearPlan):
        g1, g2, alpha = [float(x) for x in params.detach().cpu().double()]
        out = plan.loglike(g1, g2, alpha, host=True)
        ctx.save_for_backward(torch.tensor(out[1:], dtype=torch.float64))
        return torch.tensor(out[0], dtype=torch.float64)

    @staticmethod
    def backward(ctx, gout):
        (g,) = ctx.saved_tensors
        return (gout * g).to(torch.float64), None


class RenderLogPost(torch.autograd.Function):
    """Log posterior of galaxy parameters theta [n, 6] under their stamps,
    differentiable in theta.  The forward saves only theta; the gradient comes
    from the adjoint evaluation of the fit kernel (the model stamp is never
    stored)."""

    @staticmethod
    def forward(ctx, theta, data, offsets, side, psf, noise_sigma, gal_index):
        lp, g = logpost_points(data, offsets, side, psf, noise_sigma, gal_index, theta.detach().float())
        ctx.save_for_backward(g)
        return lp

    @staticmethod
    def backward(ctx, gout):
        (g,) = ctx.saved_tensors
        return (gout[:, None].to(g.dtype) * g).to(torch.float32), None, None, None, None, None, None
