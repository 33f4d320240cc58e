"""Test datasets: seeded draws from ``synth`` turned into noisy stamps by the
oracle's renderer (so no expected value or input of a parity test comes from
the CUDA path)."""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

import oracle as O
from paper_2604_22048_gb300 import synth


@dataclass
class Dataset:
    truth: synth.Truth
    theta: np.ndarray      # [n, 6] true parameters with the sheared ellipticity
    stamps: list           # list of [N, N] float64 arrays
    init: np.ndarray       # [n, n_chains, 6]
    psf: list              # oracle PSF tuples per galaxy
    sigma: np.ndarray


def psf_tuple(truth, i):
    if truth.psf_kind == "gaussian":
        return (O.PSF_GAUSSIAN, float(truth.psf_fwhm[i]))
    return (O.PSF_MOFFAT, float(truth.psf_fwhm[i]), float(truth.psf_beta))


def make_dataset(truth: synth.Truth, n_chains: int, sigma: float = 1.0, g=None, noise_seed=None,
                 pixel_scale=0.2) -> Dataset:
    g = truth.g if g is None else g
    n = truth.n
    theta = np.zeros((n, 6))
    for i in range(n):
        ep = O.shear_apply(truth.e_int[i, 0], truth.e_int[i, 1], g[0], g[1])
        theta[i] = [0.0, np.log10(truth.hlr[i]), ep[0], ep[1], truth.offset[i, 0], truth.offset[i, 1]]
    psfs = [psf_tuple(truth, i) for i in range(n)]
    unit = [None] * n
    for N in np.unique(truth.side):
        idx = np.nonzero(truth.side == N)[0]
        imgs = O.render_many(int(N), pixel_scale, [psfs[i] for i in idx], theta[idx])
        for j, i in enumerate(idx):
            unit[i] = imgs[j]
    kw = {} if noise_seed is None else {"seed": noise_seed}
    noise = synth.noise_fields(truth, sigma, **kw)
    stamps = []
    for i in range(n):
        F = truth.snr[i] * sigma / np.sqrt((unit[i] ** 2).sum())
        theta[i, 0] = np.log10(F)
        stamps.append(F * unit[i] + noise[i])
    sums = np.array([s.sum() for s in stamps])
    init = synth.initial_theta(sums, theta[:, 1], theta[:, 2:4], synth.init_offsets(truth, n_chains))
    return Dataset(truth, theta, stamps, init, psfs, np.full(n, sigma))


def pack(ds: Dataset, dtype=np.float32):
    """Flat packed stamps + int64 offsets (each start a multiple of 4)."""
    sides = np.array([s.shape[0] for s in ds.stamps])
    sizes = (sides * sides + 3) // 4 * 4
    offs = np.zeros(len(sides), dtype=np.int64)
    offs[1:] = np.cumsum(sizes)[:-1]
    flat = np.zeros(int(sizes.sum()), dtype=dtype)
    for o, s in zip(offs, ds.stamps):
        flat[o:o + s.size] = s.ravel()
    return flat, offs, sides.astype(np.int32)
