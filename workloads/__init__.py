"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This module only draws random numbers and shapes them into images and raw
filter draws.  It holds none of the OCSC method's arithmetic (no FFT-domain
solves, no projections, no normalisation of filters), so that the oracle and
the CUDA path can both consume its arrays without sharing method code.

Image recipe (stand-in for the paper's Fruit/City/House/Flower/Dog/CIFAR
images, which are preprocessed by grayscale conversion and local contrast
normalisation in Sec. IV):
  1. a Gaussian random field with 1/f amplitude spectrum (white complex
     Gaussian spectrum times 1/max(|f|, 1), DC removed),
  2. plus Poisson(6) discs with uniform centres, radius U[3, side/6] and a
     N(0, 1) piecewise-constant level,
  3. minus a Gaussian-blurred local mean (sigma = 4 px),
  4. then standardised to zero mean and unit variance.

Seeds are splitmix64-derived from (config id, image index); splitmix64 is the
published generator of Steele, Lea and Flood (OOPSLA 2014).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

_MASK = (1 << 64) - 1


def splitmix64(x: int) -> int:
    """One output of splitmix64 for state ``x`` (Steele, Lea & Flood 2014)."""
    z = (x + 0x9E3779B97F4A7C15) & _MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
    return z ^ (z >> 31)


def seed_for(config_id: int, index: int) -> int:
    return splitmix64(splitmix64(config_id) ^ (index & _MASK))


def _gauss_blur_periodic(img: np.ndarray, sigma: float) -> np.ndarray:
    h, w = img.shape
    fy = np.fft.fftfreq(h)[:, None]
    fx = np.fft.fftfreq(w)[None, :]
    g = np.exp(-2.0 * (math.pi ** 2) * (sigma ** 2) * (fy ** 2 + fx ** 2))
    return np.real(np.fft.ifft2(np.fft.fft2(img) * g))


def make_image(h: int, w: int, seed: int) -> np.ndarray:
    """One synthetic contrast-normalised image, float32 [h, w]."""
    rng = np.random.default_rng(seed)
    spec = rng.standard_normal((h, w)) + 1j * rng.standard_normal((h, w))
    fy = np.fft.fftfreq(h)[:, None] * h
    fx = np.fft.fftfreq(w)[None, :] * w
    amp = 1.0 / np.maximum(np.sqrt(fy ** 2 + fx ** 2), 1.0)
    amp[0, 0] = 0.0
    field = np.real(np.fft.ifft2(spec * amp))
    field /= max(float(field.std()), 1e-12)
    yy, xx = np.mgrid[0:h, 0:w]
    side = min(h, w)
    for _ in range(int(rng.poisson(6))):
        cy, cx = rng.uniform(0, h), rng.uniform(0, w)
        rad = rng.uniform(3.0, max(3.0, side / 6.0))
        level = rng.standard_normal()
        field[(yy - cy) ** 2 + (xx - cx) ** 2 <= rad * rad] += level
    field = field - _gauss_blur_periodic(field, 4.0)
    field = (field - field.mean()) / max(float(field.std()), 1e-12)
    return field.astype(np.float32)


def raw_filters(K: int, M: int, seed: int) -> np.ndarray:
    """Raw N(0, 1) filter draws, float32 [K, M, M] (the method normalises them)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((K, M, M)).astype(np.float32)


@dataclasses.dataclass(frozen=True)
class Workload:
    """A named OCSC workload: sizes, parameters and the image stream."""

    name: str
    config_id: int
    n_images: int
    sides: tuple          # possible square image sides
    pad: int              # zeros appended per axis before the FFT
    K: int
    M: int
    lam: float
    rho: float
    batch: int
    Jz: int
    Jd: int
    side_range: tuple = ()   # (lo, hi): sides drawn log-uniformly instead of from `sides`

    def side_of(self, index: int) -> int:
        if self.side_range:
            rng = np.random.default_rng(seed_for(self.config_id + 1000, index))
            lo, hi = self.side_range
            return int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        if len(self.sides) == 1:
            return self.sides[0]
        rng = np.random.default_rng(seed_for(self.config_id + 1000, index))
        return int(self.sides[int(rng.integers(0, len(self.sides)))])

    def image(self, index: int) -> np.ndarray:
        s = self.side_of(index)
        return make_image(s, s, seed_for(self.config_id, index))

    def filters0(self) -> np.ndarray:
        return raw_filters(self.K, self.M, seed_for(self.config_id, 1 << 40))


WORKLOADS = {
    # 20 images 64x64, circular boundary (FFT 64), K=16 filters 8x8, B=1.
    "plain_64_k16": Workload("plain_64_k16", 1, 20, (64,), 0, 16, 8, 1.0, 1.0, 1, 50, 10),
    # 1000 images 100x100 zero-padded to 128x128, K=100 filters 11x11, B=1.
    "plain_100in128_k100": Workload("plain_100in128_k100", 2, 1000, (100,), 10, 100, 11,
                                    1.0, 1.0, 1, 50, 10),
    # 4096 images of side 64/128/256, padded by 10 to FFT 128/256/512, K=100, B=64.
    "batched_mixed_k100": Workload("batched_mixed_k100", 3, 4096, (64, 128, 256), 10, 100, 11,
                                   1.0, 1.0, 64, 50, 10),
    # Requests with side log-uniform in [64, 512], each padded by 10 to its FFT
    # class, K=100 filters 11x11, dictionary update every 64 completed requests.
    "serving_k100": Workload("serving_k100", 5, 20000, (), 10, 100, 11, 1.0, 1.0, 64, 500, 10,
                             side_range=(64, 512)),
    # 2048 images 256x256 padded to FFT 288, K=256, B=128.
    "precision_256_k256": Workload("precision_256_k256", 4, 2048, (256,), 32, 256, 11,
                                   1.0, 1.0, 128, 50, 10),
}
