"""Synthetic inputs of the gene-regulatory-network classifier (784 -> 256 -> 10).

Weights are drawn once (seeded) and rounded to bfloat16, so that the values both implementations
receive are exactly representable in bf16; images are class-conditional prototypes with Gaussian
noise, clipped to [0, 1] and turned into copy numbers round(255 p). Nothing here simulates or
differentiates anything.

Initial weights (one reading of an unspecified initialisation): W1 ~ N(0, (2 / (255 sqrt(n_in)))^2),
W2 ~ N(0, 1/n_hid), b = 0, degradation rates d = 0.5 (d_min 0.25 plus 0.25), k_max = 1.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


def round_bf16(a: np.ndarray) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 (ties to even), returned as float32."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    rounded = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return rounded.astype(np.uint32).view(np.float32).copy()


@dataclass
class GRNParams:
    W1: np.ndarray      # float32 [n_hid, n_in], bf16-representable
    b1: np.ndarray      # float32 [n_hid]
    W2: np.ndarray      # float32 [n_out, n_hid], bf16-representable
    b2: np.ndarray      # float32 [n_out]
    log_d: np.ndarray   # float32 [n_hid + n_out]
    k_max: float = 1.0

    @property
    def n_in(self):
        return self.W1.shape[1]

    @property
    def n_hid(self):
        return self.W1.shape[0]

    @property
    def n_out(self):
        return self.W2.shape[0]


def grn_params(seed: int = 5, n_in: int = 784, n_hid: int = 256, n_out: int = 10, d0: float = 0.5,
               k_max: float = 1.0, w1_scale: float | None = None, w2_scale: float | None = None) -> GRNParams:
    rng = np.random.default_rng(seed)
    s1 = (2.0 / (255.0 * np.sqrt(n_in))) if w1_scale is None else w1_scale
    s2 = (1.0 / np.sqrt(n_hid)) if w2_scale is None else w2_scale
    W1 = round_bf16(rng.normal(0.0, s1, size=(n_hid, n_in)).astype(np.float32))
    W2 = round_bf16(rng.normal(0.0, s2, size=(n_out, n_hid)).astype(np.float32))
    return GRNParams(W1, np.zeros(n_hid, np.float32), W2, np.zeros(n_out, np.float32),
                     np.full(n_hid + n_out, np.log(d0), np.float32), float(k_max))


def prototype_images(seed: int = 5, n_img: int = 512, n_in: int = 784, n_classes: int = 10,
                     noise: float = 0.25) -> tuple[np.ndarray, np.ndarray]:
    """Counts int32 [n_img, n_in] in 0..255 and labels int64 [n_img] (label = index mod n_classes)."""
    rng = np.random.default_rng(seed)
    protos = (rng.random((n_classes, n_in)) < 0.2) * rng.uniform(0.5, 1.0, size=(n_classes, n_in))
    labels = np.arange(n_img) % n_classes
    p = np.clip(protos[labels] + rng.normal(0.0, noise, size=(n_img, n_in)), 0.0, 1.0)
    return np.rint(255.0 * p).astype(np.int32), labels.astype(np.int64)
