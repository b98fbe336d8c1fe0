"""Seeded synthetic workloads for the uplink and downlink system models.

This module only draws inputs: i.i.d. or exponentially correlated Rayleigh
channels, uniform bits, Gray QAM symbols and complex Gaussian noise
(Sec. II, Eq. 1). It holds none of the detection or precoding arithmetic and
is the one module that both the CUDA path and the CPU oracle consume.

Conventions (shared with the library's documented constellation):
  * SNR = U Es / N0 (Sec. II-A), so N0 = U Es 10^(-SNR/10).
  * Square Gray QAM, E|x|^2 = Es; bits b_0..b_{q/2-1} select the in-phase
    level and b_{q/2}..b_{q-1} the quadrature level, each read MSB-first as a
    Gray code of the level index.
  * Correlated channels: each user column is an AR(1) sequence over the BS
    antennas, h_0 = w_0, h_b = c h_{b-1} + sqrt(1 - c^2) w_b, which has
    covariance c^|i-j| between antennas i and j.

Two generators are provided: a NumPy PCG64 one (host arrays, used by the
tests and the oracle) and a torch one that draws on the device for the large
benchmark batches. They do not produce the same numbers for the same seed.
"""

from __future__ import annotations

import math

import numpy as np

QAM_BITS = (2, 4, 6, 8)


def snr_to_n0(snr_db: float, U: int, Es: float = 1.0) -> float:
    """N0 from the average uplink SNR U Es / N0 (Sec. II-A)."""
    return U * Es / (10.0 ** (snr_db / 10.0))


def pam_levels_by_gray_code(qam_bits: int, Es: float = 1.0) -> np.ndarray:
    """Per-axis amplitude for each Gray code word g (index g -> level)."""
    if qam_bits not in QAM_BITS:
        raise ValueError("qam_bits must be one of 2, 4, 6, 8")
    L = 1 << (qam_bits // 2)
    M = L * L
    scale = math.sqrt(3.0 * Es / (2.0 * (M - 1)))
    table = np.zeros(L)
    for j in range(L):                 # j runs over levels left to right
        table[j ^ (j >> 1)] = (2 * j - (L - 1)) * scale
    return table


def qam_map(bits: np.ndarray, qam_bits: int, Es: float = 1.0) -> np.ndarray:
    """Map bits[..., q] (0/1) to complex Gray QAM symbols[...]."""
    bits = np.asarray(bits).astype(np.int64)
    h = qam_bits // 2
    weights = 1 << np.arange(h - 1, -1, -1)
    gI = (bits[..., :h] * weights).sum(-1)
    gQ = (bits[..., h:] * weights).sum(-1)
    lv = pam_levels_by_gray_code(qam_bits, Es)
    return lv[gI] + 1j * lv[gQ]


def rayleigh(rng: np.random.Generator, n: int, B: int, U: int,
             corr: float | None = None) -> np.ndarray:
    """H[n, B, U] with CN(0, 1) entries, optionally AR(1)-correlated over B."""
    w = (rng.standard_normal((n, B, U)) + 1j * rng.standard_normal((n, B, U))) / math.sqrt(2.0)
    if corr is None or corr == 0.0:
        return w
    H = np.empty_like(w)
    H[:, 0, :] = w[:, 0, :]
    s = math.sqrt(1.0 - corr * corr)
    for b in range(1, B):
        H[:, b, :] = corr * H[:, b - 1, :] + s * w[:, b, :]
    return H


def uplink(B: int, U: int, qam_bits: int, n: int, R: int, snr_db: float,
           seed: int, Es: float = 1.0, corr: float | None = None,
           noiseless: bool = False) -> dict:
    """Uplink batch y = H x + n (Eq. 1): H[n, B, U], Y[n, R, B] complex64.

    R receive vectors (OFDM symbols) share one channel per instance.
    """
    rng = np.random.default_rng(seed)
    H = rayleigh(rng, n, B, U, corr)
    bits = rng.integers(0, 2, size=(n, R, U, qam_bits), dtype=np.uint8)
    x = qam_map(bits, qam_bits, Es)                     # [n, R, U]
    N0 = snr_to_n0(snr_db, U, Es)
    noise = (rng.standard_normal((n, R, B)) + 1j * rng.standard_normal((n, R, B))) \
        * math.sqrt(N0 / 2.0)
    y = np.matmul(H, np.swapaxes(x, 1, 2))              # [n, B, R]
    y = np.swapaxes(y, 1, 2)
    if not noiseless:
        y = y + noise
    return {"H": np.ascontiguousarray(H, dtype=np.complex64),
            "Y": np.ascontiguousarray(y, dtype=np.complex64),
            "bits": bits, "x": np.ascontiguousarray(x, dtype=np.complex64), "N0": float(N0), "Es": float(Es),
            "B": B, "U": U, "R": R, "qam_bits": qam_bits}


def downlink(B: int, U: int, qam_bits: int, n: int, R: int, snr_db: float,
             seed: int, Es: float = 1.0, corr: float | None = None) -> dict:
    """Downlink batch: uplink channel H[n, B, U] and symbols T[n, R, U] (Sec. II-B)."""
    rng = np.random.default_rng(seed)
    H = rayleigh(rng, n, B, U, corr)
    bits = rng.integers(0, 2, size=(n, R, U, qam_bits), dtype=np.uint8)
    T = qam_map(bits, qam_bits, Es)
    return {"H": np.ascontiguousarray(H, dtype=np.complex64),
            "T": np.ascontiguousarray(T, dtype=np.complex64), "bits": bits,
            "N0": float(snr_to_n0(snr_db, U, Es)), "Es": float(Es),
            "B": B, "U": U, "R": R, "qam_bits": qam_bits}


# ----------------------------------------------------------------------------
# Device-side generator for large batches
# ----------------------------------------------------------------------------

def uplink_torch(B: int, U: int, qam_bits: int, n: int, R: int, snr_db: float,
                 seed: int, device, Es: float = 1.0) -> dict:
    """Same model as uplink(), drawn with torch on `device` (i.i.d. channels)."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    f32 = torch.float32
    H = torch.complex(torch.randn((n, B, U), generator=g, device=device, dtype=f32),
                      torch.randn((n, B, U), generator=g, device=device, dtype=f32))
    H = H / math.sqrt(2.0)
    bits = torch.randint(0, 2, (n, R, U, qam_bits), generator=g, device=device,
                         dtype=torch.uint8)
    h = qam_bits // 2
    w = torch.tensor([1 << (h - 1 - t) for t in range(h)], device=device, dtype=torch.int64)
    lv = torch.tensor(pam_levels_by_gray_code(qam_bits, Es), device=device, dtype=f32)
    gI = (bits[..., :h].to(torch.int64) * w).sum(-1)
    gQ = (bits[..., h:].to(torch.int64) * w).sum(-1)
    x = torch.complex(lv[gI], lv[gQ])                   # [n, R, U]
    N0 = snr_to_n0(snr_db, U, Es)
    noise = torch.complex(torch.randn((n, R, B), generator=g, device=device, dtype=f32),
                          torch.randn((n, R, B), generator=g, device=device, dtype=f32))
    noise = noise * math.sqrt(N0 / 2.0)
    y = torch.matmul(H, x.transpose(1, 2)).transpose(1, 2) + noise
    return {"H": H.contiguous(), "Y": y.contiguous(), "bits": bits, "x": x,
            "N0": float(N0), "Es": float(Es), "B": B, "U": U, "R": R,
            "qam_bits": qam_bits}


def downlink_torch(B: int, U: int, qam_bits: int, n: int, R: int, snr_db: float,
                   seed: int, device, Es: float = 1.0) -> dict:
    """Same model as downlink(), drawn with torch on `device`."""
    d = uplink_torch(B, U, qam_bits, n, R, snr_db, seed, device, Es)
    return {"H": d["H"], "T": d["x"].contiguous(), "bits": d["bits"], "N0": d["N0"],
            "Es": Es, "B": B, "U": U, "R": R, "qam_bits": qam_bits}
