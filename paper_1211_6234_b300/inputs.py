"""Seeded synthetic inputs shared by the CUDA path, the oracle and the benchmark.

This module holds no arithmetic of the Monte Carlo method: only the recipes for
initial spin states, parameter ladders and request streams.  Spin states are
rounded to FP32 and returned as FP64 arrays so that both sides start from
bit-identical values.

The paper (arXiv:1211.6234) uses no dataset: all of its runs are synthetic
lattices (Sec. 4.1: L = 64, started from a striped or saturated state).
"""
from __future__ import annotations

import math

import numpy as np


def random_spins(L: int, R: int = 1, seed: int = 1) -> np.ndarray:
    """R independent states of unit spins uniform on S^2, shape [R, 3, L, L],
    FP32-representable values held in FP64."""
    rng = np.random.default_rng(seed)
    z = rng.uniform(-1.0, 1.0, size=(R, L, L))
    ph = rng.uniform(0.0, 2.0 * math.pi, size=(R, L, L))
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    s = np.stack([r * np.cos(ph), r * np.sin(ph), z], axis=1)
    return s.astype(np.float32).astype(np.float64)


def saturated_z(L: int, R: int = 1, sign: float = 1.0) -> np.ndarray:
    """All spins along +z (or -z), shape [R, 3, L, L]."""
    s = np.zeros((R, 3, L, L), np.float64)
    s[:, 2] = sign
    return s


def striped_z(L: int, width: int, R: int = 1) -> np.ndarray:
    """Perpendicular stripes of the given width along y (Sec. 4.1 initial state)."""
    s = np.zeros((R, 3, L, L), np.float64)
    x = np.arange(L)
    sign = np.where((x // width) % 2 == 0, 1.0, -1.0)
    s[:, 2] = sign[None, None, :]
    return s


def ladder(nT: int = 16, nK: int = 16, Tlo: float = 0.2, Thi: float = 1.2,
           ratio_lo: float = -0.5, ratio_hi: float = 0.5, K2: float = 0.8):
    """Temperature x K4/K2 ladder: list of (T, K2, K4), T-major, nT*nK entries."""
    out = []
    for T in np.linspace(Tlo, Thi, nT):
        for ratio in np.linspace(ratio_lo, ratio_hi, nK):
            out.append((float(T), float(K2), float(ratio * K2)))
    return out


def cooling_schedule(Thi: float = 1.2, Tlo: float = 0.2, step: float = 0.05):
    """Temperatures from Thi down to Tlo inclusive (21 values for the defaults)."""
    n = int(round((Thi - Tlo) / step)) + 1
    return [round(Thi - i * step, 10) for i in range(n)]


def request_stream(n: int, seed: int = 7, rate_hz: float = 1000.0,
                   sizes=(32, 48, 64, 96, 128, 256), sweeps_lo: float = 1e3,
                   sweeps_hi: float = 1e5, sweeps_scale: float = 1.0):
    """Poisson stream of simulation requests: list of dicts with arrival time (s),
    L, T, K2, K4, C_D, sweeps and a per-request seed.  `sweeps_scale` shrinks the
    log-uniform sweep counts for bounded runs."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_hz, size=n))
    reqs = []
    for i in range(n):
        sw = math.exp(rng.uniform(math.log(sweeps_lo), math.log(sweeps_hi)))
        reqs.append({
            "id": i,
            "arrival": float(t[i]),
            "L": int(rng.choice(sizes)),
            "T": float(rng.uniform(0.2, 1.2)),
            "K2": float(rng.uniform(0.5, 1.0)),
            "K4": float(rng.uniform(-0.3, 0.3)),
            "CD": 0.1,
            "J": 1.0,
            "sweeps": max(1, int(round(sw * sweeps_scale))),
            "seed": int(rng.integers(1, 2**63 - 1)),
        })
    return reqs
