"""Comparison helpers for GPU-vs-oracle parity tests (test code only)."""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from oracle import oracle as orc

F32 = lambda x: float(np.float32(x))  # noqa: E731  FP32-representable parameter


@dataclass
class TraceReport:
    compared: int = 0
    straddles: int = 0
    h_err_norm: float = 0.0     # max |h_gpu - h_orc|_inf / max |h_orc|
    h_err_elem: float = 0.0     # max elementwise relative error where |h| > 1e-3 max
    dE_err: float = 0.0
    S_err: float = 0.0
    notes: list = field(default_factory=list)


def compare_trace(gpu_tr: np.ndarray, orc_out: dict, T: float, scale: float,
                  h_tol: float = 1e-5, S_tol: float = 1e-5) -> TraceReport:
    """Compare one replica's GPU trace [n_attempts, 10] with the oracle's trace, in
    attempt order.  Decisions must be identical; a mismatch is allowed only where the
    acceptance threshold -T ln u lies within the FP32 tolerance of the oracle's dE
    (a straddle).  Comparison stops at the first straddle (the trajectories differ
    from there on)."""
    rep = TraceReport()
    q_g = gpu_tr[:, 0].astype(np.int64)
    h_g = gpu_tr[:, 1:4].astype(np.float64)
    dE_g = gpu_tr[:, 4].astype(np.float64)
    u_g = gpu_tr[:, 5].astype(np.float64)
    a_g = gpu_tr[:, 6].astype(np.int64)
    S_g = gpu_tr[:, 7:10].astype(np.float64)
    hmax = float(np.abs(orc_out["h"]).max())
    dE_tol = 2e-5 * scale
    n = len(q_g)
    stop = n
    for i in range(n):
        if a_g[i] != orc_out["acc"][i]:
            thr = -T * math.log(orc_out["u"][i]) if orc_out["u"][i] > 0 else math.inf
            if abs(orc_out["dE"][i] - thr) <= dE_tol:
                rep.straddles += 1
                rep.notes.append(f"straddle at attempt {i}: dE_orc={orc_out['dE'][i]:.9g} "
                                 f"dE_gpu={dE_g[i]:.9g} thr={thr:.9g}")
                stop = i + 1
                break
            raise AssertionError(
                f"decision mismatch at attempt {i} (q={q_g[i]}): gpu={a_g[i]} orc={orc_out['acc'][i]} "
                f"dE_gpu={dE_g[i]} dE_orc={orc_out['dE'][i]} thr={thr}")
    sl = slice(0, stop)
    np.testing.assert_array_equal(q_g[sl], orc_out["q"][sl])
    np.testing.assert_array_equal(u_g[sl], orc_out["u"][sl])
    rep.compared = stop
    dh = np.abs(h_g[sl] - orc_out["h"][sl]).max() if stop else 0.0
    rep.h_err_norm = float(dh / hmax) if hmax > 0 else float(dh)
    big = np.abs(orc_out["h"][sl]) > 1e-3 * hmax
    if big.any():
        rep.h_err_elem = float((np.abs(h_g[sl] - orc_out["h"][sl])[big] / np.abs(orc_out["h"][sl])[big]).max())
    rep.dE_err = float(np.abs(dE_g[sl] - orc_out["dE"][sl]).max()) if stop else 0.0
    rep.S_err = float(np.abs(S_g[sl] - orc_out["S"][sl]).max()) if stop else 0.0
    assert rep.h_err_norm <= h_tol, rep
    assert rep.dE_err <= dE_tol, rep
    assert rep.S_err <= S_tol, rep
    return rep


def binned_error(x: np.ndarray, min_blocks: int = 32) -> float:
    """Autocorrelation-corrected standard error by blocking: the largest error over
    block sizes 2^k that leave at least min_blocks blocks."""
    x = np.asarray(x, np.float64)
    n = len(x)
    best = x.std() / math.sqrt(max(n - 1, 1))
    b = 2
    while n // b >= min_blocks:
        m = x[: (n // b) * b].reshape(-1, b).mean(1)
        best = max(best, m.std() / math.sqrt(len(m) - 1))
        b *= 2
    return best
