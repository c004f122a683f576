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


def resync(p, W, s0, t0: int, nsw: int, gpu_tr: np.ndarray) -> dict:
    """The oracle's decision of every attempt of one replica's GPU trace
    [n_attempts, MC_TRACE_W], each sub-step decided from the GPU's pre-step state:
    the oracle decides a sub-step from its current state, then takes the GPU's
    accepted moves of that sub-step (orc_replay).  One differing decision at a
    threshold therefore does not end the comparison."""
    out = orc.replay_batch([p], W, np.asarray(s0)[None], t0, nsw, gpu_tr[None, :, 6].astype(np.int32),
                           gpu_tr[None, :, 7:10].astype(np.float64))
    return {k: v[0] for k, v in out.items()}


def compare_trace(gpu_tr: np.ndarray, orc_out: dict, T: float, scale: float,
                  h_tol: float = 1e-5, S_tol: float = 1e-5) -> TraceReport:
    """Compare one replica's GPU trace [n_attempts, 10] with the oracle's records of
    the same attempts (from `resync`): identical sites and acceptance uniforms,
    fields within h_tol normwise, dE within the FP32 tolerance, proposals within
    S_tol, and identical decisions except at a *straddle* -- the acceptance
    threshold -T ln u lies between the GPU's and the oracle's dE (up to the FP32
    rounding of the kernel's exp(-dE/T)).  Straddles are counted over the whole
    trace; any other differing decision fails."""
    rep = TraceReport()
    q_g = gpu_tr[:, 0].astype(np.int64)
    h_g = gpu_tr[:, 1:4].astype(np.float64)
    dE_g = gpu_tr[:, 4].astype(np.float64)
    u_g = gpu_tr[:, 5].astype(np.float64)
    a_g = gpu_tr[:, 6].astype(np.int64)
    S_g = gpu_tr[:, 7:10].astype(np.float64)
    np.testing.assert_array_equal(q_g, orc_out["q"])
    np.testing.assert_array_equal(u_g, orc_out["u"])
    dE_o = np.asarray(orc_out["dE"], np.float64)
    a_o = np.asarray(orc_out["acc"], np.int64)
    hmax = float(np.abs(orc_out["h"]).max()) if len(q_g) else 0.0
    dE_tol = 2e-5 * scale
    mism = a_g != a_o
    if mism.any():
        u = u_g[mism]
        thr = np.where(u > 0, -T * np.log(np.maximum(u, 1e-300)), np.inf)
        lo = np.minimum(dE_g[mism], dE_o[mism])
        hi = np.maximum(dE_g[mism], dE_o[mism])
        slack = 2.5e-7 * (np.abs(thr) + T)
        strad = (thr >= lo - slack) & (thr <= hi + slack)
        if not strad.all():
            i = int(np.nonzero(mism)[0][np.argmin(strad)])
            raise AssertionError(
                f"decision mismatch at attempt {i} (q={q_g[i]}): gpu={a_g[i]} orc={a_o[i]} "
                f"dE_gpu={dE_g[i]} dE_orc={dE_o[i]} thr={-T * math.log(u_g[i]) if u_g[i] > 0 else math.inf}")
        rep.straddles = int(strad.sum())
        for i in np.nonzero(mism)[0][:8]:
            rep.notes.append(f"straddle at attempt {i}: dE_orc={dE_o[i]:.9g} dE_gpu={dE_g[i]:.9g}")
    rep.compared = len(q_g)
    if rep.compared:
        dh = np.abs(h_g - orc_out["h"]).max()
        rep.h_err_norm = float(dh / hmax) if hmax > 0 else float(dh)
        big = np.abs(orc_out["h"]) > 1e-3 * hmax
        if big.any():
            rep.h_err_elem = float((np.abs(h_g - orc_out["h"])[big] / np.abs(orc_out["h"])[big]).max())
        rep.dE_err = float(np.abs(dE_g - dE_o).max())
        rep.S_err = float(np.abs(S_g - orc_out["S"]).max())
    assert rep.h_err_norm <= h_tol, rep
    assert rep.dE_err <= dE_tol, rep
    assert rep.S_err <= S_tol, rep
    return rep


def pooled(means) -> tuple:
    """Mean over independent replicas of their time averages, and its standard
    error from the replicas' spread (autocorrelation-corrected by construction:
    each replica's average carries its own autocorrelation)."""
    x = np.asarray(means, np.float64)
    return float(x.mean()), float(x.std(ddof=1) / math.sqrt(len(x)))


def binning_reference(x, min_blocks=32):
    """Textbook binning analysis of one time series x (Flyvbjerg and Petersen): the
    population variance, the naive error of the mean, and the autocorrelation-corrected
    error as the largest error of the means of blocks of 2^k samples over the levels that
    still hold min_blocks blocks (never below the naive one), with tau_int = (err/naive)^2 / 2."""
    x = np.asarray(x, np.float64)
    n = len(x)
    var = max(0.0, float(np.mean(x * x) - np.mean(x) ** 2))
    naive = math.sqrt(var / (n - 1))
    err, k = naive, 1
    while n >> k >= min_blocks:
        nb = n >> k
        b = x[: nb << k].reshape(nb, 1 << k).mean(axis=1)
        vk = max(0.0, float(np.mean(b * b) - np.mean(b) ** 2))
        err = max(err, math.sqrt(vk / (nb - 1)))
        k += 1
    tau = 0.5 * (err / naive) ** 2 if naive > 0 else float("nan")
    return var, naive, err, tau
