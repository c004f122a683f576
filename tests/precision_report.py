"""Error of every field path against the FP64 oracle (test infrastructure).

    python -m tests.precision_report        # on a GPU host; prints a markdown table

For each path: one traced sweep of two replicas at L = 64, l = 32 (the paper's
lattice and spacing), compared attempt by attempt with the oracle decided from the GPU's pre-step
state (field error
normwise, dE error, straddled decisions); then a 12-sweep run at L = 16, l = 8
whose trajectory equals the oracle's, with the largest deviation of the per-sweep
observable means from the oracle's.
"""
from __future__ import annotations

import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from oracle import oracle as orc  # noqa: E402
from paper_1211_6234_b300 import dipmc, inputs  # noqa: E402
from tests.parity_util import F32, compare_trace, resync  # noqa: E402

PATHS = [("direct", dipmc.MC_PATH_DIRECT), ("window_f32", dipmc.MC_PATH_WINDOW_F32),
         ("tensor_bf16x3", dipmc.MC_PATH_TENSOR), ("fft", dipmc.MC_PATH_FFT),
         ("spectral", dipmc.MC_PATH_SPECTRAL), ("incremental", dipmc.MC_PATH_INCREMENTAL),
         ("fft_cluster", dipmc.MC_PATH_FFT_CLUSTER)]


def traced(path, L=64, l=32, R=2, A=64):
    prm = [(F32(1.0), F32(0.1), F32(0.8), F32(0.0), F32(0.6)), (F32(1.0), F32(0.1), F32(0.8), F32(-0.2), F32(0.3))]
    s0 = inputs.random_spins(L, R, seed=77)
    with dipmc.Lattice(L, l, R, 5) as lat:
        lat.precompute_W(A, True)
        lat.set_field_path(path)
        for r in range(R):
            lat.set_params(*prm[r], replica=r)
        lat.init_spins(2, s0)
        tr = lat.sweep_trace(1)
    W = orc.wtilde(L, A, True)
    out = {"h": 0.0, "dE": 0.0, "straddles": 0, "attempts": 0}
    for r in range(R):
        J, CD, K2, K4, T = prm[r]
        o = resync(orc.params(L, l, J, CD, K2, K4, T, seed=5, replica=r), W, s0[r], 0, 1, tr[r])
        hmax = float(np.abs(o["h"]).max())
        rep = compare_trace(tr[r], o, T, scale=1 + abs(J) + abs(K2) + abs(K4) + CD * hmax)
        out["h"] = max(out["h"], rep.h_err_norm)
        out["dE"] = max(out["dE"], rep.dE_err)
        out["straddles"] += rep.straddles
        out["attempts"] += rep.compared
    return out


def observables(path, L=16, l=8, nsw=12):
    prm = (F32(1.0), F32(0.15), F32(0.8), F32(-0.1), F32(0.9))
    s0 = inputs.random_spins(L, 1, seed=8)
    with dipmc.Lattice(L, l, 1, 61) as lat:
        lat.precompute_W(16, True)
        lat.set_field_path(path)
        lat.set_params(*prm)
        lat.init_spins(2, s0)
        lat.sweep(nsw, 1)
        og = lat.observables(0)
        sg = lat.get_spins()[0].astype(np.float64)
    o = orc.sweeps(orc.params(L, l, *prm, seed=61, replica=0), orc.wtilde(L, 16, True), s0[0], 0, nsw,
                   trace=False, observe=True)
    if np.abs(sg - o["s"]).max() > 1e-4:
        return None
    return {nm: abs(og[nm]["mean"] - o["obs"][:, i].mean()) for i, nm in enumerate(dipmc.OBS_NAMES)}


def main():
    print("| path | field error (normwise) | max dE error | straddles / attempts | largest observable deviation |")
    print("|---|---|---|---|---|")
    for name, path in PATHS:
        t = traced(path)
        ob = observables(path)
        if ob is None:
            obs = "trajectory separated by a straddle"
        else:
            k = max(ob, key=ob.get)
            obs = f"{ob[k]:.1e} ({k})"
        print(f"| {name} | {t['h']:.1e} | {t['dE']:.1e} | {t['straddles']} / {t['attempts']} | {obs} |", flush=True)


if __name__ == "__main__":
    main()
