"""The comparison helpers of the GPU parity tests, checked on the CPU: the
oracle re-synchronised to a trajectory that is its own reproduces its own
records, and the decision comparison counts straddles and rejects any other
differing decision."""
import math

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1211_6234_b300 import inputs
from tests.parity_util import compare_trace, resync


def _as_trace(o):
    """An oracle run's records laid out as a GPU trace [n, 10] in FP32."""
    n = len(o["q"])
    tr = np.zeros((n, 10), np.float32)
    tr[:, 0] = o["q"]
    tr[:, 1:4] = o["h"]
    tr[:, 4] = o["dE"]
    tr[:, 5] = o["u"]
    tr[:, 6] = o["acc"]
    tr[:, 7:10] = o["S"]
    return tr


def test_resync_along_the_oracles_own_trajectory():
    L, l, nsw = 8, 4, 3
    W = orc.wtilde(L, 8, True)
    p = orc.params(L, l, 1.0, 0.4, 0.8, -0.1, 0.7, seed=9)
    s0 = inputs.random_spins(L, 1, seed=4)[0]
    o = orc.sweeps(p, W, s0, 0, nsw)
    tr = _as_trace(o)
    r = resync(p, W, s0, 0, nsw, tr)
    # the trajectory is the oracle's own up to the FP32 rounding of the moves
    np.testing.assert_array_equal(r["q"], o["q"])
    np.testing.assert_array_equal(r["acc"], o["acc"])
    assert np.abs(r["dE"] - o["dE"]).max() < 1e-5
    rep = compare_trace(tr, r, p.T, scale=3.0)
    assert rep.straddles == 0 and rep.compared == nsw * L * L
    # each sub-step's decisions from a given state equal that sub-step's records
    sub = orc.substep(p, W, s0, 0, 0)
    n = (L // l) ** 2
    np.testing.assert_array_equal(sub["q"], o["q"][:n])
    np.testing.assert_array_equal(sub["dE"], o["dE"][:n])


def test_substep_dE_is_a_full_energy_difference():
    """dE of every site of a sub-step from the given state equals E(after that one
    move) - E(before), both by the O(N^2) energy (Sec. 4)."""
    L, l = 6, 3
    J, CD, K2, K4, T = 1.0, 0.9, 0.8, -0.3, 2.0
    W = orc.wtilde(L, 16, True)
    s = inputs.random_spins(L, 1, seed=21)[0]
    p = orc.params(L, l, J, CD, K2, K4, T, proposal=1, seed=5)
    sub = orc.substep(p, W, s, 2, 3)
    e0 = orc.energy(W, s, J, CD, K2, K4)[3]
    for d in range(len(sub["q"])):
        t = s.copy()
        t.reshape(3, -1)[:, sub["q"][d]] = sub["S"][d]
        assert abs(orc.energy(W, t, J, CD, K2, K4)[3] - e0 - sub["dE"][d]) < 1e-11


def _toy(T, dE_o, dE_g, u, acc_o, acc_g):
    n = len(dE_o)
    o = {"q": np.arange(n, dtype=np.int32), "h": np.ones((n, 3)), "dE": np.array(dE_o, np.float64),
         "u": np.array(u, np.float64), "acc": np.array(acc_o, np.int32), "S": np.zeros((n, 3))}
    tr = np.zeros((n, 10), np.float64)
    tr[:, 0] = o["q"]
    tr[:, 1:4] = 1.0
    tr[:, 4] = dE_g
    tr[:, 5] = u
    tr[:, 6] = acc_g
    return tr, o


def test_compare_trace_counts_straddles_and_rejects_real_mismatches():
    T = 0.5
    u_thr = math.exp(-1.0 / T)              # threshold -T ln u = 1.0
    # attempt 0 straddles (1 - 4e-6 < 1 < 1 + 4e-6), attempt 1 agrees, attempt 2 straddles too
    tr, o = _toy(T, [1.0 - 4e-6, 0.5, 1.0 + 3e-6], [1.0 + 4e-6, 0.5, 1.0 - 3e-6], [u_thr, 0.25, u_thr],
                 [1, 1, 0], [0, 1, 1])
    rep = compare_trace(tr, o, T, scale=1.0)
    assert rep.straddles == 2 and rep.compared == 3
    # the same decision flip far from the threshold is an error, not a straddle
    tr, o = _toy(T, [2.0, 0.5], [2.0 + 1e-6, 0.5], [u_thr, 0.25], [0, 1], [1, 1])
    with pytest.raises(AssertionError, match="decision mismatch"):
        compare_trace(tr, o, T, scale=1.0)
    # a dE error beyond the FP32 tolerance fails even with equal decisions
    tr, o = _toy(T, [0.2], [0.2 + 1e-3], [0.25], [1], [1])
    with pytest.raises(AssertionError):
        compare_trace(tr, o, T, scale=1.0)


def test_binning_reference_on_series_of_known_autocorrelation():
    """The numpy binning analysis that the GPU error-bar tests compare every path's
    accumulators with: on independent samples its corrected error stays near the naive
    one (tau_int near 1/2); on AR(1) series x_t = rho x_(t-1) + sqrt(1 - rho^2) e_t it
    reaches the closed form tau_int = (1 + rho) / (2 (1 - rho)) of the integrated
    autocorrelation time (2^17 samples; rho = 0.5, 0.8, 0.95)."""
    from scipy.signal import lfilter

    from tests.parity_util import binning_reference
    rng = np.random.default_rng(5)
    x = rng.normal(size=1 << 16)
    var, naive, err, tau = binning_reference(x)
    assert abs(var - 1.0) < 0.03
    assert naive == pytest.approx(math.sqrt(var / (len(x) - 1)), rel=1e-12)
    assert err >= naive and 0.5 <= tau < 0.9
    for rho in (0.5, 0.8, 0.95):
        e = rng.normal(size=1 << 17)
        y = lfilter([math.sqrt(1.0 - rho * rho)], [1.0, -rho], e)
        _, _, _, tau = binning_reference(y)
        expect = (1.0 + rho) / (2.0 * (1.0 - rho))
        # the largest error over the levels leans high by the scatter of the deep levels
        assert 0.9 < tau / expect < 1.25, (rho, tau, expect)
