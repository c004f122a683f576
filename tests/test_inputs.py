"""The seeded input recipes (paper_1211_6234_b300/inputs.py) hold the synthetic
workloads both sides start from; these tests fix their shapes and laws on the CPU:
uniform unit spins on S^2 rounded to FP32, the saturated and striped states of Sec. 4.1,
the temperature x K4/K2 ladder of the batched replicas, the cooling schedule of the L = 64
scan (1.2 down to 0.2 in steps of 0.05) and the Poisson stream of serving requests."""
import math
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
from paper_1211_6234_b300 import inputs  # noqa: E402


def test_random_spins_are_unit_fp32_and_uniform_on_the_sphere():
    s = inputs.random_spins(32, 4, seed=3)
    assert s.shape == (4, 3, 32, 32) and s.dtype == np.float64
    assert np.array_equal(s, s.astype(np.float32).astype(np.float64))      # FP32-representable
    assert np.abs(np.sqrt((s ** 2).sum(axis=1)) - 1.0).max() < 1e-6
    assert np.array_equal(s, inputs.random_spins(32, 4, seed=3))           # seeded
    assert not np.array_equal(s, inputs.random_spins(32, 4, seed=4))
    # uniform on S^2: every component has mean 0 and second moment 1/3 (4096 samples each)
    for a in range(3):
        c = s[:, a].ravel()
        assert abs(c.mean()) < 4 / math.sqrt(3 * c.size)
        assert abs((c * c).mean() - 1 / 3) < 0.03
    # z uniform on [-1, 1] (Archimedes): a chi^2 over 8 bins stays well below its tail
    hist, _ = np.histogram(s[:, 2].ravel(), bins=8, range=(-1, 1))
    expect = s[:, 2].size / 8
    assert ((hist - expect) ** 2 / expect).sum() < 24.3                      # p ~ 1e-3 at 7 dof


def test_saturated_and_striped_states():
    z = inputs.saturated_z(8, 2)
    assert z.shape == (2, 3, 8, 8) and (z[:, 2] == 1).all() and (z[:, :2] == 0).all()
    assert (inputs.saturated_z(8, 1, sign=-1.0)[:, 2] == -1).all()
    st = inputs.striped_z(16, 4)
    col = st[0, 2, 0]
    assert np.array_equal(col, np.repeat([1.0, -1.0, 1.0, -1.0], 4))      # stripes of 4 along x
    assert (st[0, 2] == col[None, :]).all()                                 # constant along y
    assert (st[:, :2] == 0).all()


def test_ladder_is_temperature_major_over_the_stated_ranges():
    lad = inputs.ladder()
    assert len(lad) == 256
    T = np.array([e[0] for e in lad]).reshape(16, 16)
    K2 = np.array([e[1] for e in lad])
    ratio = np.array([e[2] / e[1] for e in lad]).reshape(16, 16)
    assert (T == T[:, :1]).all() and np.allclose(T[:, 0], np.linspace(0.2, 1.2, 16))
    assert (K2 == 0.8).all()
    assert np.allclose(ratio, np.linspace(-0.5, 0.5, 16)[None, :])


def test_cooling_schedule_is_the_21_temperatures_of_the_scan():
    Ts = inputs.cooling_schedule()
    assert len(Ts) == 21 and Ts[0] == 1.2 and Ts[-1] == 0.2
    assert np.allclose(np.diff(Ts), -0.05)


def test_request_stream_is_poisson_with_log_uniform_sweeps():
    reqs = inputs.request_stream(4000, seed=7, rate_hz=500.0)
    t = np.array([r["arrival"] for r in reqs])
    assert (np.diff(t) > 0).all()
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() * 500.0 - 1.0) < 0.05                            # rate 500 / s
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.05                       # exponential gaps
    assert {r["L"] for r in reqs} == {32, 48, 64, 96, 128, 256}
    sw = np.array([r["sweeps"] for r in reqs], dtype=np.float64)
    assert sw.min() >= 1e3 and sw.max() <= 1e5
    u = (np.log(sw) - math.log(1e3)) / (math.log(1e5) - math.log(1e3))   # uniform on [0, 1]
    assert abs(u.mean() - 0.5) < 0.02 and abs(u.var() - 1 / 12) < 0.01
    assert all(0.2 <= r["T"] <= 1.2 and 0.5 <= r["K2"] <= 1.0 and -0.3 <= r["K4"] <= 0.3 for r in reqs)
    assert len({r["seed"] for r in reqs}) == len(reqs)                      # every request its own stream
    small = inputs.request_stream(4000, seed=7, rate_hz=500.0, sweeps_scale=0.002)
    assert [r["L"] for r in small] == [r["L"] for r in reqs]                # same stream, shorter runs
    # both round the same draw: the scaled count is within half a sweep of 0.002 x the full one
    assert all(s["sweeps"] >= 1 and abs(s["sweeps"] - 0.002 * r["sweeps"]) <= 0.51 for s, r in zip(small, reqs))
