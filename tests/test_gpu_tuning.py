"""Launch shapes of the windowed tensor path (mc_set_tuning) and their autotuner.

The sub-step kernel's warp layouts change only which warps take which role, so
trajectories are bit-identical across layouts.  The split-K shape and the N-tile
change the FP32 summation order of the contraction, so each shape is checked
attempt by attempt against the oracle (re-synchronised per sub-step)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import oracle as orc  # noqa: E402
from paper_1211_6234_b300 import inputs  # noqa: E402
from tests.parity_util import F32, compare_trace, resync  # noqa: E402


@pytest.fixture(scope="module")
def dipmc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1211_6234_b300 import dipmc as d
    return d


def _ladder(R):
    lad = [(F32(1.0), F32(0.1), F32(k2), F32(k4), F32(T)) for (T, k2, k4) in inputs.ladder(16, 16)]
    return [lad[r % len(lad)] for r in range(R)]


def _run(dipmc, L, l, R, tuning, nsw, trace=False, seed=3):
    lad = _ladder(R)
    s0 = inputs.random_spins(L, R, seed=77)
    with dipmc.Lattice(L, l, R, seed) as lat:
        lat.precompute_W(16, True)
        lat.set_field_path(dipmc.MC_PATH_TENSOR)
        lat.set_tuning(**tuning)
        assert lat.tuning() == {"window": 0, **{k: 0 for k in ("tc_kblocks", "tc_ntile", "steps_layout")}, **tuning}
        for r, prm in enumerate(lad):
            lat.set_params(*prm, replica=r)
        lat.init_spins(2, s0)
        if trace:
            tr = lat.sweep_trace(nsw)
        else:
            lat.sweep(nsw, 1)
            tr = None
        return lad, s0, tr, lat.get_spins(), [lat.observables(r)["energy"] for r in range(R)]


def test_warp_layouts_give_identical_trajectories(dipmc):
    """300 replicas (a second wave of CTAs beyond 148 SMs, where layout 2 moves the
    decider) of L = 64, l = 32, 3 sweeps: every layout ends in the same spins and
    tracked energies, bit for bit."""
    ref = None
    for layout in (0, 1, 2):
        _, _, _, s, e = _run(dipmc, 64, 32, 300, {"steps_layout": layout}, 3)
        if ref is None:
            ref = (s, e)
        else:
            assert np.array_equal(s, ref[0]), layout
            assert e == ref[1], layout


@pytest.mark.parametrize("tuning", [{"tc_kblocks": 2}, {"tc_kblocks": 8, "tc_ntile": 128},
                                    {"tc_ntile": 64, "steps_layout": 2}, {"tc_kblocks": 12, "steps_layout": 1},
                                    {"window": 128}, {"window": 128, "tc_ntile": 128, "steps_layout": 1}],
                         ids=["kb2", "kb8_nt128", "nt64_layout2", "kb12_layout1", "win512", "win512_nt128_layout1"])
def test_tile_shapes_match_oracle(dipmc, tuning):
    """One traced sweep of 256 replicas of L = 64, l = 32 under a given split-K
    shape / N-tile / layout / window (128 sub-steps: 512-site windows, twelve
    M-tiles of cell-grid spectra): sampled replicas of every N-tile against the
    oracle."""
    L, l, R = 64, 32, 256
    lad, s0, tr, sg, _ = _run(dipmc, L, l, R, tuning, 1, trace=True, seed=1)
    W = orc.wtilde(L, 16, True)
    for r in (0, 63, 64, 130, 191, 255):
        J, CD, K2, K4, T = lad[r]
        p = orc.params(L, l, J, CD, K2, K4, T, proposal=0, cone=0.5, schedule=0, seed=1, replica=r)
        o = resync(p, W, s0[r], 0, 1, tr[r])
        hmax = float(np.abs(o["h"]).max())
        rep = compare_trace(tr[r], o, T, scale=1 + abs(J) + abs(K2) + abs(K4) + abs(CD) * hmax)
        assert rep.straddles == 0, rep.notes
        np.testing.assert_allclose(sg[r], o["s"], rtol=0, atol=1e-6)


def test_tuning_rejects_bad_shapes(dipmc):
    with dipmc.Lattice(64, 32, 4, 1) as lat:
        for bad in ({"tc_ntile": 100}, {"tc_ntile": 512}, {"steps_layout": 3}, {"tc_kblocks": -1}):
            with pytest.raises(dipmc.McError) as e:
                lat.set_tuning(**bad)
            assert e.value.code == dipmc.MC_EINVAL


def test_autotune_tunes_tensor_shapes_and_keeps_state(dipmc):
    L, l, R = 64, 32, 256
    s0 = inputs.random_spins(L, R, seed=4)
    with dipmc.Lattice(L, l, R, 5) as lat:
        lat.precompute_W(16, True)
        lat.init_spins(2, s0)
        lat.sweep(1, 0)
        before, t0 = lat.get_spins(), lat.sweep_counter()
        path, win = lat.autotune(1)
        tun = lat.tuning()
        assert np.array_equal(lat.get_spins(), before) and lat.sweep_counter() == t0
        if path == dipmc.MC_PATH_TENSOR:
            assert tun["tc_kblocks"] in (0, 2, 4, 6, 8, 12) and tun["tc_ntile"] in (0, 128)
            assert tun["steps_layout"] in (0, 1, 2)
        print(f"\nautotune 256 x L=64: path {path}, window {win}, tuning {tun}")
        lat.sweep(2, 1)
        assert lat.observables(0)["samples"] == 2


def test_kernel_timing_records_every_launch_of_a_call(dipmc):
    """With timing on, every launch of a call is bracketed by CUDA events (and the call
    is not replayed from a graph): two sweeps of the tensor path at 4 x L = 64, l = 32
    with 512-site windows (eight windows a sweep) record 16 tensor-core field and 16
    sub-step launches with positive times, and the sub-step kernel's clock counters
    report 32 blocks of 16 sites a launch; turning timing off clears the record."""
    with dipmc.Lattice(64, 32, 4, 3) as lat:
        lat.precompute_W(16, True)
        lat.set_field_path(dipmc.MC_PATH_TENSOR)
        lat.set_window(128)
        lat.init_spins(0)
        lat.sweep(1, 1)                  # buffers, tables and the energy anchor outside the record
        lat.set_timing(True)
        lat.sweep(2, 1)
        t = lat.timing()
        cyc = lat.window_cycles()
        lat.set_timing(False)
        t_off = lat.timing()
    assert t["tc_field"]["launches"] == 16 and t["window_steps"]["launches"] == 16
    assert t["tc_field"]["ms"] > 0 and t["window_steps"]["ms"] > 0
    assert t["sweep_direct"]["launches"] == 0
    assert cyc["blocks_per_launch"] == 32
    assert cyc["per_block"] > 0 and cyc["setup"] > 0 and cyc["tail"] > 0
    assert all(v["launches"] == 0 for v in t_off.values())
