"""Uneven lattice sizes in one persistent launch (mc_sweep_group).

Handles of L = 32, 48, 64 and 96 (one C = L / l per group) run together in one
launch of the direct kernel; every replica must end exactly where its own
handle's mc_sweep takes it: spins, tracked energy and observables bit for bit.
The direct kernel itself is checked against the oracle elsewhere; here the
oracle also checks one replica of the group's largest lattice attempt by attempt."""
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


def _make(dipmc, L, l, R, seed):
    lat = dipmc.Lattice(L, l, R, seed)
    lat.precompute_W(16, True)
    lat.set_field_path(dipmc.MC_PATH_DIRECT)
    for r in range(R):
        lat.set_params(F32(1.0), F32(0.1), F32(0.5 + 0.1 * r), F32(-0.1), F32(0.3 + 0.2 * r), replica=r)
    lat.init_spins(0)
    return lat


def _state(lat):
    obs = lat.observables_batch()
    return lat.get_spins(), [o["energy"] for o in obs], [(o["samples"], o["abs_m"]["mean"], o["e"]["mean"],
                                                        o["accepted"], o["eta"]) for o in obs]


@pytest.mark.parametrize("shapes", [((32, 16, 3), (48, 24, 2), (64, 32, 5), (96, 48, 1)),
                                    ((64, 16, 2), (96, 24, 3), (32, 8, 1)),
                                    ((16, 16, 2), (32, 32, 1)),
                                    ((48, 24, 4),)],
                         ids=["C2_L32_48_64_96", "C4_L64_96_32", "C1_exact_L16_32", "one_handle"])
def test_group_launch_equals_separate_sweeps(dipmc, shapes):
    grp = [_make(dipmc, L, l, R, 100 + L) for (L, l, R) in shapes]
    sep = [_make(dipmc, L, l, R, 100 + L) for (L, l, R) in shapes]
    try:
        for nsw, me in ((3, 1), (4, 2)):
            dipmc.sweep_group(grp, nsw, me)
            for lat in sep:
                lat.sweep(nsw, me)
        for a, b in zip(grp, sep):
            sa, ea, oa = _state(a)
            sb, eb, ob = _state(b)
            assert np.array_equal(sa, sb)
            assert ea == eb
            assert oa == ob
            assert a.sweep_counter() == b.sweep_counter() == 7
    finally:
        for lat in grp + sep:
            lat.close()


def test_group_launch_matches_oracle(dipmc):
    """After a grouped launch, one traced sweep of the L = 96 handle (direct path)
    agrees with the oracle decided from the GPU's pre-step state."""
    grp = [_make(dipmc, L, l, 1, 7 + L) for (L, l) in ((32, 16), (96, 48))]
    try:
        dipmc.sweep_group(grp, 2, 1)
        lat = grp[1]
        s0 = lat.get_spins().astype(np.float64)
        tr = lat.sweep_trace(1)
    finally:
        for g in grp:
            g.close()
    p = orc.params(96, 48, F32(1.0), F32(0.1), F32(0.5), F32(-0.1), F32(0.3), seed=7 + 96, replica=0)
    W = orc.wtilde(96, 16, True)
    o = resync(p, W, s0[0], 2, 1, tr[0])
    rep = compare_trace(tr[0], o, F32(0.3), scale=2 + 0.1 * float(np.abs(o["h"]).max()))
    assert rep.straddles == 0


def test_group_launch_rejects_mixed_shapes(dipmc):
    a = _make(dipmc, 32, 16, 1, 1)
    b = _make(dipmc, 64, 16, 1, 2)      # C = 4 against C = 2
    c = _make(dipmc, 64, 32, 1, 3)
    try:
        with pytest.raises(dipmc.McError) as e:
            dipmc.sweep_group([a, b], 1)
        assert e.value.code == dipmc.MC_EINVAL
        c.set_field_path(dipmc.MC_PATH_TENSOR)
        with pytest.raises(dipmc.McError) as e:
            dipmc.sweep_group([a, c], 1)
        assert e.value.code == dipmc.MC_EINVAL
        with pytest.raises(dipmc.McError) as e:
            dipmc.sweep_group([a, a], 1)
        assert e.value.code == dipmc.MC_EINVAL
    finally:
        for lat in (a, b, c):
            lat.close()
