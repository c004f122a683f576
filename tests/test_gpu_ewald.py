"""GPU Ewald/Harris W~ (Sec. 2.1) against the oracle's: the lattice and layers
a height z apart, installed in a handle, and one sweep with it traced against
the oracle."""
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


@pytest.mark.parametrize("L,z,eta", [(8, 0.0, 0.0), (16, 0.0, 3.0), (64, 0.0, 0.0), (8, 0.7, 0.0), (12, -2.5, 2.0)])
def test_ewald_tensor_matches_oracle(dipmc, L, z, eta):
    Wg = dipmc.wtilde_ewald(L, z, eta)
    Wo = orc.wtilde_ewald(L, z, eta)
    assert np.abs(Wg - Wo).max() <= 1e-12 * np.abs(Wo).max()


def test_ewald_in_a_handle_and_a_traced_sweep(dipmc):
    L, l, seed = 16, 8, 12
    s0 = inputs.random_spins(L, 1, seed=5)
    prm = (F32(1.0), F32(0.1), F32(0.8), F32(0.0), F32(0.6))
    with dipmc.Lattice(L, l, 1, seed) as lat:
        lat.precompute_W_ewald()
        lat.set_field_path(dipmc.MC_PATH_DIRECT)   # the direct kernel
        Wg = lat.get_W()
        lat.set_params(*prm)
        lat.init_spins(2, s0)
        tr = lat.sweep_trace(2)
    We = orc.wtilde_ewald(L)[:4]
    assert np.abs(Wg - We).max() <= 1e-12 * np.abs(We).max()
    assert np.abs(Wg - orc.wtilde(L, 64, True)).max() <= 1e-7 * np.abs(We).max()
    p = orc.params(L, l, *prm, proposal=0, cone=0.5, schedule=0, seed=seed, replica=0)
    o = resync(p, We, s0[0], 0, 2, tr[0])
    compare_trace(tr[0], o, prm[4], scale=2 + 0.1 * float(np.abs(o["h"]).max()))
