"""The allocation-free energy entry point (mc_energy_noalloc) against mc_energy.

mc_energy_noalloc serves callers that cannot call cudaMalloc (a device-memory
budget owned by a framework or a serving process, or latency-critical paths);
it keeps its field scratch in a fixed device array instead of a lattice handle.
Two calls in a row, on different lattices, must each give the energies that the
handle-based mc_energy gives for the same states.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _reference_state(dipmc, L, R, seed):
    lat = dipmc.Lattice(L, L // 2, R, seed)
    lat.precompute_W(16, True)
    coup = []
    for r in range(R):
        c = [float(np.float32(x)) for x in (1.0 - 0.1 * r, 0.1 + 0.05 * r, 0.8, -0.2 + 0.1 * r)]
        lat.set_params(*c, 0.7, replica=r)
        coup.append(c)
    lat.init_spins(0)
    ref = lat.energy()
    spins = torch.empty((R, 3, L, L), dtype=torch.float32, device="cuda")
    lat.get_spins(out=spins)
    W32 = torch.from_numpy(lat.get_W().astype(np.float32)).cuda()
    lat.close()
    return ref, spins, W32, torch.tensor(coup, dtype=torch.float32, device="cuda")


def test_energy_noalloc_matches_energy_two_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1211_6234_b300 import dipmc
    for (L, R, seed) in ((32, 5, 3), (16, 3, 4)):
        ref, spins, W32, coup = _reference_state(dipmc, L, R, seed)
        out = torch.full((R,), float("nan"), dtype=torch.float64, device="cuda")
        dipmc.energy_noalloc(L, R, W32, spins, coup, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        scale = L * L * 3.0
        np.testing.assert_allclose(got, ref, rtol=0, atol=1e-5 * scale)


def test_energy_noalloc_rejects_oversize_request():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1211_6234_b300 import dipmc
    L, R = 256, 6  # 6 * 3 * 65536 > 2^20
    t = torch.zeros(1, device="cuda")
    with pytest.raises(dipmc.McError) as e:
        dipmc.energy_noalloc(L, R, t, t, t, t)
    assert e.value.code == dipmc.MC_EINVAL
    assert "at most 5 replicas" in str(e.value)
