"""The allocation-free energy entry point (mc_energy_noalloc).

mc_energy_noalloc serves callers that cannot call cudaMalloc: code that runs
inside a device-memory budget owned by a framework's caching allocator or by a
serving process that reserves all device memory up front, and latency-critical
loops where an allocation would synchronise the device.  It keeps its field
scratch in a fixed device array instead of a lattice handle.

Checked here, on two calls in a row with different lattices: the energies equal
the CPU FP64 oracle's energy of the same states (and the handle-based
mc_energy), a call that fills the fixed scratch almost exactly gives the right
energies too, a call after warm-up changes neither the device's free memory nor
torch's allocated bytes, and oversize requests fail with MC_EINVAL naming the
bound.  This file is collected last on purpose.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import oracle as orc  # noqa: E402

A_IMG = 16


@pytest.fixture(scope="module")
def dipmc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1211_6234_b300 import dipmc as d
    return d


def _states(dipmc, L, R, seed):
    """R random states of one lattice, their couplings, the handle's mc_energy,
    and device copies of the spins, W~ (FP32) and couplings [R][4]."""
    lat = dipmc.Lattice(L, L // 2, R, seed)
    lat.precompute_W(A_IMG, True)
    coup = []
    for r in range(R):
        c = [float(np.float32(x)) for x in (1.0 - 0.01 * r, 0.1 + 0.005 * r, 0.8, -0.2 + 0.01 * r)]
        lat.set_params(*c, 0.7, replica=r)
        coup.append(c)
    lat.init_spins(0)
    handle_E = lat.energy()
    spins = torch.empty((R, 3, L, L), dtype=torch.float32, device="cuda")
    lat.get_spins(out=spins)
    W32 = torch.from_numpy(lat.get_W().astype(np.float32)).cuda()
    lat.close()
    return handle_E, spins, W32, torch.tensor(coup, dtype=torch.float32, device="cuda"), coup


def _oracle_energies(L, spins, coup, which):
    W = orc.wtilde(L, A_IMG, True)
    s = spins.cpu().numpy().astype(np.float64)
    return np.array([orc.energy(W, s[r], *coup[r])[3] for r in which])


def test_energy_noalloc_matches_oracle_two_calls(dipmc):
    for (L, R, seed) in ((32, 5, 3), (16, 3, 4)):
        handle_E, spins, W32, coup_d, coup = _states(dipmc, L, R, seed)
        out = torch.full((R,), float("nan"), dtype=torch.float64, device="cuda")
        dipmc.energy_noalloc(L, R, W32, spins, coup_d, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        ref = _oracle_energies(L, spins, coup, range(R))
        # FP32 field against the FP64 oracle: relative 1e-5 of the energy's scale
        scale = L * L * 3.0
        np.testing.assert_allclose(got, ref, rtol=0, atol=1e-5 * scale)
        np.testing.assert_allclose(got, handle_E, rtol=0, atol=1e-5 * scale)


def test_energy_noalloc_full_scratch(dipmc):
    """L = 64 with R = 85: 85 * 3 * 64^2 = 1,044,480 of the 1,048,576 scratch values."""
    L, R = 64, 85
    handle_E, spins, W32, coup_d, coup = _states(dipmc, L, R, 5)
    out = torch.full((R,), float("nan"), dtype=torch.float64, device="cuda")
    dipmc.energy_noalloc(L, R, W32, spins, coup_d, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    scale = L * L * 3.0
    np.testing.assert_allclose(got, handle_E, rtol=0, atol=1e-5 * scale)
    which = (0, 41, 84)
    np.testing.assert_allclose(got[list(which)], _oracle_energies(L, spins, coup, which), rtol=0,
                               atol=1e-5 * scale)


def test_energy_noalloc_allocates_nothing(dipmc):
    L, R = 32, 4
    _, spins, W32, coup_d, _ = _states(dipmc, L, R, 6)
    out = torch.zeros((R,), dtype=torch.float64, device="cuda")
    dipmc.energy_noalloc(L, R, W32, spins, coup_d, out)     # warm-up (module loading)
    torch.cuda.synchronize()
    first = out.clone()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    dipmc.energy_noalloc(L, R, W32, spins, coup_d, out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    assert torch.cuda.memory_allocated() == alloc0
    assert torch.equal(out, first)      # the second call sees nothing of the first


def test_energy_noalloc_rejects_oversize_request(dipmc):
    t = torch.zeros(1, device="cuda")
    with pytest.raises(dipmc.McError) as e:
        dipmc.energy_noalloc(256, 6, t, t, t, t)      # 6 * 3 * 65536 > 2^20
    assert e.value.code == dipmc.MC_EINVAL
    assert "at most 5 replicas" in str(e.value)
    with pytest.raises(dipmc.McError) as e:
        dipmc.energy_noalloc(2, 70000, t, t, t, t)    # fits the scratch, exceeds the grid rows
    assert e.value.code == dipmc.MC_EINVAL
    assert "65535" in str(e.value)
    with pytest.raises(dipmc.McError) as e:
        dipmc.energy_noalloc(8192, 1, t, t, t, t)
    assert e.value.code == dipmc.MC_EINVAL
    assert "4096" in str(e.value)
