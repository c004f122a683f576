"""GPU parity of the dipolar Ising variant (Appendix B): Ising initial states,
the reversal move on every field path, the staggered magnetisation and the
energy histogram against the oracle; the simultaneous update against the exact
sequential one (l = L) on the same lattice, as Appendix B compares them."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import oracle as orc  # noqa: E402
from tests.parity_util import F32, compare_trace, resync  # noqa: E402

# Appendix B's J/C_D = 1.7 with its energy (J/2) sum_<ij> counting each bond
# once: a coupling of 0.85 C_D per bond, where stripes of width 1 have the
# lowest energy (the library's J is the coupling per bond)
J, CD = F32(1.0), F32(1.0 / 0.85)


@pytest.fixture(scope="module")
def dipmc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1211_6234_b300 import dipmc as d
    return d


def test_ising_init_matches_oracle(dipmc):
    L, R, seed = 16, 3, 77
    with dipmc.Lattice(L, 8, R, seed) as lat:
        lat.init_spins(dipmc.INIT_ISING)
        s = lat.get_spins().astype(np.float64)
    for r in range(R):
        np.testing.assert_array_equal(s[r], orc.init_ising(L, seed, r))


PATHS = [1, 2, 3, 4, 5]


@pytest.mark.parametrize("path", PATHS, ids=["direct", "window_f32", "tensor", "fft", "spectral"])
def test_ising_trace_matches_oracle(dipmc, path):
    L, l, R, nsw, A, seed = 16, 8, 2, 2, 16, 41
    Ts = [F32(0.85 * CD), F32(0.6 * CD)]
    with dipmc.Lattice(L, l, R, seed) as lat:
        lat.precompute_W(A, True)
        lat.set_field_path(path)
        lat.set_proposal(dipmc.PROPOSAL_FLIP, 0.5)
        for r in range(R):
            lat.set_params(J, CD, 0.0, 0.0, Ts[r], replica=r)
        lat.init_spins(dipmc.INIT_ISING)
        tr = lat.sweep_trace(nsw)
        sg = lat.get_spins().astype(np.float64)
    W = orc.wtilde(L, A, True)
    for r in range(R):
        s0 = orc.init_ising(L, seed, r)
        p = orc.params(L, l, J, CD, 0.0, 0.0, Ts[r], proposal=2, schedule=0, seed=seed, replica=r)
        o = resync(p, W, s0, 0, nsw, tr[r])
        hmax = float(np.abs(o["h"]).max())
        rep = compare_trace(tr[r], o, Ts[r], scale=1 + abs(J) + abs(CD) * hmax)
        if rep.straddles == 0:
            np.testing.assert_array_equal(sg[r], o["s"])


def test_ising_observables_and_histogram_match_oracle(dipmc):
    """Same seeded run on the GPU (direct path) and in the oracle: identical
    final states, so the per-sweep m_st, |m| and E/N series agree to rounding
    and the E/N histogram of the GPU equals the oracle series binned alike."""
    L, l, nsw, A, seed = 16, 8, 40, 16, 5
    T = F32(0.9 * CD)
    lo, hi, nb = -2.0, 1.0, 60
    with dipmc.Lattice(L, l, 1, seed) as lat:
        lat.precompute_W(A, True)
        lat.set_field_path(dipmc.MC_PATH_DIRECT)
        lat.set_proposal(dipmc.PROPOSAL_FLIP, 0.5)
        lat.set_params(J, CD, 0.0, 0.0, T)
        lat.init_spins(dipmc.INIT_ISING)
        lat.set_histogram(lo, hi, nb)
        lat.sweep(nsw, 1)
        og = lat.observables(0)
        hg = lat.histogram(0)
        sg = lat.get_spins()[0].astype(np.float64)
    W = orc.wtilde(L, A, True)
    p = orc.params(L, l, J, CD, 0.0, 0.0, T, proposal=2, schedule=0, seed=seed)
    o = orc.sweeps(p, W, orc.init_ising(L, seed, 0), 0, nsw, trace=False, observe=True)
    np.testing.assert_array_equal(sg, o["s"])
    for i, nm in enumerate(dipmc.OBS_NAMES):
        assert og[nm]["mean"] == pytest.approx(o["obs"][:, i].mean(), abs=2e-6), nm
    ho, _ = np.histogram(o["obs"][:, 4], bins=nb, range=(lo, hi))
    assert hg.sum() == nsw
    assert np.abs(hg - ho).sum() <= 2          # a sample within rounding of a bin edge may move


def test_simultaneous_update_against_exact_sequential(dipmc):
    """Appendix B's test of the approximation: the simultaneous update (l = 16,
    four sites per sub-step) and the exact sequential update (l = L = 32) give
    the same m_st and E/N, within statistics, in the striped (T/C_D = 0.6, from
    horizontal stripes of width 1) and disordered (T/C_D = 1.2) phases."""
    L, R, neq, nms = 32, 48, 400, 1200
    y = np.arange(L)[:, None] * np.ones((1, L))
    s0 = np.zeros((2 * R, 3, L, L), np.float32)
    s0[:, 2] = np.where(y % 2 == 0, 1.0, -1.0)
    rng = np.random.default_rng(3)
    s0[R:, 2] = np.where(rng.random((R, L, L)) < 0.5, 1.0, -1.0)
    res = {}
    for l in (16, 32):
        with dipmc.Lattice(L, l, 2 * R, 123 + l) as lat:
            lat.precompute_W(64, True)
            lat.set_field_path(dipmc.MC_PATH_DIRECT)
            lat.set_proposal(dipmc.PROPOSAL_FLIP, 0.5)
            for r in range(2 * R):
                lat.set_params(J, CD, 0.0, 0.0, F32((0.6 if r < R else 1.2) * CD), replica=r)
            lat.init_spins(dipmc.INIT_USER, s0)
            lat.sweep(neq, 0)
            lat.reset_observables()
            lat.sweep(nms, 1)
            res[l] = [lat.observables(r) for r in range(2 * R)]
    for phase, rs in (("striped", range(R)), ("disordered", range(R, 2 * R))):
        for nm in ("m_st", "e"):
            a = np.array([res[16][r][nm]["mean"] for r in rs])
            b = np.array([res[32][r][nm]["mean"] for r in rs])
            ea = math.sqrt(np.mean([res[16][r][nm]["err"] ** 2 for r in rs]) / len(rs))
            eb = math.sqrt(np.mean([res[32][r][nm]["err"] ** 2 for r in rs]) / len(rs))
            diff = abs(a.mean() - b.mean())
            print(f"{phase} {nm}: l=16 {a.mean():.5f} +- {ea:.5f}, l=32 {b.mean():.5f} +- {eb:.5f}")
            assert diff < 3 * math.hypot(ea, eb) + 0.01 * abs(b.mean()), (phase, nm, a.mean(), b.mean(), ea, eb)
