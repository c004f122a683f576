"""GPU parity: the CUDA path (through the C ABI) against the CPU FP64 oracle on the
same seeded inputs.

Tolerances: W~ (FP64 on both sides) relative 1e-12; fields normwise relative
1e-5 (FP32 path); proposals and acceptance uniforms identical up to FP32
rounding; accept decisions identical except where the oracle's dE lies within
the FP32 tolerance of the threshold -T ln u (a straddle, counted).
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import oracle as orc  # noqa: E402
from paper_1211_6234_b300 import inputs  # noqa: E402
from tests.parity_util import F32, binning_reference, compare_trace, pooled, resync  # noqa: E402


@pytest.fixture(scope="module")
def dipmc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1211_6234_b300 import dipmc as d
    return d


_WCACHE = {}


def oracle_W(L, A):
    if (L, A) not in _WCACHE:
        _WCACHE[(L, A)] = orc.wtilde(L, A, True)
    return _WCACHE[(L, A)]


# ---------------------------------------------------------------- a0: W~
@pytest.mark.parametrize("L,A", [(2, 8), (6, 16), (12, 16), (16, 64), (64, 64)])
def test_wtilde_matches_oracle(dipmc, L, A):
    with dipmc.Lattice(L, L if L < 4 else L // 2, 1, 1) as lat:
        lat.precompute_W(A, True)
        Wg = lat.get_W()
    Wo = oracle_W(L, A)
    err = np.abs(Wg - Wo).max() / np.abs(Wo).max()
    assert err < 1e-12, err


# ---------------------------------------------------------------- full field
@pytest.mark.parametrize("L,R", [(8, 1), (16, 3), (64, 2)])
def test_full_field_matches_oracle(dipmc, L, R):
    s0 = inputs.random_spins(L, R, seed=10 + L)
    with dipmc.Lattice(L, L // 2, R, 3) as lat:
        lat.precompute_W(16 if L > 16 else 64, True)
        lat.init_spins(2, s0)
        hg = lat.get_field().astype(np.float64)
        W = lat.get_W()
    Wo = oracle_W(L, 16 if L > 16 else 64)
    for r in range(R):
        ho = orc.field(Wo, s0[r])
        err = np.abs(hg[r] - ho).max() / np.abs(ho).max()
        assert err < 1e-5, err


# ---------------------------------------------------------------- a1-a3: sweeps
CASES = [
    # L, l, R, proposal, schedule, nsweeps, A
    (16, 8, 2, 0, 0, 4, 64),    # the small L = 16 workload: l = L/2, cap 0.5 rad
    (16, 16, 1, 0, 0, 2, 64),   # l = L: exact sequential (n = 1)
    (16, 4, 2, 0, 0, 3, 64),    # C = 4: 16 simultaneous sites
    (12, 6, 2, 1, 0, 4, 16),    # non-power-of-two L, ragged thread tail, sphere proposals
    (12, 6, 1, 0, 1, 4, 16),    # the paper's with-replacement schedule
    (4, 2, 2, 0, 0, 6, 16),     # small lattice, update sites at distance 2
    (2, 2, 1, 0, 0, 8, 16),     # smallest lattice (l = L = 2)
    (48, 24, 1, 0, 0, 1, 16),   # L = 48 (2 cell offsets per thread)
    (64, 32, 2, 0, 0, 1, 16),   # the L = 64 launch configuration of the benchmark
    (64, 16, 1, 0, 0, 1, 16),   # L = 64 with 16 simultaneous sites
]


def _run_case(dipmc, L, l, R, proposal, schedule, nsw, A, params):
    seed = 1000 + 7 * L + l
    s0 = inputs.random_spins(L, R, seed=L * 31 + l)
    with dipmc.Lattice(L, l, R, seed) as lat:
        lat.precompute_W(A, True)
        lat.set_field_path(dipmc.MC_PATH_DIRECT)   # the direct kernel
        lat.set_proposal(proposal, 0.5)
        lat.set_schedule(schedule)
        for r, (J, CD, K2, K4, T) in enumerate(params):
            lat.set_params(J, CD, K2, K4, T, replica=r)
        lat.init_spins(2, s0)
        tr = lat.sweep_trace(nsw)
        sg = lat.get_spins().astype(np.float64)
        Eg_full = lat.energy()
        Eg_tracked = np.array([lat.observables(r)["energy"] * L * L for r in range(R)])
    return seed, s0, tr, sg, Eg_full, Eg_tracked


@pytest.mark.parametrize("case", CASES, ids=[f"L{c[0]}_l{c[1]}_R{c[2]}_p{c[3]}_s{c[4]}" for c in CASES])
def test_sweep_trace_matches_oracle(dipmc, case):
    L, l, R, proposal, schedule, nsw, A = case
    params = [(F32(1.0), F32(0.1), F32(0.8), F32(0.0), F32(0.6)),
              (F32(0.7), F32(0.3), F32(0.5), F32(-0.2), F32(1.1))][:R]
    seed, s0, tr, sg, Eg_full, Eg_tracked = _run_case(dipmc, L, l, R, proposal, schedule, nsw, A, params)
    W = oracle_W(L, A)
    straddles = 0
    for r in range(R):
        J, CD, K2, K4, T = params[r]
        p = orc.params(L, l, J, CD, K2, K4, T, proposal=proposal, cone=0.5, schedule=schedule,
                       seed=seed, replica=r)
        o = resync(p, W, s0[r], 0, nsw, tr[r])
        hmax = float(np.abs(o["h"]).max())
        rep = compare_trace(tr[r], o, T, scale=1 + abs(J) + abs(K2) + abs(K4) + abs(CD) * hmax)
        straddles += rep.straddles
        if rep.straddles == 0:
            assert rep.compared == nsw * L * L
            np.testing.assert_allclose(sg[r], o["s"], rtol=0, atol=1e-5)
            # tracked energy (sum of accepted dE + cross terms) against the oracle's
            # full energy of its own final state and the GPU's own full evaluation
            Eo = orc.energy(W, o["s"], J, CD, K2, K4)[3]
            assert abs(Eg_tracked[r] - Eo) < 1e-5 * (L * L) * (1 + abs(J) + abs(K2) + abs(K4) + CD * 10)
        assert abs(Eg_tracked[r] - Eg_full[r]) < 1e-5 * (L * L) * (1 + abs(J) + abs(K2) + abs(K4) + CD * 10)
    total = sum(nsw * L * L for _ in range(R))
    assert straddles / total <= 1e-6, straddles


def test_l_equals_L_gpu_matches_exact_sequential(dipmc):
    """l = L on the GPU takes the decisions of the oracle's exact sequential
    Metropolis (dE from full-energy differences), Appendix B."""
    L = 6
    s0 = inputs.random_spins(L, 1, seed=77)
    J, CD, K2, K4, T = F32(1.0), F32(0.5), F32(0.8), F32(0.2), F32(0.7)
    with dipmc.Lattice(L, L, 1, 5) as lat:
        lat.precompute_W(16, True)
        lat.set_field_path(dipmc.MC_PATH_DIRECT)   # the direct kernel
        lat.set_params(J, CD, K2, K4, T)
        lat.init_spins(2, s0)
        tr = lat.sweep_trace(3)
    p = orc.params(L, L, J, CD, K2, K4, T, proposal=0, cone=0.5, seed=5, replica=0)
    ex = orc.sweeps_exact(p, oracle_W(L, 16), s0[0], 0, 3)
    mism = np.nonzero(tr[0][:, 6].astype(int) != ex["acc"])[0]
    if len(mism):
        i = mism[0]
        thr = -T * math.log(tr[0][i, 5])
        assert abs(ex["dE"][i] - thr) < 1e-4, (i, ex["dE"][i], thr)


# ---------------------------------------------------------------- a4: observables
@pytest.mark.parametrize("T", [0.5, 2.5])
def test_observables_statistically_match_oracle(dipmc, T):
    """L = 16, 2000 sweeps measured every sweep after 300 from +z, in the ordered
    (T = 0.5) and paramagnetic (T = 2.5) phases: every observable and the cone angle
    eta, averaged over independent replicas (32 on the GPU's direct path, 16 in the
    oracle; different seeds, same law), agree within 3 combined standard errors.
    Each replica's time average carries its own autocorrelation, so the spread of
    the replica averages is an autocorrelation-corrected error of the pooled mean."""
    L, l, nsw, warm_sw, R_gpu, R_orc = 16, 8, 2000, 300, 32, 16
    J, CD, K2, K4, T = F32(1.0), F32(0.1), F32(0.8), F32(0.0), F32(T)
    with dipmc.Lattice(L, l, R_gpu, 11) as lat:
        lat.precompute_W(64, True)
        lat.set_field_path(dipmc.MC_PATH_DIRECT)   # the direct kernel
        lat.set_params(J, CD, K2, K4, T)
        lat.init_spins(1)
        lat.sweep(warm_sw, 0)
        lat.reset_observables()
        lat.sweep(nsw, 1)
        og = lat.observables_batch()
    ps = [orc.params(L, l, J, CD, K2, K4, T, proposal=0, cone=0.5, seed=99, replica=r) for r in range(R_orc)]
    W = oracle_W(L, 64)
    warm = orc.sweeps_batch(ps, W, inputs.saturated_z(L, R_orc), 0, warm_sw, observe=False)["s"]
    o = orc.sweeps_batch(ps, W, warm, warm_sw, nsw, observe=True)
    for g in og:
        assert g["samples"] == nsw
        assert 0 < g["accepted"] <= g["attempted"] == nsw * L * L
    for i, nm in enumerate(dipmc.OBS_NAMES):
        a, ea = pooled([g[nm]["mean"] for g in og])
        b, eb = pooled(o["obs"][:, :, i].mean(axis=1))
        assert abs(a - b) <= 3 * math.hypot(ea, eb) + 1e-9, (nm, a, b, ea, eb)
    a, ea = pooled([g["eta"] for g in og])
    b, eb = pooled([orc.eta(o["theta2"][r], nsw) for r in range(R_orc)])
    assert abs(a - b) <= 3 * math.hypot(ea, eb), ("eta", a, b, ea, eb)


@pytest.mark.parametrize("path", [1, 2, 3, 4, 5, 6, 7],
                         ids=["direct", "window_f32", "tensor", "fft", "spectral", "incremental", "cluster"])
def test_error_bars_equal_a_binning_analysis_of_the_samples(dipmc, path):
    """Each path's kernel keeps its own binning accumulators.  Run 128 one-sweep calls,
    measured every sweep, recover every per-sweep sample from the running means, and
    compare the library's variance, naive error, autocorrelation-corrected error and
    tau_int of every observable with a binning analysis of those samples in numpy."""
    L, l, R, n = 16, 8, 2, 128
    with dipmc.Lattice(L, l, R, 5) as lat:
        lat.precompute_W(16, True)
        lat.set_field_path(path)
        lat.set_params(F32(1.0), F32(0.15), F32(0.8), F32(-0.1), F32(0.9))
        lat.init_spins(0)
        means = np.zeros((n, R, len(dipmc.OBS_NAMES)))
        for t in range(n):
            lat.sweep(1, 1)
            a = lat.observables_arrays()
            means[t] = a["mean"]
        last = lat.observables_batch()
    cnt = np.arange(1, n + 1, dtype=np.float64)[:, None, None]
    sums = means * cnt
    x = np.diff(np.concatenate([np.zeros((1, R, means.shape[2])), sums]), axis=0)
    for r in range(R):
        assert last[r]["samples"] == n
        for i, nm in enumerate(dipmc.OBS_NAMES):
            var, naive, err, tau = binning_reference(x[:, r, i])
            got = last[r][nm]
            scale = abs(float(np.mean(x[:, r, i]))) + 1.0
            # the samples come back from FP64 running means (a few ulp of the sums each), and
            # a constant observable leaves the library rounding residue in its variance
            assert got["var"] == pytest.approx(var, rel=1e-4, abs=1e-11 * scale * scale), (nm, r)
            assert got["err_naive"] == pytest.approx(naive, rel=1e-4, abs=1e-7 * scale), (nm, r)
            assert got["err"] == pytest.approx(err, rel=1e-4, abs=1e-7 * scale), (nm, r)
            if naive > 1e-5 * scale:
                assert got["tau_int"] == pytest.approx(tau, rel=1e-3), (nm, r)


def test_error_bars_match_the_spread_of_replica_means(dipmc):
    """What the autocorrelation-corrected error estimates: over 64 independent replicas
    of one law (L = 16, T = 1.5 from +z, 3000 sweeps dropped, 16000 measured, so that the
    binning levels with at least 32 blocks reach blocks of 256 sweeps, well beyond
    tau_int of about 25), the RMS of the replicas' own binning errors of |m|, |m_z|,
    M_par and E/N equals the standard deviation of their means within the sampling
    scatter of both, where the naive errors fall short by more than half; every error is
    at least the naive one and tau_int >= 1/2."""
    L, l, R, warm, nsw = 16, 8, 64, 3000, 16000
    with dipmc.Lattice(L, l, R, 23) as lat:
        lat.precompute_W(64, True)
        lat.set_field_path(dipmc.MC_PATH_DIRECT)
        lat.set_params(F32(1.0), F32(0.1), F32(0.8), F32(0.0), F32(1.5))
        lat.init_spins(1)
        lat.sweep(warm, 0)
        lat.reset_observables()
        lat.sweep(nsw, 1)
        og = lat.observables_batch()
    for nm in ("abs_m", "abs_m_z", "m_par", "e"):
        means = np.array([g[nm]["mean"] for g in og])
        errs = np.array([g[nm]["err"] for g in og])
        naive = np.array([g[nm]["err_naive"] for g in og])
        assert np.all(errs >= naive) and np.all(naive > 0), nm
        assert all(g[nm]["tau_int"] >= 0.5 for g in og), nm
        sd = float(means.std(ddof=1))
        ratio = math.sqrt(float(np.mean(errs ** 2))) / sd
        print(f"{nm}: binning error / spread of means = {ratio:.3f}, "
              f"naive / spread = {math.sqrt(float(np.mean(naive ** 2))) / sd:.3f}")
        assert 0.7 <= ratio <= 1.35, (nm, ratio)
        assert math.sqrt(float(np.mean(naive ** 2))) / sd < 0.5, nm


# ---------------------------------------------------------------- state handling
def test_determinism_checkpoint_and_batch_invariance(dipmc):
    L, l = 16, 8
    def make(R):
        lat = dipmc.Lattice(L, l, R, 42)
        lat.precompute_W(16, True)
        lat.set_field_path(dipmc.MC_PATH_DIRECT)   # the direct kernel
        lat.init_spins(0)
        return lat
    with make(3) as a, make(3) as b, make(1) as c:
        a.sweep(20, 2); b.sweep(20, 2); c.sweep(20, 2)
        sa, sb, sc = a.get_spins(), b.get_spins(), c.get_spins()
        assert np.array_equal(sa, sb)                 # same seed, same run: bitwise
        assert np.array_equal(sa[0], sc[0])           # replica 0 alone vs in a batch
        ck = a.checkpoint()
        a.sweep(15, 1)
        s1 = a.get_spins()
        o1 = a.observables(1)
        a.restore(ck)
        assert a.sweep_counter() == 20
        a.sweep(15, 1)
        assert np.array_equal(a.get_spins(), s1)      # resume is bit-exact
        o2 = a.observables(1)
        assert o1["samples"] == o2["samples"] and o1["abs_m"]["mean"] == o2["abs_m"]["mean"]


@pytest.mark.parametrize("path", ["tensor", "spectral"])
def test_windowed_paths_checkpoint_and_batch_invariance(dipmc, path):
    """The tensor path at L = 64 (spectral operands, split-K tiles) and the windowed
    spectral path at L = 128: replica 0 of a batch equals the same replica run alone,
    bit for bit, and a restored checkpoint resumes bit-exactly (the spin spectra and
    energy anchors are rebuilt from the restored state)."""
    L, l, pid = (64, 32, dipmc.MC_PATH_TENSOR) if path == "tensor" else (128, 16, dipmc.MC_PATH_SPECTRAL)
    def make(R):
        lat = dipmc.Lattice(L, l, R, 7)
        lat.precompute_W(16, True)
        lat.set_field_path(pid)
        for r in range(R):
            lat.set_params(1.0, 0.1, 0.8, 0.1, 0.5 + 0.05 * r, replica=r)
        lat.init_spins(0)
        return lat
    with make(20) as a, make(1) as c:
        a.sweep(6, 2)
        c.sweep(6, 2)
        assert np.array_equal(a.get_spins()[0], c.get_spins()[0])
        ck = a.checkpoint()
        a.sweep(4, 1)
        s1, o1 = a.get_spins(), a.observables(3)
        a.restore(ck)
        assert a.sweep_counter() == 6
        a.sweep(4, 1)
        assert np.array_equal(a.get_spins(), s1)
        o2 = a.observables(3)
        assert o1["samples"] == o2["samples"] and o1["energy"] == o2["energy"]


@pytest.mark.parametrize("path", ["direct", "tensor"])
def test_restore_replaces_seed_proposal_and_schedule(dipmc, path):
    """A checkpoint carries the seed, the proposal kind and cone, and the site schedule.
    Restored into a handle made with another seed, which has already replayed a launch
    graph of the same call shape under the default settings, it resumes exactly as the
    handle that wrote it; a checkpoint whose header holds an invalid proposal kind is
    rejected with MC_EINVAL."""
    L, l, R = 32, 16, 4
    pid = dipmc.MC_PATH_DIRECT if path == "direct" else dipmc.MC_PATH_TENSOR
    def make(seed):
        lat = dipmc.Lattice(L, l, R, seed)
        lat.precompute_W(16, True)
        lat.set_field_path(pid)
        lat.init_spins(0)
        return lat
    with make(11) as a, make(12) as b:
        a.set_proposal(0, 0.3)
        a.set_schedule(1)
        a.sweep(3, 1)
        ck = a.checkpoint()
        a.sweep(2, 1)
        s1, o1 = a.get_spins(), a.observables(2)
        for _ in range(3):   # the shape (2 sweeps, measured every sweep) is captured and replayed
            b.sweep(2, 1)
        bad = bytearray(ck)
        bad[20:24] = (7).to_bytes(4, "little")   # the header's proposal kind
        with pytest.raises(dipmc.McError) as e:
            b.restore(bytes(bad))
        assert e.value.code == dipmc.MC_EINVAL
        b.restore(ck)
        assert b.sweep_counter() == 3
        b.sweep(2, 1)
        assert np.array_equal(b.get_spins(), s1)
        o2 = b.observables(2)
        assert o1["samples"] == o2["samples"] and o1["abs_m"]["mean"] == o2["abs_m"]["mean"]


@pytest.mark.parametrize("path", [1, 2, 3, 4, 5, 6, 7],
                         ids=["direct", "window_f32", "tensor", "fft", "spectral", "incr", "cluster"])
def test_zero_sweeps_change_nothing(dipmc, path):
    """mc_sweep with nsweeps = 0 on every path: the spins, the sweep counter and the
    observables stay as they were."""
    L, l = 32, 16
    with dipmc.Lattice(L, l, 2, 3) as lat:
        lat.precompute_W(16, True)
        lat.set_field_path(path)
        lat.init_spins(0)
        lat.sweep(2, 1)
        s0, c0, o0 = lat.get_spins(), lat.sweep_counter(), lat.observables(1)
        lat.sweep(0, 1)
        assert np.array_equal(lat.get_spins(), s0) and lat.sweep_counter() == c0
        assert lat.observables(1)["samples"] == o0["samples"]


def test_observables_batch_equals_single_reads(dipmc):
    """The batched read-back gives every replica's statistics exactly as the
    one-replica call does; an out-of-range batch is MC_EINVAL."""
    L, l, R = 16, 8, 5
    with dipmc.Lattice(L, l, R, 9) as lat:
        lat.precompute_W(16, True)
        lat.set_field_path(dipmc.MC_PATH_DIRECT)   # the direct kernel
        for r in range(R):
            lat.set_params(F32(1.0), F32(0.1), F32(0.8), F32(0.0), F32(0.4 + 0.2 * r), replica=r)
        lat.init_spins(0)
        lat.sweep(40, 1)
        one = [lat.observables(r) for r in range(R)]
        many = lat.observables_batch()
        part = lat.observables_batch(2, 2)
        def same(x, y):
            if isinstance(x, dict):
                return x.keys() == y.keys() and all(same(x[k], y[k]) for k in x)
            if isinstance(x, float) and np.isnan(x):
                return isinstance(y, float) and np.isnan(y)
            return x == y
        for r in range(R):
            assert same(one[r], many[r]), r
        assert same(part[0], many[2]) and same(part[1], many[3])
        arr = lat.observables_arrays()
        assert arr["samples"].tolist() == [m["samples"] for m in many]
        for k, nm in enumerate(dipmc.OBS_NAMES):
            np.testing.assert_array_equal(arr["mean"][:, k], [m[nm]["mean"] for m in many])
            np.testing.assert_array_equal(arr["err"][:, k], [m[nm]["err"] for m in many])
        np.testing.assert_array_equal(arr["energy"], [m["energy"] for m in many])
        with pytest.raises(dipmc.McError) as e:
            lat.observables_batch(4, 2)
        assert e.value.code == dipmc.MC_EINVAL


def test_error_codes(dipmc):
    with dipmc.Lattice(16, 8, 1, 1) as lat:
        with pytest.raises(dipmc.McError) as e:
            lat.sweep(1)
        assert e.value.code == dipmc.MC_ENOTREADY
        with pytest.raises(dipmc.McError) as e:
            lat.set_params(T=0.0)
        assert e.value.code == dipmc.MC_EINVAL
        with pytest.raises(dipmc.McError) as e:
            lat.set_proposal(0, 4.0)
        assert e.value.code == dipmc.MC_EINVAL
    with dipmc.Lattice(256, 128, 1, 1) as big:
        with pytest.raises(dipmc.McError) as e:
            big.set_field_path(dipmc.MC_PATH_DIRECT)
        assert e.value.code == dipmc.MC_ENOSYS


def test_random_init_is_uniform_on_sphere(dipmc):
    with dipmc.Lattice(64, 32, 4, 9) as lat:
        lat.init_spins(0)
        s = lat.get_spins().astype(np.float64)
    norm = np.sqrt((s**2).sum(1))
    assert np.abs(norm - 1).max() < 1e-6
    z = s[:, 2].ravel()
    assert abs(z.mean()) < 0.02 and abs((z**2).mean() - 1 / 3) < 0.02


# ---------------------------------------------------------------- benchmark configuration
def test_bench_configuration_sampled_replicas(dipmc):
    """256 replicas of L = 64, l = 32 with the temperature x K4/K2 ladder -- the launch
    configuration bench.py times (two CTAs per SM) -- one traced sweep; sampled
    replicas are compared attempt by attempt with the oracle, every replica is checked
    for self-consistent decisions."""
    L, l, R, A = 64, 32, 256, 64
    lad = [(F32(1.0), F32(0.1), F32(k2), F32(k4), F32(T)) for (T, k2, k4) in inputs.ladder(16, 16)]
    seed = 1
    s0 = inputs.random_spins(L, R, seed=2024)
    with dipmc.Lattice(L, l, R, seed) as lat:
        lat.precompute_W(A, True)
        lat.set_field_path(dipmc.MC_PATH_DIRECT)   # the direct kernel
        for r, prm in enumerate(lad):
            lat.set_params(*prm, replica=r)
        lat.init_spins(2, s0)
        tr = lat.sweep_trace(1)
        sg = lat.get_spins().astype(np.float64)
    assert tr.shape == (R, L * L, 10)
    # every replica: each site attempted once, decisions consistent with the threshold rule
    for r in range(R):
        q = tr[r, :, 0].astype(np.int64)
        assert np.array_equal(np.sort(q), np.arange(L * L))
        T = lad[r][4]
        u = tr[r, :, 5].astype(np.float64)
        thr = np.where(u > 0, -T * np.log(np.maximum(u, 1e-300)), np.inf)
        dE = tr[r, :, 4].astype(np.float64)
        acc = tr[r, :, 6].astype(np.int64)
        clear = np.abs(dE - thr) > 1e-5 * (1 + abs(dE))
        assert np.array_equal(acc[clear], (dE < thr)[clear].astype(np.int64))
    W = oracle_W(L, A)
    for r in (0, 37, 148, 255):
        J, CD, K2, K4, T = lad[r]
        p = orc.params(L, l, J, CD, K2, K4, T, proposal=0, cone=0.5, schedule=0, seed=seed, replica=r)
        o = resync(p, W, s0[r], 0, 1, tr[r])
        hmax = float(np.abs(o["h"]).max())
        rep = compare_trace(tr[r], o, T, scale=1 + abs(J) + abs(K2) + abs(K4) + abs(CD) * hmax)
        if rep.straddles == 0:
            np.testing.assert_allclose(sg[r], o["s"], rtol=0, atol=1e-5)


def test_many_replica_instance_small_lattice(dipmc):
    """More replicas than SMs selects the two-CTAs-per-SM instance also at L = 16."""
    L, l, R = 16, 8, 160
    s0 = inputs.random_spins(L, R, seed=5)
    with dipmc.Lattice(L, l, R, 8) as lat:
        lat.precompute_W(64, True)
        lat.set_field_path(dipmc.MC_PATH_DIRECT)   # the direct kernel
        lat.init_spins(2, s0)
        tr = lat.sweep_trace(2)
    W = oracle_W(L, 64)
    for r in (0, 159):
        p = orc.params(L, l, 1.0, F32(0.1), F32(0.8), 0.0, F32(0.6), seed=8, replica=r)
        o = resync(p, W, s0[r], 0, 2, tr[r])
        compare_trace(tr[r], o, F32(0.6), scale=2 + 0.1 * float(np.abs(o["h"]).max()))


# ---------------------------------------------------------------- windowed paths
WCASES = [
    # L, l, R, B (0 = automatic), schedule, nsweeps
    (16, 8, 2, 0, 0, 2),       # S_w = 128
    (16, 8, 3, 16, 0, 2),      # smaller window than the tensor path needs (F32 only)
    (16, 4, 2, 0, 0, 2),       # 16 simultaneous sites, S_w = 128
    (16, 16, 1, 0, 0, 1),      # l = L: one site per sub-step, S_w = 256
    (48, 24, 1, 0, 0, 1),      # non-power-of-two L
    (32, 16, 2, 0, 1, 1),      # the paper's with-replacement schedule
    (64, 32, 2, 0, 0, 1),      # L = 64, S_w = 512 (F32) / 256 (tensor)
    (64, 32, 2, 128, 0, 1),    # L = 64, S_w = 512 on both paths
    (80, 40, 2, 0, 0, 1),      # non-power-of-two L = 80: spectral operands (L = 2l, l % 8 == 0)
    (80, 20, 1, 0, 0, 1),      # L = 80, 16 sites per sub-step: Toeplitz operands at a large lattice
    (12, 6, 2, 12, 0, 2),      # l = 6: the 2 x 2 spectra's folds at odd l/2 = 3 (F32 only)
    (20, 10, 2, 20, 0, 2),     # l = 10: odd l/2 = 5 (F32 only)
]


# the tensor path needs windows of a multiple of 128 sites: the cases with smaller windows
# run on the FP32 window path only
WPAIRS = [(path, c) for c in WCASES for path in (2, 3) if not (path == 3 and c[3] in (12, 16, 20))]


@pytest.mark.parametrize("path,case", WPAIRS,
                         ids=[("window_f32-" if p == 2 else "tensor_bf16x3-") +
                              f"L{c[0]}_l{c[1]}_R{c[2]}_B{c[3]}_s{c[4]}" for p, c in WPAIRS])
def test_window_paths_match_oracle(dipmc, path, case):
    L, l, R, B, schedule, nsw = case
    params = [(F32(1.0), F32(0.1), F32(0.8), F32(0.0), F32(0.6)),
              (F32(0.7), F32(0.3), F32(0.5), F32(-0.2), F32(1.1)),
              (F32(1.0), F32(0.2), F32(0.8), F32(0.3), F32(0.4))][:R]
    seed = 300 + L + l
    s0 = inputs.random_spins(L, R, seed=L + 7 * l)
    A = 16
    with dipmc.Lattice(L, l, R, seed) as lat:
        lat.precompute_W(A, True)
        lat.set_window(B)
        lat.set_field_path(path)
        lat.set_schedule(schedule)
        for r, prm in enumerate(params):
            lat.set_params(*prm, replica=r)
        lat.init_spins(2, s0)
        tr = lat.sweep_trace(nsw)
        sg = lat.get_spins().astype(np.float64)
        Eg_full = lat.energy()
        Eg_tracked = np.array([lat.observables(r)["energy"] * L * L for r in range(R)])
    W = oracle_W(L, A)
    for r in range(R):
        J, CD, K2, K4, T = params[r]
        p = orc.params(L, l, J, CD, K2, K4, T, proposal=0, cone=0.5, schedule=schedule, seed=seed, replica=r)
        o = resync(p, W, s0[r], 0, nsw, tr[r])
        hmax = float(np.abs(o["h"]).max())
        rep = compare_trace(tr[r], o, T, scale=1 + abs(J) + abs(K2) + abs(K4) + abs(CD) * hmax)
        if rep.straddles == 0:
            np.testing.assert_allclose(sg[r], o["s"], rtol=0, atol=1e-5)
        assert abs(Eg_tracked[r] - Eg_full[r]) < 1e-5 * (L * L) * (1 + abs(J) + abs(K2) + abs(K4) + CD * 10)


@pytest.mark.parametrize("path", [2, 3], ids=["window_f32", "tensor_bf16x3"])
def test_window_paths_paired_replicas_odd_count(dipmc, path):
    """One replica more than the device has SMs: the sub-step kernel runs two replicas
    a CTA (even and odd warps), and the last CTA holds one.  Replicas of the first,
    a middle and the last CTA against the re-synchronised oracle."""
    import torch
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    L, l, A, R = 16, 8, 16, nsm + 1
    sample = (0, 1, R // 2, R - 2, R - 1)
    lad = [(F32(1.0), F32(0.1), F32(k2), F32(k4), F32(T)) for (T, k2, k4) in inputs.ladder(16, 16)]
    lad = [lad[r % len(lad)] for r in range(R)]
    s0 = inputs.random_spins(L, R, seed=77)
    with dipmc.Lattice(L, l, R, 12) as lat:
        lat.precompute_W(A, True)
        lat.set_field_path(path)
        for r, prm in enumerate(lad):
            lat.set_params(*prm, replica=r)
        lat.init_spins(2, s0)
        tr = lat.sweep_trace(2)
        sg = lat.get_spins().astype(np.float64)
        Eg_full = lat.energy()
        Eg_tracked = np.array([lat.observables(r)["energy"] * L * L for r in range(R)])
    W = oracle_W(L, A)
    for r in sample:
        J, CD, K2, K4, T = lad[r]
        p = orc.params(L, l, J, CD, K2, K4, T, proposal=0, cone=0.5, schedule=0, seed=12, replica=r)
        o = resync(p, W, s0[r], 0, 2, tr[r])
        hmax = float(np.abs(o["h"]).max())
        rep = compare_trace(tr[r], o, T, scale=1 + abs(J) + abs(K2) + abs(K4) + abs(CD) * hmax)
        if rep.straddles == 0:
            np.testing.assert_allclose(sg[r], o["s"], rtol=0, atol=1e-5)
    np.testing.assert_allclose(Eg_tracked, Eg_full, rtol=0, atol=1e-5 * L * L * 3)


def _resync_all(lad, L, l, seed, W, s0, tr, nsw, chunk=32):
    """Every replica's trace against the oracle re-synchronised per sub-step
    (orc_replay over all host threads, `chunk` replicas at a time); returns the
    straddle count, the attempts compared and the worst field / dE errors."""
    R = tr.shape[0]
    tot = {"straddles": 0, "compared": 0, "h_err": 0.0, "dE_err": 0.0}
    for c0 in range(0, R, chunk):
        rr = range(c0, min(R, c0 + chunk))
        ps = [orc.params(L, l, *lad[r], proposal=0, cone=0.5, schedule=0, seed=seed, replica=r) for r in rr]
        out = orc.replay_batch(ps, W, s0[c0:c0 + len(rr)], 0, nsw, tr[c0:c0 + len(rr), :, 6].astype(np.int32),
                               tr[c0:c0 + len(rr), :, 7:10].astype(np.float64))
        for i, r in enumerate(rr):
            J, CD, K2, K4, T = lad[r]
            o = {k: v[i] for k, v in out.items()}
            hmax = float(np.abs(o["h"]).max())
            rep = compare_trace(tr[r], o, T, scale=1 + abs(J) + abs(K2) + abs(K4) + abs(CD) * hmax)
            tot["straddles"] += rep.straddles
            tot["compared"] += rep.compared
            tot["h_err"] = max(tot["h_err"], rep.h_err_norm)
            tot["dE_err"] = max(tot["dE_err"], rep.dE_err)
    return tot


@pytest.mark.parametrize("path", ["tensor", "direct"])
def test_bench_shape_every_attempt_resynced(dipmc, path):
    """The benchmark's launch configuration -- 256 replicas x L = 64, l = 32, the
    16 T x 16 K4/K2 ladder -- traced over 4 sweeps on the tensor path (4.2e6
    attempts; 1 sweep on the direct path), and every attempt of every replica
    compared with the oracle decided from the GPU's pre-step state: fields within
    1e-5 normwise at every attempt, dE within the FP32 tolerance, and differing
    decisions only where the threshold straddles the two dE, at a fraction of at
    most 1e-6 of the attempts."""
    L, l, R, A = 64, 32, 256, 64
    nsw = 4 if path == "tensor" else 1
    lad = [(F32(1.0), F32(0.1), F32(k2), F32(k4), F32(T)) for (T, k2, k4) in inputs.ladder(16, 16)]
    s0 = inputs.random_spins(L, R, seed=2024)
    with dipmc.Lattice(L, l, R, 1) as lat:
        lat.precompute_W(A, True)
        lat.set_field_path(dipmc.MC_PATH_TENSOR if path == "tensor" else dipmc.MC_PATH_DIRECT)
        for r, prm in enumerate(lad):
            lat.set_params(*prm, replica=r)
        lat.init_spins(2, s0)
        tr = lat.sweep_trace(nsw)
        sg = lat.get_spins()
    assert tr.shape == (R, nsw * L * L, 10)
    tot = _resync_all(lad, L, l, 1, oracle_W(L, A), s0, tr, nsw)
    print(f"\n[{path} path, 256 x L=64, l=32, {nsw} sweep(s)] attempts compared: {tot['compared']}, "
          f"straddles: {tot['straddles']}, max field error (normwise): {tot['h_err']:.2e}, "
          f"max dE error: {tot['dE_err']:.2e}")
    assert tot["compared"] == R * nsw * L * L
    assert tot["straddles"] / tot["compared"] <= 1e-6, tot
    assert tot["h_err"] <= 1e-5
    # the final spins are the trace's last accepted proposals: replay the trace
    st = s0.astype(np.float32).copy()
    for r in range(R):
        acc = np.nonzero(tr[r, :, 6] > 0.5)[0]
        q = tr[r, acc, 0].astype(np.int64)
        _, last = np.unique(q[::-1], return_index=True)    # each site's last accepted move
        pick = acc[len(acc) - 1 - last]
        st[r].reshape(3, -1)[:, tr[r, pick, 0].astype(np.int64)] = tr[r, pick, 7:10].T
    np.testing.assert_allclose(sg, st, rtol=0, atol=1e-6)


def test_tensor_path_ragged_second_tile(dipmc):
    """300 replicas x L = 64 on the tensor path: a second, ragged N-tile of 44
    replicas; one traced sweep, sampled replicas of both tiles compared attempt by
    attempt with the re-synchronised oracle."""
    L, l, A, R = 64, 32, 64, 300
    sample = (0, 255, 256, 299)
    lad = [(F32(1.0), F32(0.1), F32(k2), F32(k4), F32(T)) for (T, k2, k4) in inputs.ladder(16, 16)]
    lad = [lad[r % len(lad)] for r in range(R)]
    s0 = inputs.random_spins(L, R, seed=2024)
    with dipmc.Lattice(L, l, R, 1) as lat:
        lat.precompute_W(A, True)
        lat.set_field_path(dipmc.MC_PATH_TENSOR)
        for r, prm in enumerate(lad):
            lat.set_params(*prm, replica=r)
        lat.init_spins(2, s0)
        tr = lat.sweep_trace(1)
        sg = lat.get_spins().astype(np.float64)
    W = oracle_W(L, A)
    worst = 0.0
    for r in sample:
        J, CD, K2, K4, T = lad[r]
        p = orc.params(L, l, J, CD, K2, K4, T, proposal=0, cone=0.5, schedule=0, seed=1, replica=r)
        o = resync(p, W, s0[r], 0, 1, tr[r])
        hmax = float(np.abs(o["h"]).max())
        rep = compare_trace(tr[r], o, T, scale=1 + abs(J) + abs(K2) + abs(K4) + abs(CD) * hmax)
        worst = max(worst, rep.h_err_norm)
        assert rep.straddles == 0
        np.testing.assert_allclose(sg[r], o["s"], rtol=0, atol=1e-6)
    assert worst < 1e-5


@pytest.mark.parametrize("R,sample", [(1, (0,)), (520, (0, 255, 256, 511, 512, 519))], ids=["R1", "R520"])
def test_tensor_path_replica_count_edges(dipmc, R, sample):
    """The tensor path at its replica-count edges: one replica (an N-tile of 16 with 15
    empty rows) and 520 replicas (two full N-tiles and a ragged third of 8): sampled
    replicas of every tile, one traced sweep, against the re-synchronised oracle."""
    L, l, A = 64, 32, 16
    lad = [(F32(1.0), F32(0.1), F32(k2), F32(k4), F32(T)) for (T, k2, k4) in inputs.ladder(16, 16)]
    lad = [lad[(7 * r) % len(lad)] for r in range(R)]
    s0 = inputs.random_spins(L, R, seed=3 * R)
    with dipmc.Lattice(L, l, R, 11) as lat:
        lat.precompute_W(A, True)
        lat.set_field_path(dipmc.MC_PATH_TENSOR)
        for r, prm in enumerate(lad):
            lat.set_params(*prm, replica=r)
        lat.init_spins(2, s0)
        tr = lat.sweep_trace(1)
        sg = lat.get_spins().astype(np.float64)
    W = oracle_W(L, A)
    for r in sample:
        J, CD, K2, K4, T = lad[r]
        p = orc.params(L, l, J, CD, K2, K4, T, proposal=0, cone=0.5, schedule=0, seed=11, replica=r)
        o = resync(p, W, s0[r], 0, 1, tr[r])
        rep = compare_trace(tr[r], o, T, scale=1 + abs(J) + abs(K2) + abs(K4) + abs(CD) * float(np.abs(o["h"]).max()))
        assert rep.straddles == 0
        np.testing.assert_allclose(sg[r], o["s"], rtol=0, atol=1e-6)


def test_tensor_path_observables_match_direct(dipmc):
    """Long runs of the tensor and direct paths sample the same law: means within
    3 combined standard errors of the replica means (L = 16, 64 independent replicas)."""
    L, l, R, nsw = 16, 8, 64, 600
    res = {}
    for path in (dipmc.MC_PATH_DIRECT, dipmc.MC_PATH_TENSOR):
        with dipmc.Lattice(L, l, R, 21 if path == 1 else 22) as lat:
            lat.precompute_W(64, True)
            lat.set_field_path(path)
            lat.set_params(F32(1.0), F32(0.1), F32(0.8), F32(0.0), F32(2.0))
            lat.init_spins(1)
            lat.sweep(100, 0)
            lat.reset_observables()
            lat.sweep(nsw, 1)
            res[path] = [lat.observables(r) for r in range(R)]
    for nm in ("abs_m", "e"):
        a, ea = pooled([o[nm]["mean"] for o in res[1]])
        b, eb = pooled([o[nm]["mean"] for o in res[3]])
        assert abs(a - b) < 3 * math.hypot(ea, eb) + 1e-9, (nm, a, b, ea, eb)


def test_tensor_path_ordered_phase_matches_oracle(dipmc):
    """A long run of the tensor path in the perpendicular ordered phase (T = 0.4,
    L = 32, l = 16: the spectral tensor operands of the benchmark's L = 2l) against
    the oracle's own runs: |m|, M_par, E/N and the cone angle eta, each averaged
    over independent replicas (64 on the GPU, 16 in the oracle, both from +z),
    agree within 3 combined standard errors of the replica means."""
    L, l, R_gpu, R_orc, neq, nms = 32, 16, 64, 16, 150, 600
    prm = (F32(1.0), F32(0.1), F32(0.8), F32(0.0), F32(0.4))
    with dipmc.Lattice(L, l, R_gpu, 71) as lat:
        lat.precompute_W(64, True)
        lat.set_field_path(dipmc.MC_PATH_TENSOR)
        lat.set_params(*prm)
        lat.init_spins(1)
        lat.sweep(neq, 0)
        lat.reset_observables()
        lat.sweep(nms, 1)
        og = lat.observables_batch()
    W = oracle_W(L, 64)
    ps = [orc.params(L, l, *prm, proposal=0, cone=0.5, schedule=0, seed=72, replica=r) for r in range(R_orc)]
    s0 = inputs.saturated_z(L, R_orc)
    warm = orc.sweeps_batch(ps, W, s0, 0, neq, observe=False)["s"]
    o = orc.sweeps_batch(ps, W, warm, neq, nms, observe=True)
    names = {"abs_m": 0, "m_par": 3, "e": 4}
    for nm, k in names.items():
        a, ea = pooled([g[nm]["mean"] for g in og])
        b, eb = pooled(o["obs"][:, :, k].mean(axis=1))
        print(f"T=0.4 {nm}: tensor {a:.6f} +- {ea:.6f}, oracle {b:.6f} +- {eb:.6f}")
        assert abs(a - b) <= 3 * math.hypot(ea, eb), (nm, a, b, ea, eb)
    a, ea = pooled([g["eta"] for g in og])
    b, eb = pooled([orc.eta(o["theta2"][r], nms) for r in range(R_orc)])
    print(f"T=0.4 eta: tensor {a:.6f} +- {ea:.6f}, oracle {b:.6f} +- {eb:.6f}")
    assert abs(a - b) <= 3 * math.hypot(ea, eb), ("eta", a, b, ea, eb)
    assert a > 0.6     # ordered perpendicular (the disordered limit is 0.4352)


def test_tensor_path_bench_lattice_low_T_matches_oracle(dipmc):
    """The benchmark's lattice on the tensor path in the ordered phase: L = 64, l = 32,
    T = 0.3 (the low end of the benchmark's temperature ladder), K2 = 0.8, K4 = 0.2 K2,
    from +z, 100 sweeps then 200 measured, 64 GPU replicas against 16 oracle replicas
    under the same protocol (so the same law at every sweep, equilibrated or not):
    |m|, M_par, E/N and eta within 3 combined standard errors of the replica means."""
    L, l, R_gpu, R_orc, neq, nms = 64, 32, 64, 16, 100, 200
    prm = (F32(1.0), F32(0.1), F32(0.8), F32(0.16), F32(0.3))
    with dipmc.Lattice(L, l, R_gpu, 81) as lat:
        lat.precompute_W(64, True)
        lat.set_field_path(dipmc.MC_PATH_TENSOR)
        lat.set_params(*prm)
        lat.init_spins(1)
        lat.sweep(neq, 0)
        lat.reset_observables()
        lat.sweep(nms, 1)
        og = lat.observables_batch()
    W = oracle_W(L, 64)
    ps = [orc.params(L, l, *prm, proposal=0, cone=0.5, schedule=0, seed=82, replica=r) for r in range(R_orc)]
    warm = orc.sweeps_batch(ps, W, inputs.saturated_z(L, R_orc), 0, neq, observe=False)["s"]
    o = orc.sweeps_batch(ps, W, warm, neq, nms, observe=True)
    for nm, k in {"abs_m": 0, "m_par": 3, "e": 4}.items():
        a, ea = pooled([g[nm]["mean"] for g in og])
        b, eb = pooled(o["obs"][:, :, k].mean(axis=1))
        print(f"L=64 T=0.3 {nm}: tensor {a:.6f} +- {ea:.6f}, oracle {b:.6f} +- {eb:.6f}")
        assert abs(a - b) <= 3 * math.hypot(ea, eb), (nm, a, b, ea, eb)
    a, ea = pooled([g["eta"] for g in og])
    b, eb = pooled([orc.eta(o["theta2"][r], nms) for r in range(R_orc)])
    print(f"L=64 T=0.3 eta: tensor {a:.6f} +- {ea:.6f}, oracle {b:.6f} +- {eb:.6f}")
    assert abs(a - b) <= 3 * math.hypot(ea, eb), ("eta", a, b, ea, eb)


# ---------------------------------------------------------------- FFT path
@pytest.mark.parametrize("L,R", [(8, 1), (16, 3), (32, 2), (64, 2), (128, 1)])
def test_fft_full_field_matches_oracle(dipmc, L, R):
    s0 = inputs.random_spins(L, R, seed=40 + L)
    A = 16
    with dipmc.Lattice(L, L // 2, R, 3) as lat:
        lat.precompute_W(A, True)
        lat.set_field_path(dipmc.MC_PATH_FFT)
        lat.init_spins(2, s0)
        hg = lat.get_field().astype(np.float64)
    Wo = oracle_W(L, A)
    for r in range(R):
        ho = orc.field(Wo, s0[r])
        err = np.abs(hg[r] - ho).max() / np.abs(ho).max()
        assert err < 1e-5, err


@pytest.mark.parametrize("L", [256, 512, 1024])
def test_fft_full_field_L256_sampled_sites(dipmc, L):
    """L = 256, 512 (odd log2 L: a radix-2 stage) and 1024 (one column pair a tile): the
    FFT field of two replicas at sampled sites against the oracle's direct sum at
    those sites."""
    R, A = 2, 8
    s0 = inputs.random_spins(L, R, seed=256)
    with dipmc.Lattice(L, 32, R, 3) as lat:
        lat.precompute_W(A, True)
        lat.init_spins(2, s0)
        hg = lat.get_field().astype(np.float64)
        Wg = lat.get_W()
    Wo = orc.wtilde(L, A, True)
    assert np.abs(Wg - Wo).max() / np.abs(Wo).max() < 1e-12
    rng = np.random.default_rng(0)
    sites = rng.integers(0, L * L, size=24)
    hmax = 0.0
    errs = []
    for r in range(R):
        for q in sites:
            qy, qx = divmod(int(q), L)
            # h_q = sum_m W~(q - m) s_m, by numpy over the whole lattice
            dy = (qy - np.arange(L)[:, None]) % L
            dx = (qx - np.arange(L)[None, :]) % L
            xx, xy, yy, zz = Wo[0][dy, dx], Wo[1][dy, dx], Wo[2][dy, dx], Wo[3][dy, dx]
            sx, sy, sz = s0[r]
            ho = np.array([(xx * sx + xy * sy).sum(), (xy * sx + yy * sy).sum(), (zz * sz).sum()])
            hmax = max(hmax, np.abs(ho).max())
            errs.append(np.abs(hg[r, :, qy, qx] - ho).max())
    assert max(errs) / hmax < 1e-5, (max(errs), hmax)


@pytest.mark.parametrize("path", [5, 7], ids=["spectral", "cluster"])
def test_spectral_path_L256_sampled_attempts(dipmc, path):
    """L = 256, l = 32 (the large-lattice configuration the spectral and cluster paths serve):
    one traced sweep of two replicas.  Every decision is consistent with its own dE
    and u; the state is replayed attempt by attempt from the trace, and at sampled
    sub-steps the recorded field and dE are compared with a direct sum over the
    replayed state (W~ from the oracle)."""
    L, l, R, A = 256, 32, 2, 8
    n, ll = (L // l) ** 2, l * l
    prm = [(F32(1.0), F32(0.1), F32(0.8), F32(0.0), F32(0.3)), (F32(1.0), F32(0.1), F32(0.8), F32(0.1), F32(0.9))]
    s0 = inputs.random_spins(L, R, seed=913)
    with dipmc.Lattice(L, l, R, 17) as lat:
        lat.precompute_W(A, True)
        lat.set_field_path(path)
        for r in range(R):
            lat.set_params(*prm[r], replica=r)
        lat.init_spins(2, s0)
        tr = lat.sweep_trace(1).astype(np.float64)
        sg = lat.get_spins().astype(np.float64)
    Wo = orc.wtilde(L, A, True)
    W0 = Wo[:, 0, 0]
    sample_k = {0, 1, 2, 37, 511, 1000, ll - 1}
    for r in range(R):
        J, CD, K2, K4, T = prm[r]
        t_r = tr[r].reshape(ll, n, -1)
        # decisions follow the recorded dE and u: accept iff dE < -T ln u
        thr = np.where(t_r[:, :, 5] > 0, -T * np.log(np.maximum(t_r[:, :, 5], 1e-300)), np.inf)
        assert np.array_equal(t_r[:, :, 6] > 0.5, t_r[:, :, 4] < thr)
        s = np.array(s0[r], np.float64)
        hmax, herr, derr = 0.0, 0.0, 0.0
        for k in range(ll):
            q = t_r[k, :, 0].astype(np.int64)
            qy, qx = q // L, q % L
            if k in sample_k:
                for d in range(0, n, 7):
                    y0, x0 = int(qy[d]), int(qx[d])
                    dy = (y0 - np.arange(L)[:, None]) % L
                    dx = (x0 - np.arange(L)[None, :]) % L
                    xx, xy, yy, zz = Wo[0][dy, dx], Wo[1][dy, dx], Wo[2][dy, dx], Wo[3][dy, dx]
                    h = np.array([(xx * s[0] + xy * s[1]).sum(), (xy * s[0] + yy * s[1]).sum(), (zz * s[2]).sum()])
                    hmax = max(hmax, np.abs(h).max())
                    herr = max(herr, np.abs(t_r[k, d, 1:4] - h).max())
                    # dE of the proposal from the replayed state (exchange, anisotropy, dipole)
                    sq = s[:, y0, x0]
                    S = t_r[k, d, 7:10]
                    dl = S - sq
                    nb = (s[:, y0, (x0 + 1) % L] + s[:, y0, (x0 - 1) % L] + s[:, (y0 + 1) % L, x0] + s[:, (y0 - 1) % L, x0])
                    ean = -K2 * S[2] ** 2 - K4 * S[2] ** 4 + K2 * sq[2] ** 2 + K4 * sq[2] ** 4
                    self_ = W0[0] * dl[0] ** 2 + 2 * W0[1] * dl[0] * dl[1] + W0[2] * dl[1] ** 2 + W0[3] * dl[2] ** 2
                    dE = -J * dl @ nb + ean + CD * (dl @ h + 0.5 * self_)
                    derr = max(derr, abs(t_r[k, d, 4] - dE))
            acc = t_r[k, :, 6] > 0.5
            s[:, qy[acc], qx[acc]] = t_r[k, acc, 7:10].T
        assert herr / hmax < 1e-5, (herr, hmax)
        assert derr < 2e-5 * (1 + abs(J) + abs(K2) + abs(K4) + CD * hmax), derr
        np.testing.assert_allclose(sg[r], s, rtol=0, atol=1e-6)   # the replay ends in the GPU's state


FCASES = [
    # path, L, l, R, schedule, nsweeps
    (4, 16, 8, 2, 0, 2),
    (4, 32, 8, 2, 0, 1),      # 16 simultaneous sites
    (4, 64, 16, 1, 1, 1),     # the paper's with-replacement schedule
    (4, 128, 64, 1, 0, 1),    # large lattice, 4 sites per sub-step
    (5, 16, 8, 2, 0, 2),      # spectral path: 2 x 2 coarse grid
    (5, 32, 8, 2, 1, 1),      # 4 x 4, with-replacement schedule
    (5, 48, 16, 2, 0, 1),     # L not a power of two, odd coarse grid (3 x 3)
    (5, 96, 12, 1, 0, 1),     # 8 x 8 coarse grid, L not a power of two
    (5, 128, 8, 1, 0, 1),     # 16 x 16 coarse grid, 256 simultaneous sites
    (5, 60, 6, 2, 0, 1),      # 10 x 10 coarse grid: 36 sub-steps, the last window partial
    (5, 50, 10, 1, 1, 1),     # odd 5 x 5 grid, with-replacement schedule (offsets repeat within windows)
    (5, 64, 2, 1, 0, 2),      # 32 x 32 coarse grid: 1024 sites per sub-step, 4-sub-step windows
    (6, 16, 8, 2, 0, 2),      # incremental field: 4 sites per sub-step
    (6, 32, 4, 2, 1, 1),      # 64 sites per sub-step, with-replacement schedule
    (6, 48, 24, 1, 0, 1),     # L not a power of two
    (6, 64, 32, 1, 0, 1),     # the paper's L and l
    (7, 16, 8, 2, 0, 2),      # cluster transform: 2 x 2 sites, two replicas (two clusters)
    (7, 16, 16, 1, 0, 1),     # l = L: one site per sub-step (exact sequential)
    (7, 16, 2, 1, 0, 1),      # 8 x 8 sites, one row per CTA
    (7, 32, 8, 2, 1, 1),      # 4 x 4 sites, with-replacement schedule
    (7, 64, 32, 1, 0, 1),     # the paper's L and l
    (7, 128, 16, 1, 0, 1),    # 8 x 8 sites of a large lattice
]


@pytest.mark.parametrize("case", FCASES, ids=[f"{ {4: 'fft', 5: 'spec', 6: 'incr', 7: 'clus'}[c[0]]}_L{c[1]}_l{c[2]}_R{c[3]}_s{c[4]}"
                                              for c in FCASES])
def test_fft_path_trace_matches_oracle(dipmc, case):
    """FFT (full-lattice transform per sub-step) and spectral (sub-lattice
    spectra) paths against the oracle's sweep: field at every update site,
    dE, decisions and final spins."""
    path, L, l, R, schedule, nsw = case
    params = [(F32(1.0), F32(0.1), F32(0.8), F32(0.0), F32(0.6)),
              (F32(0.7), F32(0.3), F32(0.5), F32(-0.2), F32(1.1))][:R]
    seed = 500 + L + l
    s0 = inputs.random_spins(L, R, seed=3 * L + l)
    A = 16
    with dipmc.Lattice(L, l, R, seed) as lat:
        lat.precompute_W(A, True)
        lat.set_field_path(path)
        lat.set_schedule(schedule)
        for r, prm in enumerate(params):
            lat.set_params(*prm, replica=r)
        lat.init_spins(2, s0)
        tr = lat.sweep_trace(nsw)
        sg = lat.get_spins().astype(np.float64)
    W = oracle_W(L, A)
    for r in range(R):
        J, CD, K2, K4, T = params[r]
        p = orc.params(L, l, J, CD, K2, K4, T, proposal=0, cone=0.5, schedule=schedule, seed=seed, replica=r)
        o = resync(p, W, s0[r], 0, nsw, tr[r])
        hmax = float(np.abs(o["h"]).max())
        rep = compare_trace(tr[r], o, T, scale=1 + abs(J) + abs(K2) + abs(K4) + abs(CD) * hmax)
        if rep.straddles == 0:
            np.testing.assert_allclose(sg[r], o["s"], rtol=0, atol=1e-5)


@pytest.mark.parametrize("other", [4, 5, 6, 7], ids=["fft", "spectral", "incremental", "cluster"])
def test_fft_path_observables_match_direct(dipmc, other):
    """The FFT and spectral paths sample the same law as the direct path (L = 16,
    pooled replicas)."""
    L, l, R, nsw = 16, 8, 32, 400
    res = {}
    for path in (dipmc.MC_PATH_DIRECT, other):
        with dipmc.Lattice(L, l, R, 31 if path == 1 else 32) as lat:
            lat.precompute_W(64, True)
            lat.set_field_path(path)
            lat.set_params(F32(1.0), F32(0.1), F32(0.8), F32(0.0), F32(2.0))
            lat.init_spins(1)
            lat.sweep(100, 0)
            lat.reset_observables()
            lat.sweep(nsw, 1)
            res[path] = [lat.observables(r) for r in range(R)]
    for o in res[other]:
        assert o["samples"] == nsw and o["attempted"] == nsw * L * L
    for nm in ("abs_m", "e"):
        a, ea = pooled([o[nm]["mean"] for o in res[1]])
        b, eb = pooled([o[nm]["mean"] for o in res[other]])
        assert abs(a - b) < 3 * math.hypot(ea, eb) + 1e-9, (nm, a, b, ea, eb)


# ---------------------------------------------------------------- graphs and autotuning
@pytest.mark.parametrize("path", [3, 4, 5, 7], ids=["tensor", "fft", "spectral", "cluster"])
def test_graph_replay_is_bit_identical(dipmc, path):
    """Repeated calls of the windowed / FFT paths replay a captured CUDA graph; three
    calls of 2 sweeps must equal one direct call of 6 sweeps bit for bit."""
    L, l, R = 32, 16, 8
    s0 = inputs.random_spins(L, R, seed=9)
    out = []
    for calls in ((2, 2, 2), (6,)):
        with dipmc.Lattice(L, l, R, 77) as lat:
            lat.precompute_W(16, True)
            lat.set_field_path(path)
            lat.init_spins(2, s0)
            for c in calls:
                lat.sweep(c, 1)
            out.append((lat.get_spins(), lat.observables(3), lat.sweep_counter()))
    assert np.array_equal(out[0][0], out[1][0])
    assert out[0][2] == out[1][2] == 6
    assert out[0][1]["samples"] == out[1][1]["samples"] == 6
    assert out[0][1]["abs_m"]["mean"] == out[1][1]["abs_m"]["mean"]


def test_autotune_keeps_state_and_picks_a_path(dipmc):
    L, l, R = 64, 32, 64
    s0 = inputs.random_spins(L, R, seed=4)
    with dipmc.Lattice(L, l, R, 5) as lat:
        lat.precompute_W(16, True)
        lat.init_spins(2, s0)
        lat.sweep(1, 0)
        before = lat.get_spins()
        t0 = lat.sweep_counter()
        path, win = lat.autotune(1)
        assert path in (dipmc.MC_PATH_DIRECT, dipmc.MC_PATH_TENSOR, dipmc.MC_PATH_FFT, dipmc.MC_PATH_SPECTRAL,
                        dipmc.MC_PATH_INCREMENTAL)
        assert np.array_equal(lat.get_spins(), before) and lat.sweep_counter() == t0
        lat.sweep(2, 1)
        assert lat.observables(0)["samples"] == 2


def test_incremental_path_energy_from_the_kept_field(dipmc):
    """The incremental path measures E from its kept field; after 13 sweeps (two
    launches, the field re-evaluated between them) it equals a full-field
    evaluation of the final state."""
    L, l, R = 32, 16, 4
    s0 = inputs.random_spins(L, R, seed=13)
    with dipmc.Lattice(L, l, R, 3) as lat:
        lat.precompute_W(16, True)
        lat.set_field_path(dipmc.MC_PATH_INCREMENTAL)
        lat.set_params(F32(1.0), F32(0.2), F32(0.8), F32(0.1), F32(0.7))
        lat.init_spins(2, s0)
        lat.sweep(13, 1)
        e_kept = np.array([lat.observables(r)["energy"] for r in range(R)]) * L * L
        e_full = lat.energy()
    np.testing.assert_allclose(e_kept, e_full, rtol=0, atol=2e-4 * L * L * 1e-2 + 1e-3)


@pytest.mark.parametrize("path", [1, 2, 3, 4, 5, 6, 7],
                         ids=["direct", "window_f32", "tensor", "fft", "spectral", "incremental", "cluster"])
def test_observables_on_identical_trajectories(dipmc, path):
    """Every path measures the observables in its own kernel: on a seeded run whose
    final state equals the oracle's (no straddled decision), the per-sweep means of
    all observables (|m|, m_z, |m_z|, M_par, E/N, m_st, walls, O_x, O_y, O_z, cone)
    equal the oracle's to rounding."""
    L, l, nsw, seed = 16, 8, 12, 61
    prm = (F32(1.0), F32(0.15), F32(0.8), F32(-0.1), F32(0.9))
    s0 = inputs.random_spins(L, 1, seed=8)
    with dipmc.Lattice(L, l, 1, seed) as lat:
        lat.precompute_W(16, True)
        lat.set_field_path(path)
        lat.set_params(*prm)
        lat.init_spins(2, s0)
        lat.sweep(nsw, 1)
        og = lat.observables(0)
        sg = lat.get_spins()[0].astype(np.float64)
    p = orc.params(L, l, *prm, proposal=0, cone=0.5, schedule=0, seed=seed, replica=0)
    o = orc.sweeps(p, oracle_W(L, 16), s0[0], 0, nsw, trace=False, observe=True)
    if np.abs(sg - o["s"]).max() > 1e-4:
        pytest.skip("a straddled decision separated the trajectories")
    assert og["samples"] == nsw
    for i, nm in enumerate(dipmc.OBS_NAMES):
        tol = 2e-5 * (1 + abs(o["obs"][:, i].mean()))
        assert og[nm]["mean"] == pytest.approx(o["obs"][:, i].mean(), abs=tol), nm
