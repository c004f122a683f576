"""Serving layer (mc_server_*): continuous batching of simulation requests.

The property that matters is that batching changes nothing: a request's final
spins and observables from the server, packed into shared launches with other
requests and advanced in quanta, equal bit for bit those of the same request run
alone on its own handle.  Around it: admission by HBM budget in arrival order,
release of running and finished requests, and argument validation.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def lone_run(dipmc, L, l, T, sweeps, seed, replicas=1, K2=0.8, K4=0.0, C_D=0.1, J=1.0, measure_every=1,
             init_mode=0, path=None, proposal=0):
    with dipmc.Lattice(L, l, replicas, seed) as lat:
        lat.set_params(J=J, C_D=C_D, K2=K2, K4=K4, T=T)
        lat.set_proposal(proposal, 0.5)
        lat.precompute_W(64, True)
        if path is not None:
            lat.set_field_path(path)
        lat.init_spins(init_mode)
        lat.sweep(sweeps, measure_every)
        obs = [lat.observables(r) for r in range(replicas)]
        return lat.get_spins(), obs


def same_obs(a, b):
    """Observables equal bit for bit (NaN where both have no samples)."""
    assert a.keys() == b.keys()
    for k, v in a.items():
        if isinstance(v, dict):
            for kk in v:
                np.testing.assert_array_equal(v[kk], b[k][kk], err_msg=f"{k}.{kk}")
        else:
            np.testing.assert_array_equal(v, b[k], err_msg=k)


# ---------------------------------------------------------------- host-only checks
def test_server_argument_validation_without_device():
    from paper_1211_6234_b300 import dipmc
    lib = dipmc.lib()
    h = C.c_void_p()
    assert lib.mc_server_create(0, 4, 10, 1e-3, C.byref(h)) == dipmc.MC_EINVAL
    assert lib.mc_server_create(1 << 20, 0, 10, 1e-3, C.byref(h)) == dipmc.MC_EINVAL
    assert lib.mc_server_create(1 << 20, 4, 0, 1e-3, C.byref(h)) == dipmc.MC_EINVAL
    assert lib.mc_server_create(1 << 20, 4, 10, 0.0, C.byref(h)) == dipmc.MC_EINVAL
    assert lib.mc_server_create(1 << 20, 4, 10, 1e-3, None) == dipmc.MC_EINVAL
    rid = C.c_uint64()
    req = dipmc.mc_request()
    assert lib.mc_server_submit(None, C.byref(req), C.byref(rid)) == dipmc.MC_EINVAL
    assert lib.mc_server_step(None) == dipmc.MC_EINVAL
    assert lib.mc_server_release(None, 1) == dipmc.MC_EINVAL
    assert lib.mc_server_destroy(None) == dipmc.MC_OK
    b = C.c_size_t()
    assert lib.mc_footprint(30, 7, 1, C.byref(b)) == dipmc.MC_EINVAL
    assert lib.mc_footprint(128, 16, 1, C.byref(b)) == dipmc.MC_OK
    one = b.value
    assert lib.mc_footprint(128, 16, 2, C.byref(b)) == dipmc.MC_OK
    assert one < b.value < 2 * one


# ---------------------------------------------------------------- GPU
gpu = pytest.mark.gpu


@pytest.fixture(scope="module")
def dipmc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1211_6234_b300 import dipmc as d
    return d


@gpu
def test_packed_requests_equal_their_lone_runs(dipmc):
    """Requests of several (L, l) groups and lengths share packed launches (direct
    packs at L = 32, 64; a spectral pack at L = 128), advanced in quanta that do not
    divide their sweep counts; every one matches its lone run bit for bit,
    multi-replica requests included."""
    specs = [
        dict(L=32, l=8, T=0.7, sweeps=61, seed=11, K4=0.1),
        dict(L=32, l=8, T=0.3, sweeps=17, seed=12, K2=0.6),
        dict(L=32, l=8, T=1.1, sweeps=40, seed=13, replicas=3),
        dict(L=64, l=32, T=0.5, sweeps=23, seed=14, K4=-0.2),
        dict(L=64, l=32, T=0.9, sweeps=9, seed=15, init_mode=1),
        dict(L=32, l=16, T=0.6, sweeps=33, seed=16),
        dict(L=128, l=16, T=0.6, sweeps=5, seed=21),
        dict(L=128, l=16, T=0.4, sweeps=3, seed=24, K4=0.2, replicas=2),
        dict(L=32, l=8, T=0.5, sweeps=19, seed=17, C_D=0.588, K2=0.0, proposal=2, init_mode=3),
    ]
    with dipmc.Server(hbm_budget_bytes=4 << 30, quantum_sweeps=2) as srv:
        ids = [srv.submit(**s) for s in specs]
        srv.run_until_done(ids, timeout_s=300)
        for rid, s in zip(ids, specs):
            info = srv.info(rid)
            assert info["state"] == dipmc.MC_REQ_DONE, info
            assert info["packed"] and info["sweeps_done"] == s["sweeps"]
            assert info["path"] == (dipmc.MC_PATH_SPECTRAL if s["L"] == 128 else dipmc.MC_PATH_DIRECT)
            spins_lone, obs_lone = lone_run(dipmc, path=info["path"], **s)   # alone, on the pack's path
            np.testing.assert_array_equal(srv.spins(rid), spins_lone)
            for r in range(s.get("replicas", 1)):
                same_obs(srv.collect(rid, r), obs_lone[r])
        st = srv.stats()
        assert st["done"] == len(specs) and st["running"] == 0 and st["queued"] == 0
        assert st["packs"] == 5 and st["lone"] == 0


@gpu
def test_mixed_lattice_sizes_share_one_launch(dipmc):
    """Requests of L = 32, 48, 64 and 96 at l = L / 2 run in the same grouped
    launches of the direct kernel (uneven L in one persistent launch), and each
    result still equals its lone run bit for bit."""
    specs = [dict(L=32, l=16, T=0.7, sweeps=21, seed=31), dict(L=48, l=24, T=0.4, sweeps=13, seed=32, K4=0.1),
             dict(L=64, l=32, T=0.9, sweeps=17, seed=33, replicas=2), dict(L=96, l=48, T=0.5, sweeps=9, seed=34),
             dict(L=48, l=24, T=1.1, sweeps=25, seed=35, init_mode=1)]
    with dipmc.Server(hbm_budget_bytes=4 << 30, quantum_sweeps=4) as srv:
        ids = [srv.submit(**s) for s in specs]
        srv.run_until_done(ids, timeout_s=300)
        st = srv.stats()
        assert st["grouped_launches"] > 0
        for rid, s in zip(ids, specs):
            info = srv.info(rid)
            assert info["state"] == dipmc.MC_REQ_DONE and info["packed"], info
            assert info["path"] == dipmc.MC_PATH_DIRECT
            spins_lone, obs_lone = lone_run(dipmc, path=dipmc.MC_PATH_DIRECT, **s)
            np.testing.assert_array_equal(srv.spins(rid), spins_lone)
            for r in range(s.get("replicas", 1)):
                same_obs(srv.collect(rid, r), obs_lone[r])


@gpu
def test_lone_handle_requests_equal_their_lone_runs(dipmc):
    """Requests with more replicas than a pack holds run on pooled lone handles
    (tensor path at L = 64, spectral path at L = 256) beside a pack and match their
    lone runs; a later request of the same shape reuses a pooled handle.  A
    shape no path serves (L = 96, l = 2: L/l = 48) fails alone, with its reason,
    and stops nothing."""
    specs = [
        dict(L=64, l=32, T=0.8, sweeps=4, seed=22, replicas=300),
        dict(L=256, l=16, T=0.7, sweeps=2, seed=25, replicas=40),
        dict(L=32, l=8, T=0.7, sweeps=12, seed=23),
        dict(L=64, l=32, T=0.5, sweeps=3, seed=26, K4=-0.1, replicas=300),
    ]
    with dipmc.Server(hbm_budget_bytes=8 << 30, quantum_sweeps=2) as srv:
        bad = srv.submit(L=96, l=2, T=0.8, sweeps=2, seed=1)
        ids = [srv.submit(**s) for s in specs]
        srv.run_until_done(ids + [bad], timeout_s=300)
        info = srv.info(bad)
        assert info["state"] == dipmc.MC_REQ_FAILED and info["error"]
        for rid, s in zip(ids, specs):
            info = srv.info(rid)
            assert info["state"] == dipmc.MC_REQ_DONE, info
            assert info["packed"] == (s["L"] == 32)
            spins_lone, obs_lone = lone_run(dipmc, path=info["path"], **s)
            np.testing.assert_array_equal(srv.spins(rid), spins_lone)
            for r in (0, s.get("replicas", 1) - 1):
                same_obs(srv.collect(rid, r), obs_lone[r])
        st = srv.stats()
        assert st["lone"] == 4 and st["failed"] == 1     # L=96 (failed), 2 x L=64, L=256
        again = dict(L=64, l=32, T=0.6, sweeps=2, seed=27, replicas=300)
        rid = srv.submit(**again)
        srv.run_until_done([rid], timeout_s=120)
        assert srv.stats()["lone"] == 4
        np.testing.assert_array_equal(srv.spins(rid), lone_run(dipmc, **again)[0])


@gpu
def test_admission_waits_for_budget_in_arrival_order(dipmc):
    """With room for one L=128 slot only, the spectral pack shrinks to one slot and
    three such requests run one after the other in arrival order; the bytes in
    use never exceed the budget; a request that can never fit is refused."""
    f1, f2 = dipmc.footprint(128, 16, 1), dipmc.footprint(128, 16, 2)
    budget = f1 + (f2 - f1) // 2
    with dipmc.Server(hbm_budget_bytes=budget, quantum_sweeps=1) as srv:
        with pytest.raises(dipmc.McError) as e:
            srv.submit(L=256, l=16, T=0.6, sweeps=1, seed=1)
        assert e.value.code == dipmc.MC_ENOMEM
        ids = [srv.submit(L=128, l=16, T=0.6 + 0.1 * i, sweeps=2, seed=30 + i) for i in range(3)]
        order, peak, states = [], 0, set()
        for _ in range(100000):
            srv.step()
            st = srv.stats()
            peak = max(peak, st["bytes_in_use"])
            assert st["running"] <= 1
            states.add((st["running"], st["queued"]))
            for rid in ids:
                if rid not in order and srv.poll(rid)[0] == dipmc.MC_REQ_DONE:
                    order.append(rid)
            if len(order) == 3:
                break
        assert order == ids
        assert peak <= budget
        assert (1, 2) in states
        for i, rid in enumerate(ids):
            spins_lone, _ = lone_run(dipmc, L=128, l=16, T=0.6 + 0.1 * i, sweeps=2, seed=30 + i)
            np.testing.assert_array_equal(srv.spins(rid), spins_lone)


@gpu
def test_release_frees_slots_for_the_next_request(dipmc):
    """Releasing a running packed request frees its slot at once and drops its record
    (the id still polls as released); a request that takes the slot (filled behind the
    launch still in flight) matches its lone run, and finished requests drop their
    results on release."""
    with dipmc.Server(hbm_budget_bytes=4 << 30, quantum_sweeps=5) as srv:
        long_id = srv.submit(L=32, l=8, T=0.7, sweeps=10**6, seed=41)
        srv.step()
        srv.step()
        assert srv.poll(long_id)[0] == dipmc.MC_REQ_RUNNING
        srv.release(long_id)
        assert srv.poll(long_id) == (dipmc.MC_REQ_RELEASED, 0)   # the record is gone, the id is known
        assert srv.info(long_id)["state"] == dipmc.MC_REQ_RELEASED
        srv.release(long_id)                                      # a second release is a no-op
        assert srv.stats()["running"] == 0
        with pytest.raises(dipmc.McError) as e:
            srv.poll(long_id + 10**6)                             # never handed out
        assert e.value.code == dipmc.MC_EINVAL
        rid = srv.submit(L=32, l=8, T=0.5, sweeps=12, seed=42)
        srv.run_until_done([rid], timeout_s=120)
        spins_lone, obs_lone = lone_run(dipmc, L=32, l=8, T=0.5, sweeps=12, seed=42, path=srv.info(rid)["path"])
        np.testing.assert_array_equal(srv.spins(rid), spins_lone)
        same_obs(srv.collect(rid), obs_lone[0])
        srv.release(rid)
        with pytest.raises(dipmc.McError) as e:
            srv.collect(rid)
        assert e.value.code == dipmc.MC_ENOTREADY
        with pytest.raises(dipmc.McError) as e:
            srv.submit(L=30, l=7, T=0.5, sweeps=1, seed=1)
        assert e.value.code == dipmc.MC_EINVAL


@gpu
def test_spacing_chosen_at_the_error_bound(dipmc):
    """l = 0 in a request takes the spacing mc_choose_spacing gives at the
    server's error bound, moved up to the first divisor the direct pack serves
    where there is one."""
    with dipmc.Server(hbm_budget_bytes=1 << 30, quantum_sweeps=4, max_error=1e-3) as srv:
        rid = srv.submit(L=64, l=0, T=0.9, sweeps=3, seed=5)
        srv.run_until_done([rid], timeout_s=120)
        assert srv.info(rid)["l"] == dipmc.choose_spacing(64, 0.1, 0.9, 1e-3)
        # L = 96 at T = 0.9: the bound allows l = 16 (L/l = 6: no direct kernel
        # instance); the next divisor the direct pack serves, l = 24 (L/l = 4), only
        # lowers the error, so the request goes to a direct pack at that spacing
        assert dipmc.choose_spacing(96, 0.1, 0.9, 1e-3) == 16
        rid = srv.submit(L=96, l=0, T=0.9, sweeps=2, seed=6)
        srv.run_until_done([rid], timeout_s=120)
        info = srv.info(rid)
        assert info["l"] == 24 and info["packed"] and info["path"] == dipmc.MC_PATH_DIRECT
        spins_lone, obs_lone = lone_run(dipmc, L=96, l=24, T=0.9, sweeps=2, seed=6, path=dipmc.MC_PATH_DIRECT)
        np.testing.assert_array_equal(srv.spins(rid), spins_lone)
        same_obs(srv.collect(rid), obs_lone[0])
        # L = 256: no direct kernel; the bound's own spacing on a spectral pack
        rid = srv.submit(L=256, l=0, T=0.9, sweeps=1, seed=7)
        srv.run_until_done([rid], timeout_s=120)
        info = srv.info(rid)
        assert info["l"] == dipmc.choose_spacing(256, 0.1, 0.9, 1e-3)
        assert info["packed"] and info["path"] == dipmc.MC_PATH_SPECTRAL
