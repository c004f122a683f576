"""Thin Python binding of libdipmc.so (C ABI in include/dipmc.h).

Argument marshalling only: every step of the sweep runs in the CUDA library.
Device buffers passed in or out are torch CUDA tensors (their data pointers);
the CUDA stream is torch's current stream unless given.  Importing this module
loads the library and raises if it has not been built -- there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdipmc.so")

MC_OK, MC_EINVAL, MC_ENOMEM, MC_ENOTREADY, MC_ETIMEOUT, MC_ECUDA, MC_ENOSYS = 0, -1, -2, -3, -4, -5, -6
MC_NOBS = 11
OBS_NAMES = ("abs_m", "m_z", "abs_m_z", "m_par", "e", "m_st", "wall", "o_x", "o_y", "o_z", "cone")
(MC_PATH_AUTO, MC_PATH_DIRECT, MC_PATH_WINDOW_F32, MC_PATH_TENSOR, MC_PATH_FFT, MC_PATH_SPECTRAL,
 MC_PATH_INCREMENTAL, MC_PATH_FFT_CLUSTER) = 0, 1, 2, 3, 4, 5, 6, 7
MC_TRACE_W = 10
PROPOSAL_CAP, PROPOSAL_SPHERE, PROPOSAL_FLIP = 0, 1, 2
INIT_RANDOM, INIT_UP, INIT_USER, INIT_ISING = 0, 1, 2, 3

# Every symbol include/dipmc.h declares.
ABI_SYMBOLS = (
    "mc_last_error", "mc_version", "mc_create_lattice", "mc_destroy", "mc_set_params",
    "mc_set_proposal", "mc_set_schedule", "mc_set_field_path", "mc_set_window", "mc_init_spins",
    "mc_precompute_W", "mc_sweep", "mc_sweep_trace", "mc_observables", "mc_observables_batch",
    "mc_reset_observables",
    "mc_get_spins", "mc_get_field", "mc_get_W", "mc_energy", "mc_get_sweep_counter",
    "mc_checkpoint", "mc_restore", "mc_energy_noalloc", "mc_set_timing", "mc_get_timing",
    "mc_choose_spacing", "mc_autotune", "mc_set_histogram", "mc_get_histogram",
    "mc_precompute_W_ewald", "mc_wtilde_ewald", "mc_set_tuning", "mc_get_tuning", "mc_sweep_group",
    "mc_get_window_cycles",
    "mc_footprint", "mc_server_create", "mc_server_submit", "mc_server_step", "mc_server_poll", "mc_server_request_info",
    "mc_server_collect", "mc_server_get_spins", "mc_server_release", "mc_server_get_stats", "mc_server_destroy",
)
MC_REQ_QUEUED, MC_REQ_RUNNING, MC_REQ_DONE, MC_REQ_FAILED, MC_REQ_RELEASED = range(5)
KERNEL_CLASSES = ("sweep_direct", "tc_field", "window_steps", "full_field", "spec_field", "spec_update", "tc_reduce")


class McError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"dipmc error {code}: {msg}")
        self.code = code


class mc_obs(C.Structure):
    _fields_ = [
        ("samples", C.c_int64),
        ("mean", C.c_double * MC_NOBS),
        ("var", C.c_double * MC_NOBS),
        ("err_naive", C.c_double * MC_NOBS),
        ("err", C.c_double * MC_NOBS),
        ("tau_int", C.c_double * MC_NOBS),
        ("eta", C.c_double),
        ("energy", C.c_double),
        ("accepted", C.c_int64),
        ("attempted", C.c_int64),
    ]

    def as_dict(self):
        d = {"samples": self.samples, "eta": self.eta, "energy": self.energy,
             "accepted": self.accepted, "attempted": self.attempted}
        for i, nm in enumerate(OBS_NAMES):
            d[nm] = {"mean": self.mean[i], "var": self.var[i], "err_naive": self.err_naive[i],
                     "err": self.err[i], "tau_int": self.tau_int[i]}
        return d


# the same record as a numpy structured type (all fields 8 bytes: no padding)
OBS_DTYPE = np.dtype([("samples", "<i8"), ("mean", "<f8", (MC_NOBS,)), ("var", "<f8", (MC_NOBS,)),
                      ("err_naive", "<f8", (MC_NOBS,)), ("err", "<f8", (MC_NOBS,)), ("tau_int", "<f8", (MC_NOBS,)),
                      ("eta", "<f8"), ("energy", "<f8"), ("accepted", "<i8"), ("attempted", "<i8")])
assert OBS_DTYPE.itemsize == C.sizeof(mc_obs)


class mc_request(C.Structure):
    _fields_ = [("L", C.c_int), ("l", C.c_int), ("replicas", C.c_int),
                ("J", C.c_double), ("C_D", C.c_double), ("K2", C.c_double), ("K4", C.c_double), ("T", C.c_double),
                ("sweeps", C.c_int64), ("measure_every", C.c_int), ("seed", C.c_uint64), ("init_mode", C.c_int),
                ("image_cutoff", C.c_int), ("proposal", C.c_int), ("cone", C.c_double)]


class mc_request_info(C.Structure):
    _fields_ = [("state", C.c_int), ("l", C.c_int), ("path", C.c_int), ("packed", C.c_int), ("sweeps_done", C.c_int64),
                ("t_submit", C.c_double), ("t_admit", C.c_double), ("t_done", C.c_double),
                ("bytes", C.c_size_t), ("error", C.c_char * 160)]


class mc_server_stats(C.Structure):
    _fields_ = [("queued", C.c_int), ("running", C.c_int), ("done", C.c_int), ("failed", C.c_int),
                ("packs", C.c_int), ("lone", C.c_int), ("completed", C.c_int64),
                ("bytes_in_use", C.c_size_t), ("budget", C.c_size_t), ("grouped_launches", C.c_int64)]


class mc_tuning(C.Structure):
    _fields_ = [("window", C.c_int), ("tc_kblocks", C.c_int), ("tc_ntile", C.c_int), ("steps_layout", C.c_int)]


class mc_timing(C.Structure):
    _fields_ = [("launches", C.c_int64 * 7), ("ms", C.c_double * 7)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is not built; run `python -m paper_1211_6234_b300.build`")
    lib = C.CDLL(LIB_PATH)
    vp, i32, f64, u64 = C.c_void_p, C.c_int, C.c_double, C.c_uint64
    sig = {
        "mc_last_error": ([], C.c_char_p),
        "mc_version": ([], i32),
        "mc_create_lattice": ([i32, i32, i32, u64, C.POINTER(vp)], i32),
        "mc_destroy": ([vp], i32),
        "mc_set_params": ([vp, i32, f64, f64, f64, f64, f64], i32),
        "mc_set_proposal": ([vp, i32, f64], i32),
        "mc_set_schedule": ([vp, i32], i32),
        "mc_set_field_path": ([vp, i32], i32),
        "mc_set_window": ([vp, i32], i32),
        "mc_init_spins": ([vp, i32, vp], i32),
        "mc_precompute_W": ([vp, i32, i32], i32),
        "mc_sweep": ([vp, i32, i32, vp], i32),
        "mc_sweep_trace": ([vp, i32, vp, C.c_size_t, vp], i32),
        "mc_observables": ([vp, i32, C.POINTER(mc_obs)], i32),
        "mc_set_histogram": ([vp, f64, f64, i32], i32),
        "mc_precompute_W_ewald": ([vp, f64], i32),
        "mc_wtilde_ewald": ([i32, f64, f64, C.POINTER(C.c_double)], i32),
        "mc_get_histogram": ([vp, i32, C.POINTER(C.c_int64)], i32),
        "mc_reset_observables": ([vp], i32),
        "mc_get_spins": ([vp, vp, i32, vp], i32),
        "mc_get_field": ([vp, vp, i32, vp], i32),
        "mc_get_W": ([vp, vp], i32),
        "mc_energy": ([vp, vp, vp], i32),
        "mc_get_sweep_counter": ([vp, C.POINTER(u64)], i32),
        "mc_checkpoint": ([vp, vp, C.POINTER(C.c_size_t)], i32),
        "mc_restore": ([vp, vp, C.c_size_t], i32),
        "mc_energy_noalloc": ([i32, i32, vp, vp, vp, vp, vp], i32),
        "mc_set_timing": ([vp, i32], i32),
        "mc_choose_spacing": ([i32, f64, f64, f64, C.POINTER(i32)], i32),
        "mc_autotune": ([vp, i32, vp, C.POINTER(i32), C.POINTER(i32)], i32),
        "mc_footprint": ([i32, i32, i32, C.POINTER(C.c_size_t)], i32),
        "mc_server_create": ([C.c_size_t, i32, i32, f64, C.POINTER(vp)], i32),
        "mc_server_submit": ([vp, C.POINTER(mc_request), C.POINTER(u64)], i32),
        "mc_server_step": ([vp], i32),
        "mc_server_poll": ([vp, u64, C.POINTER(i32), C.POINTER(C.c_int64)], i32),
        "mc_server_request_info": ([vp, u64, C.POINTER(mc_request_info)], i32),
        "mc_server_collect": ([vp, u64, i32, C.POINTER(mc_obs)], i32),
        "mc_server_get_spins": ([vp, u64, C.POINTER(C.c_float)], i32),
        "mc_server_release": ([vp, u64], i32),
        "mc_server_get_stats": ([vp, C.POINTER(mc_server_stats)], i32),
        "mc_server_destroy": ([vp], i32),
        "mc_get_timing": ([vp, C.POINTER(mc_timing)], i32),
        "mc_set_tuning": ([vp, C.POINTER(mc_tuning)], i32),
        "mc_sweep_group": ([C.POINTER(vp), i32, i32, i32, vp], i32),
        "mc_get_window_cycles": ([vp, C.POINTER(f64)], i32),
        "mc_get_tuning": ([vp, C.POINTER(mc_tuning)], i32),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    return lib


_lib = _load()


def lib():
    return _lib


def _ck(rc: int):
    if rc != MC_OK:
        raise McError(rc, _lib.mc_last_error().decode())
    return rc


def torch_float32():
    import torch
    return torch.float32


def _stream_ptr(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def energy_noalloc(L: int, R: int, W32, spins, couplings, energy, stream=None):
    """mc_energy_noalloc on torch CUDA tensors (W32 [4,L,L] f32, spins [R,3,L,L] f32,
    couplings [R,4] f32, energy [R] f64 output).  For callers that cannot allocate
    device memory; see include/dipmc.h."""
    _ck(_lib.mc_energy_noalloc(L, R, C.c_void_p(W32.data_ptr()), C.c_void_p(spins.data_ptr()),
                               C.c_void_p(couplings.data_ptr()), C.c_void_p(energy.data_ptr()),
                               _stream_ptr(stream)))


def sweep_group(lattices, nsweeps: int, measure_every: int = 0, stream=None):
    """mc_sweep_group: sweeps of handles of different L (same L / l, direct path)
    in one persistent launch; each replica's result equals its own mc_sweep."""
    arr = (C.c_void_p * len(lattices))(*[lat.h.value for lat in lattices])
    _ck(_lib.mc_sweep_group(arr, len(lattices), nsweeps, measure_every, _stream_ptr(stream)))


def choose_spacing(L: int, C_D: float, T_min: float, max_error: float) -> int:
    """Smallest update spacing l | L meeting the Sec. 3.2 error estimate (mc_choose_spacing)."""
    v = C.c_int(0)
    _ck(_lib.mc_choose_spacing(L, C_D, T_min, max_error, C.byref(v)))
    return v.value


def _np_ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


class Lattice:
    """Owner of one mc_lattice handle (R replicas of an L x L lattice, spacing l)."""

    def __init__(self, L: int, l: int, replicas: int = 1, seed: int = 1):
        h = C.c_void_p()
        _ck(_lib.mc_create_lattice(L, l, replicas, seed, C.byref(h)))
        self.h = h
        self.L, self.l, self.R, self.seed = L, l, replicas, seed

    # -- lifetime
    def close(self):
        if self.h:
            _lib.mc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def N(self):
        return self.L * self.L

    # -- set-up
    def set_params(self, J=1.0, C_D=0.1, K2=0.8, K4=0.0, T=0.6, replica=-1):
        _ck(_lib.mc_set_params(self.h, replica, J, C_D, K2, K4, T))

    def set_proposal(self, kind=0, cone=0.5):
        _ck(_lib.mc_set_proposal(self.h, kind, cone))

    def set_schedule(self, kind=0):
        _ck(_lib.mc_set_schedule(self.h, kind))

    def set_field_path(self, path=MC_PATH_AUTO):
        _ck(_lib.mc_set_field_path(self.h, path))

    def set_window(self, B=0):
        _ck(_lib.mc_set_window(self.h, B))

    def set_tuning(self, window=0, tc_kblocks=0, tc_ntile=0, steps_layout=0):
        """Launch shapes of the windowed tensor path (mc_set_tuning)."""
        t = mc_tuning(window, tc_kblocks, tc_ntile, steps_layout)
        _ck(_lib.mc_set_tuning(self.h, C.byref(t)))

    def tuning(self) -> dict:
        t = mc_tuning()
        _ck(_lib.mc_get_tuning(self.h, C.byref(t)))
        return {k: getattr(t, k) for k, _ in mc_tuning._fields_}

    def init_spins(self, mode=0, user=None):
        if mode == 2:
            a = np.ascontiguousarray(user, np.float32)
            assert a.size == self.R * 3 * self.N
            _ck(_lib.mc_init_spins(self.h, 2, _np_ptr(a)))
        else:
            _ck(_lib.mc_init_spins(self.h, mode, None))

    def precompute_W_ewald(self, eta=0.0):
        _ck(_lib.mc_precompute_W_ewald(self.h, eta))

    def precompute_W(self, image_cutoff=64, tail_correction=True):
        _ck(_lib.mc_precompute_W(self.h, image_cutoff, int(bool(tail_correction))))

    # -- run
    def sweep(self, nsweeps, measure_every=0, stream=None):
        _ck(_lib.mc_sweep(self.h, nsweeps, measure_every, _stream_ptr(stream)))

    def sweep_trace(self, nsweeps, stream=None):
        """Run nsweeps and return the per-attempt trace as a numpy array
        [R, nsweeps * L*L, MC_TRACE_W] (device buffer from torch)."""
        import torch
        nf = self.R * nsweeps * self.N * MC_TRACE_W
        buf = torch.empty(nf, dtype=torch.float32, device="cuda")
        _ck(_lib.mc_sweep_trace(self.h, nsweeps, C.c_void_p(buf.data_ptr()), nf, _stream_ptr(stream)))
        torch.cuda.synchronize()
        return buf.cpu().numpy().reshape(self.R, nsweeps * self.N, MC_TRACE_W)

    # -- read back
    def observables(self, replica=0) -> dict:
        o = mc_obs()
        _ck(_lib.mc_observables(self.h, replica, C.byref(o)))
        return o.as_dict()

    def observables_arrays(self, first=0, count=None) -> np.ndarray:
        """Observables of replicas first .. first+count-1 with one read-back, as a numpy
        record array of OBS_DTYPE (fields samples, mean/var/err_naive/err/tau_int
        [count][MC_NOBS] in OBS_NAMES order, eta, energy, accepted, attempted)."""
        if count is None:
            count = self.R - first
        out = np.zeros(max(count, 1), OBS_DTYPE)
        _ck(_lib.mc_observables_batch(self.h, first, count, out.ctypes.data_as(C.POINTER(mc_obs))))
        return out[:count]

    def observables_batch(self, first=0, count=None) -> list:
        """observables() of replicas first .. first+count-1 with one read-back."""
        a = self.observables_arrays(first, count)
        cols = {f: a[f].tolist() for f in OBS_DTYPE.names}
        res = []
        for i in range(len(a)):
            d = {"samples": cols["samples"][i], "eta": cols["eta"][i], "energy": cols["energy"][i],
                 "accepted": cols["accepted"][i], "attempted": cols["attempted"][i]}
            for k, nm in enumerate(OBS_NAMES):
                d[nm] = {"mean": cols["mean"][i][k], "var": cols["var"][i][k], "err_naive": cols["err_naive"][i][k],
                         "err": cols["err"][i][k], "tau_int": cols["tau_int"][i][k]}
            res.append(d)
        return res

    def reset_observables(self):
        _ck(_lib.mc_reset_observables(self.h))

    def set_histogram(self, lo, hi, nbins):
        """Histogram of E/N over the measured sweeps: nbins bins on [lo, hi)."""
        _ck(_lib.mc_set_histogram(self.h, lo, hi, nbins))
        self._hist_bins = nbins

    def histogram(self, replica=0) -> np.ndarray:
        a = np.zeros(self._hist_bins, np.int64)
        _ck(_lib.mc_get_histogram(self.h, replica, a.ctypes.data_as(C.POINTER(C.c_int64))))
        return a

    def get_spins(self, out=None, stream=None) -> np.ndarray:
        """Spins [R][3][L][L]; into `out` if given: a torch tensor on the device or in
        (pinned) host memory, or a float32 numpy array of that size."""
        if isinstance(out, np.ndarray):
            assert out.dtype == np.float32 and out.flags.c_contiguous and out.size == self.R * 3 * self.N
            _ck(_lib.mc_get_spins(self.h, _np_ptr(out), 0, _stream_ptr(stream)))
            return out
        if out is not None:  # torch tensor
            assert out.dtype == torch_float32() and out.is_contiguous() and out.numel() == self.R * 3 * self.N
            _ck(_lib.mc_get_spins(self.h, C.c_void_p(out.data_ptr()), 1 if out.is_cuda else 0, _stream_ptr(stream)))
            return out
        a = np.empty((self.R, 3, self.L, self.L), np.float32)
        _ck(_lib.mc_get_spins(self.h, _np_ptr(a), 0, _stream_ptr(stream)))
        return a

    def get_field(self, stream=None) -> np.ndarray:
        a = np.empty((self.R, 3, self.L, self.L), np.float32)
        _ck(_lib.mc_get_field(self.h, _np_ptr(a), 0, _stream_ptr(stream)))
        return a

    def get_W(self) -> np.ndarray:
        a = np.empty((4, self.L, self.L), np.float64)
        _ck(_lib.mc_get_W(self.h, _np_ptr(a)))
        return a

    def energy(self, stream=None) -> np.ndarray:
        a = np.empty(self.R, np.float64)
        _ck(_lib.mc_energy(self.h, _np_ptr(a), _stream_ptr(stream)))
        return a

    def set_timing(self, enable=True):
        _ck(_lib.mc_set_timing(self.h, int(bool(enable))))

    def timing(self) -> dict:
        """Per-kernel-class launches and device milliseconds since set_timing."""
        t = mc_timing()
        _ck(_lib.mc_get_timing(self.h, C.byref(t)))
        return {nm: {"launches": t.launches[i], "ms": t.ms[i]} for i, nm in enumerate(KERNEL_CLASSES)}

    def window_cycles(self) -> dict:
        """mc_get_window_cycles: SM cycles per 16-site decision block, set-up and tail
        of the sub-step kernel, averaged over its CTAs and launches while timing."""
        out = (C.c_double * 4)()
        _ck(_lib.mc_get_window_cycles(self.h, out))
        return {"per_block": out[0], "setup": out[1], "tail": out[2], "blocks_per_launch": out[3]}
    def autotune(self, nsweeps_trial=2, stream=None):
        """Time the supported paths on a copy of the state; keep the fastest.
        Returns (path, window)."""
        pth, win = C.c_int(0), C.c_int(0)
        _ck(_lib.mc_autotune(self.h, nsweeps_trial, _stream_ptr(stream), C.byref(pth), C.byref(win)))
        return pth.value, win.value

    def sweep_counter(self) -> int:
        v = C.c_uint64()
        _ck(_lib.mc_get_sweep_counter(self.h, C.byref(v)))
        return v.value

    def checkpoint(self) -> bytes:
        n = C.c_size_t(0)
        _ck(_lib.mc_checkpoint(self.h, None, C.byref(n)))
        buf = C.create_string_buffer(n.value)
        _ck(_lib.mc_checkpoint(self.h, buf, C.byref(n)))
        return buf.raw[: n.value]

    def restore(self, data: bytes):
        buf = C.create_string_buffer(data, len(data))
        _ck(_lib.mc_restore(self.h, buf, len(data)))


def wtilde_ewald(L: int, z: float = 0.0, eta: float = 0.0) -> np.ndarray:
    """W~ by the Ewald/Harris split on the GPU, [6][L][L] FP64 (xx, xy, yy, zz, xz, yz)."""
    a = np.zeros((6, L, L), np.float64)
    _ck(_lib.mc_wtilde_ewald(L, z, eta, a.ctypes.data_as(C.POINTER(C.c_double))))
    return a


def footprint(L: int, l: int, replicas: int = 1) -> int:
    """Device bytes of a handle (the server's admission estimate)."""
    b = C.c_size_t()
    _ck(_lib.mc_footprint(L, l, replicas, C.byref(b)))
    return b.value


class Server:
    """Continuous-batching service (mc_server_*).  Requests of the same (L, l)
    share packed launches; each request's result equals its lone run."""

    def __init__(self, hbm_budget_bytes=8 << 30, max_active=4096, quantum_sweeps=50, max_error=1e-3):
        h = C.c_void_p()
        _ck(_lib.mc_server_create(int(hbm_budget_bytes), max_active, quantum_sweeps, max_error, C.byref(h)))
        self.h = h
        self._shape = {}

    def close(self):
        if self.h:
            _lib.mc_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def submit(self, L, T, sweeps, seed, l=0, replicas=1, J=1.0, C_D=0.1, K2=0.8, K4=0.0,
               measure_every=1, init_mode=0, image_cutoff=64, proposal=0, cone=0.5) -> int:
        r = mc_request(L, l, replicas, J, C_D, K2, K4, T, int(sweeps), measure_every, int(seed), init_mode,
                       image_cutoff, proposal, cone)
        rid = C.c_uint64()
        _ck(_lib.mc_server_submit(self.h, C.byref(r), C.byref(rid)))
        self._shape[rid.value] = (max(1, replicas), L)
        return rid.value

    def step(self):
        _ck(_lib.mc_server_step(self.h))

    def poll(self, rid):
        st, done = C.c_int(), C.c_int64()
        _ck(_lib.mc_server_poll(self.h, rid, C.byref(st), C.byref(done)))
        return st.value, done.value

    def info(self, rid) -> dict:
        i = mc_request_info()
        _ck(_lib.mc_server_request_info(self.h, rid, C.byref(i)))
        return {"state": i.state, "l": i.l, "path": i.path, "packed": bool(i.packed), "sweeps_done": i.sweeps_done,
                "t_submit": i.t_submit, "t_admit": i.t_admit, "t_done": i.t_done, "bytes": i.bytes,
                "error": i.error.decode()}

    def collect(self, rid, replica=0) -> dict:
        o = mc_obs()
        _ck(_lib.mc_server_collect(self.h, rid, replica, C.byref(o)))
        return o.as_dict()

    def spins(self, rid) -> np.ndarray:
        R, L = self._shape[rid]
        a = np.empty((R, 3, L, L), np.float32)
        _ck(_lib.mc_server_get_spins(self.h, rid, a.ctypes.data_as(C.POINTER(C.c_float))))
        return a

    def release(self, rid):
        _ck(_lib.mc_server_release(self.h, rid))

    def stats(self) -> dict:
        s = mc_server_stats()
        _ck(_lib.mc_server_get_stats(self.h, C.byref(s)))
        return {k: getattr(s, k) for k, _ in mc_server_stats._fields_}

    def run_until_done(self, ids, timeout_s=600.0, on_done=None):
        """Step until every id in `ids` is DONE or FAILED; on_done(id) when each ends."""
        import time
        left = set(ids)
        t_end = time.monotonic() + timeout_s
        while left:
            self.step()
            for rid in list(left):
                st, _ = self.poll(rid)
                if st in (MC_REQ_DONE, MC_REQ_FAILED):
                    left.discard(rid)
                    if on_done:
                        on_done(rid)
            if time.monotonic() > t_end:
                raise TimeoutError(f"{len(left)} requests unfinished")
