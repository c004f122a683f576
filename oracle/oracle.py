"""Python access to the CPU FP64 oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  This module never
imports the CUDA package and the CUDA package never imports it.

Every function is a literal wrapper around the C definitions; see the header
of oracle.c for the readings of the paper (arXiv:1211.6234) they follow.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")


# per-sweep observables: |m|, m_z, |m_z|, M_par, E/N, m_st (Appendix B staggered magnetisation),
# wall density, orientational order O_x, O_y, O_z and the cone angle of one state (Sec. 4.1)
NOBS = 11


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so with gcc (IEEE FP64, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-fno-fast-math", "-ffp-contract=off", "-fopenmp", "-fPIC",
             "-shared", "-std=c11", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Params(C.Structure):
    """Mirror of orc_params in oracle.c."""
    _fields_ = [
        ("L", C.c_int), ("l", C.c_int),
        ("J", C.c_double), ("CD", C.c_double), ("K2", C.c_double), ("K4", C.c_double),
        ("T", C.c_double),
        ("proposal", C.c_int), ("cone", C.c_double),
        ("schedule", C.c_int),
        ("seed", C.c_uint64), ("replica", C.c_uint32),
    ]


def params(L, l, J=1.0, CD=0.1, K2=0.8, K4=0.0, T=0.6, proposal=0, cone=0.5, schedule=0,
           seed=1, replica=0) -> Params:
    return Params(L, l, J, CD, K2, K4, T, proposal, cone, schedule, seed, replica)


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        d = C.POINTER(C.c_double)
        i32 = C.POINTER(C.c_int32)
        u32 = C.POINTER(C.c_uint32)
        _lib.orc_philox4x32_10.argtypes = [u32, u32, u32]
        _lib.orc_wtilde.argtypes = [C.c_int, C.c_int, C.c_int, d]
        _lib.orc_wtilde.restype = C.c_int
        _lib.orc_wtilde_ewald.argtypes = [C.c_int, C.c_double, C.c_double, d]
        _lib.orc_wtilde_ewald.restype = C.c_int
        _lib.orc_field.argtypes = [C.c_int, d, d, d]
        _lib.orc_energy.argtypes = [C.c_int, d, d, C.c_double, C.c_double, C.c_double,
                                    C.c_double, d]
        _lib.orc_dipole_energy_pairs.argtypes = [C.c_int, C.c_int, C.c_int, d, C.c_double]
        _lib.orc_dipole_energy_pairs.restype = C.c_double
        _lib.orc_offset.argtypes = [C.c_uint64, C.c_int, C.c_int, C.c_uint32, C.c_uint32]
        _lib.orc_offset.restype = C.c_uint32
        _lib.orc_sweeps.argtypes = [C.POINTER(Params), d, d, C.c_uint32, C.c_int, i32, d, d, d,
                                    i32, d, d, d]
        _lib.orc_sweeps.restype = C.c_int
        _lib.orc_sweeps_batch.argtypes = [C.c_int, C.POINTER(Params), d, d, C.c_uint32, C.c_int,
                                          d, d]
        _lib.orc_sweeps_batch.restype = C.c_int
        _lib.orc_substep.argtypes = [C.POINTER(Params), d, d, C.c_uint32, C.c_uint32, i32, d, d, d, i32, d]
        _lib.orc_substep.restype = None
        _lib.orc_replay_batch.argtypes = [C.c_int, C.POINTER(Params), d, d, C.c_uint32, C.c_int, i32, d,
                                          i32, d, d, d, i32, d]
        _lib.orc_replay_batch.restype = C.c_int
        _lib.orc_sweeps_exact.argtypes = [C.POINTER(Params), d, d, C.c_uint32, C.c_int, d, i32]
        _lib.orc_sweeps_exact.restype = C.c_int
        _lib.orc_init_random.argtypes = [C.c_int, C.c_uint64, C.c_uint32, d]
        _lib.orc_init_ising.argtypes = [C.c_int, C.c_uint64, C.c_uint32, d]
        _lib.orc_eta.argtypes = [C.c_int, d, C.c_double]
        _lib.orc_eta.restype = C.c_double
        _lib.orc_eps12.argtypes = [d, d, d, C.c_double]
        _lib.orc_eps12.restype = C.c_double
        _lib.orc_eps_total.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_int, C.c_int]
        _lib.orc_eps_total.restype = C.c_double
        _lib.orc_propose.argtypes = [C.c_int, C.c_double, d, C.c_double, C.c_double, d]
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a: np.ndarray):
    assert a.dtype == np.int32 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def philox(ctr, key):
    """Philox4x32-10 of a 4-word counter under a 2-word key."""
    c = (C.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (C.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (C.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return [int(x) for x in o]


def wtilde(L: int, A: int = 64, tail: bool = True) -> np.ndarray:
    """Replica-summed dipole tensor, shape [4, L, L] (xx, xy, yy, zz; [rho_y, rho_x])."""
    W = np.zeros((4, L, L), np.float64)
    if lib().orc_wtilde(L, A, int(bool(tail)), _dp(W)) != 0:
        raise ValueError("bad arguments")
    return W


def wtilde_ewald(L: int, z: float = 0.0, eta: float = 0.0) -> np.ndarray:
    """W~ by the Ewald/Harris split (Sec. 2.1), [6][L][L]: xx, xy, yy, zz, xz, yz
    for two layers a height z apart; eta = 0 takes L / 4."""
    W = np.zeros((6, L, L), np.float64)
    if lib().orc_wtilde_ewald(L, float(z), float(eta) if eta > 0 else L / 4.0, _dp(W)) != 0:
        raise ValueError("bad arguments")
    return W


def field(W: np.ndarray, s: np.ndarray) -> np.ndarray:
    L = W.shape[-1]
    W = np.ascontiguousarray(W, np.float64)
    s = np.ascontiguousarray(s, np.float64)
    h = np.zeros((3, L, L), np.float64)
    lib().orc_field(L, _dp(W), _dp(s), _dp(h))
    return h


def energy(W, s, J, CD, K2, K4):
    """(exchange, anisotropy, dipole, total) energy of state s."""
    L = W.shape[-1]
    W = np.ascontiguousarray(W, np.float64)
    s = np.ascontiguousarray(s, np.float64)
    out = np.zeros(4, np.float64)
    lib().orc_energy(L, _dp(W), _dp(s), J, CD, K2, K4, _dp(out))
    return tuple(float(x) for x in out)


def dipole_energy_pairs(L, A, tail, s, CD):
    s = np.ascontiguousarray(s, np.float64)
    return float(lib().orc_dipole_energy_pairs(L, A, int(bool(tail)), _dp(s), CD))


def offset(seed, l, kind, t, k) -> int:
    return int(lib().orc_offset(seed, l, kind, t, k))


def sweeps(p: Params, W, s, t0: int, nsweeps: int, trace: bool = True, observe: bool = False):
    """Approximated parallel sweeps on a copy of s.  Returns a dict with the final
    state and, if requested, the per-attempt trace and per-sweep observables."""
    L, l = p.L, p.l
    n = (L // l) ** 2
    W = np.ascontiguousarray(W, np.float64)
    s = np.array(s, np.float64, copy=True, order="C")
    ntr = nsweeps * l * l * n if trace else 0
    out = {}
    null = None
    if trace:
        out["q"] = np.zeros(ntr, np.int32)
        out["h"] = np.zeros((ntr, 3), np.float64)
        out["dE"] = np.zeros(ntr, np.float64)
        out["u"] = np.zeros(ntr, np.float64)
        out["acc"] = np.zeros(ntr, np.int32)
        out["S"] = np.zeros((ntr, 3), np.float64)
    if observe:
        out["obs"] = np.zeros((nsweeps, NOBS), np.float64)
        out["theta2"] = np.zeros(L * L, np.float64)
    rc = lib().orc_sweeps(
        C.byref(p), _dp(W), _dp(s), t0, nsweeps,
        _ip(out["q"]) if trace else null, _dp(out["h"]) if trace else null,
        _dp(out["dE"]) if trace else null, _dp(out["u"]) if trace else null,
        _ip(out["acc"]) if trace else null, _dp(out["S"]) if trace else null,
        _dp(out["obs"]) if observe else null, _dp(out["theta2"]) if observe else null)
    if rc != 0:
        raise ValueError("bad arguments")
    out["s"] = s
    return out


def substep(p: Params, W, s, t: int, k: int):
    """Decisions of sub-step k of sweep t from state s (unchanged): per update
    site d, q, h[3], dE, u, accept, S[3]."""
    n = (p.L // p.l) ** 2
    W = np.ascontiguousarray(W, np.float64)
    s = np.ascontiguousarray(s, np.float64)
    out = {"q": np.zeros(n, np.int32), "h": np.zeros((n, 3)), "dE": np.zeros(n), "u": np.zeros(n),
           "acc": np.zeros(n, np.int32), "S": np.zeros((n, 3))}
    lib().orc_substep(C.byref(p), _dp(W), _dp(s), t, k, _ip(out["q"]), _dp(out["h"]), _dp(out["dE"]),
                      _dp(out["u"]), _ip(out["acc"]), _dp(out["S"]))
    return out


def replay_batch(ps, W, s, t0: int, nsweeps: int, ext_acc, ext_S):
    """Decisions of every sub-step, each from the pre-step state of another
    trajectory (orc_replay): s is [R, 3, L, L] (copied); ext_acc [R, n_att] and
    ext_S [R, n_att, 3] are that trajectory's decisions and proposals in trace
    order (n_att = nsweeps * L^2).  Returns the oracle's q, h, dE, u, acc, S per
    attempt, [R, n_att, ...], and the final state (the other trajectory's)."""
    R = len(ps)
    arr = (Params * R)(*ps)
    L = ps[0].L
    m = nsweeps * L * L
    W = np.ascontiguousarray(W, np.float64)
    s = np.array(s, np.float64, copy=True, order="C")
    ea = np.ascontiguousarray(ext_acc, np.int32).reshape(R, m)
    eS = np.ascontiguousarray(ext_S, np.float64).reshape(R, m, 3)
    out = {"q": np.zeros((R, m), np.int32), "h": np.zeros((R, m, 3)), "dE": np.zeros((R, m)),
           "u": np.zeros((R, m)), "acc": np.zeros((R, m), np.int32), "S": np.zeros((R, m, 3))}
    rc = lib().orc_replay_batch(R, arr, _dp(W), _dp(s), t0, nsweeps, _ip(ea), _dp(eS), _ip(out["q"]),
                                _dp(out["h"]), _dp(out["dE"]), _dp(out["u"]), _ip(out["acc"]), _dp(out["S"]))
    if rc != 0:
        raise ValueError("bad arguments")
    out["s"] = s
    return out


def sweeps_batch(ps, W, s, t0, nsweeps, observe=True):
    """Independent replicas over all host threads; s is [R, 3, L, L] (copied)."""
    R = len(ps)
    arr = (Params * R)(*ps)
    W = np.ascontiguousarray(W, np.float64)
    s = np.array(s, np.float64, copy=True, order="C")
    L = ps[0].L
    obs = np.zeros((R, nsweeps, NOBS), np.float64) if observe else None
    th = np.zeros((R, L * L), np.float64) if observe else None
    rc = lib().orc_sweeps_batch(R, arr, _dp(W), _dp(s), t0, nsweeps,
                                _dp(obs) if observe else None, _dp(th) if observe else None)
    if rc != 0:
        raise ValueError("bad arguments")
    return {"s": s, "obs": obs, "theta2": th}


def sweeps_exact(p: Params, W, s, t0, nsweeps):
    """Exact sequential Metropolis with dE from two full-energy evaluations."""
    N = p.L * p.L
    W = np.ascontiguousarray(W, np.float64)
    s = np.array(s, np.float64, copy=True, order="C")
    dE = np.zeros(nsweeps * N, np.float64)
    acc = np.zeros(nsweeps * N, np.int32)
    lib().orc_sweeps_exact(C.byref(p), _dp(W), _dp(s), t0, nsweeps, _dp(dE), _ip(acc))
    return {"s": s, "dE": dE, "acc": acc}


def init_random(L, seed, replica=0):
    s = np.zeros((3, L, L), np.float64)
    lib().orc_init_random(L, seed, replica, _dp(s))
    return s


def init_ising(L, seed, replica=0):
    """Random Ising state s = (0, 0, +-1) from the seed (Appendix B)."""
    s = np.zeros((3, L, L), np.float64)
    lib().orc_init_ising(L, seed, replica, _dp(s))
    return s


def propose(kind, cone, s, u1, u2):
    s = np.ascontiguousarray(s, np.float64)
    S = np.zeros(3, np.float64)
    lib().orc_propose(kind, cone, _dp(s), u1, u2, _dp(S))
    return S


def eta(theta2, count):
    theta2 = np.ascontiguousarray(theta2, np.float64)
    return float(lib().orc_eta(theta2.size, _dp(theta2), float(count)))


def eps12(d1, d2, r, CD=1.0):
    a = np.ascontiguousarray(d1, np.float64)
    b = np.ascontiguousarray(d2, np.float64)
    c = np.ascontiguousarray(r, np.float64)
    return float(lib().orc_eps12(_dp(a), _dp(b), _dp(c), CD))


def eps_total(L, l, CD, T, mode, A=64):
    return float(lib().orc_eps_total(L, l, CD, T, mode, A))
