"""Host-side checks of the C-ABI library that need no GPU: it loads, it exports
every entry point include/dipmc.h declares, and argument validation that
precedes any CUDA call reports the documented error codes."""
import ctypes as C
import math
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dipmc.h")


def declared_symbols():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(mc_\w+)\s*\(", text, re.M)))


def test_header_declares_the_abi():
    syms = declared_symbols()
    for s in ("mc_create_lattice", "mc_set_params", "mc_precompute_W", "mc_sweep", "mc_observables"):
        assert s in syms


def test_library_exports_every_declared_symbol():
    from paper_1211_6234_b300 import dipmc
    out = subprocess.run(["nm", "-D", "--defined-only", dipmc.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if ln.strip()}
    missing = [s for s in declared_symbols() if s not in exported]
    assert not missing, missing
    assert set(dipmc.ABI_SYMBOLS) == set(declared_symbols())
    for s in declared_symbols():
        getattr(dipmc.lib(), s)


def test_validation_before_any_device_call():
    from paper_1211_6234_b300 import dipmc
    lib = dipmc.lib()
    h = C.c_void_p()
    assert lib.mc_create_lattice(16, 5, 1, 1, C.byref(h)) == dipmc.MC_EINVAL
    assert b"L % l" in lib.mc_last_error()
    assert lib.mc_create_lattice(16, 1, 1, 1, C.byref(h)) == dipmc.MC_EINVAL
    assert lib.mc_create_lattice(1, 1, 1, 1, C.byref(h)) == dipmc.MC_EINVAL
    assert lib.mc_create_lattice(16, 8, 0, 1, C.byref(h)) == dipmc.MC_EINVAL
    assert lib.mc_create_lattice(16, 8, 1, 1, None) == dipmc.MC_EINVAL
    assert lib.mc_sweep(None, 1, 0, None) == dipmc.MC_EINVAL
    assert lib.mc_observables(None, 0, None) == dipmc.MC_EINVAL
    assert lib.mc_destroy(None) == dipmc.MC_OK
    assert lib.mc_version() >= 1


def test_binding_raises_instead_of_falling_back():
    """The binding wraps non-zero codes in McError; there is no CPU path."""
    from paper_1211_6234_b300 import dipmc
    with pytest.raises(dipmc.McError) as e:
        dipmc.Lattice(16, 5, 1, 1)
    assert e.value.code == dipmc.MC_EINVAL


@pytest.mark.parametrize("L,CD,T,err", [(64, 0.1, 0.2, 1e-3), (64, 0.1, 0.6, 1e-3), (256, 0.1, 0.3, 1e-3),
                                        (256, 0.2, 0.3, 1e-4), (48, 0.1, 0.5, 1e-3), (16, 0.1, 0.6, 1e-2)])
def test_choose_spacing_against_oracle_error_estimate(L, CD, T, err):
    """The spacing chooser (host logic of the library) against the oracle's own
    evaluation of the Sec. 3.2 error estimate summed over the update sublattice:
    the chosen l meets the bound and every smaller divisor of L violates it."""
    from oracle import oracle as orc
    from paper_1211_6234_b300 import dipmc
    l = dipmc.choose_spacing(L, CD, T, err)
    assert L % l == 0 and l >= 2
    tail = lambda ll: 2 * CD * 4 * math.sqrt(2) / ((64 * (L // ll) + 0.5) * ll**3 * T)  # noqa: E731
    if l < L:
        assert orc.eps_total(L, l, CD, T, 1, 64) + tail(l) <= err * (1 + 1e-9)
    for m in range(2, l):
        if L % m == 0:
            assert orc.eps_total(L, m, CD, T, 1, 64) + tail(m) > err


def test_binding_without_the_library_fails_to_import(tmp_path):
    """A copy of the package without libdipmc.so: importing the binding raises
    ImportError naming the missing library, so no call can run anywhere but in it."""
    import shutil
    import sys
    pkg = tmp_path / "paper_1211_6234_b300"
    pkg.mkdir()
    for f in ("__init__.py", "dipmc.py", "inputs.py"):
        shutil.copy(os.path.join(ROOT, "paper_1211_6234_b300", f), pkg / f)
    code = ("import sys; sys.path.insert(0, sys.argv[1])\n"
            "try:\n    import paper_1211_6234_b300.dipmc\nexcept ImportError as e:\n"
            "    print('IMPORT-ERROR', e); sys.exit(0)\nsys.exit(3)\n")
    r = subprocess.run([sys.executable, "-c", code, str(tmp_path)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, (r.stdout, r.stderr)
    assert "IMPORT-ERROR" in r.stdout and "libdipmc.so" in r.stdout and "not built" in r.stdout
