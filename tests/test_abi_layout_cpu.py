"""The binding's view of the C ABI against the header itself, on the CPU: a small C
program compiled against include/dipmc.h prints the size of every public struct and
the offset of every field, and the values of the numeric #define constants; the
ctypes structures and constants of paper_1211_6234_b300/dipmc.py must agree."""
import ctypes as C
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dipmc.h")
STRUCTS = ("mc_obs", "mc_timing", "mc_tuning", "mc_request", "mc_request_info", "mc_server_stats")


def header_constants():
    text = open(HEADER).read()
    return {m.group(1): int(m.group(2)) for m in re.finditer(r"^#define\s+(MC_\w+)\s+\(?(-?\d+)\)?", text, re.M)}


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    from paper_1211_6234_b300 import dipmc
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "dipmc.h"', "int main(void) {"]
    for s in STRUCTS:
        lines.append(f'    printf("{s} size %zu\\n", sizeof({s}));')
        for name, _ in getattr(dipmc, s)._fields_:
            lines.append(f'    printf("{s} {name} %zu %zu\\n", offsetof({s}, {name}), sizeof((({s} *)0)->{name}));')
    lines += ["    return 0;", "}"]
    d = tmp_path_factory.mktemp("abi")
    src, exe = d / "layout.c", d / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    sizes, fields = {}, {}
    for ln in out.splitlines():
        p = ln.split()
        if p[1] == "size":
            sizes[p[0]] = int(p[2])
        else:
            fields[(p[0], p[1])] = (int(p[2]), int(p[3]))
    return sizes, fields


@pytest.mark.parametrize("name", STRUCTS)
def test_ctypes_structs_match_the_header(c_layout, name):
    from paper_1211_6234_b300 import dipmc
    sizes, fields = c_layout
    st = getattr(dipmc, name)
    assert C.sizeof(st) == sizes[name], name
    for f, _ in st._fields_:
        desc = getattr(st, f)
        assert (desc.offset, desc.size) == fields[(name, f)], (name, f)


def test_binding_constants_match_the_header():
    from paper_1211_6234_b300 import dipmc
    consts = header_constants()
    assert len(consts) > 20
    shared = [k for k in consts if hasattr(dipmc, k)]
    for k in shared:
        assert getattr(dipmc, k) == consts[k], k
    # every error code, field path and request state the header defines is in the binding
    for k in consts:
        if re.match(r"MC_(OK|E[A-Z]+|PATH_\w+|REQ_\w+|NOBS)$", k):
            assert k in shared, k


def test_observable_and_kernel_class_orders_match_the_header():
    """OBS_NAMES and KERNEL_CLASSES index the header's MC_OBS_* and MC_K_* arrays."""
    from paper_1211_6234_b300 import dipmc
    consts = header_constants()
    obs = {k[len("MC_OBS_"):]: v for k, v in consts.items() if k.startswith("MC_OBS_")}
    names = {"ABS_M": "abs_m", "MZ": "m_z", "ABS_MZ": "abs_m_z", "MPAR": "m_par", "E": "e", "MST": "m_st",
             "WALL": "wall", "OX": "o_x", "OY": "o_y", "OZ": "o_z", "CONE": "cone"}
    assert len(obs) == consts["MC_NOBS"] == len(dipmc.OBS_NAMES)
    for k, v in obs.items():
        assert dipmc.OBS_NAMES[v] == names[k], k
    kc = {k[len("MC_K_"):].lower(): v for k, v in consts.items() if k.startswith("MC_K_")}
    assert len(kc) == consts["MC_NKCLASS"] == len(dipmc.KERNEL_CLASSES)
    for k, v in kc.items():
        assert dipmc.KERNEL_CLASSES[v] == k, k
