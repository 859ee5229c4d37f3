"""Host-side checks of the C-ABI library (no GPU needed): it builds for sm_103a, loads,
exports every function include/eik.h declares, and the binding refuses CPU tensors."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?!typedef)[A-Za-z_][\w\s\*]*?\b([A-Za-z_]\w*)\s*\([^;{]*\)\s*;", text, re.M):
            names.append(m.group(1))
    return sorted(set(names))


@pytest.fixture(scope="module")
def libeik():
    from paper_2609_14982_b300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("eik_forward", "tangent_build", "tangent_apply", "tangent_apply_T", "tangent_solve",
              "tangent_solve_T", "tangent_stats", "tangent_export", "tangent_free", "sweep_apply"):
        assert n in names


def test_library_exports_every_declared_symbol(libeik):
    missing = [n for n in _declared() if not hasattr(libeik, n)]
    assert not missing, missing


def test_binding_lists_match_header():
    from paper_2609_14982_b300 import eik
    assert sorted(eik.EXPORTED) == _declared()


def test_version_and_defaults(libeik):
    from paper_2609_14982_b300 import eik
    libeik.eik_version.restype = ctypes.c_char_p
    assert b"sm_103a" in libeik.eik_version()
    o = eik.default_opts()
    assert o.schedule == eik.SCHED_PERSISTENT and o.wait_timeout_s > 0 and o.lu_pivot_tol > 0
    assert o.block_lu_min == 0


def test_binding_rejects_host_tensors():
    import torch
    from paper_2609_14982_b300 import eik
    with pytest.raises(TypeError):
        eik._dev(torch.zeros(4), name="x")


def test_binding_structs_match_header_layout(tmp_path):
    """The ctypes mirrors of eik_grid, eik_opts and eik_stats have the header's field
    offsets and sizes (compiled with the host C compiler)."""
    import subprocess
    from paper_2609_14982_b300 import eik
    structs = {"eik_grid": eik.Grid_, "eik_opts": eik.Opts, "eik_stats": eik.Stats}
    lines = ['#include <stdio.h>', '#include "eik.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {(a, b): int(c) for a, b, c in (ln.split() for ln in out if ln)}
    for cname, py in structs.items():
        assert got[(cname, "sizeof")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)
