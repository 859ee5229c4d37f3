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


def test_binding_rejects_host_tensors():
    import torch
    from paper_2609_14982_b300 import eik
    with pytest.raises(TypeError):
        eik._dev(torch.zeros(4), name="x")
