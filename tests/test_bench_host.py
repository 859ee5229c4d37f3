"""Host-side logic of bench.py (no GPU): the algorithmic-bytes model behind the roofline
fraction, and the traffic record that is used only while the kernel source matches the
hash it was captured from."""
import hashlib
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_algorithmic_bytes_closed_form(bench):
    """At R = 64 FP32 with ~2.96 edges per node: the forward call reads the shared model p
    once (4 / S bytes per node-update), writes dT (4) and reads the structure once, shared
    by the R columns; the reverse call writes lam (4) and g once (4 / S), reads the
    receiver data and the structure.  The per-source-input figure 8 + 36/R is kept beside."""
    S, N, R, n_rec = 25, 1000, 64, 10
    st = [{"edges": 2960} for _ in range(S)]
    ab = bench.algorithmic_bytes(st, R, 4, S, N, n_rec)
    struct = 16 + 2.96 * 8
    assert ab["updates"] == S * N * R
    assert ab["fwd_per_update"] == pytest.approx(4 + 4 / S + struct / R + n_rec * 4 / N, rel=1e-12)
    assert ab["bwd_per_update"] == pytest.approx(4 + struct / R + n_rec * 4 / N + 4 / S, rel=1e-12)
    assert ab["fwd_per_update_input_per_source"] == pytest.approx(8 + struct / R + n_rec * 4 / N, rel=1e-12)
    # the method's per-update bytes of the 3-D workload (R = 64, S = 25): about 4.78
    assert 4.7 < 4 + 4 / S + struct / R < 4.85


def test_traffic_record_requires_matching_source_hash(bench, tmp_path, monkeypatch):
    """measured_traffic reads profiles/traffic.txt only for the kernel and direction it
    names and only while the traversal kernels' sources still hash to the recorded value."""
    h = hashlib.sha256()
    for name in ("eik_apply.cu", "eik_trav.h", "eik_vec.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2609_14982_b300", "csrc", name), "rb").read())
    digest = h.hexdigest()
    assert bench.kernel_source_digest() == digest
    got = bench.measured_traffic("fwd", "k_traverse_persistent<float,4,false>")
    rec = open(os.path.join(ROOT, "profiles", "traffic.txt")).read()
    if digest in rec:
        assert got is not None and 4.0 < got < 12.0
    else:
        assert got is None
    assert bench.measured_traffic("fwd", "no_such_kernel") is None
    # a record for another source hash is ignored
    fake = tmp_path / "profiles"
    fake.mkdir()
    (fake / "traffic.txt").write_text("direction=fwd kernel=k bytes_per_update=7.0 source_sha256=" + "0" * 64 + "\n")
    csrc = tmp_path / "paper_2609_14982_b300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "eik_apply.cu").write_text("// other source\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_traffic("fwd", "k") is None
