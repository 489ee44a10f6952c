"""C-ABI library: builds for sm_103a, loads without a GPU, exports every entry
point declared in include/*.h, and rejects bad arguments before touching the
device."""
import ctypes as C
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1003_3896_gb300 import build
    path = build.build()
    return C.CDLL(path)


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(nb_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_core_calls():
    names = declared_functions()
    for required in ["nb_create", "nb_load", "nb_accel", "nb_step", "nb_energy",
                     "nb_get_state", "nb_destroy", "nb_last_error"]:
        assert required in names


def test_every_declared_symbol_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_abi_version_and_defaults(lib):
    from paper_1003_3896_gb300 import nbsym
    assert nbsym.nb_abi_version() == 3
    p = nbsym.Params()
    nbsym.nb_params_default(C.byref(p))
    assert p.G == 1.0 and p.eps == 0.0 and p.precision == nbsym.NB_DS
    assert (p.Md, p.ad, p.bd, p.Mb, p.ab) == (100.0, 6.5, 0.26, 15.0, 0.7)
    assert (p.Mbh, p.eps_bh) == (0.0, 0.0)
    nbsym.nb_params_default(None)   # NULL-safe


@pytest.mark.parametrize("field,value", [("G", 0.0), ("G", float("nan")), ("eps", -1.0),
                                         ("precision", 7), ("bd", 0.0), ("Mbh", -1.0),
                                         ("Mbh", float("inf")), ("eps_bh", -0.5)])
def test_create_rejects_bad_params_without_gpu(lib, field, value):
    from paper_1003_3896_gb300 import nbsym
    p = nbsym.Params()
    nbsym.nb_params_default(C.byref(p))
    p.ext_on = 1
    setattr(p, field, value)
    h = C.c_void_p()
    rc = nbsym.nb_create(C.byref(p), 16, C.byref(h))
    assert rc == nbsym.NB_EINVAL
    assert not h.value
    assert nbsym.nb_last_error()


NULL_CALLS = r"""
import sys
sys.path.insert(0, %r)
from paper_1003_3896_gb300 import nbsym as nb
E = nb.NB_EINVAL
calls = {
    "nb_create": nb.nb_create(None, 16, None),
    "nb_create_batch": nb.nb_create_batch(None, 1, None, None),
    "nb_set_cluster_params": nb.nb_set_cluster_params(None, None, None),
    "nb_clusters": nb.nb_clusters(None),
    "nb_load": nb.nb_load(None, 1, None, None, None),
    "nb_load_device": nb.nb_load_device(None, 1, None, None, None),
    "nb_accel": nb.nb_accel(None, None),
    "nb_accel_device": nb.nb_accel_device(None, None),
    "nb_step": nb.nb_step(None, 2, 0.1, 1),
    "nb_energy": nb.nb_energy(None, None),
    "nb_energy_clusters": nb.nb_energy_clusters(None, None),
    "nb_torque": nb.nb_torque(None, None),
    "nb_get_state": nb.nb_get_state(None, None, None),
    "nb_get_state_device": nb.nb_get_state_device(None, None, None),
    "nb_size": nb.nb_size(None),
    "nb_set_precision": nb.nb_set_precision(None, 0),
    "nb_prof_enable": nb.nb_prof_enable(None, 1),
    "nb_prof_read": nb.nb_prof_read(None, None),
    "nb_accel_static": nb.nb_accel_static(None, 16, None, None, None),
    "nb_accel_range": nb.nb_accel_range(None, 0, 1, None),
    "nb_accel_symmetric": nb.nb_accel_symmetric(None, None, None),
    "nb_substep_range": nb.nb_substep_range(None, 0, 1, 0.0, 0.1),
    "nb_stage_weights": nb.nb_stage_weights(6, None),
    "nb_set_state": nb.nb_set_state(None, None, None),
    "nb_set_state_device": nb.nb_set_state_device(None, None, None),
    "nb_tune": nb.nb_tune(None, 2, None),
    "nb_pair_shape": nb.nb_pair_shape(None, None, None, None, None),
    "nb_server_create": nb.nb_server_create(None, None),
    "nb_server_submit": nb.nb_server_submit(None, None, None, None, None, None),
    "nb_server_poll": nb.nb_server_poll(None, 1, None),
    "nb_server_wait": nb.nb_server_wait(None, 1, 0.0, None),
    "nb_server_result": nb.nb_server_result(None, 1, None, None),
    "nb_server_cancel": nb.nb_server_cancel(None, 1),
    "nb_server_forget": nb.nb_server_forget(None, 1),
    "nb_server_stats": nb.nb_server_stats(None, None),
}
nb.nb_destroy(None)
nb.nb_server_destroy(None)
nb.nb_params_default(None)
nb.nb_server_params_default(None)
bad = {k: v for k, v in calls.items() if v != E}
print("checked", len(calls), "bad", bad)
sys.exit(1 if bad else 0)
"""


def test_null_handles_are_rejected(lib):
    """Every entry point that takes a context, a server, parameters or an
    output pointer returns NB_EINVAL for NULL without touching the device, and
    the destroy / defaults calls are NULL-safe.  Run in a child process, so a
    missing check shows as a crash report instead of ending the test run."""
    import subprocess
    import sys
    r = subprocess.run([sys.executable, "-c", NULL_CALLS % ROOT], capture_output=True,
                       text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "checked 35 bad {}" in r.stdout


def test_oracle_is_not_on_the_product_path():
    """The product package never imports or loads the oracle."""
    pkg = os.path.join(ROOT, "paper_1003_3896_gb300")
    for f in glob.glob(os.path.join(pkg, "**", "*.*"), recursive=True):
        if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
            assert "oracle" not in open(f).read().replace("Oracle", "").lower() or \
                f.endswith("ics.py"), f


def test_tuning_table_files_without_gpu(lib, tmp_path):
    """The tuned-shape table round-trips through its text file; malformed
    files and shapes this build lacks are rejected and merge nothing."""
    from paper_1003_3896_gb300 import nbsym
    nbsym.tune_clear()
    assert nbsym.tune_entries() == 0
    good = tmp_path / "good.txt"
    good.write_text("nbsym-tune 2\n152 1 1 65536 512 4 128 6\n152 0 512 1289617 64 1 32 8\n")
    assert nbsym.tune_load(str(good)) == 2
    assert nbsym.tune_entries() == 2
    out = tmp_path / "out.txt"
    nbsym.tune_save(str(out))
    lines = [ln for ln in out.read_text().splitlines() if ln]
    assert lines[0] == "nbsym-tune 2" and len(lines) == 3
    nbsym.tune_clear()
    assert nbsym.tune_load(str(out)) == 2
    nbsym.tune_clear()
    bad = tmp_path / "bad.txt"
    for text in ("nbsym-tune 2\n152 1 1 65536 512 3 128 6\n",  # no kernel with I = 3
                 "nbsym-tune 2\n152 1 1 65536 512 4 48 6\n",   # j-tile must divide 128
                 "nbsym-tune 2\n152 1 1 65536\n",              # truncated entry
                 "nbsym-tune 1\n",                              # unknown version
                 "garbage\n"):
        bad.write_text(text)
        assert nbsym.nb_tune_load(os.fsencode(str(bad))) == nbsym.NB_EINVAL
        assert nbsym.tune_entries() == 0
    assert nbsym.nb_tune_load(None) == nbsym.NB_EINVAL
    assert nbsym.nb_tune_save(None) == nbsym.NB_EINVAL
    assert nbsym.nb_tune(None, 2, None) == nbsym.NB_EINVAL
    assert nbsym.nb_pair_shape(None, None, None, None, None) == nbsym.NB_EINVAL


def test_traffic_record_keys_on_code_not_comments():
    """The benchmark reports the captured DRAM traffic of the pair kernel only
    while pair.cu's code is the captured code: comment and layout edits keep
    the digest, any code edit changes it (and the bench then reports null)."""
    import bench
    src = "int f(int a) {\n    return a + 1;   // one\n}\n/* block\n comment */\n"
    same = "int f(int a)\n{\n  return a + 1;   // another comment\n}\n"
    other = "int f(int a) {\n    return a + 2;\n}\n"
    assert bench.code_digest(src) == bench.code_digest(same)
    assert bench.code_digest(src) != bench.code_digest(other)
    assert len(bench.pair_source_digest()) == 16


def test_static_entry_point_validates_like_create(lib):
    """nb_accel_static applies nb_create's parameter rules and says what was
    wrong (no stale message from an earlier call), all before the device."""
    from paper_1003_3896_gb300 import nbsym
    p = nbsym.Params()
    nbsym.nb_params_default(C.byref(p))
    cases = [(16385, {}, "n must be in [1, 16384]"), (0, {}, "n must be in"),
             (16, {"G": float("inf")}, "G must be finite"),
             (16, {"eps": float("inf")}, "eps must be finite"),
             (16, {"ext_on": 1, "Md": float("nan")}, "external field needs"),
             (16, {"precision": 9}, "precision must be")]
    for n, change, msg in cases:
        q = nbsym.Params()
        C.pointer(q)[0] = p
        for k, v in change.items():
            setattr(q, k, v)
        nbsym.nb_create(None, 16, None)          # leaves another message behind
        assert nbsym.nb_accel_static(C.byref(q), n, 8, 8, 8) == nbsym.NB_EINVAL
        assert msg in nbsym.nb_last_error().decode(), (change, nbsym.nb_last_error())
    assert nbsym.nb_accel_static(C.byref(p), 16, None, 8, 8) == nbsym.NB_EINVAL
    assert "NULL" in nbsym.nb_last_error().decode()


class _FakeTensor:
    """Stands in for a device tensor: only what the binding inspects."""

    def __init__(self, numel, dtype="torch.float64", contiguous=True):
        self._n, self.dtype, self._c = numel, dtype, contiguous

    def numel(self):
        return self._n

    def is_contiguous(self):
        return self._c

    def data_ptr(self):
        return 0x1000


def test_binding_checks_buffers_before_the_library(lib):
    """Device buffers too small, of another dtype or not contiguous, and
    per-cluster arrays of the wrong length, are refused by the binding before
    any pointer reaches the library."""
    from paper_1003_3896_gb300 import nbsym

    class Sized(nbsym.Context):
        n = 5
        clusters = 2

        def __init__(self):
            self._h = None

    c = Sized()
    ok = _FakeTensor(15)
    for bad in (_FakeTensor(14), _FakeTensor(15, "torch.float32"),
                _FakeTensor(15, contiguous=False)):
        with pytest.raises(ValueError):
            c.load_device(5, bad, ok, _FakeTensor(5))
        with pytest.raises(ValueError):
            c.accel_device(bad)
        with pytest.raises(ValueError):
            c.get_state_device(ok, bad)
    with pytest.raises(ValueError):
        c.load_device(5, ok, ok, _FakeTensor(4))
    with pytest.raises(ValueError):
        c.set_cluster_params(eps=[0.1, 0.2, 0.3])
    with pytest.raises(ValueError):
        c.set_cluster_params(dt_scale=[1.0])


def test_binding_fails_loudly_without_the_library(tmp_path):
    """With no built libnbsym.so beside it the binding raises ImportError at
    import: there is no CPU or library fallback to fall into."""
    import shutil
    import subprocess
    import sys
    shutil.copy(os.path.join(ROOT, "paper_1003_3896_gb300", "nbsym.py"), tmp_path / "nbsym.py")
    code = ("import sys; sys.path.insert(0, %r)\n"
            "try:\n    import nbsym\nexcept ImportError as e:\n    print('ImportError:', e)\n"
            "else:\n    print('imported')\n") % str(tmp_path)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, r.stderr
    assert r.stdout.startswith("ImportError:") and "libnbsym.so is missing" in r.stdout
