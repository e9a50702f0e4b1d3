"""The tuned-launch-parameter cache (host only, no CUDA call): the in-process
table, its text file (header line, "key<TAB>value" lines, rewritten whole on
every store), reloading in another process, the STBEM_TUNE_CACHE variable and
the rejection of malformed entries."""
import os
import subprocess
import sys

import pytest

from paper_1811_05224_gb300 import capi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture()
def lib():
    try:
        L = capi.load()
    except OSError as e:          # library not built here
        pytest.skip(str(e))
    yield L
    L.stbem_tune_cache_path(None)
    L.stbem_tune_cache_clear()


def _get(L, key, cap=256):
    import ctypes
    buf = ctypes.create_string_buffer(cap)
    code = L.stbem_tune_cache_get(key.encode(), buf, cap)
    return code, buf.value.decode()


def test_memory_table_round_trip(lib):
    assert lib.stbem_tune_cache_path(None) == capi.STBEM_OK
    lib.stbem_tune_cache_clear()
    assert _get(lib, "dev|k|nt=4")[0] == capi.STBEM_ERR_ARG
    assert lib.stbem_tune_cache_put(b"dev|k|nt=4", b"bn=128") == capi.STBEM_OK
    assert _get(lib, "dev|k|nt=4") == (capi.STBEM_OK, "bn=128")
    assert lib.stbem_tune_cache_put(b"dev|k|nt=4", b"bn=256") == capi.STBEM_OK   # replaced
    assert _get(lib, "dev|k|nt=4") == (capi.STBEM_OK, "bn=256")
    assert _get(lib, "dev|k|nt=4", cap=4)[0] == capi.STBEM_ERR_NOMEM
    lib.stbem_tune_cache_clear()
    assert _get(lib, "dev|k|nt=4")[0] == capi.STBEM_ERR_ARG


def test_rejects_malformed_entries(lib):
    for k, v in [(b"a\tb", b"x"), (b"a", b"x\ny"), (b"", b"x"), (b"a", b""), (b"a\rb", b"x")]:
        assert lib.stbem_tune_cache_put(k, v) == capi.STBEM_ERR_ARG


def test_file_persists_across_processes(lib, tmp_path):
    f = tmp_path / "tune.txt"
    assert lib.stbem_tune_cache_path(str(f).encode()) == capi.STBEM_OK     # missing file: empty table
    lib.stbem_tune_cache_clear()
    assert lib.stbem_tune_cache_put(b"GB300|sm152|cc10.3|tc_plain|nt=512|nx=512|rhs=8", b"bn=128") == capi.STBEM_OK
    assert lib.stbem_tune_cache_put(b"GB300|sm152|cc10.3|ragged_apply|prec=f32", b"tiles32=1 lpc=32") == 0
    lines = f.read_text().splitlines()
    assert lines[0].startswith("#") and len(lines) == 3
    assert "GB300|sm152|cc10.3|tc_plain|nt=512|nx=512|rhs=8\tbn=128" in lines
    assert not (tmp_path / "tune.txt.tmp").exists()
    # forget the process's table, reload from the file
    lib.stbem_tune_cache_clear()
    assert _get(lib, "GB300|sm152|cc10.3|tc_plain|nt=512|nx=512|rhs=8")[0] == capi.STBEM_ERR_ARG
    assert lib.stbem_tune_cache_path(str(f).encode()) == capi.STBEM_OK
    assert _get(lib, "GB300|sm152|cc10.3|tc_plain|nt=512|nx=512|rhs=8") == (capi.STBEM_OK, "bn=128")
    # another process, through the environment variable; it adds an entry
    code = ("from paper_1811_05224_gb300 import capi; import ctypes; L = capi.load(); "
            "b = ctypes.create_string_buffer(64); "
            "assert L.stbem_tune_cache_get(b'GB300|sm152|cc10.3|ragged_apply|prec=f32', b, 64) == 0; "
            "print(b.value.decode()); "
            "assert L.stbem_tune_cache_put(b'other|key', b'v=1') == 0")
    env = dict(os.environ, STBEM_TUNE_CACHE=str(f), PYTHONPATH=ROOT)
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stderr
    assert out.stdout.strip() == "tiles32=1 lpc=32"
    # this process's next store merges the other process's entry
    assert lib.stbem_tune_cache_put(b"third", b"v=3") == capi.STBEM_OK
    text = f.read_text()
    assert "other|key\tv=1" in text and "third\tv=3" in text and "tiles32=1 lpc=32" in text


def test_unwritable_file_is_reported(lib, tmp_path):
    f = tmp_path / "no_such_dir" / "tune.txt"
    assert lib.stbem_tune_cache_path(str(f).encode()) == capi.STBEM_OK
    assert lib.stbem_tune_cache_put(b"k", b"v") == capi.STBEM_ERR_ARG
    assert _get(lib, "k") == (capi.STBEM_OK, "v")       # the in-process entry stands
