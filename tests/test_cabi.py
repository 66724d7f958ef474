"""C-ABI checks that need no GPU: the library builds for sm_103a, loads, exports
every function include/sem.h declares, and refuses work before sem_init."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(sem_[a-z_0-9]+)\s*\(", text, re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2606_12650_gb300 import build, sem
    build.build()
    return sem.load()


def test_header_declares_the_boundary():
    names = _declared("sem.h")
    for must in ("sem_init", "sem_update", "sem_run", "sem_sync", "sem_finalize"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    for name in _declared("sem.h"):
        assert hasattr(lib, name), name


def test_binding_names_match_exports():
    from paper_2606_12650_gb300 import sem
    assert set(sem.EXPORTS) <= set(_declared("sem.h"))


def test_calls_before_init_return_einit(lib):
    from paper_2606_12650_gb300 import sem
    if sem._keep.get("initialised"):
        pytest.skip("libsem was initialised by an earlier test in this process")
    buf = (ctypes.c_double * 4)()
    assert lib.sem_update(ctypes.cast(buf, ctypes.c_void_p), 0, 4, 8, sem.SEM_TO) == sem.SEM_EINIT
    assert "not initialised" in sem.last_error()
    assert lib.sem_run(b"ax", 0, None) == sem.SEM_EINIT
    assert lib.sem_sync() == sem.SEM_EINIT
    assert lib.sem_finalize() == sem.SEM_EINIT
    assert lib.sem_set_stream(None) == sem.SEM_EINIT


def test_allocator_hooks_must_come_in_pairs(lib):
    from paper_2606_12650_gb300 import sem
    if sem._keep.get("initialised"):
        pytest.skip("libsem was initialised by an earlier test in this process")
    fn = sem.ALLOC_FN(lambda n, c: 0)
    assert lib.sem_set_allocator(ctypes.cast(fn, ctypes.c_void_p), None, None) == sem.SEM_EARG
    assert lib.sem_set_allocator(None, None, None) == sem.SEM_OK


def test_marshalling_kinds():
    import numpy as np
    from paper_2606_12650_gb300 import sem
    assert sem._marshal(3).kind == sem.ARG_INT
    assert sem._marshal(2.5).kind == sem.ARG_DOUBLE
    assert sem._marshal(None).kind == sem.ARG_NONE
    assert sem._marshal(np.zeros(4)).kind == sem.ARG_MAPPED
    assert sem._marshal(sem.OutInt()).kind == sem.ARG_OUT_INT
    assert sem._marshal(sem.OutDouble()).kind == sem.ARG_OUT_DOUBLE
    assert sem._marshal(sem.DevicePtr(256)).kind == sem.ARG_DEVICE
    with pytest.raises(TypeError):
        sem._marshal(True)
    with pytest.raises(ValueError):
        sem._marshal(np.zeros((4, 4))[:, 1])


def test_product_path_fails_loudly_without_library(tmp_path):
    from paper_2606_12650_gb300 import sem
    with pytest.raises(RuntimeError, match="libsem.so not found"):
        sem._open(str(tmp_path / "missing.so"))


def test_autotune_table_is_checked_at_init(lib, tmp_path):
    """--autotune-table: every entry is validated before the device is
    touched (kind, N in [1, 9], variant available for the kind, elements per
    block fitting one block); a bad file fails sem_init with SEM_EARG."""
    from paper_2606_12650_gb300 import sem
    if sem._keep.get("initialised"):
        pytest.skip("libsem was initialised by an earlier test in this process")

    def init(*args):
        arr = (ctypes.c_char_p * len(args))(*[a.encode() for a in args])
        return lib.sem_init(len(args), arr)

    assert init(f"--autotune-table={tmp_path / 'missing.txt'}") == sem.SEM_EARG
    assert "cannot read" in sem.last_error()
    bad = tmp_path / "bad.txt"
    bad.write_text("# comment\n0 7 1 2 10.0\n0 7 9 1\n")
    assert init(f"--autotune-table={bad}") == sem.SEM_EARG
    assert "line 3" in sem.last_error()
    for entry in ("1 7 0 0",      # column kernel is FP64 only
                  "0 7 2 0",      # persistent kernel is FP32 only
                  "0 7 4 2",      # staged factors: FP32 only
                  "1 7 3 4",      # register prefetch: BF16 factors only
                  "0 10 1 1",     # N above 9
                  "0 0 1 1",      # N below 1
                  "0 7 1 600",    # 600 elements of 64 threads do not fit a block
                  "0 7 1 0",      # line kernel needs elements per block
                  "3 7 1 1",      # no such kind
                  "0 7"):         # too few fields
        f = tmp_path / "one.txt"
        f.write_text(entry + "\n")
        assert init(f"--autotune-table={f}") == sem.SEM_EARG, entry
    good = tmp_path / "good.txt"
    good.write_text("# kind N variant epb us\n0 7 1 2 1800.5\n2 7 1 4\n1 3 2 0\n\n")
    rc = init(f"--autotune-table={good}")
    if rc == sem.SEM_OK:          # a GPU is present
        assert lib.sem_finalize() == sem.SEM_OK
    else:                         # the table passed; the device query failed
        assert rc == sem.SEM_ECUDA, sem.last_error()
