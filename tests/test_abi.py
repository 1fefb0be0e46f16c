"""The C ABI library loads and exports every function include/pa.h declares
(no GPU needed: nothing here calls into CUDA)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "pa.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(pa_[A-Za-z0-9_]+)\s*\(", text)
    return sorted(set(names))


def _library():
    from paper_1704_01888_gb300 import build

    try:
        return build.build()
    except (OSError, RuntimeError) as e:  # no nvcc in this environment
        pytest.skip(f"cannot build the CUDA library here: {e}")


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("pa_init", "pa_sweep", "pa_energy", "pa_resample", "pa_observables"):
        assert required in names


def test_library_exports_every_declared_symbol():
    path = _library()
    lib = ctypes.CDLL(path)
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    import paper_1704_01888_gb300 as pa

    assert sorted(pa.EXPORTED) == _declared_functions()


def test_status_strings_and_validation_without_gpu():
    import paper_1704_01888_gb300 as pa

    _library()
    lib = pa.load_library()
    assert lib.pa_status_str(pa.PA_ERR_CAPACITY) == b"population exceeds capacity"
    # invalid configurations are rejected before any CUDA call
    ctx = ctypes.c_void_p()
    for bad in (dict(q=1, L=16, R=10), dict(q=10, L=15, R=10), dict(q=129, L=16, R=10),
                dict(q=10, L=16, R=0), dict(q=10, L=16, R=10, R_cap=5), dict(q=10, L=16, R=10, stream=256)):
        cfg = pa.Config(bad["q"], bad["L"], bad["R"], bad.get("R_cap", 0), 1, 0, 0, 0.0, 0, bad.get("stream", 0))
        assert lib.pa_init(ctypes.byref(cfg), None, ctypes.byref(ctx)) == pa.PA_ERR_INVALID
        assert not ctx.value
    # replicas whose bit planes exceed a block's shared memory (204800 bytes):
    # q = 128 (7 planes) at L = 458, q = 20 (5 planes) at L = 570, q = 10 (4
    # planes) at L = 642 and 1024
    for q, L in ((128, 458), (20, 570), (10, 642), (10, 1024)):
        cfg = pa.Config(q, L, 10, 0, 1, 0, 0, 0.0, 0, 0)
        assert lib.pa_init(ctypes.byref(cfg), None, ctypes.byref(ctx)) == pa.PA_ERR_TOO_LARGE
        assert not ctx.value
    assert lib.pa_kernel_launch_count() == 0


def test_checkpoint_loader_rejects_bad_files_before_device_work(tmp_path):
    """pa_load validates header, sizes and checksum on the host first."""
    import paper_1704_01888_gb300 as pa

    _library()
    lib = pa.load_library()
    ctx = ctypes.c_void_p()
    missing = str(tmp_path / "none.ckpt").encode()
    assert lib.pa_load(missing, None, ctypes.byref(ctx)) == pa.PA_ERR_INVALID
    junk = tmp_path / "junk.ckpt"
    junk.write_bytes(b"PAGB300\x01" + bytes(400))
    assert lib.pa_load(str(junk).encode(), None, ctypes.byref(ctx)) == pa.PA_ERR_INVALID
    assert not ctx.value
