"""The C-ABI library builds, loads and exports every symbol its header
declares; host-only calls behave without a GPU (CPU only)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for h in sorted(os.listdir(inc)):
        if h.endswith(".h"):
            src = re.sub(r"/\*.*?\*/", "", open(os.path.join(inc, h)).read(), flags=re.S)
            names |= set(re.findall(r"\b(dvl_[a-z_]+)\s*\(", src))
    return sorted(names)


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["dvl_create", "dvl_destroy", "dvl_load_amr", "dvl_build_order", "dvl_set_tf",
              "dvl_update", "dvl_read_bins"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    import paper_2306_11612_b300 as dvl
    lib = ctypes.CDLL(dvl._LIB_PATH)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(dvl.EXPORTS) == set(_declared())


def test_status_strings_and_null_handles():
    import paper_2306_11612_b300 as dvl
    L = dvl.lib
    for code in range(-7, 1):
        assert L.dvl_status_string(code).decode()
    assert L.dvl_status_string(99).decode() == "unknown status"
    assert L.dvl_last_error(None).decode() == ""
    L.dvl_destroy(None)                      # no-op
    assert L.dvl_update(None, None) == dvl.ERR_ARG
    assert L.dvl_sync(None) == dvl.ERR_ARG
    assert L.dvl_read_bins_all(None, None) == dvl.ERR_ARG
    assert L.dvl_set_tfs(None, 4, None, 256, None) == dvl.ERR_ARG
    assert L.dvl_create(None, 0, None) == dvl.ERR_ARG


def test_create_fails_loudly_without_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_2306_11612_b300 as dvl
    with pytest.raises(dvl.DVLError) as e:
        dvl.DVL(0)
    assert e.value.status == dvl.ERR_CUDA


def test_kernels_are_built_for_sm103a():
    # the build passes only -gencode arch=compute_103a,code=sm_103a
    from paper_2306_11612_b300 import _build
    assert "arch=compute_103a,code=sm_103a" in _build.ARCH
    assert "-fmad=false" in _build.COMMON


def test_serving_rules_without_gpu():
    # batch-size buckets and memory admission are pure host functions
    import paper_2306_11612_b300 as dvl
    L = dvl.lib
    assert [L.dvl_serve_bucket(k, 64) for k in (0, 1, 2, 3, 5, 9, 33, 64, 100)] == [0, 1, 2, 4, 8, 16, 64, 64, 64]
    assert L.dvl_serve_bucket(40, 48) == 48 and L.dvl_serve_bucket(17, 48) == 32
    GB = 1 << 30
    # room for everything: all queued requests up to max_batch
    assert L.dvl_serve_admit(5, 64, 0, GB, 0, 100 * GB) == 5
    assert L.dvl_serve_admit(200, 64, 0, GB, 0, 100 * GB) == 64
    # growth to a bucket of 8 needs 8 GB; only 5 GB left -> bucket 4
    assert L.dvl_serve_admit(7, 64, 0, GB, 95 * GB, 100 * GB) == 4
    # buffers already hold 4 slots: a batch of 4 needs no new memory
    assert L.dvl_serve_admit(7, 64, 4, GB, 100 * GB, 100 * GB) == 4
    # nothing allocated and not even one slot fits
    assert L.dvl_serve_admit(3, 64, 0, GB, 100 * GB - 1, 100 * GB) == 0
    assert L.dvl_serve_admit(0, 64, 0, GB, 0, 100 * GB) == 0
    assert L.dvl_server_create(None, 0, None) == dvl.ERR_ARG
    L.dvl_server_destroy(None)


def test_read_bins_all_checks_buffer_sizes_on_the_host():
    """The binding refuses buffers smaller than n_fields x W (W for count)
    before it calls into the library."""
    import numpy as np
    import paper_2306_11612_b300 as dvl
    ctx = object.__new__(dvl.DVL)          # no device context: the check runs first
    ctx.M, ctx.W, ctx._h = 4, 100, None
    for name, arr in [("mean", np.empty(399, np.float32)), ("sum", np.empty(399, np.float64)),
                      ("count", np.empty(99, np.uint32)), ("y", np.empty(200, np.float64)[:199])]:
        with pytest.raises(ValueError):
            ctx.read_bins_all({name: arr})
