"""The C-ABI library builds, loads and exports every declared entry point
(no GPU needed: nothing here launches a kernel)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "ipls.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\**\s+\**(ipls\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ["iplsCreate", "iplsDestroy", "iplsScratchBytes", "iplsSort", "iplsSortSegmented",
                 "iplsSubmit", "iplsPoll", "iplsWait", "iplsLastError", "iplsGetStats"]:
        assert want in names


def test_library_exports_every_declared_symbol():
    import paper_2208_06902_gb300 as p
    lib = p.load()
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert ctypes.cast(getattr(lib, name), ctypes.c_void_p).value


def test_host_side_validation_without_gpu():
    # argument checks happen before any CUDA call
    import paper_2208_06902_gb300 as p
    lib = p.load()
    assert lib.iplsDefaultConfig(None) == -1
    assert lib.iplsSort(None, None, -5, 0) == -1
    assert lib.iplsSort(None, None, 10, 7) == -1
    assert lib.iplsSort(None, None, 2**32, 0) == -1
    assert lib.iplsSort(None, None, 10, 0) == -1      # NULL keys
    assert "NULL" in p.iplsLastError()
    assert lib.iplsSort(None, ctypes.c_void_p(0x1004), 10, 0) == -1   # f64 keys not 8-aligned
    assert "aligned" in p.iplsLastError()
    assert lib.iplsSortSegmented(None, None, None, -1, 0) == -1
    assert lib.iplsSortSegmented(None, None, None, 0, 0) == 0   # nothing to do
    # host batches: count, dtype, NULL arrays and sizes are checked first
    P = (ctypes.c_void_p * 2)(None, None)
    N = (ctypes.c_int64 * 2)(10, 5)
    assert lib.iplsSortHostBatch(None, P, N, 0, 0) == 0           # nothing to do
    assert lib.iplsSortHostBatch(None, P, N, -1, 0) == -1
    assert lib.iplsSortHostBatch(None, P, N, 2, 9) == -1          # unknown dtype
    assert lib.iplsSortHostBatch(None, None, N, 2, 0) == -1
    assert lib.iplsSortHostBatch(None, P, N, 2, 0) == -1          # NULL array of 10 keys
    assert "NULL" in p.iplsLastError()
    N2 = (ctypes.c_int64 * 2)(2**32, 1)
    assert lib.iplsSortHostBatch(None, P, N2, 2, 0) == -1         # above 2^32 - 1 keys
    cfg = p.iplsDefaultConfig()
    assert (cfg.k, cfg.cutoff, cfg.sync) == (256, 32, 1)
    n = p.iplsScratchBytes(None, 1 << 28, 0)
    assert n >= (1 << 28) * 8


def test_product_package_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2208_06902_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "ipls_oracle" not in text, f


def test_config_validation_without_gpu():
    # iplsCreate checks the configuration before any CUDA call
    import paper_2208_06902_gb300 as p
    lib = p.load()
    ctx = ctypes.c_void_p()
    for bad in (1, 3, 96, 2048, -2):
        cfg = p.iplsDefaultConfig()
        cfg.pl2_leaves = bad
        assert lib.iplsCreate(ctypes.byref(ctx), ctypes.byref(cfg), None, None, None, None) == -1
        assert "pl2_leaves" in p.iplsLastError()
    for good in (0, 2, 64, 1024):
        cfg = p.iplsDefaultConfig()
        cfg.pl2_leaves = good
        rc = lib.iplsCreate(ctypes.byref(ctx), ctypes.byref(cfg), None, None, None, None)
        assert rc != -1 or "pl2_leaves" not in p.iplsLastError()
        if rc == 0:
            lib.iplsDestroy(ctx)
