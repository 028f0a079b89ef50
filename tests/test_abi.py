"""The C ABI library builds, loads, and exports every symbol include/mipwa.h
declares (no GPU needed: nothing here launches work)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "mipwa.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(mipwa_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1703_03284_gb300 import build, _lib
    build.build()
    return _lib.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("mipwa_set_events", "mipwa_set_norm_sample", "mipwa_set_model", "mipwa_nll",
              "mipwa_nll_grad"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_declares_every_symbol():
    from paper_1703_03284_gb300 import _lib
    bound = {n for n, _, _ in _lib.SIGNATURES}
    assert bound == set(declared_functions())


def test_constants_match_header():
    from paper_1703_03284_gb300 import _lib
    src = open(os.path.join(ROOT, "include", "mipwa.h")).read()
    for name, val in (("MIPWA_MAX_RES", _lib.MAX_RES), ("MIPWA_MAX_KNOTS", _lib.MAX_KNOTS)):
        assert int(re.search(rf"#define {name} (\d+)", src).group(1)) == val
    for name in ("OK", "EINVAL", "EOUTSIDE", "ENONPOS", "ECUDA", "ETIMEOUT", "ESTATE", "ENOMEM"):
        m = re.search(rf"MIPWA_{name} = (-?\d+)", src)
        assert int(m.group(1)) == getattr(_lib, name)
    for name in ("FFMA", "FFMA2", "DFMA", "MUFU"):
        m = re.search(rf"#define MIPWA_PROBE_{name} (\d+)", src)
        assert int(m.group(1)) == getattr(_lib, f"PROBE_{name}")


def test_toys_config_layout_matches_header():
    """mipwa_toys_config: two int64 chunks, then two ints (24 bytes)."""
    from paper_1703_03284_gb300 import _lib
    src = open(os.path.join(ROOT, "include", "mipwa.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    body = re.search(r"typedef struct \{([^{}]*)\} mipwa_toys_config;", src).group(1)
    fields = re.findall(r"(int64_t|int)\s+(\w+);", body)
    assert [n for _, n in fields] == [n for n, _ in _lib.ToysConfig._fields_]
    assert ctypes.sizeof(_lib.ToysConfig) == 24


def test_null_context_is_rejected(lib):
    assert lib.mipwa_num_params(None) == -1
    assert lib.mipwa_nll(None, None, None) == -1
    assert lib.mipwa_set_masses(None, 1.0, 0.1, 0.1) == -1
    lib.mipwa_destroy(None)
    assert lib.mipwa_last_error(None) == b"null context"


def test_create_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    assert lib.mipwa_create(ctypes.byref(h), 0, 0) == -4
    assert not h.value
