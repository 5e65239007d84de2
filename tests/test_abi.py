"""C-ABI checks that need no GPU: the library loads, exports every entry point that
include/me.h declares, and rejects bad arguments with status codes before touching a
device."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2312_02898_b300 import binding
    if not os.path.exists(binding.LIB_PATH):
        from paper_2312_02898_b300 import build
        build.build(verbose=False)
    return binding.load()


def declared_functions():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(me_[a-z0-9_]+)\s*\(", txt))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for f in ("me_init", "me_compute", "me_info", "me_last_error", "me_free"):
        assert f in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2312_02898_b300 import binding
    names = declared_functions()
    for n in names:
        assert hasattr(lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", binding.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(l.split()[-1] for l in out.splitlines() if l.strip())
    assert set(names) <= exported
    assert set(binding.EXPORTS) <= set(names)


def test_defaults(lib):
    from paper_2312_02898_b300 import binding
    p = binding.default_params()
    assert (p.mZ, p.wZ, p.mt, p.wt, p.aEWM1, p.Gf, p.alphas_default) == (91.188, 2.4414, 173.0, 1.4915, 132.5,
                                                                         1.16639e-5, 0.118)
    assert p.precision == 0 and p.zero_width_tchan == 0


def test_init_argument_errors_without_gpu(lib):
    from paper_2312_02898_b300 import binding
    p = binding.default_params()
    h = ctypes.c_void_p()
    assert lib.me_init(b"g g > t t~ q", ctypes.byref(p), ctypes.byref(h)) == binding.ME_ERR_ARG
    assert h.value is None
    assert b"unknown process" in lib.me_last_error(None)
    assert lib.me_init(None, ctypes.byref(p), ctypes.byref(h)) == binding.ME_ERR_ARG
    bad = binding.default_params()
    bad.mt = -1.0
    assert lib.me_init(b"g g > t t~", ctypes.byref(bad), ctypes.byref(h)) == binding.ME_ERR_ARG
    bad = binding.default_params()
    bad.precision = 7
    assert lib.me_init(b"g g > t t~", ctypes.byref(bad), ctypes.byref(h)) == binding.ME_ERR_ARG


def test_compute_argument_errors_without_gpu(lib):
    from paper_2312_02898_b300 import binding
    assert lib.me_compute(None, 10, None, None, None, None, None, None, None, None) == binding.ME_ERR_ARG
    assert lib.me_compute_host(None, 10, None, None, None, None, None, None, None, None) == binding.ME_ERR_ARG
    assert lib.me_info(None, None, None, None, None, None) == binding.ME_ERR_ARG
    assert lib.me_flops(None, None, None) == binding.ME_ERR_ARG
    assert lib.me_set_config(None, 0) == binding.ME_ERR_ARG
    lib.me_free(None)  # no-op


def test_product_has_no_cpu_path():
    # the product package never imports the oracle and has no fallback implementation
    pkg = os.path.join(ROOT, "paper_2312_02898_b300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "me_oracle" not in txt, f
