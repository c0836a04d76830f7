"""CPU checks of the C ABI: the library builds, loads and exports every symbol
include/cls.h declares; the product package never reaches the oracle."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    with open(os.path.join(ROOT, "include", "cls.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cls_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    from paper_1708_00765_gb300 import _native, build
    build.build()
    lib = _native.load()
    names = declared_symbols()
    assert len(names) >= 16
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(_native.EXPORTED)


def test_strerror_names_every_code():
    from paper_1708_00765_gb300 import _native
    for code in range(0, -7, -1):
        assert _native.strerror(code) != "unknown error"
    assert _native.strerror(-99) == "unknown error"


def test_no_device_is_an_error_not_a_fallback():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_1708_00765_gb300 as cls
    with pytest.raises(cls.ClsError) as e:
        cls.Problem([0.5, 5, 2, 0.5, 0.5, 0.9, 10, 1, 100])
    assert e.value.code == cls._native.CLS_E_NODEVICE


def test_product_package_does_not_use_the_oracle():
    pkg = os.path.join(ROOT, "paper_1708_00765_gb300")
    for dirpath, _, files in os.walk(pkg):
        if "_build" in dirpath:
            continue
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                with open(os.path.join(dirpath, f)) as fh:
                    src = fh.read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", src, re.M), f
                assert "cls_oracle" not in src, f


def test_workload_generator_is_deterministic():
    from paper_1708_00765_gb300 import workloads
    a = workloads.batch_sweep(256, seed=7)
    b = workloads.batch_sweep(256, seed=7)
    assert (a == b).all()
    assert set(a[:, 7]) <= {1.0, 3.0} and set(a[:, 6]) <= {0.1, 1.0, 10.0}
    assert a[:, 0:2].min() >= 0.02 and a[:, 0:2].max() <= 10
    assert a[:, 2:4].min() >= 0.05 and a[:, 2:4].max() <= 10


def test_binding_constants_equal_the_header():
    """Every CLS_* value the Python binding uses is the one include/cls.h defines, and
    every ctypes signature has the declared number of parameters."""
    from paper_1708_00765_gb300 import _native
    with open(os.path.join(ROOT, "include", "cls.h")) as f:
        text = f.read()
    defines = {m.group(1): int(m.group(2)) for m in
               re.finditer(r"#define\s+(CLS_[A-Z0-9_]+)\s+\(?(-?\d+)\)?", text)}
    bound = {k: v for k, v in vars(_native).items() if k.startswith("CLS_") and isinstance(v, int)}
    assert len(bound) >= 30
    for k, v in bound.items():
        assert k in defines, k
        assert defines[k] == v, k
    code = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    lib = _native.load()
    for m in re.finditer(r"\b(cls_[a-z_]+)\s*\(([^)]*)\)\s*;", code):
        params = [p for p in m.group(2).split(",") if p.strip() and p.strip() != "void"]
        fn = getattr(lib, m.group(1))
        assert len(fn.argtypes) == len(params), m.group(1)
