"""Host-side checks of the C ABI: the CUDA library builds for sm_103a,
loads, and exports every function that include/steiner.h declares; the
Python binding binds exactly those names.  No compute call (no GPU here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "steiner.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(steiner_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2205_14503_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["steiner_load_graph", "steiner_query", "steiner_query_batch",
                     "steiner_submit", "steiner_poll", "steiner_voronoi", "steiner_free_graph",
                     "steiner_result_free"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, f"not exported: {missing}"


def test_binding_covers_the_header(lib):
    from paper_2205_14503_gb300 import steiner
    assert sorted(steiner.SIGNATURES) == declared_functions()
    steiner.load_library()
    assert steiner.steiner_version().startswith("gb300-steiner")


def test_binding_fails_loudly_without_the_library(tmp_path):
    from paper_2205_14503_gb300 import steiner
    saved = steiner._lib
    steiner._lib = None
    try:
        with pytest.raises(RuntimeError, match="not built"):
            steiner.load_library(str(tmp_path / "missing.so"))
    finally:
        steiner._lib = saved


def test_status_codes_match_header():
    from paper_2205_14503_gb300 import steiner
    text = open(HEADER).read()
    for name, val in re.findall(r"#define (STEINER_[A-Z]+)\s+(-?\d+)", text):
        assert getattr(steiner, name) == int(val)


def test_kernels_compile_for_sm103a():
    """Every kernel source compiles with -gencode arch=compute_103a,code=sm_103a."""
    from paper_2205_14503_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in build.ARCH
    assert os.path.exists(build.build())


def test_autotune_fingerprint_is_stable_and_sensitive():
    import paper_2205_14503_gb300.workloads as wl
    from paper_2205_14503_gb300 import autotune
    a = wl.grid(50, 40, 100, seed=1)
    b = wl.grid(50, 40, 100, seed=1)
    c = wl.grid(50, 40, 100, seed=2)
    assert autotune.fingerprint(a) == autotune.fingerprint(b)
    assert autotune.fingerprint(a) != autotune.fingerprint(c)
