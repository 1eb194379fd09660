"""The C-ABI library loads on a machine without a GPU and exports every entry
point include/tdk.h declares; host-side argument checks need no GPU."""
import ctypes
import os
import re

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _declared_functions():
    names = []
    for fname in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fname.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fname)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", text, flags=re.M):
            name = m.group(1)
            if name not in ("if", "while", "sizeof") and not name.startswith("TDK"):
                names.append(name)
    return sorted(set(names))


@pytest.fixture(scope="module")
def L():
    import paper_1412_1885_gb300 as t
    from paper_1412_1885_gb300 import build

    build.build()
    return t.lib()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for must in ("tucker_sketch", "tucker_core", "ffcp_als", "tdk_ctx_create", "tdk_ctx_destroy"):
        assert must in names, names


def test_library_exports_every_declared_symbol(L):
    for name in _declared_functions():
        assert hasattr(L, name), name


def test_test_hooks_live_only_in_the_test_build(L):
    """The product library exports no test hook; libtdk_test.so, the same
    sources built with -DTDK_TESTING, exports them and every public symbol."""
    import paper_1412_1885_gb300 as t

    for name in t.TEST_EXPORTS:
        assert not hasattr(L, name), name
    T = t.lib_test()
    for name in t.TEST_EXPORTS + _declared_functions():
        assert hasattr(T, name), name


def test_python_binding_names_match_header():
    import paper_1412_1885_gb300 as t

    assert set(t.EXPORTS) <= set(_declared_functions())


def test_strerror_and_argument_checks_without_gpu(L):
    import paper_1412_1885_gb300 as t

    assert t.strerror(t.TDK_EINVAL).startswith("invalid")
    assert t.strerror(t.TDK_WRANKDEF).startswith("warning")
    # null context / descriptor are rejected before any CUDA call
    assert L.tucker_sketch(None, None, None, None, None, None, None) == t.TDK_EINVAL
    assert L.tucker_core(None, None, None, None, None, None) == t.TDK_EINVAL
    assert L.ffcp_als(None, None, None, None, None, None, None, None, None, None) == t.TDK_EINVAL
    assert L.tdk_ctx_create(None, 0, None) == t.TDK_EINVAL


def test_struct_layouts_match_header():
    import paper_1412_1885_gb300 as t

    # int N, dtype, prec, p; int64 I[8]; int R[8]; uint64 seed
    assert ctypes.sizeof(t.TuckerDesc) == 16 + 64 + 32 + 8
    assert t.TuckerDesc.seed.offset == 112
    # int R, max_sweeps; double tol; int nonneg, init, check_every, form; double timeout_s, l1
    assert ctypes.sizeof(t.AlsOpts) == 4 + 4 + 8 + 4 * 4 + 8 + 8
    # int sweeps, status; double fit_core, fit_Y, ms; int form, grid
    assert ctypes.sizeof(t.AlsReport) == 4 + 4 + 8 * 3 + 4 + 4


def test_desc_validation_rules():
    import paper_1412_1885_gb300 as t

    d = t.make_desc((10, 12, 14), t.F32, (3, 3, 3), 2)
    assert d.N == 3 and d.I[2] == 14 and d.R[1] == 3
    with pytest.raises(ValueError):
        t.make_desc((10, 12), t.F32, (3, 3, 3), 2)


def test_descriptor_edge_cases_without_gpu(L):
    """The descriptor rules every entry point applies before any CUDA call:
    empty modes, ranks beyond the mode or the sketch-width limit, negative
    oversampling, unknown types, orders outside 2..8, element-count overflow."""
    import paper_1412_1885_gb300 as t

    ok, bad = t.TDK_OK, t.TDK_EINVAL
    chk = t.tucker_check
    assert chk((10, 12, 14), t.F32, (3, 3, 3), 2) == ok
    assert chk((5, 7), t.F64, (2, 3), 1) == ok                       # matrices (N = 2)
    assert chk((3,) * 8, t.F32, (1,) * 8, 2) == ok                    # 8 modes, Rt = I
    assert chk((70, 64, 80), t.BF16, (60, 60, 60), 4) == ok           # Rt = 64, the limit
    assert chk((70, 64, 80), t.BF16, (60, 61, 60), 4) == bad          # Rt = 65
    assert chk((10, 0, 14), t.F32, (3, 3, 3), 2) == bad               # empty mode
    assert chk((10, 12, 14), t.F32, (3, 0, 3), 2) == bad              # zero rank
    assert chk((10, 12, 4), t.F32, (3, 3, 3), 2) == bad               # Rt > I
    assert chk((10, 12, 14), t.F32, (3, 3, 3), -1) == bad             # p < 0
    assert chk((10,), t.F32, (3,), 2) == bad                          # N = 1
    assert chk((10, 12, 14), 7, (3, 3, 3), 2) == bad                  # dtype
    assert chk((10, 12, 14), t.F32, (3, 3, 3), 2, prec=5) == bad      # form
    assert chk((1 << 21,) * 3, t.F32, (3, 3, 3), 2) == bad            # 2^63 elements
