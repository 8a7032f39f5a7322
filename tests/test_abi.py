"""The C ABI: libcholqr.so builds, loads without a GPU, exports every function
include/cholqr.h declares, and rejects bad arguments before touching CUDA."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cholqr.h")


def header_functions(path=HEADER):
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    # a declaration: type, then whitespace or '*', then the name and '(' (a
    # function-pointer member such as "int (*f)(...)" is not one)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_]\w*(?:\s+|\s*\*+\s*)([A-Za-z_]\w*)\s*\(", text, flags=re.M)
    return [n for n in names if n not in ("if", "while", "defined")]


@pytest.fixture(scope="module")
def cq():
    import paper_2507_07788_gb300 as cq
    from paper_2507_07788_gb300 import _build
    _build.build()
    return cq


def test_header_parses():
    names = header_functions()
    for must in ("cholqr_factor", "basis_create", "basis_append", "basis_free"):
        assert must in names


def test_every_declared_symbol_is_exported(cq):
    L = C.CDLL(cq.LIB_PATH)
    for name in header_functions():
        assert hasattr(L, name), name


def test_binding_covers_header(cq):
    assert set(header_functions()) == set(cq.exported_symbols())


def test_default_opts_and_status_strings(cq):
    o = cq.default_opts()
    assert o.tol == 1e-13 and o.max_iter == 10 and o.update_min_iter == 2
    assert o.shift_policy == cq.SHIFT_SCHOLQR3 and o.precision == cq.PREC_FP64
    assert cq.status_string(cq.OK) == "ok"
    assert "breakdown" in cq.status_string(cq.ERR_BREAKDOWN).lower()


@pytest.mark.parametrize("m,n,lda,ldq,ldr", [
    (10, 0, 10, 10, 1),      # n = 0
    (3, 5, 3, 3, 5),         # m < n
    (10, 4, 9, 10, 4),       # lda < m
    (10, 4, 10, 9, 4),       # ldq < m
    (10, 4, 10, 10, 3),      # ldr < n
    (1000, 513, 1000, 1000, 513),  # n > CQR_MAX_N
])
def test_factor_rejects_bad_sizes_without_gpu(cq, m, n, lda, ldq, ldr):
    fake = C.c_void_p(0x1000)
    info = cq.Info()
    st = cq.cholqr_factor(None, m, n, fake, lda, C.c_void_p(0x2000000), ldq, C.c_void_p(0x3000000),
                          ldr, C.byref(info), None)
    assert st == cq.ERR_INVALID


def test_factor_rejects_null_and_bad_opts(cq):
    st = cq.cholqr_factor(None, 10, 2, None, 10, C.c_void_p(0x1000), 10, C.c_void_p(0x2000), 2, None, None)
    assert st == cq.ERR_INVALID
    bad = cq.default_opts(max_iter=0)
    st = cq.cholqr_factor(C.byref(bad), 10, 2, C.c_void_p(0x1000), 10, C.c_void_p(0x9000), 10,
                          C.c_void_p(0x20000), 2, None, None)
    assert st == cq.ERR_INVALID
    bad = cq.default_opts(shift_policy=7)
    st = cq.cholqr_factor(C.byref(bad), 10, 2, C.c_void_p(0x1000), 10, C.c_void_p(0x9000), 10,
                          C.c_void_p(0x20000), 2, None, None)
    assert st == cq.ERR_INVALID


def test_factor_rejects_partial_overlap(cq):
    # Q starts inside A but is not A itself
    base = 0x100000
    st = cq.cholqr_factor(None, 100, 4, C.c_void_p(base), 100, C.c_void_p(base + 8 * 50), 100,
                          C.c_void_p(0x900000), 4, None, None)
    assert st == cq.ERR_INVALID
    # in place with different leading dimensions
    st = cq.cholqr_factor(None, 100, 4, C.c_void_p(base), 100, C.c_void_p(base), 101,
                          C.c_void_p(0x900000), 4, None, None)
    assert st == cq.ERR_INVALID


def test_factor_host_rejects_overlap_without_gpu(cq):
    # the host entry point writes Q while its input copy may still read A
    base = 0x100000
    for qoff, ldq in ((0, 100), (8 * 50, 100)):
        st = cq.cholqr_factor_host(None, 100, 4, C.c_void_p(base), 100, C.c_void_p(base + qoff), ldq,
                                   C.c_void_p(0x900000), 4, None, None)
        assert st == cq.ERR_INVALID


@pytest.mark.parametrize("m,n,r,lda,ldq,ldr", [
    (100, 8, 0, 100, 100, 8),       # r = 0
    (100, 8, 9, 100, 100, 8),       # r > n
    (2000, 1000, 1, 2000, 2000, 1000),  # panel of 1000 columns > CQR_MAX_N
    (5, 8, 2, 5, 5, 8),             # m < n
    (100, 8, 2, 99, 100, 8),        # lda < m
    (100, 8, 2, 100, 100, 7),       # ldr < n
    (5000, 1100, 10, 5000, 5000, 1100),  # n > CQR_MAX_BASIS
])
def test_pn_rejects_bad_sizes_without_gpu(cq, m, n, r, lda, ldq, ldr):
    st = cq.lib().cholqr_pn(None, m, n, r, C.c_void_p(0x1000), lda, C.c_void_p(0x20000000), ldq,
                            C.c_void_p(0x30000000), ldr, None, None)
    assert st == cq.ERR_INVALID


def test_pn_rejects_overlap_without_gpu(cq):
    base = 0x100000
    st = cq.lib().cholqr_pn(None, 100, 4, 2, C.c_void_p(base), 100, C.c_void_p(base), 100,
                            C.c_void_p(0x900000), 4, None, None)
    assert st == cq.ERR_INVALID


def test_basis_null_handles(cq):
    L = cq.lib()
    assert L.basis_free(None) == cq.OK
    assert L.basis_cols(None) == -1
    assert L.basis_append(None, 4, C.c_void_p(0x1000), 10, None, None) == cq.ERR_INVALID
    h = C.c_void_p()
    assert L.basis_create(0, 4, None, None, C.byref(h)) == cq.ERR_INVALID
    assert L.basis_create(10, 0, None, None, C.byref(h)) == cq.ERR_INVALID
    assert L.basis_create(10, cq.MAX_BASIS + 1, None, None, C.byref(h)) == cq.ERR_INVALID
    assert L.basis_create(10, 4, None, None, None) == cq.ERR_INVALID


def test_product_path_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_2507_07788_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src, f
                assert "cholqr_oracle" not in src, f
