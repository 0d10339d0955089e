"""C-ABI checks that need no GPU: the library builds, loads, exports every
symbol include/rqlp.h declares, and rejects invalid arguments before any
device work."""
import ctypes
import os
import re

import pytest

from paper_2110_01011_gb300 import build, rqlp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(rqlp_\w+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def lib():
    build.build()
    return rqlp.load()


def test_exports_every_declared_symbol(lib):
    declared = _declared_symbols()
    assert declared, "no declarations found"
    for name in sorted(declared):
        assert hasattr(lib, name), name
    assert declared == set(rqlp.EXPORTED)


def test_host_only_calls(lib):
    assert rqlp.rqlp_version() >= 100
    assert rqlp.rqlp_status_string(0) == "ok"
    assert "breakdown" in rqlp.rqlp_status_string(3).lower()
    o = rqlp.rqlp_default_opts()
    assert o.precision == rqlp.PREC_FP32 and o.small_fp64 == 0
    assert o.test_stall == 0 and o.bf16_parts == 0 and o.literal_step5 == 0 and o.fused_power == 0
    assert list(o.reserved) == [0] * 2


@pytest.mark.parametrize("m,n,k,p,q", [(0, 10, 1, 0, 0), (10, 10, 0, 1, 0), (10, 10, 8, 3, 0),
                                       (300, 300, 250, 10, 0), (10, 10, 2, -1, 0),
                                       (10, 10, 2, 1, -1)])
def test_workspace_rejects_bad_sizes(lib, m, n, k, p, q):
    assert rqlp.rqlp_workspace_bytes(m, n, k, p, q) == 0


def test_workspace_grows_with_size(lib):
    a = rqlp.rqlp_workspace_bytes(1000, 1000, 20, 5, 1)
    b = rqlp.rqlp_workspace_bytes(4000, 2000, 20, 5, 1)
    assert 0 < a < b
    assert rqlp.rqlp_host_workspace_bytes(1000, 1000, 20, 5, 1) > a + 4 * 1000 * 1000


def test_bad_opts_rejected(lib):
    o = rqlp.rqlp_default_opts()
    o.reserved[0] = 1
    assert rqlp.rqlp_workspace_bytes(100, 100, 5, 5, 0, o) == 0
    o = rqlp.rqlp_default_opts()
    o.test_stall = 1                 # the fault-injection hook belongs to the batched form only
    assert rqlp.rqlp_workspace_bytes(100, 100, 5, 5, 0, o) == 0
    o = rqlp.rqlp_default_opts()
    o.precision = 7
    assert rqlp.rqlp_workspace_bytes(100, 100, 5, 5, 0, o) == 0
    o = rqlp.rqlp_default_opts()
    o.bf16_parts = 3                 # BF16 parts belong to the BF16X3 form only
    assert rqlp.rqlp_workspace_bytes(100, 100, 5, 5, 0, o) == 0
    o.precision = rqlp.PREC_BF16X3
    for parts, ok in ((0, True), (1, False), (2, True), (3, True), (4, False)):
        o.bf16_parts = parts
        assert (rqlp.rqlp_workspace_bytes(100, 100, 5, 5, 0, o) > 0) == ok, parts
    o = rqlp.rqlp_default_opts()
    o.fused_power = 2
    assert rqlp.rqlp_workspace_bytes(100, 100, 5, 5, 0, o) == 0
    o.fused_power = 1
    assert rqlp.rqlp_workspace_bytes(100, 100, 5, 5, 2, o) > 0
    o = rqlp.rqlp_default_opts()
    o.literal_step5 = 2
    assert rqlp.rqlp_workspace_bytes(100, 100, 5, 5, 0, o) == 0
    o.literal_step5 = 1
    assert rqlp.rqlp_workspace_bytes(100, 100, 5, 5, 0, o) > 0
    o = rqlp.rqlp_default_opts()
    o.precision = rqlp.PREC_BF16X3
    # the third part of A costs half as much workspace again as the two halves
    o.bf16_parts = 2
    two = rqlp.rqlp_workspace_bytes(1000, 1000, 5, 5, 0, o)
    o.bf16_parts = 3
    assert rqlp.rqlp_workspace_bytes(1000, 1000, 5, 5, 0, o) >= two + 2 * 1000 * 1024


def test_factor_argument_errors_without_device_work(lib):
    """Invalid sizes, strides and null pointers return RQLP_ERR_ARG before
    anything is enqueued (the fake pointers are never dereferenced)."""
    fake = 0x1000
    o = rqlp.rqlp_default_opts()
    base = dict(A=fake, m=100, n=80, lda=80, k=10, p=5, q=1, Omega=fake, ldo=15, Q=fake, ldq=15,
                L=fake, ldl=15, P=fake, ldp=15, workspace=fake, ws_bytes=1 << 30, d_info=fake,
                d_diag=None, opts=o, stream=None)

    def call(**kw):
        a = dict(base)
        a.update(kw)
        return rqlp.rqlp_factor(**a)

    assert call(lda=79) == 1          # lda < n
    assert call(ldo=14) == 1          # ldo < d
    assert call(A=None) == 1
    assert call(d_info=None) == 1
    assert call(k=0) == 1
    assert call(k=78, p=5) == 1       # d > min(m, n)
    assert call(ws_bytes=10) == 6     # workspace too small
    assert call(workspace=fake + 8) == 6   # misaligned


def test_sparse_workspace_rules(lib):
    """Sizing of the sparse path: the chain's workspace plus A^T in CSR form;
    FP32 only; invalid descriptors size to 0 (no device pointer is read)."""
    fake = 0x1000
    m, n, nnz = 1000, 800, 12000
    csr = rqlp.Csr(m, n, nnz, fake, fake, fake)
    o = rqlp.rqlp_default_opts()
    nb = rqlp.rqlp_sparse_workspace_bytes(csr, 20, 5, 1, o)
    dense = rqlp.rqlp_workspace_bytes(m, n, 20, 5, 1, o)
    assert nb >= dense + 8 * (n + 1) + 8 * nnz + 4 * n
    o.precision = rqlp.PREC_BF16X3
    assert rqlp.rqlp_sparse_workspace_bytes(csr, 20, 5, 1, o) == 0
    o = rqlp.rqlp_default_opts()
    assert rqlp.rqlp_sparse_workspace_bytes(rqlp.Csr(m, n, nnz, None, fake, fake), 20, 5, 1, o) == 0
    assert rqlp.rqlp_sparse_workspace_bytes(rqlp.Csr(0, n, nnz, fake, fake, fake), 20, 5, 1, o) == 0
    assert rqlp.rqlp_sparse_workspace_bytes(csr, 790, 20, 1, o) == 0     # d > min(m, n)
