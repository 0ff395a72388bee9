"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every entry point include/chfsi.h declares, and rejects bad arguments on the
host before anything is queued."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2110_15853_gb300 import build
    build.build()
    import paper_2110_15853_gb300 as P
    return P.load()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "chfsi.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(chfsi_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["chfsi_filter", "chfsi_filter_backward", "chfsi_rayleigh_ritz", "chfsi_lanczos_bounds"]:
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2110_15853_gb300 import _abi
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in _abi.SIGNATURES, f"{name} has no ctypes signature"


def test_binding_constants_match_the_header():
    """Every integer #define CHFSI_* of include/chfsi.h has the same value in the
    binding (status codes, layouts, precisions, product flags)."""
    from paper_2110_15853_gb300 import _abi
    text = open(os.path.join(ROOT, "include", "chfsi.h")).read()
    defs = dict(re.findall(r"^#define (CHFSI_[A-Z0-9_]+) (\d+)", text, flags=re.M))
    assert len(defs) >= 24 and "CHFSI_F40_OZAKI" in defs
    for name, value in defs.items():
        assert getattr(_abi, name) == int(value), name


def test_status_strings(lib):
    assert lib.chfsi_version() >= 10000
    for code in range(10):
        s = lib.chfsi_status_string(code)
        assert s and s != b"unknown status"
    assert lib.chfsi_status_string(99) == b"unknown status"


def _csr_desc(N=8, nnz=8):
    from paper_2110_15853_gb300 import _abi
    m = _abi.chfsi_matrix()
    m.kind = _abi.CHFSI_CSR
    # fake (never dereferenced) device pointers: host validation only
    m.csr = _abi.chfsi_csr(N, nnz, 0x1000, 0x2000, 0x3000)
    return m


def test_workspace_sizes_are_host_arithmetic(lib):
    from paper_2110_15853_gb300 import _abi
    desc = _csr_desc(1000, 5000)
    sz = ctypes.c_size_t()
    assert lib.chfsi_filter_workspace_size(ctypes.byref(desc), 64, 10, None, ctypes.byref(sz)) == 0
    ldw = 64
    assert sz.value >= 2 * 1000 * ldw * 8
    # m = 1 needs no iterate buffers
    assert lib.chfsi_filter_workspace_size(ctypes.byref(desc), 64, 1, None, ctypes.byref(sz)) == 0
    assert sz.value <= 4096
    # a mixed schedule adds FP32 iterates and an FP32 copy of H
    prec = (ctypes.c_int32 * 10)(*([_abi.CHFSI_F32] * 6 + [_abi.CHFSI_F64] * 4))
    sch = _abi.chfsi_schedule(10, ctypes.cast(prec, ctypes.POINTER(ctypes.c_int32)))
    sz2 = ctypes.c_size_t()
    assert lib.chfsi_filter_workspace_size(ctypes.byref(desc), 64, 10, ctypes.byref(sch), ctypes.byref(sz2)) == 0
    assert sz2.value >= 2 * 1000 * 64 * 8 + 3 * 1000 * 64 * 4 + 5000 * 4
    # a low-precision step after an FP64 step is rejected
    bad = (ctypes.c_int32 * 10)(*([_abi.CHFSI_F64] + [_abi.CHFSI_F32] * 9))
    schb = _abi.chfsi_schedule(10, ctypes.cast(bad, ctypes.POINTER(ctypes.c_int32)))
    assert lib.chfsi_filter_workspace_size(ctypes.byref(desc), 64, 10, ctypes.byref(schb),
                                           ctypes.byref(sz2)) == _abi.CHFSI_ERR_ARG
    assert lib.chfsi_filter_backward_workspace_size(ctypes.byref(desc), 64, 16, 0, ctypes.byref(sz)) == 0


def test_workspace_is_sized_for_one_column_slab(lib):
    """A CSR filter (and its adjoint) over more than 512 states runs in 512-state
    column slabs, so its workspace does not grow with n beyond one slab; a BSR
    operator keeps the full width (the tensor-core step's copy is block-major)."""
    from paper_2110_15853_gb300 import _abi
    desc = _csr_desc(1000, 5000)
    sizes = {}
    for n in (512, 513, 2000, 6000):
        sz = ctypes.c_size_t()
        assert lib.chfsi_filter_workspace_size(ctypes.byref(desc), n, 10, None, ctypes.byref(sz)) == 0
        sizes[n] = sz.value
    assert sizes[513] == sizes[2000] == sizes[6000] == sizes[512]
    assert sizes[512] >= 2 * 1000 * 512 * 8
    bw = []
    for n in (512, 4096):
        sz = ctypes.c_size_t()
        assert lib.chfsi_filter_backward_workspace_size(ctypes.byref(desc), n, 16, 0, ctypes.byref(sz)) == 0
        bw.append(sz.value)
    assert bw[0] == bw[1]
    b = _abi.chfsi_matrix()
    b.kind = _abi.CHFSI_BSR
    b.bsr = _abi.chfsi_bsr(16, 40, 64, 0x1000, 0x2000, 0x3000)    # N = 1024
    s1, s2 = ctypes.c_size_t(), ctypes.c_size_t()
    assert lib.chfsi_filter_workspace_size(ctypes.byref(b), 512, 10, None, ctypes.byref(s1)) == 0
    assert lib.chfsi_filter_workspace_size(ctypes.byref(b), 2048, 10, None, ctypes.byref(s2)) == 0
    assert s2.value >= 2 * 1024 * 2048 * 8 > s1.value


def test_host_validation_rejects_before_queueing(lib):
    from paper_2110_15853_gb300 import _abi
    desc = _csr_desc()
    ws = 0x10000
    # bounds: a0 < a < b required
    rc = lib.chfsi_filter(ctypes.byref(desc), 0x4000, 4, 0x8000, 4, 4, 3, 1.0, 2.0, 1.5, None, ws, 1 << 20, None)
    assert rc == _abi.CHFSI_ERR_BOUNDS
    rc = lib.chfsi_filter(ctypes.byref(desc), 0x4000, 4, 0x8000, 4, 4, 3, 1.0, float("nan"), 0.0, None, ws, 1 << 20,
                          None)
    assert rc == _abi.CHFSI_ERR_BOUNDS
    # degree m >= 1
    rc = lib.chfsi_filter(ctypes.byref(desc), 0x4000, 4, 0x8000, 4, 4, 0, 1.0, 2.0, 0.0, None, ws, 1 << 20, None)
    assert rc == _abi.CHFSI_ERR_ARG
    # NULL / misaligned blocks, ld < n, aliasing
    rc = lib.chfsi_filter(ctypes.byref(desc), None, 4, 0x8000, 4, 4, 3, 1.0, 2.0, 0.0, None, ws, 1 << 20, None)
    assert rc == _abi.CHFSI_ERR_ARG
    rc = lib.chfsi_filter(ctypes.byref(desc), 0x4008, 4, 0x8000, 4, 4, 3, 1.0, 2.0, 0.0, None, ws, 1 << 20, None)
    assert rc == _abi.CHFSI_ERR_ARG
    rc = lib.chfsi_filter(ctypes.byref(desc), 0x4000, 2, 0x8000, 4, 4, 3, 1.0, 2.0, 0.0, None, ws, 1 << 20, None)
    assert rc == _abi.CHFSI_ERR_ARG
    rc = lib.chfsi_filter(ctypes.byref(desc), 0x4000, 4, 0x4000, 4, 4, 3, 1.0, 2.0, 0.0, None, ws, 1 << 20, None)
    assert rc == _abi.CHFSI_ERR_ARG
    # workspace too small
    rc = lib.chfsi_filter(ctypes.byref(desc), 0x4000, 4, 0x8000, 4, 4, 3, 1.0, 2.0, 0.0, None, ws, 16, None)
    assert rc == _abi.CHFSI_ERR_NOMEM
    # malformed descriptors
    bad = _csr_desc(0, 8)
    rc = lib.chfsi_filter(ctypes.byref(bad), 0x4000, 4, 0x8000, 4, 4, 3, 1.0, 2.0, 0.0, None, ws, 1 << 20, None)
    assert rc == _abi.CHFSI_ERR_ARG
    m = _abi.chfsi_matrix()
    m.kind = 7
    assert lib.chfsi_filter(ctypes.byref(m), 0x4000, 4, 0x8000, 4, 4, 3, 1.0, 2.0, 0.0, None, ws, 1 << 20,
                            None) == _abi.CHFSI_ERR_ARG
    b = _abi.chfsi_matrix()
    b.kind = _abi.CHFSI_BSR
    b.bsr = _abi.chfsi_bsr(2, 4, 32, 0x1000, 0x2000, 0x3000)      # bdim must be 64
    assert lib.chfsi_filter(ctypes.byref(b), 0x4000, 4, 0x8000, 4, 4, 3, 1.0, 2.0, 0.0, None, ws, 1 << 20,
                            None) == _abi.CHFSI_ERR_ARG
    # the backward pass and the Lanczos bounds take CSR only
    b.bsr.bdim = 64
    sz = ctypes.c_size_t()
    assert lib.chfsi_filter_backward_workspace_size(ctypes.byref(b), 4, 3, 0, ctypes.byref(sz)) == \
        _abi.CHFSI_ERR_UNSUPPORTED
    assert lib.chfsi_lanczos_workspace_size(ctypes.byref(b), 20, ctypes.byref(sz)) == _abi.CHFSI_ERR_UNSUPPORTED
    # Lanczos: n_wanted must be in [1, N)
    a_, b_, c_ = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    assert lib.chfsi_lanczos_bounds(ctypes.byref(desc), 20, 0x4000, 8, ctypes.byref(a_), ctypes.byref(b_),
                                    ctypes.byref(c_), ws, 1 << 20, None) == _abi.CHFSI_ERR_ARG


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    import paper_2110_15853_gb300._abi as abi
    monkeypatch.setattr(abi, "_lib", None)
    monkeypatch.setattr(abi, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(ImportError):
        abi.load()


def test_ozaki_schedules_validated_on_host(lib):
    """Filter schedules with 40-bit Ozaki steps (CHFSI_F40_OZAKI): they join the Ozaki
    tail in any order with FP64-accurate Ozaki steps, after an optional low-precision
    prefix, and need the same workspace; they mix neither with plain FP64 steps nor with
    a later low-precision step, and need 64 x 64 blocks."""
    from paper_2110_15853_gb300 import _abi
    F40, OZ, F64, F32 = _abi.CHFSI_F40_OZAKI, _abi.CHFSI_F64_OZAKI, _abi.CHFSI_F64, _abi.CHFSI_F32
    b = _abi.chfsi_matrix()
    b.kind = _abi.CHFSI_BSR
    b.bsr = _abi.chfsi_bsr(16, 40, 64, 0x1000, 0x2000, 0x3000)    # N = 1024

    def size(desc, steps):
        prec = (ctypes.c_int32 * len(steps))(*steps)
        sch = _abi.chfsi_schedule(len(steps), ctypes.cast(prec, ctypes.POINTER(ctypes.c_int32)))
        sz = ctypes.c_size_t()
        rc = lib.chfsi_filter_workspace_size(ctypes.byref(desc), 200, len(steps), ctypes.byref(sch),
                                             ctypes.byref(sz))
        return rc, sz.value

    rc, full = size(b, [OZ] * 10)
    assert rc == 0
    for steps in ([F40] * 6 + [OZ] * 4, [F40] * 10, [OZ] * 5 + [F40] * 5, [OZ, F40] * 5):
        assert size(b, steps) == (0, full)
    assert size(b, [F32] * 3 + [F40] * 5 + [OZ] * 2)[0] == 0
    for steps in ([F40] * 5 + [F64] * 5, [F64] * 5 + [F40] * 5, [F40] * 3 + [F32] * 7):
        assert size(b, steps)[0] == _abi.CHFSI_ERR_ARG
    assert size(_csr_desc(1000, 5000), [F40] * 4)[0] == _abi.CHFSI_ERR_UNSUPPORTED
