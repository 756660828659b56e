"""The C ABI library loads on a machine without a GPU, exports every entry
point its header declares, and rejects bad arguments on the host (before any
CUDA call)."""
import ctypes
import os
import re

import pytest

from paper_2607_24959_b300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    if build.is_stale():
        build.build()
    return _lib.load()


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(cs_[a-z0-9_]+)\s*\(", txt))
    return names


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert {"cs_solve_fwd", "cs_solve_adjoint", "cs_solve_fused"} <= names
    raw = ctypes.CDLL(_lib.LIB_PATH)
    missing = [n for n in sorted(names) if not hasattr(raw, n)]
    assert not missing, missing
    unbound = [n for n in sorted(names) if n not in _lib._SIGS]
    assert not unbound, unbound


def test_struct_sizes_match_header(lib):
    assert ctypes.sizeof(_lib.CsBatch) == 96
    assert ctypes.sizeof(_lib.CsOptions) == 16
    assert ctypes.sizeof(_lib.CsState) == 40
    from paper_2607_24959_b300.workloads import INST_DTYPE
    assert INST_DTYPE.itemsize == 40


def _batch(**kw):
    b = _lib.CsBatch()
    b.n, b.nv_max, b.m_max = 4, 18, 128
    fake = 0x10000
    b.inst = b.M = b.J = b.qfrc = b.aref = b.D = fake
    b.total_M = b.total_J = b.total_v = b.total_r = 1000
    for k, v in kw.items():
        setattr(b, k, v)
    return b


def _opts(**kw):
    o = _lib.CsOptions()
    o.tol, o.max_iter, o.keep_factor, o.warps_per_block = 1e-8, 50, 1, 0
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _fused(lib, b, o, ws_bytes=256, ws=0x20000):
    f = 0x30000
    return lib.cs_solve_fused(ctypes.byref(b), ctypes.byref(o), f, None, f, f, f, f, f, f,
                              ws, ws_bytes, None)


def test_host_validation_codes(lib):
    assert _fused(lib, _batch(n=-1), _opts()) == _lib.CS_EINVAL
    assert _fused(lib, _batch(n=0), _opts()) == _lib.CS_OK        # no-op, no CUDA
    assert _fused(lib, _batch(nv_max=129), _opts()) == _lib.CS_EUNSUPPORTED
    # fits the CTA kernel's shared memory only up to about 45k words
    assert _fused(lib, _batch(nv_max=128, m_max=1024), _opts()) == _lib.CS_EUNSUPPORTED
    assert b"shared memory" in lib.cs_last_error()
    assert _fused(lib, _batch(nv_max=0), _opts()) == _lib.CS_EUNSUPPORTED
    assert _fused(lib, _batch(m_max=1025), _opts()) == _lib.CS_EUNSUPPORTED
    assert _fused(lib, _batch(M=None), _opts()) == _lib.CS_EINVAL
    assert _fused(lib, _batch(J=None), _opts()) == _lib.CS_EINVAL
    assert _fused(lib, _batch(total_J=-1), _opts()) == _lib.CS_EINVAL
    assert _fused(lib, _batch(), _opts(tol=-1.0)) == _lib.CS_EINVAL
    assert _fused(lib, _batch(), _opts(max_iter=-1)) == _lib.CS_EINVAL
    assert _fused(lib, _batch(), _opts(warps_per_block=9)) == _lib.CS_EINVAL
    assert _fused(lib, _batch(), _opts(), ws_bytes=8) == _lib.CS_EINVAL
    assert _fused(lib, _batch(), _opts(), ws=0x20004) == _lib.CS_EINVAL   # misaligned
    assert b"workspace" in lib.cs_last_error()
    assert lib.cs_solve_fwd(None, None, None, None, None) == _lib.CS_EINVAL
    o = _opts()
    b = _batch()
    assert lib.cs_solve_fwd(ctypes.byref(b), ctypes.byref(o), None, None, None) == _lib.CS_EINVAL
    assert lib.cs_solve_adjoint(ctypes.byref(b), ctypes.byref(o), None, None, None, None,
                                None, None, None) == _lib.CS_EINVAL


def test_strerror_and_version(lib):
    assert lib.cs_version() >= 100
    for code in (0, -1, -2, -3, -4, -5, -6, 1):
        assert lib.cs_strerror(code)
    assert lib.cs_strerror(-99) == b"unknown error code"


def test_python_layer_fails_loudly_without_library(tmp_path):
    saved = _lib._lib
    try:
        _lib._lib = None
        with pytest.raises(RuntimeError, match="no CPU fallback"):
            _lib.load(str(tmp_path / "missing.so"))
    finally:
        _lib._lib = saved


def test_serve_argument_checks_without_gpu(lib):
    h = ctypes.c_void_p(None)
    assert lib.cs_serve_create(None, ctypes.byref(h)) == _lib.CS_EINVAL
    c = _lib.CsServeConfig()
    c.arena_bytes, c.streams, c.max_batch, c.policy, c.max_iter = 1 << 30, 0, 16, 0, 50
    assert lib.cs_serve_create(ctypes.byref(c), ctypes.byref(h)) == _lib.CS_EINVAL
    c.streams = 4
    c.arena_bytes = 1 << 20                     # < 1 MiB per stream
    assert lib.cs_serve_create(ctypes.byref(c), ctypes.byref(h)) == _lib.CS_EINVAL
    c.arena_bytes, c.policy, c.fixed_batch = 1 << 30, 1, 0
    assert lib.cs_serve_create(ctypes.byref(c), ctypes.byref(h)) == _lib.CS_EINVAL
    t = ctypes.c_uint64(0)
    assert lib.cs_serve_submit(None, None, ctypes.byref(t)) == _lib.CS_EINVAL
    assert lib.cs_serve_poll(None, 1, None) == _lib.CS_EINVAL


def test_library_owned_state_without_gpu(lib):
    """The library-owned form of the adjoint state (cs_state_create,
    cs_solve_fwd_alloc, cs_state_status, cs_state_free): argument checks on
    the host, and the whole life cycle of an empty state, which needs no
    device memory."""
    P = ctypes.POINTER(_lib.CsState)
    st = P()
    b = _batch()
    assert lib.cs_state_create(ctypes.byref(b), 1, None) == _lib.CS_EINVAL
    assert lib.cs_state_create(None, 1, ctypes.byref(st)) == _lib.CS_EINVAL
    assert not st
    assert lib.cs_state_create(ctypes.byref(_batch(n=-1)), 1, ctypes.byref(st)) == _lib.CS_EINVAL
    assert lib.cs_state_create(ctypes.byref(b), 2, ctypes.byref(st)) == _lib.CS_EINVAL
    # a caller-built cs_state is not a library-owned one
    mine = _lib.CsState()
    assert lib.cs_state_status(ctypes.byref(mine), None, None, None) == _lib.CS_EINVAL
    assert b"cs_state_create" in lib.cs_last_error()
    lib.cs_state_free(ctypes.cast(ctypes.byref(mine), P))     # ignored
    lib.cs_state_free(None)                                   # ignored
    o = _opts()
    assert lib.cs_solve_fwd_alloc(ctypes.byref(b), ctypes.byref(o), None, None,
                                  None) == _lib.CS_EINVAL
    other = ctypes.cast(ctypes.byref(mine), P)
    assert lib.cs_solve_fwd_alloc(ctypes.byref(b), ctypes.byref(o), 0x30000, ctypes.byref(other),
                                  None) == _lib.CS_EINVAL
    # an empty batch: the state owns no device memory
    e = _batch(n=0, total_M=0, total_J=0, total_v=0, total_r=0)
    assert lib.cs_state_create(ctypes.byref(e), 0, ctypes.byref(st)) == _lib.CS_OK
    assert st and not st.contents.L
    assert lib.cs_state_status(st, None, None, None) == _lib.CS_OK
    lib.cs_state_free(st)
    # after cs_state_free the pointer is no longer a state of the library
    assert lib.cs_state_status(st, None, None, None) == _lib.CS_EINVAL


def test_cta_sized_comparator_and_round_cone_checks_without_gpu(lib):
    """The unrolled comparator and the round cone take CTA-sized batches
    (nv <= 128, m <= 1024) and refuse, on the host, the ones whose instance
    does not fit one CTA's shared memory; argument checks come first."""
    f = ctypes.c_void_p(0x30000)
    big = _batch(nv_max=128, m_max=1024)
    o = _opts()
    # unrolled forward: NULL outputs are refused before any size question
    assert lib.cs_unrolled_fwd(ctypes.byref(_batch(nv_max=96, m_max=64)), ctypes.byref(o),
                               None, None, None, None, None, None) == _lib.CS_EINVAL
    assert lib.cs_unrolled_fwd(ctypes.byref(big), ctypes.byref(o), f, f, f, f, f,
                               None) == _lib.CS_EUNSUPPORTED
    assert b"shared memory" in lib.cs_last_error()
    assert lib.cs_unrolled_fwd(ctypes.byref(_batch(m_max=1025)), ctypes.byref(o), f, f, f, f, f,
                               None) == _lib.CS_EUNSUPPORTED
    # round cone: the same size rule
    assert lib.cs_solve_fused_elliptic(ctypes.byref(big), ctypes.byref(o), f, f, None, f, f, f,
                                       f, f, f, f, f, f, ctypes.c_void_p(0x20000), 256,
                                       None) == _lib.CS_EUNSUPPORTED
    assert b"shared memory" in lib.cs_last_error()
    # the trace sizes are host arithmetic on the batch totals
    b = _batch(nv_max=96, m_max=64)
    assert lib.cs_unrolled_trace_floats(ctypes.byref(b), 5) == 5 * (1000 + 4 * 1000 + 2 * 4)
    assert lib.cs_unrolled_mask_bytes(ctypes.byref(b), 5) == 5 * 1000
