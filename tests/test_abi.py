"""The C-ABI library loads and exports every entry point of include/ddm.h.

Host-only checks: no call here launches GPU work.  Argument errors are
detected before any CUDA call, so they are checked on the CPU as well.
"""
import ctypes
import os
import re

import pytest

import paper_1309_3458_gb300 as ddm
from paper_1309_3458_gb300 import build as B

HEADER = os.path.join(B.INCLUDE, "ddm.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return ddm.lib()


def declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ddm_[a-z_0-9]+)\s*\(", text)))


def test_header_declarations_match_binding():
    assert declared() == sorted(ddm.SIGNATURES)


def test_every_symbol_exported(lib):
    for name in declared():
        assert hasattr(lib, name), name


def test_strerror(lib):
    for code in range(9):
        assert ddm.ddm_strerror(code)
    assert ddm.ddm_strerror(99) == "unknown error"


def test_argument_errors_without_gpu(lib):
    k = ctypes.c_uint64(0)
    assert lib.ddm_create(None, 0) == ddm.DDM_ERR_ARG
    assert lib.ddm_destroy(None) == ddm.DDM_OK
    assert lib.ddm_count(None, 1, None, None, 0, None, None, 0, 0, ctypes.byref(k), None) == ddm.DDM_ERR_ARG
    assert lib.ddm_match(None, 1, None, None, 0, None, None, 0, 0, None, 0, ctypes.byref(k), None) == ddm.DDM_ERR_ARG
    assert lib.ddm_build(None, 1, None, None, 0, None) == ddm.DDM_ERR_ARG
    assert lib.ddm_plan(None, None, None, 0, 0, None, None, None) == ddm.DDM_ERR_ARG
    assert lib.ddm_write(None, 0, 0, None, 0, None, None) == ddm.DDM_ERR_ARG
    e = ctypes.c_uint32(0)
    assert lib.ddm_chunk_end(None, 0, 0, ctypes.byref(e), None) == ddm.DDM_ERR_ARG
    assert lib.ddm_tree_shape(None, None, None, None) == ddm.DDM_ERR_ARG
    assert lib.ddm_tree_export(None, None, None, None, None) == ddm.DDM_ERR_ARG
    assert lib.ddm_debug_set_alloc_limit(None, 0) == ddm.DDM_ERR_ARG


def test_every_call_refuses_a_null_context_without_gpu(lib):
    """The remaining entry points check their context (and pointers) on the
    host before any CUDA call: DDM_ERR_ARG, no GPU needed."""
    k = ctypes.c_uint64(0)
    e = ctypes.c_uint32(0)
    A = ddm.DDM_ERR_ARG
    assert lib.ddm_match_range(None, 1, None, None, 0, None, None, 0, 0, 0, 0, None, 0,
                               ctypes.byref(k), None) == A
    assert lib.ddm_refit(None, None, None, None) == A
    assert lib.ddm_attach(None, None) == A
    assert lib.ddm_plan_async(None, None, None, 0, 0, None) == A
    assert lib.ddm_write_async(None, 0, 0, None, 0, None, None, None) == A
    assert lib.ddm_pair_offsets_async(None, None, 0, None, None) == A
    assert lib.ddm_match_moved(None, None, None, 0, None, 0, None, 0, ctypes.byref(k), None) == A
    assert lib.ddm_plan_stats(None, ctypes.byref(k)) == A
    assert lib.ddm_plan_order(None, None, None, None) == A
    assert lib.ddm_write_ordered(None, 0, 0, None, 0, ctypes.byref(k), None) == A
    assert lib.ddm_write_ordered_ids(None, 0, 0, None, 0, ctypes.byref(k), None) == A
    assert lib.ddm_chunk_end_ordered(None, 0, 0, ctypes.byref(e), None) == A
    assert lib.ddm_set_replay_budget(None, 0) == A
    assert lib.ddm_set_tuning(None, 0, 8, 1) == A
    assert lib.ddm_set_update_id_base(None, 5) == A
    assert lib.ddm_set_tiling(None, 32, 24) == A
    assert lib.ddm_debug_wait_timeout(None, 1, None) == A
    assert lib.ddm_batch_match(None, 1, 1, None, None, None, 0, None, None, None, 0, 0, None, 0,
                               None, ctypes.byref(k), None) == A
    assert lib.ddm_batch_match_async(None, 1, 1, None, None, None, 0, None, None, None, 0, 0, None,
                                     0, None, None, None, None) == A
    assert lib.ddm_scan_counts_noalloc(None, 0, None, None) == A
    assert lib.ddm_scan_counts_noalloc(None, ddm.DDM_NOALLOC_MAX_UPDATES + 1, None, None) == A


def test_create_reports_missing_device(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    assert lib.ddm_create(ctypes.byref(h), 0) == ddm.DDM_ERR_CUDA
    assert h.value is None


def test_product_path_does_not_import_oracle():
    # The binding, the kernels and the build script never load the oracle.
    pkg = os.path.dirname(ddm.__file__)
    pat = re.compile(r"^\s*(import\s+oracle|from\s+oracle\b)|libddm_oracle|ddm_oracle\.c|oracle_[a-z]+\(",
                     re.M)
    for root, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                assert not pat.search(open(os.path.join(root, f)).read()), f


def test_binding_rejects_host_and_mistyped_arrays():
    """The kernels read coordinates directly: the binding refuses pageable
    host tensors, wrong dtypes and mismatched shapes before any library call
    (no GPU needed)."""
    import torch
    lo = torch.zeros((2, 8), dtype=torch.float32)
    hi = torch.ones((2, 8), dtype=torch.float32)
    with pytest.raises(ValueError):
        ddm.ddm_count(0, lo, hi, lo, hi)                        # host memory
    with pytest.raises(TypeError):
        ddm.ddm_count(0, lo.double(), hi.double(), lo, hi)      # float64
    with pytest.raises(ValueError):
        ddm.ddm_count(0, lo, hi[:, :4], lo, hi)                 # shapes differ
    with pytest.raises(ValueError):
        ddm.ddm_count(0, lo, hi, lo[:1], hi[:1])                # d differs
    with pytest.raises(TypeError):
        ddm.ddm_write_ordered_ids(0, 0, 1, torch.zeros((4, 2), dtype=torch.int32))  # not 1-D
    with pytest.raises(TypeError):
        ddm.ddm_write_ordered_ids(0, 0, 1, torch.zeros(4, dtype=torch.int64))       # int64
    with pytest.raises(ValueError):
        ddm.ddm_write_ordered_ids(0, 0, 1, torch.zeros(4, dtype=torch.int32))       # host


class _FakeCuda:
    """Stands in for a CUDA tensor on `index` (no GPU needed): the binding's
    checks only read these attributes, and every check below fails before
    any pointer reaches the library."""

    def __init__(self, shape, dtype, index):
        import torch
        self.shape = torch.Size(shape)
        self.dtype = dtype
        self.is_cuda = True
        self.device = torch.device("cuda", index)

    def dim(self):
        return len(self.shape)

    def numel(self):
        n = 1
        for s in self.shape:
            n *= s
        return n

    def element_size(self):
        import torch
        return torch.empty(0, dtype=self.dtype).element_size()

    def is_contiguous(self):
        return True

    def data_ptr(self):
        return 0


class _NoLibrary:
    """Takes the library's place: any call into it fails the test."""

    def __getattr__(self, name):
        raise AssertionError(f"{name} was called although a check should have failed")


def test_binding_rejects_tensors_on_another_device(monkeypatch):
    """A context lives on one GPU; its kernels would dereference a peer GPU's
    pointer.  The binding records each context's device and refuses tensors
    on any other one before calling the library (no GPU needed: fake handles
    and tensors)."""
    import torch
    fake_ctx = 0x5151
    monkeypatch.setitem(ddm._CTX_DEVICE, fake_ctx, 0)
    monkeypatch.setattr(ddm, "_lib", _NoLibrary())
    f32 = torch.float32
    on0 = _FakeCuda((2, 8), f32, 0)
    on1 = _FakeCuda((2, 8), f32, 1)
    with pytest.raises(ValueError, match="cuda:1"):
        ddm.ddm_count(fake_ctx, on1, on1, on1, on1)
    with pytest.raises(ValueError, match="cuda:1"):
        ddm.ddm_build(fake_ctx, on1, on1)
    with pytest.raises(ValueError, match="cuda:1"):
        ddm.ddm_plan(fake_ctx, on1, on1)
    with pytest.raises(ValueError, match="cuda:1"):  # sets fine, pair buffer elsewhere
        ddm.ddm_match(fake_ctx, on0, on0, on0, on0, _FakeCuda((16, 2), torch.int32, 1))
    with pytest.raises(ValueError, match="cuda:1"):
        ddm.ddm_write_ordered_ids(fake_ctx, 0, 1, _FakeCuda((16,), torch.int32, 1))
    with pytest.raises(ValueError, match="cuda:1"):
        ddm.ddm_plan_order(fake_ctx, _FakeCuda((8,), torch.int32, 1))
    # the allocation-free scan runs on the current device
    monkeypatch.setattr(torch.cuda, "current_device", lambda: 0)
    with pytest.raises(ValueError, match="cuda:1"):
        ddm.ddm_scan_counts_noalloc(_FakeCuda((8,), torch.int32, 1),
                                    _FakeCuda((9,), torch.int64, 0))


def test_binding_rejects_counts_the_c_abi_cannot_carry(monkeypatch):
    """Sizes go to uint32 arguments: the binding refuses what would be
    truncated, and mistyped counts, before any library call."""
    import torch
    monkeypatch.setattr(ddm, "_lib", _NoLibrary())
    big = _FakeCuda((ddm.DDM_NOALLOC_MAX_UPDATES + 1,), torch.int32, 0)
    off = _FakeCuda((ddm.DDM_NOALLOC_MAX_UPDATES + 2,), torch.int64, 0)
    with pytest.raises(ValueError, match="at most"):
        ddm.ddm_scan_counts_noalloc(big, off)
    with pytest.raises(ValueError, match="at most"):
        ddm.ddm_scan_counts_noalloc(_FakeCuda(((1 << 32) + 3,), torch.int32, 0), off)
    with pytest.raises(TypeError):
        ddm.ddm_scan_counts_noalloc(_FakeCuda((8,), torch.float32, 0),
                                    _FakeCuda((9,), torch.int64, 0))
    with pytest.raises(TypeError):
        ddm.ddm_scan_counts_noalloc(_FakeCuda((8,), torch.int32, 0),
                                    _FakeCuda((9,), torch.int32, 0))
    huge = _FakeCuda((1, ddm.DDM_MAX_EXTENTS + 1), torch.float32, 0)
    with pytest.raises(ValueError, match="at most"):
        ddm.ddm_build(0x5151, huge, huge)


def test_checked_build_exports_every_symbol():
    """The bounds-checking variant (libddm_checked.so) builds and exports the
    same entry points (no GPU needed)."""
    path = B.build(checked=True)
    L = ctypes.CDLL(path)
    for name in declared():
        assert hasattr(L, name), name
    L.ddm_strerror.restype = ctypes.c_char_p
    assert b"bounds" in L.ddm_strerror(ddm.DDM_ERR_INTERNAL)
