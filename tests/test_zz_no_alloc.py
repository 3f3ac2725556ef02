"""The allocation-free unstable index (rtg_unstable_index_static) against the context-based
rtg_unstable_index, through the C ABI.

rtg_unstable_index_static exists for callers that must not allocate device memory, such
as a thread running beside the real-time mapping loop, where cudaMalloc could stall the
device, or a program whose memory budget is already held by its own pool.  Its scratch
is a fixed array inside the library, so these tests also check that two calls in a row
do not see each other's leftovers and that sizes beyond the array are refused.

This file is collected last on purpose: a run that stops at the first failure has then
already run every other test.
"""

import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _lib():
    from paper_2404_19706_b300 import _lib as L
    return L, L.load()


def _context_index(lib, flags):
    """ids and count from the existing entry point, which uses a context's workspace."""
    L, _ = _lib()
    n = flags.numel()
    cap = L.rtg_capacity(max(n, 1), 1, 16, 16, 3, 1024)
    ctx = ctypes.c_void_p()
    assert lib.rtg_create(ctypes.byref(ctx), ctypes.byref(cap)) == L.RTG_OK
    ids = torch.full((max(n, 1),), -7, dtype=torch.int32, device="cuda")
    nu = torch.zeros(1, dtype=torch.int64, device="cuda")
    st = lib.rtg_unstable_index(ctx, n, flags.data_ptr(), ids.data_ptr(), nu.data_ptr(), None)
    torch.cuda.synchronize()
    lib.rtg_destroy(ctx)
    assert st == L.RTG_OK
    k = int(nu.item())
    return ids[:k].cpu().numpy(), k


def _static_index(lib, flags, fill):
    L, _ = _lib()
    n = flags.numel()
    ids = torch.full((max(n, 1),), fill, dtype=torch.int32, device="cuda")
    nu = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    st = lib.rtg_unstable_index_static(n, flags.data_ptr(), ids.data_ptr(), nu.data_ptr(), None)
    torch.cuda.synchronize()
    assert st == L.RTG_OK
    k = int(nu.item())
    return ids[:k].cpu().numpy(), k


def test_static_index_matches_context_index_two_calls_in_a_row():
    L, lib = _lib()
    rng = np.random.default_rng(11)
    # two different inputs back to back: the second must not inherit the first's scratch
    for n, p in ((3_000_000, 0.2), (1_234_567, 0.65)):
        flags = torch.tensor((rng.random(n) < p).astype(np.uint8), device="cuda")
        ref_ids, ref_nu = _context_index(lib, flags)
        got_ids, got_nu = _static_index(lib, flags, fill=-3)
        assert got_nu == ref_nu == int(flags.sum().item())
        np.testing.assert_array_equal(got_ids, ref_ids)


def test_static_index_edge_sizes_and_limit():
    L, lib = _lib()
    ones = torch.ones(1025, dtype=torch.uint8, device="cuda")  # one full block plus one
    got_ids, got_nu = _static_index(lib, ones, fill=-1)
    assert got_nu == 1025 and (got_ids == np.arange(1025)).all()
    empty = torch.zeros(0, dtype=torch.uint8, device="cuda")
    nu = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    assert lib.rtg_unstable_index_static(0, None, None, nu.data_ptr(), None) == L.RTG_OK
    torch.cuda.synchronize()
    assert int(nu.item()) == 0 and empty.numel() == 0
    # beyond the fixed scratch: refused before any launch (pointers are never touched)
    assert lib.rtg_unstable_index_static((1 << 24) + 1, None, None, nu.data_ptr(), None) == L.RTG_ERR_ARG
    dummy = torch.zeros(1, dtype=torch.uint8, device="cuda")
    assert lib.rtg_unstable_index_static((1 << 24) + 1, dummy.data_ptr(), dummy.data_ptr(), nu.data_ptr(),
                                         None) == L.RTG_ERR_WORKSPACE
