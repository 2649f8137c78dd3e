"""psp_apply_noalloc (the allocation-free variant of psp_apply) against psp_apply, through the C ABI.

Callers that cannot allocate device memory while they run (a framework allocator already holding
the free memory, a fixed memory budget, a loop timed as one stream-ordered region) use
psp_apply_noalloc, whose work vectors live in a fixed 16 MiB device array inside the library.
This file is collected last so that a run stopping at the first failure has run everything else.
"""
import ctypes

import numpy as np
import pytest

from paper_1204_0111_gb300 import workloads as wl

from _cases import small_cases

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1204_0111_gb300 import psp  # noqa: E402

TOL = 1e-10  # the apply parity tolerance of the other GPU tests


def _make(case, precision="c128"):
    c = torch.from_numpy(case.c).cuda()
    return psp.SweepingPreconditioner(c, case.h, case.omega, case.gamma, case.depth, pad=case.pad, leaf=case.leaf,
                                      pml_C=case.C, alpha=case.alpha, faces=case.faces, precision=precision)


def _noalloc(P, rhs, out):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    nrhs = rhs.numel() // P.N
    return psp.lib().psp_apply_noalloc(P._h, ctypes.c_void_p(rhs.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                       nrhs, stream)


def _rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


def test_noalloc_apply_matches_apply_on_two_calls_in_a_row():
    case = small_cases()[0]
    P = _make(case)
    r = torch.from_numpy(wl.random_vector(case.N, 2, seed=31)).cuda()
    ref = torch.empty_like(r)
    P.apply(r, ref)
    for call in range(2):
        out = torch.from_numpy(wl.random_vector(case.N, 2, seed=40 + call)).cuda()   # stale contents
        assert _noalloc(P, r, out) == 0, psp.lib().psp_last_error()
        torch.cuda.synchronize()
        assert _rel(out, ref) < TOL, call
    inplace = r.clone()
    assert _noalloc(P, inplace, inplace) == 0
    torch.cuda.synchronize()
    assert _rel(inplace, ref) < TOL
    P.close()


def test_noalloc_second_problem_after_first():
    # the shared array keeps the previous call's contents; a different problem must not see them
    cases = small_cases()
    for case in (cases[1], cases[0]):
        P = _make(case)
        r = torch.from_numpy(wl.random_vector(case.N, 1, seed=7)).cuda()
        ref = torch.empty_like(r)
        P.apply(r, ref)
        out = torch.zeros_like(r)
        assert _noalloc(P, r, out) == 0
        torch.cuda.synchronize()
        assert _rel(out, ref) < TOL
        P.close()


def test_noalloc_rejects_host_pointers_and_oversize_requests():
    case = small_cases()[2]
    P = _make(case)
    L = psp.lib()
    host = wl.random_vector(case.N, 1, seed=1)
    hout = np.zeros_like(host)
    st = L.psp_apply_noalloc(P._h, ctypes.c_void_p(host.ctypes.data), ctypes.c_void_p(hout.ctypes.data), 1, None)
    assert st == 1 and b"device pointers" in L.psp_last_error()
    big = torch.zeros((64, case.N), dtype=torch.complex128, device="cuda")
    st = _noalloc(P, big, big)
    assert st == 1 and b"use psp_apply" in L.psp_last_error()
    P.close()


def test_noalloc_complex64_handle_matches_apply():
    # complex64 fronts and work vectors (8-byte elements in the shared array)
    case = small_cases()[2]
    P = _make(case, precision="c64")
    r = torch.from_numpy(wl.random_vector(case.N, 3, seed=5)).cuda()
    ref = torch.empty_like(r)
    P.apply(r, ref)
    for call in range(2):
        out = torch.from_numpy(wl.random_vector(case.N, 3, seed=60 + call)).cuda()
        assert _noalloc(P, r, out) == 0, psp.lib().psp_last_error()
        torch.cuda.synchronize()
        assert _rel(out, ref) < TOL, call      # same kernels and schedule as psp_apply
    P.close()


def test_noalloc_batch_of_two_problems_matches_apply():
    # a batch handle: each problem's work vectors sit at their own offset inside the shared array
    cases = small_cases()[:2]
    probs = [dict(c=torch.from_numpy(cs.c).cuda(), h=cs.h, omega=cs.omega, gamma=cs.gamma, panel_depth=cs.depth)
             for cs in cases]
    B = psp.SweepingPreconditionerBatch(probs, leaf=16)
    nrhs = 2
    r = torch.from_numpy(wl.random_vector(B.N * nrhs, 1, seed=9).reshape(-1)).cuda()
    ref = torch.empty_like(r)
    B.apply(r, ref)
    for call in range(2):
        out = torch.zeros_like(r)
        assert _noalloc(B, r, out) == 0, psp.lib().psp_last_error()
        torch.cuda.synchronize()
        assert _rel(out, ref) < TOL, call
    B.close()
