"""The allocation-free inverse propagation (hcgs_asm_propagate_noalloc).

Callers that cannot call cudaMalloc (an application whose device memory is
all owned by its own pool allocator, or a display loop that must not stall
on allocation mid-frame) get this one entry point; its working memory is a
fixed static device array.  The test calls it through the C ABI several times
in a row and compares each result with the context-based
hcgs_asm_propagate(sign=-1, reduce_planes=0), within the propagation
tolerance of the other tests (relative L2 1e-5).  This file is collected
last so that a run stopping at the first failure has run every other test.
"""
import ctypes

import numpy as np
import pytest

import hcgs_synth as S

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def _call(P, x, B, optics, out):
    fn = P._lib.hcgs_asm_propagate_noalloc
    return fn(ctypes.c_void_p(x.data_ptr()), B, ctypes.byref(P.make_optics(optics)),
              ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_noalloc_matches_context_path_on_consecutive_calls():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2506_08350_b300 as P
    ctx = P.Context(0)
    cases = [((120, 200, 3, 2, 2), 11),  # ragged 2^a 3^b 5^c sizes, two views
             ((120, 200, 3, 2, 2), 12),  # same shape, new input: nothing stale may leak
             ((256, 256, 2, 1, 1), 13)]  # another shape
    for (H, W, L, C, B), seed in cases:
        wl = S.WAVELENGTHS_RGB[:C] if C > 1 else (515e-9,)
        o = S.Optics(H, W, wl, tuple(np.linspace(1e-3, 9e-3, L)))
        x = torch.from_numpy(S.random_complex((B, C, H, W), seed=seed)).cuda()
        ref = torch.empty((B, L, C, H, W), dtype=torch.complex64, device="cuda")
        ctx.asm_propagate(x, B, o, -1, 0, ref)
        out = torch.full((B, L, C, H, W), float("nan"), dtype=torch.complex64, device="cuda")
        assert _call(P, x, B, o, out) == 0
        torch.cuda.synchronize()
        e = _rel(out.cpu().numpy(), ref.cpu().numpy())
        assert e < 1e-5, e


def test_noalloc_rejects_requests_beyond_its_scratch():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2506_08350_b300 as P
    H, W, L, C, B = 1080, 1920, 2, 3, 1  # 6.2 Mi complex values > 4 Mi
    o = S.Optics(H, W, S.WAVELENGTHS_RGB, (0.0, 1e-3))
    x = torch.zeros((B, C, H, W), dtype=torch.complex64, device="cuda")
    out = torch.zeros((B, L, C, H, W), dtype=torch.complex64, device="cuda")
    assert _call(P, x, B, o, out) == -3  # HCGS_ERR_CAPACITY, before any launch


def test_noalloc_rejects_overlapping_input_and_output():
    # `out` is written while `in` is still being read, so a partial overlap is
    # as wrong as `in == out`: both are refused before any launch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2506_08350_b300 as P
    H, W, L, C, B = 64, 64, 2, 1, 1
    o = S.Optics(H, W, (515e-9,), (0.0, 1e-3))
    n = B * C * H * W
    buf = torch.zeros(n * (L + 2), dtype=torch.complex64, device="cuda")
    x = buf[:n]
    for start in (0, n // 2, n - 1):
        out = buf[start:start + n * L]
        assert _call(P, x, B, o, out) == -1  # HCGS_ERR_INVALID_ARG
    # adjacent, not overlapping: accepted
    assert _call(P, x, B, o, buf[n:n + n * L]) == 0
    torch.cuda.synchronize()
