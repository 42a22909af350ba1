"""CPU checks of the C-ABI library: it loads, exports every entry point that
include/hcgs.h declares, and rejects bad arguments before touching CUDA."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hcgs.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hcgs_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as E
    path = E._build_module().build()
    return ctypes.CDLL(path)


def test_header_declares_the_path():
    names = _declared()
    for n in ("hcgs_project", "hcgs_rasterize_planes", "hcgs_asm_propagate", "hcgs_render_view",
              "hcgs_project_backward", "hcgs_rasterize_planes_backward", "hcgs_asm_propagate_backward",
              "hcgs_render_view_backward"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_lists_every_export():
    import paper_2506_08350_b300 as P
    assert sorted(P.EXPORTS) == _declared()


def test_status_strings(lib):
    lib.hcgs_status_string.restype = ctypes.c_char_p
    lib.hcgs_status_string.argtypes = [ctypes.c_int]
    assert lib.hcgs_status_string(0) == b"HCGS_OK"
    assert lib.hcgs_status_string(-4) == b"HCGS_ERR_UNSUPPORTED_SIZE"
    assert lib.hcgs_status_string(-7) == b"HCGS_ERR_STATE"


def test_null_context_is_rejected_without_cuda(lib):
    # every entry point checks its context first and returns
    # HCGS_ERR_INVALID_ARG (-1) without any CUDA call
    for name in ("hcgs_project", "hcgs_rasterize_planes", "hcgs_asm_propagate", "hcgs_render_view",
                 "hcgs_rasterize_planes_backward", "hcgs_project_backward", "hcgs_render_view_backward",
                 "hcgs_focal_stack_loss", "hcgs_adam_step", "hcgs_mlp_forward", "hcgs_mlp_backward",
                 "hcgs_asm_propagate_backward", "hcgs_adam_step_multi", "hcgs_adan_step_multi"):
        f = getattr(lib, name)
        f.restype = ctypes.c_int
        args = [None] * 20
        assert f(*args) == -1, name
    lib.hcgs_saved_create.restype = ctypes.c_int
    assert lib.hcgs_saved_create(None, None) == -1
    lib.hcgs_ctx_create.restype = ctypes.c_int
    assert lib.hcgs_ctx_create(None, 0) == -1


def test_torch_complex_gradient_convention():
    # The ABI passes upstream gradients as g = dL/dRe + j dL/dIm; torch's
    # complex autograd hands backward() the same quantity for a real loss.
    import torch
    z = torch.tensor([0.3 - 1.2j, 2.0 + 0.5j], dtype=torch.complex128, requires_grad=True)
    L = (z.real ** 2 * 3.0 + z.imag * 5.0 - z.real * z.imag).sum()
    L.backward()
    x, y = z.detach().real, z.detach().imag
    expect = (6 * x - y) + 1j * (5.0 - x)
    assert torch.allclose(z.grad, expect)


def test_checked_build_exports_the_same_entry_points():
    # the bounds-checked variant (HCGS_CHECKED) is the same ABI; only
    # hcgs_is_checked_build tells them apart (callable without a GPU)
    import __graft_entry__ as E
    checked = ctypes.CDLL(E._build_module().build(checked=True))
    regular = ctypes.CDLL(E._build_module().build())
    for name in _declared():
        assert hasattr(checked, name), name
    checked.hcgs_is_checked_build.restype = ctypes.c_int
    regular.hcgs_is_checked_build.restype = ctypes.c_int
    assert checked.hcgs_is_checked_build() == 1 and regular.hcgs_is_checked_build() == 0
    for lib_ in (checked, regular):
        lib_.hcgs_check_status.restype = ctypes.c_int
        assert lib_.hcgs_check_status(None, None) == -1  # NULL context, no CUDA call
