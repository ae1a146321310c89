"""Argument checks of the Python binding that run before the library is
called (no GPU needed): a bad tensor must raise ValueError without reaching
the C ABI, where it would be read as a device pointer of another layout."""
import pytest
import torch

import paper_2110_07670_gb300 as ace


@pytest.fixture
def no_library(monkeypatch):
    """Any call into the library fails the test."""
    def boom(*a, **k):
        raise AssertionError("the library was called")
    monkeypatch.setattr(ace, "load", boom)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32, torch.complex32 if hasattr(torch, "complex32")
                                   else torch.float16])
def test_apply_noalloc_rejects_real_dtypes(no_library, dtype):
    """A real tensor would be taken as complex with n_pw_half = its width and
    read twice its size on the device."""
    x = torch.zeros((4, 16), dtype=dtype)
    with pytest.raises(ValueError, match="complex64"):
        ace.ace_apply_noalloc(x, x.clone(), x.clone())


def test_apply_noalloc_rejects_host_tensors(no_library):
    x = torch.zeros((4, 16), dtype=torch.complex64)
    with pytest.raises(ValueError):
        ace.ace_apply_noalloc(x, x.clone(), x.clone())


def test_apply_noalloc_rejects_mixed_dtypes(no_library):
    x = torch.zeros((4, 16), dtype=torch.complex64)
    y = torch.zeros((4, 16), dtype=torch.complex128)
    with pytest.raises(ValueError):
        ace.ace_apply_noalloc(x, y, y.clone())
