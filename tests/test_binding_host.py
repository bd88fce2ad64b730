"""Argument marshalling of the Python binding that runs without a GPU: smearing coefficient structs,
link arguments (complex128 torch tensors pass through, anything else becomes a contiguous complex128
array), raw pointers."""
import ctypes

import numpy as np
import pytest
import torch

import paper_2111_10354_gb300 as h


def test_smear_coeffs_struct():
    c = h.smear_coeffs(c1=0.5, c3=0.25, c5=0.125, c7=0.0625, cL=-1.0, cN=-1 / 24)
    assert (c.one_link, c.three_staple, c.five_staple, c.seven_staple, c.lepage, c.naik) == \
        (0.5, 0.25, 0.125, 0.0625, -1.0, -1 / 24)
    assert ctypes.sizeof(h.hisq_smear_coeffs) == 6 * 8  # six doubles, as the C struct
    d = h._coeffs(dict(c1=1.0, cN=2.0))
    assert (d.one_link, d.three_staple, d.naik) == (1.0, 0.0, 2.0)
    assert h._coeffs(c) is c


def test_links_argument():
    t = torch.zeros((4, 4, 3, 3), dtype=torch.complex128)
    assert h._links_arg(t) is t
    with pytest.raises(TypeError):
        h._links_arg(t.to(torch.complex64))
    a = h._links_arg(np.zeros((2, 4, 3, 3), np.float64)[:, ::2])
    assert a.dtype == np.complex128 and a.flags.c_contiguous


def test_pointers():
    assert h._ptr(None) is None
    a = np.zeros(4)
    assert h._ptr(a).value == a.ctypes.data
    with pytest.raises(ValueError):
        h._ptr(np.zeros((4, 4))[:, ::2])
    t = torch.zeros(4)
    assert h._ptr(t).value == t.data_ptr()
    with pytest.raises(TypeError):
        h._ptr("not an array")
