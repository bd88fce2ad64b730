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


def test_struct_layouts_match_the_header(tmp_path):
    """The binding's ctypes structs against the C header, compiled by the host compiler: the size of each
    struct and the offset of every field the binding declares (a field added on one side only would
    shift everything after it)."""
    import os
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    structs = {"hisq_solver_opts": h.hisq_solver_opts, "hisq_solver_stats": h.hisq_solver_stats,
               "hisq_smear_coeffs": h.hisq_smear_coeffs}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "hisq.h"', 'int main(void) {']
    for name, cls in structs.items():
        lines.append('  printf("%s size %%zu\\n", sizeof(%s));' % (name, name))
        for field, _ in cls._fields_:
            lines.append('  printf("%s %s %%zu\\n", offsetof(%s, %s));' % (name, field, name, field))
    lines += ['  return 0;', '}']
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(root, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l}
    for name, cls in structs.items():
        assert got[(name, "size")] == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert got[(name, field)] == getattr(cls, field).offset, (name, field)
