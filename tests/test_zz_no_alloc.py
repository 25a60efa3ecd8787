"""ps_overlap_noalloc: the overlap for callers that cannot allocate device memory.

The call takes two device buffers and a device output and uses a fixed
scratch array inside the library instead of a handle's cudaMalloc'd buffer.
It must agree with ps_overlap (same kernels, same summation order) on every
call, including a second call right after the first with other inputs,
since all calls share the one scratch array.  This file is collected last on
purpose, so that a run stopping at its first failure has run everything else.
"""
import numpy as np
import pytest
import torch

import paper_2504_17881_gb300 as ps
from paper_2504_17881_gb300 import inputs

pytestmark = pytest.mark.gpu

TDT = {ps.PS_C128: torch.complex128, ps.PS_C64: torch.complex64}


def _state(n, dtype, seed):
    st = ps.StateVector(n, dtype=TDT[dtype])
    st.load(inputs.gaussian_state(n, seed))
    return st


def _noalloc(n, dtype, a, b, out):
    ps.ps_overlap_noalloc(n, dtype, a.tensor.data_ptr(), b.tensor.data_ptr(),
                          torch.cuda.current_stream().cuda_stream, out.data_ptr())
    torch.cuda.current_stream().synchronize()
    return complex(out[0].item(), out[1].item())


@pytest.mark.parametrize("dtype", [ps.PS_C128, ps.PS_C64])
def test_noalloc_overlap_matches_ps_overlap_twice(dtype):
    n = 18
    a, b = _state(n, dtype, 1), _state(n, dtype, 2)
    c, d = _state(n, dtype, 3), _state(n, dtype, 4)
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    # tolerance of the reduction tests: 1e-14 * sqrt(2^n)
    tol = 1e-14 * np.sqrt(1 << n)
    first = _noalloc(n, dtype, a, b, out)
    assert abs(first - b.overlap(a)) < tol
    second = _noalloc(n, dtype, c, d, out)
    assert abs(second - d.overlap(c)) < tol
    assert abs(second - first) > 1e-6  # the second call saw its own inputs


def test_noalloc_overlap_rejects_out_of_range_sizes():
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    a = _state(4, ps.PS_C64, 5)
    with pytest.raises(ps.PsError) as e:
        ps.ps_overlap_noalloc(41, ps.PS_C64, a.tensor.data_ptr(), a.tensor.data_ptr(), 0, out.data_ptr())
    assert "outside" in str(e.value)
    with pytest.raises(ps.PsError):
        ps.ps_overlap_noalloc(4, ps.PS_C64, 0, a.tensor.data_ptr(), 0, out.data_ptr())
