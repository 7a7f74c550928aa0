"""rt_transport_static: radiative transport for callers that cannot allocate
device memory (their allocator owns the GPU, or an allocation would grow the
footprint or synchronise the device mid-run).  Its only scratch is a static
device array inside the library, so these checks call it through the C ABI
and compare it with the allocating path (rt_step with no absorber, no source
and no chemistry change, i.e. pure transport), on two calls in a row.

This file is collected last on purpose: it must pass both alone in a fresh
process and after every other test.
"""
import ctypes as C

import numpy as np
import pytest

from paper_1508_07888_b300 import binding as B
from paper_1508_07888_b300 import inputs as I

pytestmark = pytest.mark.gpu

TABLE0 = {"sigN": [0.0] * 4, "sigE": [0.0] * 4, "Eavg": [0.0] * 4, "frac": [0.25] * 4}


def entry():
    f = B.lib().rt_transport_static
    f.restype = C.c_int
    f.argtypes = [C.POINTER(B.rt_params), C.POINTER(B.rt_box), C.c_int, C.c_void_p]
    return f


def params(G, prec, bc):
    return B.make_params(G, TABLE0, 0.1 * I.C_LIGHT, isothermal=True, rates_const=True,
                         bc=bc, precision=prec)


def allocating_path(U0, G, prec, bc, dx, nsteps):
    """The existing entry point: rt_create + rt_step (transport + identity chemistry)."""
    import torch
    fp = torch.float64 if prec != B.RT_PREC_SPLIT else torch.float32
    shape = U0.shape[1:4]
    st = B.BoxState(U=torch.as_tensor(U0, dtype=fp, device="cuda").contiguous(),
                    xHI=torch.ones(shape, dtype=torch.float64, device="cuda"),
                    T=torch.full(shape, 1e4, dtype=torch.float64, device="cuda"),
                    n0=torch.full(shape, 1e-3, dtype=fp, device="cuda"), dx=dx, nunit=1.0)
    s = B.Solver(params(G, prec, bc), [st])
    assert s.step(nsteps) == B.RT_OK
    out = st.U.double().cpu().numpy()
    s.close()
    return out


def static_path(Ut, G, prec, bc, dx, nsteps):
    import torch
    box = B.rt_box()
    box.nz, box.ny, box.nx = Ut.shape[1:4]
    box.dx, box.nunit = dx, 1.0
    box.U = Ut.data_ptr()
    p = params(G, prec, bc)
    code = entry()(C.byref(p), C.byref(box), nsteps, C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert code == B.RT_OK, code
    return Ut.double().cpu().numpy()


def normwise(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("prec,tol", [(B.RT_PREC_SPLIT, 3e-6), (B.RT_PREC_FP64, 1e-14),
                                      (B.RT_PREC_FP64_STRICT, 0.0)])
@pytest.mark.parametrize("bc", [[0] * 6, [2, 1, 2, 1, 1, 1]])
def test_static_transport_matches_allocating_path_two_calls_in_a_row(prec, tol, bc):
    import torch
    G, shape, dx = 2, (20, 24, 37), 3e20
    U0 = I.f32(I.random_realizable_state(shape, G, 41))
    fp = torch.float64 if prec != B.RT_PREC_SPLIT else torch.float32
    Ut = torch.as_tensor(U0, dtype=fp, device="cuda").contiguous()
    first = static_path(Ut, G, prec, bc, dx, 3)           # odd count: result copied back
    assert normwise(first, allocating_path(U0, G, prec, bc, dx, 3)) <= tol
    second = static_path(Ut, G, prec, bc, dx, 2)          # continues from the first call
    assert normwise(second, allocating_path(U0, G, prec, bc, dx, 5)) <= tol
    assert not np.array_equal(first, second)


@pytest.mark.parametrize("side", [256, 1 << 20])
def test_static_transport_rejects_a_box_beyond_its_scratch(side):
    """256^3 x 16 B = 256 MiB is over the 32 MiB scratch; at 2^20 cells per
    axis the byte count of the box overflows 64 bits, which the check must not
    let wrap past the limit.  Both return before any work is queued."""
    import torch
    Ut = torch.zeros(16, dtype=torch.float32, device="cuda")
    box = B.rt_box()
    box.nx = box.ny = box.nz = side
    box.dx, box.nunit = 3e20, 1.0
    box.U = Ut.data_ptr()
    p = params(1, B.RT_PREC_SPLIT, [0] * 6)
    assert entry()(C.byref(p), C.byref(box), 1, None) == B.RT_ERR_TOO_LARGE
    assert "does not fit" in B.rt_last_error(None)
    torch.cuda.synchronize()
    assert torch.count_nonzero(Ut).item() == 0
