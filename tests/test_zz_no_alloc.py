"""The allocation-free step entry point (lbm_step_static_f32).

Some callers cannot allocate device memory: a host framework that owns the
whole device-memory pool, a time loop that must not stall on the allocator,
a program held to a fixed memory budget.  They advance caller-owned FP32
buffers with lbm_step_static_f32, whose scratch psi field is a static device
array.  This file is collected last so that a run stopping at the first
failure has run every other test; it passes alone in a fresh process and
after the others.
"""
import ctypes as C

import numpy as np
import pytest

import oracle as O
from helpers import lbm_mod, rel_err

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("lat,ext", [("D3Q19", (40, 24, 16)), ("D2Q9", (64, 40, 1))])
def test_static_step_matches_context_step_twice(lat, ext):
    import torch
    assert torch.cuda.is_available()
    lbm = lbm_mod()
    nx, ny, nz = ext
    tau, G = 0.9, -5.0
    bub = (np.array([[10, 8, 6, 4.0], [28, 16, 10, 5.0]]) if lat == "D3Q19"
           else np.array([[16, 12, 0, 6.0], [44, 26, 0, 7.0]]))
    # reference: the existing context API on the two-pass path, plain FP32 values
    ref = lbm.Lattice(lat, nx, ny, nz, tau=tau, G=G, storage="f32", kernel="two_pass",
                      rho_ref=0.0)
    ref.seed_bubbles(bub, 2.0, 0.15, 2.0, 1e-3, 3)
    f0 = ref.read("f")
    # caller-owned device buffers (the caller allocates; the entry point does not)
    a = torch.tensor(f0.astype(np.float32).reshape(-1), device="cuda")
    b = torch.empty_like(a)
    stream = torch.cuda.current_stream().cuda_stream
    for step in (1, 2):                      # two calls in a row
        lbm.step_static_f32(lat, nx, ny, nz, tau, G, 1.0, a.data_ptr(), b.data_ptr(), stream)
        ref.step(1)
        torch.cuda.synchronize()
        got = b.cpu().numpy().astype(np.float64).reshape(f0.shape)
        want = ref.read("f")
        assert rel_err(got, want) < 1e-5, (step, rel_err(got, want))
        a, b = b, a
    # and both agree with the FP64 oracle from the same start
    fo = O.run(O.D3Q19 if lat == "D3Q19" else O.D2Q9, f0, 2, tau, G)
    assert rel_err(a.cpu().numpy().astype(np.float64).reshape(f0.shape), fo) < 1e-5
    ref.close()


def test_static_step_rejects_oversize_and_aliasing():
    lbm = lbm_mod()
    lib = lbm.lib()
    p = C.c_void_p(1 << 20)
    q = C.c_void_p(1 << 21)
    assert lib.lbm_step_static_f32(1, 256, 128, 128, 0.9, -5.0, 1.0, p, q, None) == lbm.EINVAL
    assert "2097152" in lib.lbm_last_error().decode()
    assert lib.lbm_step_static_f32(1, 16, 16, 16, 0.9, -5.0, 1.0, p, p, None) == lbm.EINVAL
