"""The allocation-free residual entry point, for callers that cannot allocate device memory.

evp_stress_residual_noalloc keeps its scratch in a fixed array inside the library instead of a
caller-supplied buffer. This file is collected last so that a run stopping at the first failure
has already run every other test. It checks, through the C ABI, that two calls in a row agree
with the allocating entry point evp_stress_residual on the same inputs.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1509_04953_gb300 import build
    build.build()
    from paper_1509_04953_gb300 import evp
    L = evp.load()
    L.evp_stress_residual_noalloc.argtypes = [C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    L.evp_stress_residual_noalloc.restype = C.c_int
    return torch, evp, L


@pytest.mark.parametrize("n,prec", [(32, "fp64"), (64, "fp32")])
def test_noalloc_matches_allocating_entry_point_on_two_calls(env, n, prec):
    torch, evp, L = env
    dt = torch.float64 if prec == "fp64" else torch.float32
    cd = torch.complex128 if prec == "fp64" else torch.complex64
    code = 0 if prec == "fp64" else 1
    stream = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(2024 + n)
    for call in range(2):            # the second call runs on the contents the first one left
        sig = torch.tensor(rng.standard_normal((6, n, n, n)) * 40.0 + 10.0 * call, dtype=dt, device="cuda")
        spec_ref, out_ref = evp.stress_residual(sig)
        spec = torch.empty((6, n, n, n // 2 + 1), dtype=cd, device="cuda")
        out = torch.empty(7, dtype=torch.float64, device="cuda")
        rc = L.evp_stress_residual_noalloc(n, code, sig.data_ptr(), spec.data_ptr(), out.data_ptr(), stream)
        assert rc == 0
        torch.cuda.synchronize()
        tol = 1e-12 if prec == "fp64" else 2e-6
        a, b = out.cpu().numpy(), out_ref.cpu().numpy()
        assert np.abs(a - b).max() <= tol * np.abs(b).max()
        assert torch.allclose(spec, spec_ref, rtol=tol, atol=tol * spec_ref.abs().max().item())


def test_noalloc_rejects_sizes_beyond_its_array(env):
    torch, evp, L = env
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    for bad_n in (512, 12, 2):
        assert L.evp_stress_residual_noalloc(bad_n, 0, x.data_ptr(), x.data_ptr(), x.data_ptr(), None) == -1
