"""nsrgs_step_static: the allocation-free variant of nsrgs_step.

It serves callers that cannot allocate device memory where they run an
iteration.  This file is collected last so that a run that stops at the first
failure has already run every other test.  The entry point is called directly
through the C ABI (ctypes) and compared with nsrgs_step, with a caller
workspace, on two calls in a row (the second call reuses the shared array
left over from the first).
"""
import ctypes

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import __graft_entry__

    __graft_entry__.build()
    import paper_2604_07372_gb300 as P

    return P


def _static_step(P, pa, eta, K, Xin, Xout, upd=None):
    fn = P.lib().nsrgs_step_static
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.POINTER(P._lib._A), ctypes.c_float, ctypes.c_int] + [ctypes.c_void_p] * 4
    a = pa.struct()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    un = ctypes.c_void_p(upd.data_ptr()) if upd is not None else None
    return fn(ctypes.byref(a), eta, K, ctypes.c_void_p(Xin.data_ptr()), ctypes.c_void_p(Xout.data_ptr()), un, stream)


# (300, 3) FP32 and (1000, 2) BF16 run the panel stream with the per-block
# epilogue in registers; (900, 16) BF16 runs the tile-upper tensor-core stream
# and the shared-memory epilogue, whose scratch (X^T tiles, float64 partials)
# also lives in the array.
@pytest.mark.parametrize("n,d,storage", [(300, 3, 0), (1000, 2, 1), (900, 16, 1)])
def test_static_step_matches_workspace_step_twice(P, n, d, storage):
    inst = synth.make_instance(n, d, synth.sigma_rule(0.3, n, d), seed=n + d, dtype=np.float32)
    pa = P.nsrgs_pack_upper(torch.from_numpy(inst.upper).cuda(), n, d, storage)
    rng = np.random.default_rng(1)
    Xa = torch.from_numpy(np.linalg.qr(rng.standard_normal((n, d, d)))[0].reshape(n * d, d).astype(np.float32)).cuda()
    eta, K = 1.0 / n, 2
    ref_un = torch.zeros(2, dtype=torch.float64, device="cuda")
    got_un = torch.zeros(2, dtype=torch.float64, device="cuda")
    ref1 = P.nsrgs_step(pa, eta, K, Xa, torch.empty_like(Xa), upd_norm=ref_un[0:1])
    ref2 = P.nsrgs_step(pa, eta, K, ref1, torch.empty_like(Xa), upd_norm=ref_un[1:2])
    got1 = torch.empty_like(Xa)
    got2 = torch.empty_like(Xa)
    assert _static_step(P, pa, eta, K, Xa, got1, got_un[0:1]) == 0, P.lib().nsrgs_last_error()
    assert _static_step(P, pa, eta, K, got1, got2, got_un[1:2]) == 0, P.lib().nsrgs_last_error()
    torch.cuda.synchronize()
    assert torch.max(torch.abs(got1 - ref1)).item() <= 2e-5
    assert torch.max(torch.abs(got2 - ref2)).item() <= 2e-5
    # the update norms written through the static scratch match the workspace call's
    r, g = ref_un.cpu().numpy(), got_un.cpu().numpy()
    assert np.all(r > 0) and np.allclose(g, r, rtol=1e-5, atol=0)


def test_static_step_allocates_no_device_memory(P):
    """After the first call on the device (which loads the module holding the
    array), further calls leave the device's free memory unchanged."""
    n, d = 300, 3
    inst = synth.make_instance(n, d, synth.sigma_rule(0.3, n, d), seed=7, dtype=np.float32)
    pa = P.nsrgs_pack_upper(torch.from_numpy(inst.upper).cuda(), n, d, 0)
    rng = np.random.default_rng(2)
    Xa = torch.from_numpy(np.linalg.qr(rng.standard_normal((n, d, d)))[0].reshape(n * d, d).astype(np.float32)).cuda()
    Xb = torch.empty_like(Xa)
    un = torch.zeros(1, dtype=torch.float64, device="cuda")
    assert _static_step(P, pa, 1.0 / n, 2, Xa, Xb, un) == 0, P.lib().nsrgs_last_error()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(5):
        assert _static_step(P, pa, 1.0 / n, 2, Xa, Xb, un) == 0, P.lib().nsrgs_last_error()
        assert _static_step(P, pa, 1.0 / n, 2, Xb, Xa, un) == 0, P.lib().nsrgs_last_error()
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_static_step_rejects_sizes_beyond_the_array(P):
    fn = P.lib().nsrgs_step_static
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.POINTER(P._lib._A), ctypes.c_float, ctypes.c_int] + [ctypes.c_void_p] * 4
    a = P._lib._A(16, 200000, 4, 0)  # workspace far above 8 MiB; rejected before any device access
    assert fn(ctypes.byref(a), 0.1, 2, None, None, None, None) == 1
    assert b"8 MiB" in P.lib().nsrgs_last_error()
