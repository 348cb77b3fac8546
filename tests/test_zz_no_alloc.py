"""The allocation-free entry point unravel_grad_noalloc (for callers that must
not allocate device memory during a call) against the allocating unravel_grad,
through the C ABI, on two calls in a row.  This file is collected last on
purpose: a failure here leaves every other test already run."""
import ctypes

import numpy as np
import pytest

from paper_2508_05745_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_noalloc_matches_unravel_grad_twice():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2508_05745_gb300 import build, lemps as L
    build.build()
    lib = L.load()
    stream = torch.cuda.current_stream().cuda_stream
    for seed, chi, dt in ((31, 16, np.complex128), (32, 8, np.complex64)):
        w = I.workload_adjoint(seed=seed, batch=300, chi=chi, dtype=dt)
        th = torch.from_numpy(w["theta"]).cuda()
        p = torch.from_numpy(w["p"]).cuda()
        h = torch.from_numpy(w["H"]).cuda()
        cost_ref, grad_ref, _ = L.unravel_grad(th, p, h)
        cost = torch.full_like(cost_ref, float("nan"))
        grad = torch.full_like(grad_ref, float("nan"))
        st = lib.unravel_grad_noalloc(th.data_ptr(), 1 if dt == np.complex128 else 0, th.shape[0], chi,
                                      p.data_ptr(), h.data_ptr(), cost.data_ptr(), grad.data_ptr(), stream)
        assert st == L.LEMPS_OK, lib.lemps_last_error()
        torch.cuda.synchronize()
        assert torch.allclose(cost, cost_ref, rtol=0, atol=1e-12)
        assert torch.allclose(grad, grad_ref, rtol=0, atol=1e-12)


def test_noalloc_rejects_batches_above_its_maximum():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2508_05745_gb300 import build, lemps as L
    build.build()
    lib = L.load()
    dummy = torch.zeros(4, dtype=torch.float64, device="cuda")
    st = lib.unravel_grad_noalloc(dummy.data_ptr(), 1, 16385, 4, dummy.data_ptr(), dummy.data_ptr(),
                                  dummy.data_ptr(), None, None)
    assert st == L.LEMPS_EINVAL
    assert b"16384" in lib.lemps_last_error()
