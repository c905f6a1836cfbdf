"""The allocation-free batched SVD entry point against the ordinary one.

ptebd_svd_batched_noalloc is meant for callers that cannot allocate device
memory (for example code that is only handed its input and output buffers by
a host framework); its scratch lives in a fixed device array inside the
library.  It must give the same singular values and vectors as
ptebd_svd_batched on the same inputs, on consecutive calls that reuse that
array, and refuse a batch that does not fit.

This file sorts last so that a run stopping at the first failure has already
run every other test."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2312_02667_gb300 import ptebd
    fn = ptebd.lib.ptebd_svd_batched_noalloc
    P = ctypes.c_void_p
    fn.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, P, ctypes.c_int32, P, P,
                   ctypes.c_int32, P, ctypes.c_int32]
    fn.restype = ctypes.c_int
    return torch, ptebd, fn


def run_both(torch, ptebd, fn, a, prec):
    batch, rows, cols = a.shape
    am = a.transpose(1, 2).contiguous()  # column-major per matrix
    dt = a.dtype
    s_ref = torch.empty((batch, cols), dtype=torch.float64, device="cuda")
    u_ref = torch.empty((batch, cols, rows), dtype=dt, device="cuda")
    wb = ptebd.ptebd_svd_workspace_bytes(prec, batch, rows, cols)
    ws = torch.empty(wb, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    ptebd.ptebd_svd_batched(prec, batch, rows, cols, am.data_ptr(), rows, s_ref.data_ptr(), u_ref.data_ptr(),
                            rows, ws.data_ptr(), wb, stream, 1)
    s_na = torch.empty_like(s_ref)
    u_na = torch.empty_like(u_ref)
    rc = fn(prec, batch, rows, cols, am.data_ptr(), rows, s_na.data_ptr(), u_na.data_ptr(), rows, stream, 1)
    assert rc == 0, rc
    torch.cuda.synchronize()
    return s_ref.cpu().numpy(), u_ref.cpu().numpy(), s_na.cpu().numpy(), u_na.cpu().numpy()


@pytest.mark.parametrize("prec,shape,tol", [(1, (6, 512, 512), 1e-5), (0, (3, 256, 200), 1e-10)])
def test_noalloc_matches_batched(env, prec, shape, tol):
    torch, ptebd, fn = env
    dt = torch.complex64 if prec == 1 else torch.complex128
    for call in range(2):  # two calls in a row: the shared scratch is reused
        rng = np.random.default_rng(10 + call)
        a = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
        at = torch.from_numpy(a / np.sqrt(shape[1])).to(dt).cuda()
        s_ref, u_ref, s_na, u_na = run_both(torch, ptebd, fn, at, prec)
        assert np.abs(s_na - s_ref).max() <= tol * s_ref.max()
        # both entry points run the same kernels on the same data; only the
        # scratch differs, so leftovers of an earlier call would show up as a
        # difference in any bit
        assert np.array_equal(s_na, s_ref)
        assert np.array_equal(u_na, u_ref)


def test_noalloc_rejects_oversize(env):
    torch, ptebd, fn = env
    big = torch.zeros((64, 512, 512), dtype=torch.complex64, device="cuda")
    s = torch.empty((64, 512), dtype=torch.float64, device="cuda")
    rc = fn(1, 64, 512, 512, big.data_ptr(), 512, s.data_ptr(), None, 512,
            torch.cuda.current_stream().cuda_stream, 1)
    assert rc == -3  # PTEBD_ERR_MEMORY
