"""The allocation-free tensor-core product (tz_op_cgemm_static): for callers
that cannot call cudaMalloc, the library keeps the product's scratch in its
own fixed-size device array. Its results must equal those of tz_op_cgemm,
which takes caller-supplied scratch, on two calls in a row (the second call
must not see the first call's leftovers). This file sorts last so a run that
stops at the first failure has already run every other test; it also passes
alone in a fresh process."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _c64(torch, rng, shape):
    x = (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex64)
    return torch.from_numpy(x.view(np.float32).copy()).cuda()


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3", "fp16x3"])
def test_static_scratch_matches_caller_scratch(prec):
    import torch
    import paper_1907_11217_gb300 as tz
    from paper_1907_11217_gb300._lib import PRECISIONS, check, lib
    assert torch.cuda.is_available()
    L = lib()
    p = PRECISIONS[prec]
    rng = np.random.default_rng(11)
    # three calls in a row: the largest prepared B first, then a product
    # whose long K is split across CTAs (its partials go to the static
    # array too), then a small one; each must read nothing of what an
    # earlier call left in the array
    for (batch, m, n, k) in [(1, 512, 128, 64), (1, 128, 8, 4096), (2, 256, 24, 16)]:
        dA = _c64(torch, rng, (batch, m, k))
        dB = _c64(torch, rng, (batch, n, k))
        ref = torch.zeros(batch * m * n * 2, dtype=torch.float32, device="cuda")
        got = torch.full_like(ref, float("nan"))
        nbytes = tz.tz_op_cgemm_scratch_bytes(prec, batch, m, n, k)
        scratch = torch.empty(nbytes // 4 + 64, dtype=torch.float32, device="cuda")
        tz.tz_op_cgemm(prec, batch, m, n, k, dA, m * k, dB, n * k, ref, m * n, scratch=scratch)
        tz.tz_op_cgemm_status(prec, scratch)
        check(L.tz_op_cgemm_static(p, batch, m, n, k, ctypes.c_void_p(dA.data_ptr()), m * k,
                                   ctypes.c_void_p(dB.data_ptr()), n * k, ctypes.c_void_p(got.data_ptr()), m * n,
                                   ctypes.c_void_p(0)))
        tz.tz_op_cgemm_static_status()
        torch.cuda.synchronize()
        r = ref.cpu().numpy()
        g = got.cpu().numpy()
        # the same kernels on the same inputs, with a fixed summation order
        # (split-K partials are added in a fixed order): equal bit for bit
        assert np.all(np.isfinite(g))
        assert np.array_equal(g.view(np.uint32), r.view(np.uint32)), (batch, m, n, k)


def test_static_scratch_rejects_oversize():
    import torch
    from paper_1907_11217_gb300._lib import TZ_EINVAL, TZ_TF32X3, lib
    assert torch.cuda.is_available()
    L = lib()
    d = torch.zeros(16, dtype=torch.float32, device="cuda")
    # the prepared B of batch 64 x n 512 x k 256 complex is 1024 real rows
    # of 512 FP32 values per batch, 128 MiB for its hi copy and as much for
    # its lo copy: 256 MiB against the array's 16 MiB
    rc = L.tz_op_cgemm_static(TZ_TF32X3, 64, 128, 512, 256, ctypes.c_void_p(d.data_ptr()), 128 * 256,
                              ctypes.c_void_p(d.data_ptr()), 512 * 256, ctypes.c_void_p(d.data_ptr()), 128 * 512,
                              ctypes.c_void_p(0))
    assert rc == TZ_EINVAL
    assert b"static scratch" in L.tz_last_error()
