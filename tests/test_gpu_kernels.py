"""Per-kernel parity on the GPU, through the C ABI (tz_op_*), against the
plain definitions in oracle.linalg."""
import numpy as np
import pytest

from oracle import linalg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    import paper_1907_11217_gb300 as tz
    assert torch.cuda.is_available()
    return tz, torch


def c64(torch, rng, shape):
    x = (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex64)
    return x, torch.from_numpy(x.view(np.float32).copy()).cuda()


@pytest.mark.parametrize("rank", [0, 1, 3, 5, 9, 10, 11, 14, 17, 22])
def test_permute_bit_exact(env, rank):
    tz, torch = env
    rng = np.random.default_rng(rank)
    x, dx = c64(torch, rng, 1 << rank)
    perms = [list(range(rank)), list(range(rank))[::-1], list(rng.permutation(rank))]
    if rank > 6:
        p = list(range(rank))
        p[:3], p[-3:] = p[-3:], p[:3]
        perms.append(p)
    for perm in perms:
        dy = torch.empty_like(dx)
        tz.tz_op_permute(dx, dy, perm)
        torch.cuda.synchronize()
        y = dy.cpu().numpy().view(np.complex64)
        assert np.array_equal(y, linalg.bit_permute(x, perm)), perm


@pytest.mark.parametrize("batch,m,n,k", [(1, 1, 1, 1), (1, 7, 3, 5), (3, 64, 64, 8), (2, 130, 17, 33),
                                         (1, 1000, 2, 4), (5, 33, 80, 1), (1, 4096, 16, 64), (16, 256, 256, 256),
                                         (1, 1, 300, 9), (3, 4096, 1, 2), (1, 512, 4, 16), (2, 300, 3, 5),
                                         (1, 1 << 16, 2, 8), (8192, 1, 1, 1024), (16, 8, 8, 64), (3, 2, 3, 200)])
def test_cgemm_simt(env, batch, m, n, k):
    tz, torch = env
    rng = np.random.default_rng(m * 7 + n)
    A, dA = c64(torch, rng, (batch, m, k))
    B, dB = c64(torch, rng, (batch, n, k))
    dC = torch.zeros(batch * m * n * 2, dtype=torch.float32, device="cuda")
    tz.tz_op_cgemm("c64", batch, m, n, k, dA, m * k, dB, n * k, dC, m * n)
    torch.cuda.synchronize()
    C = dC.cpu().numpy().view(np.complex64).reshape(batch, m, n)
    ref = linalg.cgemm(A, B)
    bound = linalg.cgemm(np.abs(A).astype(np.complex128), np.abs(B).astype(np.complex128)).real
    # FP32 products summed over k: |err| <= ~ (k + 2) * 2^-24 * sum |a||b| per component
    assert np.all(np.abs(C - ref) <= 4 * (k + 2) * 2.0 ** -24 * bound + 1e-30)


@pytest.mark.parametrize("batch,m,n,k", [(1, 128, 1, 2), (1, 128, 8, 16), (2, 256, 64, 32), (1, 1024, 128, 64),
                                         (3, 128, 4, 4), (1, 512, 256, 128), (4, 384, 24, 10), (1, 8192, 16, 256),
                                         (2, 256, 24, 100)])
def test_cgemm_tf32x3(env, batch, m, n, k):
    """Split-TF32 tcgen05 product: hi*hi + hi*lo + lo*hi with round-to-nearest
    splits leaves < 2^-20 |a||b| per product, plus FP32 accumulation."""
    tz, torch = env
    rng = np.random.default_rng(m + 3 * n + 7 * k)
    A, dA = c64(torch, rng, (batch, m, k))
    B, dB = c64(torch, rng, (batch, n, k))
    dC = torch.zeros(batch * m * n * 2, dtype=torch.float32, device="cuda")
    nbytes = tz.tz_op_cgemm_scratch_bytes("tf32x3", batch, m, n, k)
    scratch = torch.empty(nbytes // 4 + 64, dtype=torch.float32, device="cuda")
    tz.tz_op_cgemm("tf32x3", batch, m, n, k, dA, m * k, dB, n * k, dC, m * n, scratch=scratch)
    torch.cuda.synchronize()
    C = dC.cpu().numpy().view(np.complex64).reshape(batch, m, n)
    ref = linalg.cgemm(A, B)
    bound = linalg.cgemm(np.abs(A).astype(np.complex128), np.abs(B).astype(np.complex128)).real
    err = np.abs(C - ref)
    assert np.all(err <= (2.0 ** -18 + 4 * (k + 2) * 2.0 ** -24) * bound + 1e-30), float(np.max(err / bound))
    # and it is genuinely more accurate than one TF32 product would be
    assert np.max(err / bound) < 2.0 ** -14


@pytest.mark.parametrize("batch,m,n,k", [(1, 128, 8, 16), (2, 256, 64, 32), (1, 1024, 128, 64), (3, 128, 4, 4),
                                         (1, 512, 256, 128), (4, 384, 24, 12), (1, 8192, 16, 256), (37, 256, 40, 8),
                                         (2, 256, 24, 100)])
def test_cgemm_bf16x3(env, batch, m, n, k):
    """Split-BF16 product: hi and lo carry 8+8 significand bits, so the
    dropped lo*lo term and the lo roundings leave ~2^-16 |a||b| per product."""
    tz, torch = env
    rng = np.random.default_rng(m + 5 * n + 11 * k)
    A, dA = c64(torch, rng, (batch, m, k))
    B, dB = c64(torch, rng, (batch, n, k))
    dC = torch.zeros(batch * m * n * 2, dtype=torch.float32, device="cuda")
    nbytes = tz.tz_op_cgemm_scratch_bytes("bf16x3", batch, m, n, k)
    scratch = torch.empty(nbytes // 4 + 64, dtype=torch.float32, device="cuda")
    tz.tz_op_cgemm("bf16x3", batch, m, n, k, dA, m * k, dB, n * k, dC, m * n, scratch=scratch)
    torch.cuda.synchronize()
    C = dC.cpu().numpy().view(np.complex64).reshape(batch, m, n)
    ref = linalg.cgemm(A, B)
    bound = linalg.cgemm(np.abs(A).astype(np.complex128), np.abs(B).astype(np.complex128)).real
    err = np.abs(C - ref)
    assert np.all(err <= (2.0 ** -14 + 4 * (k + 2) * 2.0 ** -24) * bound + 1e-30), float(np.max(err / bound))
    assert np.max(err / bound) < 2.0 ** -10   # far better than one BF16 product


def _fp16x3(tz, torch, A, B):
    batch, m, k = A.shape
    n = B.shape[1]
    dA = torch.from_numpy(A.astype(np.complex64).view(np.float32).copy()).cuda()
    dB = torch.from_numpy(B.astype(np.complex64).view(np.float32).copy()).cuda()
    dC = torch.zeros(batch * m * n * 2, dtype=torch.float32, device="cuda")
    nbytes = tz.tz_op_cgemm_scratch_bytes("fp16x3", batch, m, n, k)
    scratch = torch.empty(nbytes // 4 + 64, dtype=torch.float32, device="cuda")
    tz.tz_op_cgemm("fp16x3", batch, m, n, k, dA, m * k, dB, n * k, dC, m * n, scratch=scratch)
    torch.cuda.synchronize()
    return dC.cpu().numpy().view(np.complex64).reshape(batch, m, n)


@pytest.mark.parametrize("batch,m,n,k,ea,eb", [(1, 128, 8, 16, 0, 0), (2, 256, 64, 32, -40, -35),
                                               (1, 1024, 128, 64, 30, -20), (3, 128, 4, 4, -60, 10),
                                               (1, 512, 256, 128, -20, -20), (4, 384, 24, 12, 5, 5),
                                               (1, 8192, 16, 256, -35, 0), (37, 256, 40, 8, 0, -50),
                                               (2, 256, 24, 100, -10, 12)])
def test_cgemm_fp16x3(env, batch, m, n, k, ea, eb):
    """Split-FP16 product with per-tensor power-of-two scaling (the paper's
    amplitudes, near 2^(-n/2), lie below FP16's normal range): operands
    multiplied by 2^ea and 2^eb, far outside FP16's range for most cases, must
    come back with 11+11 significand bits, i.e. split-TF32 accuracy."""
    tz, torch = env
    rng = np.random.default_rng(m + 5 * n + 11 * k + ea)
    A = (rng.standard_normal((batch, m, k)) + 1j * rng.standard_normal((batch, m, k))) * 2.0 ** ea
    B = (rng.standard_normal((batch, n, k)) + 1j * rng.standard_normal((batch, n, k))) * 2.0 ** eb
    A, B = A.astype(np.complex64), B.astype(np.complex64)
    C = _fp16x3(tz, torch, A, B)
    ref = linalg.cgemm(A, B)
    bound = linalg.cgemm(np.abs(A).astype(np.complex128), np.abs(B).astype(np.complex128)).real
    err = np.abs(C - ref)
    assert np.all(err <= (2.0 ** -18 + 4 * (k + 2) * 2.0 ** -24) * bound), float(np.max(err / bound))
    assert np.max(err / bound) < 2.0 ** -16   # one FP16 product would leave ~2^-11


def test_cgemm_fp16x3_zero_and_wide_range(env):
    """A zero operand gives an exact zero product; an operand whose entries
    span 2^-30..2^0 keeps its small entries to the error of its largest."""
    tz, torch = env
    rng = np.random.default_rng(7)
    batch, m, n, k = 2, 256, 16, 64
    A = (rng.standard_normal((batch, m, k)) + 1j * rng.standard_normal((batch, m, k))).astype(np.complex64)
    B0 = np.zeros((batch, n, k), np.complex64)
    assert not np.any(_fp16x3(tz, torch, A, B0))
    B = (rng.standard_normal((batch, n, k)) + 1j * rng.standard_normal((batch, n, k)))
    B *= 2.0 ** -rng.integers(0, 31, size=(batch, n, k))
    B = B.astype(np.complex64)
    C = _fp16x3(tz, torch, A, B)
    ref = linalg.cgemm(A, B)
    bound = linalg.cgemm(np.abs(A).astype(np.complex128), np.abs(B).astype(np.complex128)).real
    scale = np.max(np.abs(A)) * np.max(np.abs(B)) * k
    err = np.abs(C - ref)
    assert np.all(err <= (2.0 ** -18 + 4 * (k + 2) * 2.0 ** -24) * bound + 2.0 ** -36 * scale)


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3", "fp16x3"])
def test_cgemm_tc_many_tiles_scatter_free(env, prec):
    """More tiles than SMs, so each persistent CTA walks several tiles and
    both accumulator buffers are reused."""
    tz, torch = env
    batch, m, n, k = 8, 2048, 256, 64
    rng = np.random.default_rng(99)
    A, dA = c64(torch, rng, (batch, m, k))
    B, dB = c64(torch, rng, (batch, n, k))
    dC = torch.zeros(batch * m * n * 2, dtype=torch.float32, device="cuda")
    nbytes = tz.tz_op_cgemm_scratch_bytes(prec, batch, m, n, k)
    scratch = torch.empty(nbytes // 4 + 64, dtype=torch.float32, device="cuda")
    tz.tz_op_cgemm(prec, batch, m, n, k, dA, m * k, dB, n * k, dC, m * n, scratch=scratch)
    torch.cuda.synchronize()
    C = dC.cpu().numpy().view(np.complex64).reshape(batch, m, n)
    ref = linalg.cgemm(A, B)
    bound = linalg.cgemm(np.abs(A).astype(np.complex128), np.abs(B).astype(np.complex128)).real
    tol = 2.0 ** -14 if prec == "bf16x3" else 2.0 ** -18
    assert np.all(np.abs(C - ref) <= (tol + 4 * (k + 2) * 2.0 ** -24) * bound)


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3", "fp16x3"])
@pytest.mark.parametrize("batch,m,n,k", [(2, 128, 16, 4096), (64, 128, 32, 2048), (1, 256, 8, 1024)])
def test_cgemm_tc_split_k(env, prec, batch, m, n, k):
    """Few output tiles and a long K: the product splits K across CTAs (2 to
    16 ranges for these shapes) and sums the partials in a fixed order, so two
    runs agree bit for bit."""
    tz, torch = env
    rng = np.random.default_rng(batch + m + n + k)
    A, dA = c64(torch, rng, (batch, m, k))
    B, dB = c64(torch, rng, (batch, n, k))
    nbytes = tz.tz_op_cgemm_scratch_bytes(prec, batch, m, n, k)
    scratch = torch.empty(nbytes // 4 + 64, dtype=torch.float32, device="cuda")
    outs = []
    for _ in range(2):
        dC = torch.full((batch * m * n * 2,), float("nan"), dtype=torch.float32, device="cuda")
        tz.tz_op_cgemm(prec, batch, m, n, k, dA, m * k, dB, n * k, dC, m * n, scratch=scratch)
        torch.cuda.synchronize()
        outs.append(dC.cpu().numpy().view(np.complex64).reshape(batch, m, n))
    assert np.array_equal(outs[0], outs[1])
    C = outs[0]
    ref = linalg.cgemm(A, B)
    bound = linalg.cgemm(np.abs(A).astype(np.complex128), np.abs(B).astype(np.complex128)).real
    tol = 2.0 ** -14 if prec == "bf16x3" else 2.0 ** -18
    err = np.abs(C - ref)
    assert np.all(err <= (tol + 4 * (k + 2) * 2.0 ** -24) * bound), float(np.max(err / bound))


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3", "fp16x3"])
def test_cgemm_tc_accumulation_bias(env, prec):
    """The tensor cores' FP32 accumulation rounds toward zero, so a product
    summed over K real values in one accumulator comes out smaller by about
    6e-9 K (2.5e-5 measured for 4096 values per accumulator). The kernel adds
    ranges of 128 real values in FP32 registers instead: over K = 16384
    complex the mean shrink (the error's component along the exact result)
    stays near 6e-9 x 128, checked below 3e-6."""
    tz, torch = env
    batch, m, n, k = 2, 256, 16, 16384
    rng = np.random.default_rng(4242)
    A, dA = c64(torch, rng, (batch, m, k))
    B, dB = c64(torch, rng, (batch, n, k))
    dC = torch.zeros(batch * m * n * 2, dtype=torch.float32, device="cuda")
    nbytes = tz.tz_op_cgemm_scratch_bytes(prec, batch, m, n, k)
    scratch = torch.empty(nbytes // 4 + 64, dtype=torch.float32, device="cuda")
    tz.tz_op_cgemm(prec, batch, m, n, k, dA, m * k, dB, n * k, dC, m * n, scratch=scratch)
    torch.cuda.synchronize()
    C = dC.cpu().numpy().view(np.complex64).reshape(batch, m, n).astype(np.complex128)
    ref = linalg.cgemm(A, B)
    d = C - ref
    shrink = float(np.sum((d * np.conj(ref)).real) / np.sum(np.abs(ref) ** 2))
    rel = float(np.sqrt(np.sum(np.abs(d) ** 2) / np.sum(np.abs(ref) ** 2)))
    print(f"{prec} K={k}: mean shrink {shrink:.2e}, relative error {rel:.2e}")
    assert abs(shrink) < 3e-6
    assert rel < 1e-5


def test_cgemm_tc_rejects_unsupported(env):
    tz, torch = env
    with pytest.raises(tz.TzError) as e:
        tz.tz_op_cgemm_scratch_bytes("tf32x3", 1, 64, 8, 8)   # M below one 128-row tile
    assert e.value.code == -6


@pytest.mark.parametrize("batch,m,n,k", [(1, 7, 3, 5), (3, 64, 64, 8), (2, 130, 17, 33), (1, 4, 1, 4096)])
def test_cgemm_c128(env, batch, m, n, k):
    """complex128 product (FP64 FMA): agrees with the complex128 definition
    to FP64 rounding."""
    tz, torch = env
    rng = np.random.default_rng(m * 13 + k)
    A = rng.standard_normal((batch, m, k)) + 1j * rng.standard_normal((batch, m, k))
    B = rng.standard_normal((batch, n, k)) + 1j * rng.standard_normal((batch, n, k))
    dA = torch.from_numpy(A.view(np.float64).copy()).cuda()
    dB = torch.from_numpy(B.view(np.float64).copy()).cuda()
    dC = torch.zeros(batch * m * n * 2, dtype=torch.float64, device="cuda")
    tz.tz_op_cgemm("c128", batch, m, n, k, dA, m * k, dB, n * k, dC, m * n)
    torch.cuda.synchronize()
    C = dC.cpu().numpy().view(np.complex128).reshape(batch, m, n)
    ref = linalg.cgemm(A, B)
    bound = linalg.cgemm(np.abs(A), np.abs(B)).real
    assert np.all(np.abs(C - ref) <= 4 * (k + 2) * 2.0 ** -53 * bound)


def test_accumulate_fp64(env):
    tz, torch = env
    rng = np.random.default_rng(5)
    part, dpart = c64(torch, rng, 1000)
    acc0 = (rng.standard_normal(1000) + 1j * rng.standard_normal(1000)) * 1e-12
    dacc = torch.from_numpy(acc0.view(np.float64).copy()).cuda()
    s = 0.25 - 0.5j
    tz.tz_op_accumulate(dpart, dacc, 1000, s)
    torch.cuda.synchronize()
    got = dacc.cpu().numpy().view(np.complex128)
    ref = linalg.accumulate(acc0, part, s)
    assert np.max(np.abs(got - ref)) <= 1e-15 * np.max(np.abs(ref))


@pytest.mark.parametrize("prec", ["bf16x3", "fp16x3"])
@pytest.mark.parametrize("batch,m,n,k", [(2, 256, 64, 32), (1, 1024, 128, 64), (3, 512, 100, 72),
                                         (1, 256, 64, 8192), (2, 4096, 256, 512)])
def test_cgemm_pairs_match_single_cta(env, prec, batch, m, n, k):
    """Products on pairs of CTAs (cta_group::2: M = 256 per pair, each CTA
    loading half of the B tile) against the same products on single CTAs and
    against the complex128 definition: ragged column tiles (n = 100), a
    ragged last k-block (k = 72), split K (k = 8192 over two tiles)."""
    tz, torch = env
    rng = np.random.default_rng(m + 13 * n + 17 * k)
    A, dA = c64(torch, rng, (batch, m, k))
    B, dB = c64(torch, rng, (batch, n, k))
    nbytes = tz.tz_op_cgemm_scratch_bytes(prec, batch, m, n, k)
    scratch = torch.empty(nbytes // 4 + 64, dtype=torch.float32, device="cuda")
    out = {}
    try:
        for mode in (0, 1):
            tz.tz_tune_tc_pairs(mode)
            dC = torch.full((batch * m * n * 2,), float("nan"), dtype=torch.float32, device="cuda")
            tz.tz_op_cgemm(prec, batch, m, n, k, dA, m * k, dB, n * k, dC, m * n, scratch=scratch)
            tz.tz_op_cgemm_status(prec, scratch)
            out[mode] = dC.cpu().numpy().view(np.complex64).reshape(batch, m, n)
    finally:
        tz.tz_tune_tc_pairs(-1)
    ref = linalg.cgemm(A, B)
    bound = linalg.cgemm(np.abs(A).astype(np.complex128), np.abs(B).astype(np.complex128)).real
    for mode, C in out.items():
        assert np.all(np.isfinite(C)), mode
        err = np.abs(C - ref)
        assert np.all(err <= (2.0 ** -14 + 4 * (k + 2) * 2.0 ** -24) * bound + 1e-30), (mode, float(np.max(err / bound)))
    # the same splits and the same accumulation ranges: the two forms agree to
    # the FP32 rounding of the accumulation
    diff = np.abs(out[1] - out[0])
    print(f"{prec} {batch}x{m}x{n}x{k}: pairs vs single CTA max |diff|/bound {np.max(diff / bound):.2e}, "
          f"bit-identical {np.array_equal(out[1], out[0])}")
    assert np.all(diff <= 4 * (k + 2) * 2.0 ** -24 * bound + 1e-30)
