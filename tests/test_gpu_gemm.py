"""The tcgen05 BF16 GEMM (hesp_gemm_bf16) against a float64 matmul of the same
bf16 operands: fp32 outputs within a relative error set by fp32 accumulation
over K, bf16 outputs within one bf16 rounding step; ragged M, N; every
epilogue (fp32, bias + ReLU with the transposed copy, ReLU-mask)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.mlp_ref import bf16_round  # noqa: E402
from paper_1602_05510_b300 import hesp  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1602_05510_b300 import build
    build.build()


def rand_bf16(shape, rng, scale=1.0):
    return bf16_round(rng.standard_normal(shape) * scale)


def dev(x, dtype=torch.bfloat16):
    return torch.from_numpy(np.asarray(x, np.float32)).to(dtype).cuda()


SHAPES = [(128, 128, 64), (256, 128, 128), (300, 200, 192), (128, 384, 1024), (1000, 512, 512), (4096, 512, 2496)]


@pytest.mark.parametrize("M,N,K", SHAPES)
def test_gemm_f32(M, N, K):
    rng = np.random.default_rng(M + N + K)
    A, B = rand_bf16((M, K), rng), rand_bf16((N, K), rng)
    C = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    hesp.gemm_bf16(dev(A), dev(B), hesp.GEMM_F32, C=C, err=err)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    ref = A @ B.T
    got = C.cpu().numpy().astype(np.float64)
    tol = 1e-5 * np.sqrt(K) * (np.abs(A) @ np.abs(B).T + 1e-3)
    assert np.all(np.abs(got - ref) <= tol)


@pytest.mark.parametrize("M,N,K", SHAPES[:4])
def test_gemm_bias_relu_and_transpose(M, N, K):
    rng = np.random.default_rng(7 + M)
    A, B = rand_bf16((M, K), rng), rand_bf16((N, K), rng)
    bias = rng.standard_normal(N).astype(np.float32)
    out = torch.zeros((M, N), dtype=torch.bfloat16, device="cuda")
    out_t = torch.zeros((N, M), dtype=torch.bfloat16, device="cuda")
    hesp.gemm_bf16(dev(A), dev(B), hesp.GEMM_BIAS_RELU, bias=torch.from_numpy(bias).cuda(), out=out, out_t=out_t)
    torch.cuda.synchronize()
    ref = np.maximum(A @ B.T + bias.astype(np.float64), 0)
    got = out.float().cpu().numpy().astype(np.float64)
    assert np.array_equal(got, out_t.float().cpu().numpy().T)
    # one bf16 rounding of an fp32 sum: within one bf16 step of the exact value
    assert np.all(np.abs(got - ref) <= 2 ** -7 * np.abs(ref) + 1e-6 * np.sqrt(K))
    assert np.mean(got == bf16_round(ref)) > 0.98


def test_gemm_mask():
    rng = np.random.default_rng(3)
    M, N, K = 384, 256, 256
    A, B = rand_bf16((M, K), rng), rand_bf16((N, K), rng)
    mask = bf16_round(rng.standard_normal((M, N)))
    out = torch.zeros((M, N), dtype=torch.bfloat16, device="cuda")
    hesp.gemm_bf16(dev(A), dev(B), hesp.GEMM_MASK, mask=dev(mask), out=out)
    torch.cuda.synchronize()
    ref = (A @ B.T) * (mask > 0)
    got = out.float().cpu().numpy().astype(np.float64)
    assert np.all(np.abs(got - ref) <= 2 ** -7 * np.abs(ref) + 1e-6 * np.sqrt(K))
    assert (got[mask <= 0] == 0).all()


def test_gemm_rejects_bad_shapes():
    a = torch.zeros((128, 100), dtype=torch.bfloat16, device="cuda")
    C = torch.zeros((128, 128), dtype=torch.float32, device="cuda")
    with pytest.raises(hesp.HespError):
        hesp.gemm_bf16(a, a, hesp.GEMM_F32, C=C)   # K = 100 not a multiple of 64


# The persistent kernel runs min(tiles, SMs) CTAs, each walking output tiles
# of 128 x 256; these shapes give every CTA several tiles (both TMEM
# accumulators, the epilogue of one tile under the next tile's main loop, and
# the mbarrier phases carried across tiles): 65,536 x 512 is 1,024 tiles (the
# surrogate's inference chunk, K = 2,496 for the 816-task one-hot layer and
# K = 512 for layer 2); 512 x 23,936 with K = 512 is 376 tiles (the
# weight-gradient GEMM dW1 = dZ1^T X of the 5,984-task, 4-level first layer);
# 40,000 x 640 is ragged in both M and N.
MULTI = [(65536, 512, 2496), (65536, 512, 512), (512, 23936, 512), (40000, 640, 256)]


def _ref64(A, B):
    return torch.from_numpy(A).double() @ torch.from_numpy(B).double().T


def _absbound(A, B):
    return torch.from_numpy(np.abs(A)).double() @ torch.from_numpy(np.abs(B)).double().T


@pytest.mark.parametrize("M,N,K", MULTI)
def test_gemm_f32_multi_tile(M, N, K):
    rng = np.random.default_rng(M + 3 * N + K)
    A, B = rand_bf16((M, K), rng).astype(np.float32), rand_bf16((N, K), rng).astype(np.float32)
    C = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    hesp.gemm_bf16(dev(A), dev(B), hesp.GEMM_F32, C=C, err=err)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    ref = _ref64(A, B)
    bound = _absbound(A, B)
    got = C.cpu().double()
    # every element: fp32 accumulation over K of exact bf16 products
    assert bool(torch.all((got - ref).abs() <= 1e-5 * np.sqrt(K) * (bound + 1e-3)))


@pytest.mark.parametrize("M,N,K", MULTI[:2] + MULTI[3:])
def test_gemm_bias_relu_multi_tile(M, N, K):
    rng = np.random.default_rng(11 + M + N)
    A, B = rand_bf16((M, K), rng).astype(np.float32), rand_bf16((N, K), rng).astype(np.float32)
    bias = rng.standard_normal(N).astype(np.float32)
    out = torch.zeros((M, N), dtype=torch.bfloat16, device="cuda")
    out_t = torch.zeros((N, M), dtype=torch.bfloat16, device="cuda")
    hesp.gemm_bf16(dev(A), dev(B), hesp.GEMM_BIAS_RELU, bias=torch.from_numpy(bias).cuda(), out=out, out_t=out_t)
    torch.cuda.synchronize()
    ref = torch.clamp(_ref64(A, B) + torch.from_numpy(bias).double(), min=0)
    got = out.cpu().double()
    assert torch.equal(out.cpu(), out_t.cpu().T)
    # got = bf16(relu(s)) with s the fp32 sum, |s - exact| <= e (the bound of
    # the fp32 test); relu is 1-Lipschitz and the bf16 rounding moves a value
    # by at most 2^-8 of it, so |got - ref| <= 2^-8 (|ref| + e) + e
    e = 1e-5 * np.sqrt(K) * (_absbound(A, B) + torch.from_numpy(np.abs(bias).astype(np.float64))[None, :] + 1e-3)
    assert bool(torch.all((got - ref).abs() <= 2 ** -7 * ref.abs() + 2 * e))
    assert float((got == torch.from_numpy(bf16_round(ref.numpy()))).double().mean()) > 0.98


def test_gemm_mask_multi_tile():
    rng = np.random.default_rng(5)
    M, N, K = 65536, 512, 512
    A, B = rand_bf16((M, K), rng).astype(np.float32), rand_bf16((N, K), rng).astype(np.float32)
    mask = bf16_round(rng.standard_normal((M, N))).astype(np.float32)
    out = torch.zeros((M, N), dtype=torch.bfloat16, device="cuda")
    out_t = torch.zeros((N, M), dtype=torch.bfloat16, device="cuda")
    hesp.gemm_bf16(dev(A), dev(B), hesp.GEMM_MASK, mask=dev(mask), out=out, out_t=out_t)
    torch.cuda.synchronize()
    keep = torch.from_numpy(mask > 0)
    ref = _ref64(A, B) * keep
    got = out.cpu().double()
    assert torch.equal(out.cpu(), out_t.cpu().T)
    e = 1e-5 * np.sqrt(K) * (_absbound(A, B) + 1e-3)
    assert bool(torch.all((got - ref).abs() <= 2 ** -7 * ref.abs() + 2 * e))
    assert bool(torch.all(got[~keep] == 0))
