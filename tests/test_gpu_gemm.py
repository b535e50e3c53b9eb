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
