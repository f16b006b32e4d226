"""The tcgen05 BF16 GEMM against a float64 matmul of the same bf16-rounded operands."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_01844_gb300 import binding, build

    build.build()
    return binding


def _bf16(a):
    return torch.from_numpy(a.astype(np.float32)).to(torch.bfloat16)


@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (256, 128, 256), (384, 256, 4096),
                                   (1024, 384, 256), (256, 512, 192), (128, 4096, 128),
                                   (19456, 256, 128), (9728, 512, 256)])
@pytest.mark.parametrize("relu", [0, 1])
def test_gemm_matches_float64(B, M, N, K, relu):
    """The last two shapes fill the GPU's SMs with 128 x 256 tiles, the others use 128 x 128."""
    rng = np.random.default_rng(M + N + K)
    a = _bf16(rng.standard_normal((M, K)))
    b = _bf16(rng.standard_normal((N, K)))
    bias = torch.from_numpy(rng.standard_normal(N).astype(np.float32))
    want = a.double() @ b.double().T + bias.double()
    if relu:
        want = want.clamp_min(0)
    da, db, dbias = a.cuda(), b.cuda(), bias.cuda()
    c32 = torch.empty((M, N), device="cuda")
    c16 = torch.empty((M, N), dtype=torch.bfloat16, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    B.check(B.lib().gs_gemm_bf16(B.ptr(da), B.ptr(db), M, N, K, B.ptr(dbias), relu, B.ptr(c32),
                                 B.ptr(c16), N, B.ptr(err),
                                 torch.cuda.current_stream().cuda_stream), "gemm")
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    got = c32.cpu().double()
    # FP32 accumulation of K products of bf16 values: error ~ K * 2^-24 * sum|a b|
    bound = 2e-6 * K ** 0.5 * (a.double().abs() @ b.double().abs().T) + 1e-6
    assert bool(((got - want).abs() <= bound).all()), float((got - want).abs().max())
    assert torch.allclose(c16.cpu().double(), got, rtol=1e-2, atol=1e-2)


@pytest.mark.parametrize("M,N,K", [(118016, 256, 4096), (256, 4096, 118016)])
def test_gemm_mlp_full_shapes_sampled(B, M, N, K):
    """The benchmark's largest layer shapes (the first layer's forward over 118,016 bricks and
    its weight gradient with K = 118,016), 512 sampled outputs against float64 dot products of
    the same bf16-rounded rows."""
    rng = np.random.default_rng(M + 7 * N)
    a = _bf16(rng.standard_normal((M, K), dtype=np.float32))
    b = _bf16(rng.standard_normal((N, K), dtype=np.float32))
    da, db = a.cuda(), b.cuda()
    c32 = torch.empty((M, N), device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    B.check(B.lib().gs_gemm_bf16(B.ptr(da), B.ptr(db), M, N, K, None, 0, B.ptr(c32), None, N,
                                 B.ptr(err), torch.cuda.current_stream().cuda_stream), "gemm")
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    i = rng.integers(0, M, 512)
    j = rng.integers(0, N, 512)
    got = c32[torch.from_numpy(i).cuda(), torch.from_numpy(j).cuda()].cpu().double()
    ra, rb = a[torch.from_numpy(i)].double(), b[torch.from_numpy(j)].double()
    want = (ra * rb).sum(dim=1)
    bound = 2e-6 * K ** 0.5 * (ra.abs() * rb.abs()).sum(dim=1) + 1e-6
    assert bool(((got - want).abs() <= bound).all()), float((got - want).abs().max())


def test_gemm_rejects_bad_shapes(B):
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    x = torch.zeros((128, 64), dtype=torch.bfloat16, device="cuda")
    rc = B.lib().gs_gemm_bf16(B.ptr(x), B.ptr(x), 100, 128, 64, None, 0, B.ptr(x), None, 128,
                              B.ptr(err), torch.cuda.current_stream().cuda_stream)
    assert rc == B.GS_ERR_ARG


@pytest.mark.parametrize("ldc", [260, 264])
def test_gemm_row_stride(B, ldc):
    """Outputs with a row stride wider than N: ldc % 8 == 0 takes the 16-byte store epilogue,
    other strides the per-element one; both leave the padding columns untouched."""
    M, N, K = 256, 256, 128
    rng = np.random.default_rng(ldc)
    a = _bf16(rng.standard_normal((M, K)))
    b = _bf16(rng.standard_normal((N, K)))
    want = a.double() @ b.double().T
    c32 = torch.full((M, ldc), 7.0, device="cuda")
    c16 = torch.full((M, ldc), 7.0, dtype=torch.bfloat16, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    da, db = a.cuda(), b.cuda()  # held: the library reads them after the call returns
    B.check(B.lib().gs_gemm_bf16(B.ptr(da), B.ptr(db), M, N, K, None, 0, B.ptr(c32),
                                 B.ptr(c16), ldc, B.ptr(err),
                                 torch.cuda.current_stream().cuda_stream), "gemm")
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    got = c32[:, :N].cpu().double()
    bound = 2e-6 * K ** 0.5 * (a.double().abs() @ b.double().abs().T) + 1e-6
    assert bool(((got - want).abs() <= bound).all())
    assert torch.allclose(c16[:, :N].cpu().double(), got, rtol=1e-2, atol=1e-2)
    assert bool((c32[:, N:] == 7.0).all()) and bool((c16[:, N:] == 7.0).all())
