"""The allocation-free SSIM2D entry point (gs_ssim2d_loss_noalloc) against the workspace
version (gs_ssim2d_loss), through the C ABI.

gs_ssim2d_loss_noalloc serves callers that cannot allocate device memory themselves (a host
framework that owns the device memory budget, or a loop where an allocation's implicit
synchronisation is not acceptable): its scratch is a fixed array inside the library.  Two
calls in a row must each match the workspace version, which also shows that the shared
scratch keeps no state that leaks from one call into the next.  Kept in a file of its own that
pytest collects last.
"""
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


def _inputs(seed, shape):
    rng = np.random.default_rng(seed)
    y = rng.random(shape, dtype=np.float32)
    x = np.clip(y + 0.1 * rng.standard_normal(shape).astype(np.float32), 0, None)
    return torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(), float(y.max())


def _workspace_version(B, x, y, L, weight, grad0=None, with_loss=True):
    n, H, W = x.shape
    loss = torch.zeros(1, device="cuda")
    grad = torch.zeros_like(x) if grad0 is None else grad0.clone()
    ws = torch.empty(B.lib().gs_ssim_workspace_size(x.numel()), dtype=torch.uint8, device="cuda")
    B.check(B.lib().gs_ssim2d_loss(B.ptr(x), B.ptr(y), n, H, W, L, weight,
                                   B.ptr(loss) if with_loss else None, B.ptr(grad),
                                   0 if grad0 is None else 1, B.ptr(ws), ws.numel(),
                                   torch.cuda.current_stream().cuda_stream), "gs_ssim2d_loss")
    return loss, grad


def _noalloc_version(B, x, y, L, weight, grad0=None, with_loss=True):
    n, H, W = x.shape
    loss = torch.zeros(1, device="cuda")
    grad = torch.zeros_like(x) if grad0 is None else grad0.clone()
    B.check(B.lib().gs_ssim2d_loss_noalloc(B.ptr(x), B.ptr(y), n, H, W, L, weight,
                                           B.ptr(loss) if with_loss else None, B.ptr(grad),
                                           0 if grad0 is None else 1,
                                           torch.cuda.current_stream().cuda_stream),
            "gs_ssim2d_loss_noalloc")
    return loss, grad


def test_noalloc_matches_workspace_version_twice(B):
    # two calls in a row with different sizes; the second is smaller, so any stale scratch
    # from the first would show up if the kernels read entries they did not write
    for seed, shape in ((0, (8, 512, 512)), (1, (3, 77, 45))):
        x, y, L = _inputs(seed, shape)
        want_loss, want_grad = _workspace_version(B, x, y, L, 0.25)
        got_loss, got_grad = _noalloc_version(B, x, y, L, 0.25)
        torch.cuda.synchronize()
        assert abs(float(got_loss) - float(want_loss)) <= 1e-5 * max(1.0, abs(float(want_loss)))
        scale = float(want_grad.abs().max())
        assert float((got_grad - want_grad).abs().max()) <= 1e-5 * scale


def test_noalloc_accumulates_and_takes_no_loss_pointer(B):
    """accumulate = 1 adds onto a non-zero gradient, and d_loss = NULL computes the gradient
    alone; both equal the workspace version called the same way."""
    x, y, L = _inputs(3, (4, 96, 80))
    grad0 = torch.randn_like(x)
    want_loss, want_grad = _workspace_version(B, x, y, L, 0.5, grad0=grad0)
    got_loss, got_grad = _noalloc_version(B, x, y, L, 0.5, grad0=grad0)
    torch.cuda.synchronize()
    assert abs(float(got_loss) - float(want_loss)) <= 1e-5 * max(1.0, abs(float(want_loss)))
    scale = float(want_grad.abs().max())
    assert float((got_grad - want_grad).abs().max()) <= 1e-5 * scale
    assert float((got_grad - grad0).abs().max()) > 0
    _, want_grad = _workspace_version(B, x, y, L, 0.5, with_loss=False)
    loss, got_grad = _noalloc_version(B, x, y, L, 0.5, with_loss=False)
    torch.cuda.synchronize()
    assert float(loss) == 0.0
    assert float((got_grad - want_grad).abs().max()) <= 1e-5 * float(want_grad.abs().max())


def test_noalloc_rejects_oversize(B):
    x, y, L = _inputs(2, (1, 8, 8))
    loss = torch.zeros(1, device="cuda")
    grad = torch.zeros_like(x)
    # 9 images of 512 x 512 = 2,359,296 pixels > GS_SSIM2D_NOALLOC_MAX_PIXELS (2,097,152);
    # rejected on the host from the sizes alone, before any kernel touches the buffers
    rc = B.lib().gs_ssim2d_loss_noalloc(B.ptr(x), B.ptr(y), 9, 512, 512, L, 1.0, B.ptr(loss),
                                        B.ptr(grad), 0, torch.cuda.current_stream().cuda_stream)
    assert rc == B.GS_ERR_CAPACITY
    assert b"GS_SSIM2D_NOALLOC_MAX_PIXELS" in B.lib().gs_last_error()
