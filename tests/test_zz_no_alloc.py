"""The allocation-free reconstruction entry point against the allocating one.

ttice_reconstruct_noalloc exists for callers that cannot allocate device memory at the moment they
reconstruct (for example while capturing a CUDA graph that must contain no allocation nodes); it
keeps its intermediates in a fixed array inside the library.  Its output must equal that of
ttice_reconstruct, on two calls in a row (the second call reuses the array the first one left
behind), and a request larger than the fixed array must be refused.
"""
import numpy as np
import pytest
import torch

from tt_streams import blob_video

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2211_12487_gb300 import ttice

    return ttice


def test_noalloc_reconstruct_matches_allocating_one(T):
    view = (6, 8, 8, 8, 3)
    Y = blob_video(0, 16, height=48, width=64, n_blobs=5, sigma=(3, 10), view=view, seed=21).cuda()
    g = T.TTICE(view, 0.05, input_dtype=torch.float32, max_batch=8)
    for k in range(0, 16, 8):
        g.update(Y[k:k + 8])
    for dtype in (torch.float64, torch.float32):
        ref = torch.empty((16,) + view, dtype=dtype, device="cuda")
        T.ttice_reconstruct(g.h, 0, 16, ref)
        for _ in range(2):  # two calls in a row through the same fixed scratch
            out = torch.full((16,) + view, float("nan"), dtype=dtype, device="cuda")
            T.ttice_reconstruct_noalloc(g.h, 0, 16, out)
            torch.cuda.synchronize()
            a, b = out.double().cpu().numpy(), ref.double().cpu().numpy()
            tol = 1e-12 if dtype == torch.float64 else 1e-6
            assert np.isfinite(a).all()
            assert np.abs(a - b).max() <= tol * np.abs(b).max()
        # a sub-range, also twice
        ref2 = torch.empty((5,) + view, dtype=dtype, device="cuda")
        T.ttice_reconstruct(g.h, 7, 5, ref2)
        for _ in range(2):
            out2 = torch.empty((5,) + view, dtype=dtype, device="cuda")
            T.ttice_reconstruct_noalloc(g.h, 7, 5, out2)
            torch.cuda.synchronize()
            assert torch.allclose(out2.double(), ref2.double(), rtol=0, atol=float(tol * ref2.abs().max()))
    g.close()


def test_noalloc_rejects_requests_beyond_its_scratch(T):
    view = (20, 24, 20, 32, 3)  # 921600 elements per observation
    Y = blob_video(0, 8).cuda()
    g = T.TTICE(view, 0.1, input_dtype=torch.float32, max_batch=8)
    g.update(Y)
    n_fit = T.TTICE_NOALLOC_MAX_ELEMS // (20 * 24 * 20 * 32 * 3)
    assert 1 <= n_fit < 8
    out = torch.empty((8,) + view, dtype=torch.float32, device="cuda")
    with pytest.raises(T.TTICEError) as ei:
        T.ttice_reconstruct_noalloc(g.h, 0, 8, out)
    assert ei.value.code == T.TTICE_EINVAL
    ref = torch.empty((n_fit,) + view, dtype=torch.float32, device="cuda")
    T.ttice_reconstruct(g.h, 0, n_fit, ref)
    T.ttice_reconstruct_noalloc(g.h, 0, n_fit, out[:n_fit])
    torch.cuda.synchronize()
    assert torch.allclose(out[:n_fit], ref, rtol=0, atol=1e-6 * float(ref.abs().max()))
    g.close()
