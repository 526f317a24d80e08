"""The large workloads on the FP32 path: the 1080x1920x3 video (27x40x48x40x3, batches of 32,
eps = 0.05, scene cut) and the 128^3 x 4 Fourier flow (batches of 16, eps = 0.05 and 0.01).

The oracle cannot run these sizes in a test's time, so the checks are the paper's guarantees on the
GPU result itself: every increment is represented within eps (Theorem 1 / Corollary 1, measured
from the GPU reconstruction in FP64), earlier observations are unchanged by later updates
(Theorem 2), and every core is orthonormal.  These runs exercise Gram sides above 1000, more new
directions in one update than one Rayleigh-Ritz problem holds (chunked append) and the generic
first-pass path for n_1 = 128.
"""
import math

import numpy as np
import pytest
import torch

from tt_streams import blob_video, fourier_flow

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2211_12487_gb300 import ttice

    return ttice


def _run(T, frames_fn, dims, b, eps, n_inc, max_rank=512):
    g = T.TTICE(dims, eps, precision="fp32", input_dtype=torch.float32, max_batch=b, max_rank=max_rank)
    first = None
    for k in range(n_inc):
        Y = frames_fn(k * b, b)
        g.update(Y)
        rec = g.reconstruct(k * b, b)
        err = math.sqrt(float(((Y.double() - rec) ** 2).sum()) / float((Y.double() ** 2).sum()))
        assert err <= eps * (1 + 1e-6), (k, err)
        if k == 0:
            first = rec.clone()
        else:  # Theorem 2: the first increment's reconstruction is unchanged by later updates
            again = g.reconstruct(0, b)
            assert float((again - first).abs().max()) <= 1e-9 * float(first.abs().max())
        del Y, rec
    for i in range(1, len(dims) + 1):
        U = g.core(i)
        assert np.abs(U.T @ U - np.eye(U.shape[1])).max() < 1e-9
    ranks = g.ranks()
    g.close()
    return ranks


def test_large_video_27x40x48x40x3(T):
    """40 blobs on 1080x1920x3 frames.  At the video stream's pixel noise (0.01) these sparse frames
    are ~9% noise by energy, above the 5% target, so TT-ICE has to represent the noise and the
    ranks run to the capacity within one increment; the test uses noise 0.002 (signal-dominated
    frames) to keep ranks within a test-sized capacity."""
    dims = (27, 40, 48, 40, 3)

    def frames(t0, n):
        return blob_video(t0, n, height=1080, width=1920, n_blobs=40, view=dims, scene_len=500,
                          noise_std=0.002, seed=1004, device="cuda")

    ranks = _run(T, frames, dims, 32, 0.05, 2, max_rank=1024)
    assert ranks[1] >= 1


@pytest.mark.parametrize("eps", [0.05, 0.01])
def test_flow_128cubed_x4(T, eps):
    """The simulation-shaped stream at both of its workload's tolerances (eps = 0.01 keeps more
    modes: larger ranks and Gram sides on the inner cores)."""
    dims = (128, 128, 128, 4)

    def frames(t0, n):
        return fourier_flow(t0, n, device="cuda")

    ranks = _run(T, frames, dims, 16, eps, 2, max_rank=2048)
    assert ranks[1] <= 33  # cos/sin of at most 17 distinct |k_1| values per mode-1 fibre
