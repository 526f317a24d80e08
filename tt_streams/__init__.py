"""Seeded synthetic tensor streams shaped like the paper's workloads.

The paper evaluates TT-ICE on ATARI game frames (Sec. 5.2.1), self-oscillating gel simulations
(Sec. 5.2.2) and an exactly low-rank synthetic TT stream (Appendix B).  None of those datasets is
available, so these generators stand in for them.  This module holds none of the TT-ICE arithmetic:
it only draws inputs.  Both the CPU oracle and the CUDA path consume its output, so every stream is
produced once (on any torch device, in float64) and then cast to the requested dtype.

Every frame is a pure function of (seed, frame index): a stream can be generated in any chunking and
on any device and describes the same signal (the Gaussian noise draws use one torch generator per
frame, so CPU and CUDA noise differ; parity tests therefore copy one generated tensor to both sides).

Streams (observation shape, then the layout of one observation in memory, C order):

* ``cp_cosine``      -- sum of R rank-1 terms with cosine coefficients plus Gaussian noise
                        (exactly rank R up to the noise).  16^4, R=6 is the small FP64 workload.
* ``blob_video``     -- frames of moving Gaussian blobs, H x W x 3, viewed as a 5-way tensor
                        (480x640x3 -> 20x24x20x32x3; 1080x1920x3 -> 27x40x48x40x3).
* ``fourier_flow``   -- G^3 grid x F fields, each a sum of Fourier modes with |k|^(-5/3) amplitude
                        advected at constant velocity (a simulation-shaped, exactly low-rank stream).
* ``random_tt``      -- slices along the last mode of a random tensor train with prescribed TT-ranks
                        (the Appendix B test bed: 10x15x20x500, ranks [1,2,3,5,1] or [1,4,10,30,1]).
"""
from __future__ import annotations

import math

import torch

__all__ = [
    "cp_cosine",
    "blob_video",
    "fourier_flow",
    "random_tt",
    "STREAMS",
]


def _gen(device, *keys: int) -> torch.Generator:
    """A torch generator on ``device`` seeded from a tuple of small non-negative integers."""
    s = 0x9E3779B97F4A7C15
    for k in keys:
        s = (s ^ (int(k) & 0xFFFFFFFFFFFF)) * 0x100000001B3 & 0xFFFFFFFFFFFFFFFF
    g = torch.Generator(device=device)
    g.manual_seed(s & 0x7FFFFFFFFFFFFFFF)
    return g


def _params_gen(*keys: int) -> torch.Generator:
    # stream parameters are always drawn on the CPU so that every device sees the same signal
    return _gen("cpu", *keys)


def _noise(frames, t_index, seed, std, device):
    """Add N(0, std^2) noise to each frame from a generator keyed by (seed, frame index)."""
    if std == 0.0:
        return frames
    for i, t in enumerate(t_index):
        g = _gen(device, seed, 0xA0A0, int(t))
        frames[i] += std * torch.randn(frames[i].shape, generator=g, device=device, dtype=frames.dtype)
    return frames


def cp_cosine(t0: int, count: int, *, dims=(16, 16, 16, 16), rank: int = 6, freq: float = 0.05,
              noise_std: float = 1e-6, seed: int = 1000, dtype=torch.float64, device="cpu"):
    """Frames t = t0+1 .. t0+count of  Y_t = sum_j cos(freq*j*t + phi_j) a_j (x) b_j (x) ... + noise.

    Factor vectors are N(0,1) draws normalised to unit length, phases phi_j ~ U[0, 2pi).
    Returns a tensor of shape (count, *dims).
    """
    g = _params_gen(seed, 1)
    factors = []
    for n in dims:
        f = torch.randn(n, rank, generator=g, dtype=torch.float64)
        factors.append((f / f.norm(dim=0, keepdim=True)).to(device))
    phi = (2 * math.pi * torch.rand(rank, generator=g, dtype=torch.float64)).to(device)
    t = torch.arange(t0 + 1, t0 + count + 1, dtype=torch.float64, device=device)
    j = torch.arange(1, rank + 1, dtype=torch.float64, device=device)
    coef = torch.cos(freq * t[:, None] * j[None, :] + phi[None, :])  # (count, rank)
    # explicit outer product, one mode at a time: shape (count, rank, n1, n2, ...)
    x = coef.reshape(count, rank)
    for f in factors:
        x = x.unsqueeze(-1) * f.T.reshape((1, rank) + (1,) * (x.dim() - 2) + (f.shape[0],))
    frames = x.sum(dim=1)
    frames = _noise(frames, range(t0 + 1, t0 + count + 1), seed, noise_std, device)
    return frames.to(dtype)


def blob_video(t0: int, count: int, *, height: int = 480, width: int = 640, channels: int = 3,
               n_blobs: int = 12, sigma=(8.0, 40.0), speed: float = 2.0, noise_std: float = 0.01,
               scene_len: int = 0, view=(20, 24, 20, 32, 3), seed: int = 1001,
               dtype=torch.float32, device="cpu", compute_dtype=torch.float64):
    """Frames t0 .. t0+count-1 of moving Gaussian blobs, returned with shape (count, *view).

    Each blob has sigma ~ U[sigma], per-channel amplitude ~ U(0,1), a start position uniform in the
    frame and a velocity ~ U(-speed, speed) px/frame per axis; positions reflect at the borders.
    With ``scene_len > 0`` every ``scene_len`` frames start a new scene with freshly drawn blobs.
    The frame is H x W x C in C order, then viewed as ``view`` (same memory order).
    ``compute_dtype`` is the arithmetic of the frame synthesis (blob parameters are always drawn in
    float64): float64 by default; float32 gives the same stream to ~1e-7 relative at a fraction of
    the cost on GPUs with slow FP64 (large frames for benchmarks, never for oracle comparisons,
    which copy one generated tensor to both sides anyway).
    """
    assert math.prod(view) == height * width * channels
    cdt = compute_dtype
    out = torch.empty((count, height, width, channels), dtype=cdt, device=device)
    yy = torch.arange(height, dtype=cdt, device=device)
    xx = torch.arange(width, dtype=cdt, device=device)

    def reflect(p, size):
        q = torch.remainder(p, 2.0 * size)
        return torch.where(q < size, q, 2.0 * size - q)

    t = t0
    while t < t0 + count:
        scene = t // scene_len if scene_len > 0 else 0
        scene_end = (scene + 1) * scene_len if scene_len > 0 else t0 + count
        stop = min(t0 + count, scene_end)
        g = _params_gen(seed, 2, scene)
        sig = sigma[0] + (sigma[1] - sigma[0]) * torch.rand(n_blobs, generator=g, dtype=torch.float64)
        amp = torch.rand(n_blobs, channels, generator=g, dtype=torch.float64)
        py0 = height * torch.rand(n_blobs, generator=g, dtype=torch.float64)
        px0 = width * torch.rand(n_blobs, generator=g, dtype=torch.float64)
        vy = speed * (2 * torch.rand(n_blobs, generator=g, dtype=torch.float64) - 1)
        vx = speed * (2 * torch.rand(n_blobs, generator=g, dtype=torch.float64) - 1)
        sig, amp, py0, px0, vy, vx = (a.to(device) for a in (sig, amp, py0, px0, vy, vx))
        local = torch.arange(t, stop, dtype=torch.float64, device=device) - (scene * scene_len if scene_len > 0 else 0)
        py = reflect(py0[None, :] + vy[None, :] * local[:, None], height)  # (k, nb)
        px = reflect(px0[None, :] + vx[None, :] * local[:, None], width)
        inv = (1.0 / (2.0 * sig * sig)).to(cdt)
        py, px, amp = py.to(cdt), px.to(cdt), amp.to(cdt)
        gy = torch.exp(-((yy[None, None, :] - py[:, :, None]) ** 2) * inv[None, :, None])  # (k, nb, H)
        gx = torch.exp(-((xx[None, None, :] - px[:, :, None]) ** 2) * inv[None, :, None])  # (k, nb, W)
        # frame[h, w, c] = sum_b amp[b, c] gy[b, h] gx[b, w]
        gyc = gy[:, :, :, None] * amp[None, :, None, :]  # (k, nb, H, C)
        out[t - t0:stop - t0] = torch.einsum("kbhc,kbw->khwc", gyc, gx)
        t = stop
    out = _noise(out, range(t0, t0 + count), seed, noise_std, device)
    return out.reshape((count,) + tuple(view)).to(dtype)


def fourier_flow(t0: int, count: int, *, grid: int = 128, fields: int = 4, modes: int = 64,
                 kmax: int = 16, velocity=(0.3, 0.1, 0.2), seed: int = 1002,
                 dtype=torch.float32, device="cpu"):
    """Snapshots t0 .. t0+count-1 of f_c(x,t) = sum_m |k_m|^(-5/3) cos(2 pi k_m.(x - v t)/G + phi_cm).

    Wave vectors have integer components U{-kmax..kmax} (|k| >= 1), drawn independently per field;
    phases phi ~ U[0, 2pi).  Returns shape (count, G, G, G, fields), field index fastest.
    """
    g = _params_gen(seed, 3)
    k = torch.randint(-kmax, kmax + 1, (fields, modes, 3), generator=g)
    while True:  # redraw all-zero wave vectors
        zero = (k == 0).all(dim=-1)
        if not zero.any():
            break
        k[zero] = torch.randint(-kmax, kmax + 1, (int(zero.sum()), 3), generator=g)
    phi = 2 * math.pi * torch.rand(fields, modes, generator=g, dtype=torch.float64)
    kf = k.to(torch.float64)
    amp = kf.norm(dim=-1) ** (-5.0 / 3.0)
    kf, phi, amp = kf.to(device), phi.to(device), amp.to(device)
    v = torch.tensor(velocity, dtype=torch.float64, device=device)
    x = torch.arange(grid, dtype=torch.float64, device=device)
    w = 2 * math.pi / grid
    e = [torch.polar(torch.ones_like(kf[..., a, None] * x), w * kf[..., a, None] * x) for a in range(3)]  # (F,M,G)
    out = torch.empty((count, grid, grid, grid, fields), dtype=torch.float64, device=device)
    for i, t in enumerate(range(t0, t0 + count)):
        ph = phi - w * t * (kf @ v)  # (F, M)
        c = torch.polar(amp, ph)  # complex amplitude per (field, mode)
        for f in range(fields):
            ab = torch.einsum("m,ma,mb->mab", c[f], e[0][f], e[1][f])  # (M, G, G)
            out[i, :, :, :, f] = torch.einsum("mab,mc->abc", ab, e[2][f]).real
    return out.to(dtype)


def random_tt(t0: int, count: int, *, dims=(10, 15, 20), ranks=(1, 2, 3, 5, 1), length: int = 500,
              seed: int = 1003, dtype=torch.float64, device="cpu"):
    """Slices t0 .. t0+count-1 along the last mode of a random TT tensor of shape dims x length.

    ``ranks`` are the TT-ranks [r_0, .., r_d, r_{d+1}=1] of the (d+1)-way tensor; cores are N(0,1).
    Returns shape (count, *dims).
    """
    d = len(dims)
    assert len(ranks) == d + 2 and ranks[0] == 1 and ranks[-1] == 1
    g = _params_gen(seed, 4)
    cores = [torch.randn(ranks[i], n, ranks[i + 1], generator=g, dtype=torch.float64)
             for i, n in enumerate(tuple(dims) + (length,))]
    x = cores[0].reshape(dims[0], ranks[1])
    for i in range(1, d):
        x = (x @ cores[i].reshape(ranks[i], -1)).reshape(-1, ranks[i + 1])
    last = cores[d].reshape(ranks[d], length)[:, t0:t0 + count]  # (r_d, count)
    out = (x @ last).T.contiguous().reshape((count,) + tuple(dims))
    return out.to(device=device, dtype=dtype).contiguous()


STREAMS = {
    "cp_cosine": cp_cosine,
    "blob_video": blob_video,
    "fourier_flow": fourier_flow,
    "random_tt": random_tt,
}
