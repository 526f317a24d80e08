"""Continuous-batching serving loop: every stream's result is the same alone and in the mix.

Streams of different shapes, batch sizes and tolerances are first run alone (one after the other,
one update at a time); then the same increments are submitted, interleaved, to a ServingEngine
whose slots run updates of different streams concurrently on separate CUDA streams.  Ranks must be
identical and reconstructions equal within 1e-10 relative (FP64 path) / 1e-5 (FP32 path: the only
differences come from the order of FP64 atomic additions in reductions).  A second run with a
memory budget that fits one stream at a time checks admission by projected core memory.
"""
import numpy as np
import pytest
import torch

from tt_streams import blob_video, cp_cosine, fourier_flow

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2211_12487_gb300 import serving, ttice

    return serving, ttice


def _workload(precision):
    dt = torch.float32
    specs, incs = [], {}
    view_v = (6, 8, 8, 8, 3)
    yv = blob_video(0, 24, height=48, width=64, n_blobs=5, sigma=(3, 10), view=view_v, seed=31)
    yc = cp_cosine(0, 12, dims=(8, 8, 8, 8), seed=32).to(dt)
    yf = fourier_flow(0, 8, grid=16, fields=2, modes=8, kmax=4, seed=33)
    for name, y, b, eps in (("video", yv, 4, 0.1), ("cosine", yc, 1, 0.05), ("flow", yf, 2, 0.01),
                            ("video2", yv.flip(0).contiguous(), 8, 0.3)):
        specs.append((name, tuple(y.shape[1:]), eps, b))
        incs[name] = [y[k:k + b].cuda() for k in range(0, y.shape[0], b)]
    return specs, incs


def _alone(ttice, specs, incs, precision):
    out = {}
    for name, dims, eps, b in specs:
        h = ttice.TTICE(dims, eps, precision=precision, input_dtype=torch.float32, max_batch=b)
        for Y in incs[name]:
            h.update(Y)
        n = sum(Y.shape[0] for Y in incs[name])
        out[name] = (h.ranks(), h.reconstruct(0, n).cpu().numpy())
        h.close()
    return out


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp32", 1e-5)])
@pytest.mark.parametrize("budget", ["roomy", "one_at_a_time"])
def test_same_alone_and_in_the_mix(mods, precision, tol, budget):
    serving, ttice = mods
    specs, incs = _workload(precision)
    ref = _alone(ttice, specs, incs, precision)
    sp = [serving.StreamSpec(name, dims, eps, b, precision=precision) for name, dims, eps, b in specs]
    mem = None
    if budget == "one_at_a_time":
        mem = max(serving.projected_core_bytes(s) for s in sp) + 1
    eng = serving.ServingEngine(sp, slots=3, mem_budget=mem)
    try:
        # interleave the submissions of all streams, round robin
        k = 0
        while any(k < len(incs[n]) for n, *_ in specs):
            for name, *_ in specs:
                if k < len(incs[name]):
                    eng.submit(serving.Request(name, incs[name][k]))
            k += 1
            if budget == "one_at_a_time":
                # close a stream once all of its increments are in, so the next can be admitted
                pass
        if budget == "one_at_a_time":
            # streams finish in admission order; release each when done so the next is admitted
            order = [n for n, *_ in specs]
            for name in order:
                while True:
                    with eng.lock:
                        done = name in eng.handles and not eng.pending[name] and name not in eng.busy
                    if done:
                        break
                    eng.drain(timeout=0.05)
                h = eng.handles[name]
                n = sum(Y.shape[0] for Y in incs[name])
                got = (h.ranks(), h.reconstruct(0, n).cpu().numpy())
                assert got[0] == ref[name][0], name
                err = np.abs(got[1] - ref[name][1]).max() / np.abs(ref[name][1]).max()
                assert err < tol, (name, err)
                eng.release(name)
        else:
            assert eng.drain(timeout=300)
            for name, dims, eps, b in specs:
                h = eng.handles[name]
                n = sum(Y.shape[0] for Y in incs[name])
                assert h.ranks() == ref[name][0], name
                rec = h.reconstruct(0, n).cpu().numpy()
                err = np.abs(rec - ref[name][1]).max() / np.abs(ref[name][1]).max()
                assert err < tol, (name, err)
        assert all(r.error is None for r in eng.completed)
        lat = eng.latencies_ms()
        assert len(lat) == sum(len(v) for v in incs.values())
    finally:
        eng.close()
