"""GPU path (libttice through its C ABI) against the FP64 CPU oracle on identical seeded inputs.

Bars: identical ranks and skip / subselection decisions on every increment; reconstructions and
projections within 1e-10 relative on the FP64 path; epsilon met on every increment on every path
(Theorem 1 / Corollary 1); mixed-precision paths within a tolerance derived from FP32 rounding.
"""
import json
import math
import os

import numpy as np
import pytest
import torch

from oracle import ttice_oracle as O
from tt_streams import blob_video, cp_cosine, fourier_flow, random_tt

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2211_12487_gb300 import ttice

    return ttice


def _relmax(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _interface_projectors(cores, max_rows=2048):
    """Projectors onto the spans of the left interface matrices (first i cores contracted);
    gauge-free, so they can be compared across implementations.  Stops once they get large."""
    A = np.ones((1, 1))
    out = []
    for U in cores:
        if U.shape[1] == 0 or A.shape[1] == 0 or A.shape[0] * (U.shape[0] // A.shape[1]) > max_rows:
            break
        A = np.kron(A, np.eye(U.shape[0] // A.shape[1])) @ U
        out.append(A @ A.T)
    return out


def run_pair(T, frames, batch, eps, *, precision="fp64", tol=1e-10, check_eps=True,
             oracle_kw=None, gpu_kw=None, stats_out=None, orth_tol=1e-12, oracle_eps=None, err2_tol=None):
    """Stream `frames` through the GPU and the oracle; compare after every increment.  With
    `stats_out` (a list), the GPU's per-update statistics are appended to it.  `oracle_eps`: the
    oracle's tolerance when the GPU mode decides at another one than its eps (the errors are still
    checked against eps); `err2_tol`: absolute bound on the difference of the squared batch errors
    before each update (instead of `tol` relative to the error)."""
    dims = frames.shape[1:]
    in_dtype = frames.dtype
    g = T.TTICE(dims, eps, precision=precision, input_dtype=in_dtype, max_batch=batch,
                **(gpu_kw or {}))
    o = O.TTICEOracle(dims, eps if oracle_eps is None else oracle_eps, **(oracle_kw or {}))
    dev = frames.to("cuda")
    for k in range(0, frames.shape[0], batch):
        Yk = frames[k:k + batch]
        st = g.update(dev[k:k + batch])
        if stats_out is not None:
            stats_out.append((st.krylov_solves, st.krylov_fallbacks, list(st.new_dirs[:len(dims)])))
        so = o.update(Yk.double().numpy(), check_error=check_eps)
        assert list(st.ranks[:len(dims) + 1]) == so.ranks[:len(dims) + 1], (k, list(st.ranks[:len(dims) + 2]), so.ranks)
        assert bool(st.skipped) == so.skipped, k
        assert st.n_selected == so.n_selected, k
        if err2_tol is None:
            assert st.rel_err_before == pytest.approx(so.rel_err_before, rel=max(tol, 1e-9), abs=1e-12)
        else:
            assert abs(st.rel_err_before ** 2 - so.rel_err_before ** 2) <= err2_tol, (k, st.rel_err_before, so.rel_err_before)
        if check_eps:
            rec = g.reconstruct(k, Yk.shape[0]).cpu().numpy()
            Y64 = Yk.double().numpy()
            err = math.sqrt(((Y64 - rec) ** 2).sum() / max((Y64 ** 2).sum(), 1e-300))
            assert err <= eps * (1 + 1e-9), (k, err)
    n = frames.shape[0]
    rec = g.reconstruct(0, n).cpu().numpy()
    ref = o.reconstruct(0, n)
    assert _relmax(rec, ref) < tol, _relmax(rec, ref)
    Pg = _interface_projectors([g.core(i + 1) for i in range(len(dims))])
    Po = _interface_projectors(o.U)
    for a, b in zip(Pg, Po):
        assert np.abs(a - b).max() < max(tol, 1e-12) * 100
    for i in range(len(dims)):
        Ug = g.core(i + 1)
        assert np.abs(Ug.T @ Ug - np.eye(Ug.shape[1])).max() < orth_tol, i
    g.close()
    return o


def test_cp_stream_fp64(T):
    """16^4 cosine stream, FP64 input, eps=0.1, 200 single-tensor increments."""
    Y = cp_cosine(0, 200)
    run_pair(T, Y, 1, 0.1, check_eps=False)


def test_cp_stream_fp64_eps_checked(T):
    Y = cp_cosine(0, 30)
    run_pair(T, Y, 1, 0.1)


@pytest.mark.parametrize("batch", [1, 4])
def test_video_small_fp64(T, batch):
    Y = blob_video(0, 24, height=48, width=64, n_blobs=5, sigma=(3, 10), view=(6, 8, 8, 8, 3), seed=7)
    run_pair(T, Y, batch, 0.1)


def test_video_small_ragged_batches(T):
    """Batches of different sizes in one stream, including a ragged tail."""
    Y = blob_video(0, 23, height=48, width=64, n_blobs=5, sigma=(3, 10), view=(6, 8, 8, 8, 3), seed=8)
    g = T.TTICE(Y.shape[1:], 0.05, input_dtype=torch.float32, max_batch=8)
    o = O.TTICEOracle(Y.shape[1:], 0.05)
    dev = Y.cuda()
    k = 0
    for b in (1, 8, 3, 5, 2, 4):
        st = g.update(dev[k:k + b])
        so = o.update(Y[k:k + b].double().numpy())
        assert list(st.ranks[:6]) == so.ranks[:6]
        k += b
    assert _relmax(g.reconstruct(0, k).cpu().numpy(), o.reconstruct(0, k)) < 1e-10


def test_video_c1_prefix_fp64(T):
    """Full-size video frames 480x640x3 as 20x24x20x32x3, batches of 8 (first three increments)."""
    Y = blob_video(0, 24)
    run_pair(T, Y, 8, 0.1)


def test_tt_ice_plain_and_paper_variants(T):
    Y = blob_video(0, 16, height=48, width=64, n_blobs=5, sigma=(3, 10), view=(6, 8, 8, 8, 3), seed=9)
    run_pair(T, Y, 4, 0.1, oracle_kw=dict(skip_mode=O.SKIP_NONE, subselect=False, tau=math.inf),
             gpu_kw=dict(skip_mode="none", subselect=False, tau=math.inf))
    run_pair(T, Y, 4, 0.1, check_eps=False, oracle_kw=dict(skip_mode=O.SKIP_MEAN, eps_upd_mode=O.EPS_UPD_APPROX, tau=0.8),
             gpu_kw=dict(skip_mode="mean", eps_upd="approx", tau=0.8))


def test_appendix_b_rank_recovery_gpu(T):
    """Exactly low-rank 10x15x20 stream with TT-ranks [1,2,3,5,1] at eps = 1e-8 (Appendix B)."""
    Y = random_tt(0, 120, ranks=(1, 2, 3, 5, 1), seed=11)
    g = T.TTICE((10, 15, 20), 1e-8, input_dtype=torch.float64, max_batch=1)
    dev = Y.cuda()
    for k in range(120):
        g.update(dev[k:k + 1])
    assert g.ranks() == [1, 2, 3, 5, 1]
    rec = g.reconstruct(0, 120).cpu().numpy()
    Yn = Y.numpy()
    assert math.sqrt(((rec - Yn) ** 2).sum() / (Yn ** 2).sum()) < 1e-8


def test_project_matches_oracle(T):
    Y = blob_video(0, 12, height=48, width=64, n_blobs=5, sigma=(3, 10), view=(6, 8, 8, 8, 3), seed=7)
    Z = blob_video(100, 6, height=48, width=64, n_blobs=5, sigma=(3, 10), view=(6, 8, 8, 8, 3), seed=7)
    g = T.TTICE(Y.shape[1:], 0.1, input_dtype=torch.float32, max_batch=6)
    o = O.TTICEOracle(Y.shape[1:], 0.1)
    for k in range(0, 12, 6):
        g.update(Y[k:k + 6].cuda())
        o.update(Y[k:k + 6].double().numpy())
    coeffs, rel = g.project(Z.cuda())
    c_o, rho2, y2 = o.errors(Z.double().numpy())
    assert _relmax(coeffs.cpu().numpy(), c_o) < 1e-10
    np.testing.assert_allclose(rel.cpu().numpy(), np.sqrt(rho2 / y2), rtol=1e-9)


@pytest.mark.parametrize("grid", [64, 128])
def test_first_pass_tensor_cores_flow(T, grid):
    """FP32 path whose first pass runs on the tensor cores at n_1 = 64 and 128 (four 32-row chunks,
    r_1 = 33): new snapshots projected onto cores loaded from the oracle give the oracle's
    coefficients to FP32 accuracy, and per-observation relative errors (stage residuals by
    Pythagoras) within 2e-3 relative: ||X||^2 - ||U^T X||^2 carries the ~1e-6 relative rounding of
    the tensor-core sums times ||X||^2 / ||R||^2 (~100 here)."""
    b = 2
    Y = fourier_flow(0, 2 * b, grid=grid, seed=21)
    o = O.TTICEOracle(Y.shape[1:], 0.05)
    o.update(Y[:b].double().numpy())
    assert 32 < o.ranks[1] <= 64
    g = T.TTICE(Y.shape[1:], 0.05, precision="fp32", input_dtype=torch.float32, max_batch=b)
    last = np.zeros((len(o.last), o.ranks[-1]))
    for j, c in enumerate(o.last):
        last[j, :c.shape[0]] = c
    g.load(o.ranks, o.U, last)
    Z = Y[b:]
    coeffs, rel = g.project(Z.cuda())
    c_o, rho2, y2 = o.errors(Z.double().numpy())
    assert _relmax(coeffs.cpu().numpy(), c_o) < 1e-5
    np.testing.assert_allclose(rel.cpu().numpy(), np.sqrt(rho2 / y2), rtol=2e-3)
    g.close()


def test_subselect_golden_gpu(T):
    g_ = json.load(open(os.path.join(GOLDEN, "subselect_example.json")))
    e = g_["expect"]
    g = T.TTICE(g_["dims"], g_["eps"], input_dtype=torch.float64, max_batch=2)
    g.update(torch.tensor(g_["increment_1"], dtype=torch.float64).cuda())
    st = g.update(torch.tensor(g_["increment_2"], dtype=torch.float64).cuda())
    assert st.n_selected == 1
    assert st.eps_upd == pytest.approx(e["eps_upd_exact"], abs=1e-15)
    assert st.eps_core == pytest.approx(e["eps_core_exact"], abs=1e-15)
    assert g.ranks() == e["ranks"]
    np.testing.assert_allclose(g.core(1), np.array(e["U1"]), atol=1e-14)
    np.testing.assert_allclose(g.core(2), np.array(e["U2"]), atol=1e-14)
    np.testing.assert_allclose(g.last_core().T, np.array(e["last_core"]), atol=1e-14)


def test_zero_observation_and_skip(T):
    Y = cp_cosine(0, 3)
    Y[1] = 0.0
    g = T.TTICE((16, 16, 16, 16), 0.1, input_dtype=torch.float64, max_batch=2)
    st = g.update(Y[:2].cuda())
    assert st.n_selected == 1
    assert np.abs(g.last_core()[1]).max() == 0.0
    r = g.ranks()
    st = g.update(Y[:1].cuda())  # same tensor again: represented exactly, skipped
    assert st.skipped and g.ranks() == r


def test_invalid_and_nonfinite_leave_state(T):
    Y = cp_cosine(0, 4)
    g = T.TTICE((16, 16, 16, 16), 0.1, input_dtype=torch.float64, max_batch=2)
    g.update(Y[:1].cuda())
    r = g.ranks()
    last = g.last_core().copy()
    with pytest.raises(T.TTICEError) as ei:
        T.ttice_update(g.h, Y[:3].cuda(), 3)
    assert ei.value.code == T.TTICE_EINVAL
    bad = Y[1:2].clone()
    bad[0, 0, 0, 0, 0] = float("nan")
    with pytest.raises(T.TTICEError) as ei:
        g.update(bad.cuda())
    assert ei.value.code == T.TTICE_ENONFINITE
    assert g.ranks() == r
    np.testing.assert_array_equal(g.last_core(), last)


def test_capacity_exceeded_rolls_back(T):
    Y = blob_video(0, 8, height=48, width=64, n_blobs=5, sigma=(3, 10), view=(6, 8, 8, 8, 3), seed=7)
    g = T.TTICE(Y.shape[1:], 0.01, input_dtype=torch.float32, max_batch=4, max_rank=3)
    with pytest.raises(T.TTICEError) as ei:
        g.update(Y[:4].cuda())
    assert ei.value.code == T.TTICE_ECAPACITY
    assert g.ranks() == [1, 0, 0, 0, 0, 0, 1]
    for i in range(1, 6):
        assert g.core(i).size == 0


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp32", 1e-5)])
def test_capacity_growth_matches_roomy_handle(T, precision, tol):
    """A handle created with rank capacity 2, grown by ttice_reserve_rank to the rank that each
    failed update names, ends in the state of a handle created with room to spare: the failed
    update leaves ranks and cores as they were, the repeated one gives the same ranks, and the
    reconstructions agree (up to the order of FP64 atomic additions)."""
    Y = blob_video(0, 16, height=48, width=64, n_blobs=5, sigma=(3, 10), view=(6, 8, 8, 8, 3), seed=7)
    dims = Y.shape[1:]
    roomy = T.TTICE(dims, 0.05, precision=precision, input_dtype=torch.float32, max_batch=4)
    g = T.TTICE(dims, 0.05, precision=precision, input_dtype=torch.float32, max_batch=4, max_rank=2,
                obs_reserve=2)
    bytes0 = g.device_bytes()
    assert bytes0 > 0 and g.capacities() == [1, 2, 2, 2, 2, 2]
    grown = 0
    for k in range(0, 16, 4):
        Yk = Y[k:k + 4].cuda()
        roomy.update(Yk)
        while True:
            r_before = g.ranks()
            core_before = g.core(1)
            try:
                g.update(Yk)
                break
            except T.TTICEError as e:
                assert e.code == T.TTICE_ECAPACITY
                assert g.ranks() == r_before
                kk, need = g.capacity_miss()
                caps = g.capacities()
                assert 1 <= kk <= len(dims) and need > caps[kk]
                g.reserve_rank(kk, need)
                assert g.capacities()[kk] == need
                assert g.ranks() == r_before
                np.testing.assert_array_equal(g.core(1), core_before)
                grown += 1
        assert g.capacity_miss() == (0, 0)
        assert g.ranks() == roomy.ranks(), k
    assert grown >= 3 and g.device_bytes() > bytes0
    g.reserve_rank(1, 1)  # below the current capacity: no-op
    assert _relmax(g.reconstruct(0, 16).cpu().numpy(), roomy.reconstruct(0, 16).cpu().numpy()) < tol
    g.close()
    roomy.close()


def test_lockstep_load(T):
    """Load the oracle's state mid-stream, apply one increment on both sides, compare."""
    Y = blob_video(0, 16, height=48, width=64, n_blobs=5, sigma=(3, 10), view=(6, 8, 8, 8, 3), seed=12)
    o = O.TTICEOracle(Y.shape[1:], 0.1)
    for k in range(0, 12, 4):
        o.update(Y[k:k + 4].double().numpy())
    g = T.TTICE(Y.shape[1:], 0.1, input_dtype=torch.float32, max_batch=4)
    last = np.zeros((len(o.last), o.ranks[-1]))
    for j, c in enumerate(o.last):
        last[j, :c.shape[0]] = c
    g.load(o.ranks, o.U, last)
    assert _relmax(g.reconstruct(0, 12).cpu().numpy(), o.reconstruct(0, 12)) < 1e-12
    st = g.update(Y[12:16].cuda())
    so = o.update(Y[12:16].double().numpy())
    assert list(st.ranks[:6]) == so.ranks[:6]
    assert _relmax(g.reconstruct(0, 16).cpu().numpy(), o.reconstruct(0, 16)) < 1e-10


def test_fp32_projection_mode(T):
    """FP32 projections (FP64 Gram / eigen-solve / CGS2 / norms): epsilon met on every increment,
    ranks equal to the oracle's, reconstructions within FP32-level error."""
    Y = blob_video(0, 24, height=48, width=64, n_blobs=5, sigma=(3, 10), view=(6, 8, 8, 8, 3), seed=7)
    run_pair(T, Y, 4, 0.1, precision="fp32", tol=1e-4)


def test_video_c1_prefix_fp32(T):
    """Full-size video frames on the FP32 path (Krylov / Jacobi eigen-solves with FP64 Rayleigh-Ritz):
    ranks and decisions equal to the oracle's, eps met on every increment, and the block-Krylov
    solver (Gram sides above 96) both runs and certifies its result."""
    Y = blob_video(0, 32)
    stats = []
    run_pair(T, Y, 8, 0.1, precision="fp32", tol=1e-4, stats_out=stats)
    assert sum(x[0] for x in stats) >= 1, stats


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-14), ("fp32", 1e-6)])
def test_skip_mean_golden_gpu(T, precision, tol):
    """The hand-derived increment on which the paper's mean-error skip and the exact batch error
    disagree (Sec. 4.3): same decision, ranks, cores and last core as derived by hand."""
    g_ = json.load(open(os.path.join(GOLDEN, "skip_mean_example.json")))
    dt = torch.float64 if precision == "fp64" else torch.float32
    for mode, key in (("mean", "expect_mean"), ("exact", "expect_exact")):
        e = g_[key]
        g = T.TTICE(g_["dims"], g_["eps"], skip_mode=mode, precision=precision, input_dtype=dt, max_batch=4)
        g.update(torch.tensor(g_["increment_1"], dtype=dt).cuda())
        st = g.update(torch.tensor(g_["increment_2"], dtype=dt).cuda())
        assert bool(st.skipped) == e["skipped"]
        assert st.rel_err_before == pytest.approx(e["rel_err_before"], rel=max(tol, 1e-12))
        assert g.ranks() == e["ranks"]
        np.testing.assert_allclose(g.core(1), np.array(e["U1"]), atol=tol)
        np.testing.assert_allclose(g.last_core().T, np.array(e["last_core"]), atol=tol * 10)
        g.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-14), ("fp32", 1e-6)])
def test_occupancy_golden_gpu(T, precision, tol):
    """The hand-derived increment on which occupancy tau = 0.8 keeps a core at occupancy 0.8 and
    tau = 1 expands it (Eq. 16), with the core element count of Eq. 22."""
    g_ = json.load(open(os.path.join(GOLDEN, "occupancy_example.json")))
    dt = torch.float64 if precision == "fp64" else torch.float32
    for tau, key in ((0.8, "expect_tau_0.8"), (1.0, "expect_tau_1")):
        e = g_[key]
        g = T.TTICE(g_["dims"], g_["eps"], tau=tau, precision=precision, input_dtype=dt, max_batch=2)
        g.update(torch.tensor(g_["increment_1"], dtype=dt).cuda())
        st = g.update(torch.tensor(g_["increment_2"], dtype=dt).cuda())
        assert st.eps_core == pytest.approx(g_["eps_core"], rel=max(tol, 1e-12))
        assert g.ranks() == e["ranks"]
        np.testing.assert_allclose(g.core(1), np.array(e["U1"], dtype=float), atol=tol)
        np.testing.assert_allclose(g.core(2), np.array(e["U2"], dtype=float), atol=tol)
        np.testing.assert_allclose(g.last_core().T, np.array(e["last_core"]), atol=tol * 10)
        assert st.core_elems == e["core_elements"]
        g.close()


@pytest.mark.parametrize("ranks", [[1, 37, 300, 90, 8], [1, 3, 17, 64, 5]])
def test_projection_kernel_shapes(T, ranks):
    """The tensor-core projection of the mixed path (W = U^T X per stage, residual norms by
    Pythagoras) against the oracle's sequential projection (Algorithm 2 'project', Eq. 12) and its
    direct per-observation errors (Eq. 17), on cores loaded into the handle: ragged K chunks (m not a
    multiple of 32), ragged column tiles (L not a multiple of 128), several N tiles (r_2 = 300 > 256,
    the last one partial), r not a multiple of 16, and a batch of 3."""
    dims = (40, 20, 36, 8)
    rng = np.random.default_rng(5)
    cores = []
    for i, n in enumerate(dims):
        q, _ = np.linalg.qr(rng.normal(size=(ranks[i] * n, ranks[i + 1])))
        cores.append(q)
    o = O.TTICEOracle(dims, 0.1)
    o.ranks = list(ranks[:len(dims) + 1])
    o.U = [c.copy() for c in cores]
    # data: half inside the span of the cores (small residuals), half generic
    C = rng.normal(size=(3, ranks[len(dims)]))
    Y = o.expand(C) + 0.05 * rng.normal(size=(3,) + dims)
    last = np.zeros((1, ranks[len(dims)]))
    c_o, rho2, y2 = o.errors(Y)
    for precision, tol_c, tol_e in (("fp64", 1e-12, 1e-10), ("fp32", 1e-5, 1e-3)):
        g = T.TTICE(dims, 0.1, precision=precision, input_dtype=torch.float32, max_batch=4, max_rank=512)
        g.load(ranks[:len(dims) + 1], cores, last)
        Yd = torch.tensor(Y, dtype=torch.float32).cuda()
        coeffs, rel = g.project(Yd)
        Y32 = Yd.double().cpu().numpy()
        c32, rho32, y32 = o.errors(Y32)
        assert _relmax(coeffs.cpu().numpy(), c32) < tol_c, (precision, _relmax(coeffs.cpu().numpy(), c32))
        np.testing.assert_allclose(rel.cpu().numpy(), np.sqrt(rho32 / y32), rtol=tol_e)
        g.close()


# decision tolerance of the TF32 mode: eps sqrt(1 - 1/16), the rest of eps^2 left to its projections
TF32_SHARE = 1.0 / 16.0


def test_tf32_mode_projection_budget(T):
    """TTICE_TF32 (one TF32 product per stage projection) against the oracle's FP64 projection of the
    same FP32 data onto the same cores (Eq. 12 per stage, Eq. 17 per observation): per observation,
    the error of its squared residual plus the squared error of its coefficients stays within the
    mode's budget, 1/16 of eps^2 ||y||^2; and the mode is visibly less accurate than the split
    products of TTICE_FP32, so the one-product path is the one that ran (stages 1 and 2 here: 740 x
    288 and 10800 x 8 per observation).  Shapes as in test_projection_kernel_shapes (ragged K chunks
    and column tiles, several N tiles)."""
    dims, ranks, eps = (40, 20, 36, 8), [1, 37, 300, 90, 8], 0.1
    rng = np.random.default_rng(6)
    cores = [np.linalg.qr(rng.normal(size=(ranks[i] * n, ranks[i + 1])))[0] for i, n in enumerate(dims)]
    o = O.TTICEOracle(dims, eps)
    o.ranks = list(ranks)
    o.U = [c.copy() for c in cores]
    C = rng.normal(size=(4, ranks[-1]))
    Y = o.expand(C) + 0.05 * rng.normal(size=(4,) + dims)
    Yd = torch.tensor(Y, dtype=torch.float32).cuda()
    c32, rho32, y32 = o.errors(Yd.double().cpu().numpy())
    err = {}
    for precision in ("fp32", "tf32"):
        g = T.TTICE(dims, eps, precision=precision, input_dtype=torch.float32, max_batch=4, max_rank=512)
        g.load(ranks, cores, np.zeros((1, ranks[-1])))
        coeffs, rel = g.project(Yd)
        coeffs, rel = coeffs.cpu().numpy(), rel.cpu().numpy()
        drho = np.abs(rel ** 2 * y32 - rho32)
        dc2 = ((coeffs - c32) ** 2).sum(axis=1)
        assert np.all(drho + dc2 <= TF32_SHARE * eps ** 2 * y32), (precision, drho / y32, dc2 / y32)
        err[precision] = _relmax(coeffs, c32)
        g.close()
    assert err["tf32"] > 10 * err["fp32"], err


@pytest.mark.parametrize("stream", ["small", "c1_prefix"])
def test_tf32_mode_stream(T, stream):
    """TTICE_TF32 through whole updates: decisions and ranks equal to the oracle's at the mode's
    decision tolerance eps sqrt(15/16), squared batch errors before each update within the mode's
    share of eps^2, eps itself met on every increment (measured in FP64 from the reconstruction),
    cores orthonormal, reconstructions within the TF32 rounding of the oracle's.  On the 480x640
    frames (20x24x20x32x3) the second stage (r_1 24 rows x 1920 columns per frame) takes one product;
    the small stream's stages are all below the size rule (the decision tolerance alone differs)."""
    if stream == "small":
        Y, b = blob_video(0, 24, height=48, width=64, n_blobs=5, sigma=(3, 10), view=(6, 8, 8, 8, 3), seed=7), 4
    else:
        Y, b = blob_video(0, 24), 8
    eps = 0.1
    run_pair(T, Y, b, eps, precision="tf32", tol=2e-3, oracle_eps=eps * math.sqrt(1.0 - TF32_SHARE),
             err2_tol=TF32_SHARE * eps ** 2)


def test_blocked_reorthogonalisation(T):
    """Increments that add more directions to a core than one chunk holds (~240 per increment to the
    third core of a 8 x 16 x 16 x 16 Gaussian-noise stream at eps = 0.3) take the blocked
    tensor-core re-orthogonalisation (forced here for every shape): the block against the core's
    earlier columns in one pass, then each 96-column chunk against the chunks of its block already
    appended.  Same ranks and decisions as the oracle on every increment, eps met, reconstructions and
    interface projectors within FP32-level error, cores orthonormal to 2e-7."""
    g = torch.Generator().manual_seed(11)
    Y = torch.randn((48, 8, 16, 16, 16), generator=g, dtype=torch.float32)
    stats = []
    try:
        T.ttice_test_tc_cgs_min(0.0)
        run_pair(T, Y, 16, 0.3, precision="fp32", tol=1e-4, orth_tol=2e-7, stats_out=stats,
                 gpu_kw={"max_rank": 1024})
    finally:
        T.ttice_test_tc_cgs_min(-1.0)
    assert all(x[2][2] > 96 for x in stats[1:]), stats


def test_large_gram_block_krylov(T):
    """Gram sides of 1024 (core 2 of a 16 x 80 x 64 stream, batches of 16) take the block Krylov
    solver with its 768-vector basis in global memory: on a random TT stream (ranks 16, 40, 48)
    with 1e-3 noise, same ranks and decisions as the oracle on every increment, eps met, and the
    Krylov result certified (no fall-back to the full Jacobi solver)."""
    from tt_streams import random_tt

    Y = random_tt(0, 32, dims=(16, 80, 64), ranks=(1, 16, 40, 48, 1), length=64)
    g = torch.Generator().manual_seed(3)
    Y = (Y + 1e-3 * Y.std() * torch.randn(Y.shape, generator=g, dtype=Y.dtype)).float()
    stats = []
    run_pair(T, Y, 16, 0.1, precision="fp32", tol=1e-4, stats_out=stats)
    assert sum(x[0] for x in stats) >= 1 and sum(x[1] for x in stats) == 0, stats


def test_transposed_stage_projection_and_growth(T):
    """Stages with 3 columns per observation (not a multiple of 4: no tile layout of the projection
    kernel takes them) run as a transposed tensor-core projection with FP64 sums across K splits.
    On seeded orthonormal cores loaded into the handle and the oracle (ranks [1,8,160,400,600,60];
    stage 3 has m = 16000, L = 3, r = 600): coefficients and per-observation errors equal to the
    oracle's (Eq. 12, Eq. 17) at FP32 accuracy.  Then one update (tensor-core forms forced) of data
    with four rank-one tensors outside the cores' span: the inner cores gain columns, and the new
    rows of the L = 3 and L = 1 stages are projected from an offset into the core (Algorithm 2, last
    steps).  Same ranks as the oracle, the batch's reconstruction within FP32-level error of the
    oracle's and within eps."""
    dims = (8, 20, 20, 40, 3)
    ranks = [1, 8, 160, 400, 600, 60]
    rng = np.random.default_rng(17)
    cores = [np.linalg.qr(rng.normal(size=(ranks[i] * n, ranks[i + 1])))[0] for i, n in enumerate(dims)]
    o = O.TTICEOracle(dims, 0.1)
    o.ranks = list(ranks)
    o.U = [c.copy() for c in cores]
    o.last = [np.zeros(ranks[-1])]  # the handle is loaded with one (zero) observation
    b = 8
    Y = o.expand(rng.normal(size=(b, ranks[-1]))) + 0.005 * rng.normal(size=(b,) + dims)
    Y32 = torch.tensor(Y, dtype=torch.float32)
    g = T.TTICE(dims, 0.1, precision="fp32", input_dtype=torch.float32, max_batch=b, max_rank=1024)
    g.load(ranks, cores, np.zeros((1, ranks[-1])))
    coeffs, rel = g.project(Y32.cuda())
    c_o, rho2, y2 = o.errors(Y32.double().numpy())
    assert _relmax(coeffs.cpu().numpy(), c_o) < 1e-5, _relmax(coeffs.cpu().numpy(), c_o)
    np.testing.assert_allclose(rel.cpu().numpy(), np.sqrt(rho2 / y2), rtol=2e-3)

    def rank_one():
        v = [rng.normal(size=n) for n in dims]
        t = v[0] / np.linalg.norm(v[0])
        for x in v[1:]:
            t = np.multiply.outer(t, x / np.linalg.norm(x))
        return t

    P = np.stack([rank_one() for _ in range(4)])
    Z = o.expand(rng.normal(size=(b, ranks[-1]))) + np.einsum("zp,p...->z...", 3.0 * rng.normal(size=(b, 4)), P)
    Z32 = torch.tensor(Z, dtype=torch.float32)
    try:
        T.ttice_test_tc_cgs_min(0.0)
        st = g.update(Z32.cuda())
    finally:
        T.ttice_test_tc_cgs_min(-1.0)
    so = o.update(Z32.double().numpy())
    assert list(st.ranks[:len(dims) + 1]) == so.ranks[:len(dims) + 1]
    assert st.new_dirs[3] > 0 and st.new_dirs[4] > 0
    rec = g.reconstruct(1, b).cpu().numpy()
    ref = o.reconstruct(1, b)
    assert _relmax(rec, ref) < 1e-4, _relmax(rec, ref)
    err = math.sqrt(((Z - rec) ** 2).sum() / (Z ** 2).sum())
    assert err <= 0.1 * (1 + 1e-6), err
    g.close()


def test_bounded_wait_expiry_returns_etimeout(T):
    """A wait inside the tensor-core projection that runs out (a copy the producer was told not to
    issue, with a 20 ms wait limit) ends the kernel cleanly: ttice_update returns TTICE_ETIMEOUT, the
    decomposition is as it was (ranks, stored observations, reconstructions), and the next update
    with the default limit succeeds and agrees with an undisturbed handle."""
    view = (8, 16, 12, 8)
    Y = blob_video(0, 12, height=64, width=64, n_blobs=4, sigma=(3, 8), view=view, seed=17).cuda()
    g = T.TTICE(view, 0.1, precision="fp32", input_dtype=torch.float32, max_batch=4)
    ref = T.TTICE(view, 0.1, precision="fp32", input_dtype=torch.float32, max_batch=4)
    g.update(Y[:4])
    ref.update(Y[:4])
    r0 = g.ranks()
    rec0 = g.reconstruct(0, 4)
    try:
        T.ttice_test_wait_limit_ns(20_000_000)
        T.ttice_test_drop_copy(0)
        with pytest.raises(T.TTICEError) as ei:
            g.update(Y[4:8])
        assert ei.value.code == T.TTICE_ETIMEOUT
    finally:
        T.ttice_test_drop_copy(-1)
        T.ttice_test_wait_limit_ns(0)
    torch.cuda.synchronize()
    assert g.ranks() == r0 and g.stats().n_obs == 4
    assert torch.equal(g.reconstruct(0, 4), rec0)
    for k in (4, 8):
        g.update(Y[k:k + 4])
        ref.update(Y[k:k + 4])
    assert g.ranks() == ref.ranks()
    a, b = g.reconstruct(0, 12), ref.reconstruct(0, 12)
    assert float((a - b).abs().max()) <= 1e-5 * float(b.abs().max())
    g.close()
    ref.close()


def test_tensor_core_cgs_matches_oracle(T):
    """The tensor-core re-orthogonalisation of new directions, CGS2 and CholQR2, and the transposed
    projection of the narrow stages (all forced wherever the shapes allow), on the 480p video
    prefix: same decisions and ranks as the oracle on every increment, eps met, batch errors within
    2e-4 relative (the forced narrow stages' residual norms by Pythagoras carry FP32 rounding
    amplified by ||x||^2 / ||R||^2), and cores orthonormal to 2e-7.  The column norms are FP64 sums; the
    coupling left between columns is the tensor core's FP32 summation of products (~2^-23 of the
    products' magnitudes per 8-term MMA), largest for short columns with a few large entries (here
    m is a few hundred and entries reach 0.2: ~1e-7; ~1e-9 for the delocalised columns of length
    ~5e4 of the 1080p stream)."""
    frames = blob_video(0, 16)
    try:
        T.ttice_test_tc_cgs_min(0.0)
        run_pair(T, frames, 8, 0.1, precision="fp32", tol=2e-4, orth_tol=2e-7)
    finally:
        T.ttice_test_tc_cgs_min(-1.0)


def test_projection_kernel_packed_observations(T):
    """Stages with fewer than 128 columns per observation (L = 64 and 4 here, dividing 128) pack
    128 / L observations into one tile of the tensor-core projection: 40 observations fill 20 tiles
    at L = 64 (two per tile, each spanning two warps) and two at L = 4 (32 + 8).  Coefficients and
    per-observation errors against the oracle's projection (Eq. 12, Eq. 17)."""
    dims = (12, 10, 16, 4)
    ranks = [1, 12, 70, 40, 4]
    rng = np.random.default_rng(9)
    cores = []
    for i, n in enumerate(dims):
        q, _ = np.linalg.qr(rng.normal(size=(ranks[i] * n, ranks[i + 1])))
        cores.append(q)
    o = O.TTICEOracle(dims, 0.1)
    o.ranks = list(ranks)
    o.U = [c.copy() for c in cores]
    C = rng.normal(size=(40, ranks[-1]))
    Y = o.expand(C) + 0.05 * rng.normal(size=(40,) + dims)
    g = T.TTICE(dims, 0.1, precision="fp32", input_dtype=torch.float32, max_batch=40, max_rank=128)
    g.load(ranks, cores, np.zeros((1, ranks[-1])))
    Yd = torch.tensor(Y, dtype=torch.float32).cuda()
    coeffs, rel = g.project(Yd)
    c32, rho32, y32 = o.errors(Yd.double().cpu().numpy())
    assert _relmax(coeffs.cpu().numpy(), c32) < 1e-5
    np.testing.assert_allclose(rel.cpu().numpy(), np.sqrt(rho32 / y32), rtol=1e-3)
    g.close()
