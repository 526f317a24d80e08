"""Life cycle of a GPU decomposition through the C ABI: checkpoint / resume, the memory projection
of a handle, and out-of-memory paths with host-injected allocation failures.  ttice_save writes the state, ttice_open recreates it on the device, and the resumed handle
continues the stream exactly as the uninterrupted one does (same decisions and ranks;
reconstructions equal up to the order of FP64 atomic additions, which on the FP32 path can move FP32
roundings).  ttice_projected_bytes, a dry run of the creation code, equals what a handle holds."""
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


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp32", 1e-5)])
def test_save_open_resume(T, tmp_path, precision, tol):
    Y = blob_video(0, 16, height=48, width=64, n_blobs=5, sigma=(3, 10), view=(6, 8, 8, 8, 3), seed=9).cuda()
    g = T.TTICE(Y.shape[1:], 0.1, precision=precision, input_dtype=torch.float32, max_batch=4)
    for k in range(0, 8, 4):
        g.update(Y[k:k + 4])
    path = str(tmp_path / "s.ttck")
    g.save(path)
    r = T.TTICE.open(path, max_batch=4)
    assert r.ranks() == g.ranks() and r.dims == g.dims
    np.testing.assert_array_equal(r.last_core(), g.last_core())
    for i in range(1, len(g.dims) + 1):
        np.testing.assert_array_equal(r.core(i), g.core(i))
    np.testing.assert_array_equal(r.reconstruct(0, 8).cpu().numpy(), g.reconstruct(0, 8).cpu().numpy())
    for k in range(8, 16, 4):
        s1 = g.update(Y[k:k + 4])
        s2 = r.update(Y[k:k + 4])
        assert list(s1.ranks[:7]) == list(s2.ranks[:7])
        assert (s1.skipped, s1.n_selected) == (s2.skipped, s2.n_selected)
    a, b = g.reconstruct(0, 16).cpu().numpy(), r.reconstruct(0, 16).cpu().numpy()
    assert np.abs(a - b).max() <= tol * np.abs(a).max()
    g.close()
    r.close()


def test_projected_bytes_equal_device_bytes(T):
    """The dry run of the creation code counts exactly what a handle allocates, also after growth."""
    dims = (6, 8, 8, 8, 3)
    for precision in ("fp64", "fp32"):
        g = T.TTICE(dims, 0.1, precision=precision, input_dtype=torch.float32, max_batch=4, max_rank=8)
        h = T.ttice_default_heuristics()
        h.precision = T.PRECISIONS[precision]
        c = T.ttice_default_capacity()
        c.max_batch, c.max_rank = 4, 8
        assert g.device_bytes() == T.ttice_projected_bytes(dims, h, c)
        g.reserve_rank(2, 40)
        assert g.capacities()[2] == 40
        assert g.device_bytes() == T.ttice_projected_bytes(dims, h, c, g.capacities())
        g.close()


def test_injected_allocation_failures(T):
    """Out-of-memory paths, with the failure injected on the host (ttice_test_fail_alloc): a
    creation that fails at any of its allocations returns TTICE_ENOMEM and leaks nothing; a failed
    capacity growth leaves the handle as it was and usable; an update whose last-core growth fails
    leaves the decomposition as it was, and the repeated update gives the uninterrupted result."""
    dims = (6, 8, 8, 8, 3)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    created = False
    try:
        for k in range(1, 200):
            T.ttice_test_fail_alloc(k)
            try:
                g = T.TTICE(dims, 0.1, precision="fp32", input_dtype=torch.float32, max_batch=4)
            except T.TTICEError as e:
                assert e.code == T.TTICE_ENOMEM
                continue
            T.ttice_test_fail_alloc(0)
            g.close()
            created = True
            break
    finally:
        T.ttice_test_fail_alloc(0)
    assert created and k > 10
    torch.cuda.synchronize()
    assert abs(torch.cuda.mem_get_info()[0] - free0) < 64 << 20

    Y = blob_video(0, 12, height=48, width=64, n_blobs=5, sigma=(3, 10), view=dims, seed=9).cuda()
    ref = T.TTICE(dims, 0.05, precision="fp64", input_dtype=torch.float32, max_batch=4, obs_reserve=4)
    g = T.TTICE(dims, 0.05, precision="fp64", input_dtype=torch.float32, max_batch=4, max_rank=2,
                obs_reserve=4)
    ref.update(Y[:4])
    with pytest.raises(T.TTICEError) as ei:
        g.update(Y[:4])
    assert ei.value.code == T.TTICE_ECAPACITY
    kk, need = g.capacity_miss()
    caps = g.capacities()
    T.ttice_test_fail_alloc(1)
    try:
        with pytest.raises(T.TTICEError) as ei:
            g.reserve_rank(kk, need)
        assert ei.value.code == T.TTICE_ENOMEM
    finally:
        T.ttice_test_fail_alloc(0)
    assert g.capacities() == caps and g.ranks() == [1, 0, 0, 0, 0, 0, 1]
    for i in range(1, 6):
        g.reserve_rank(i, 512)
    g.update(Y[:4])
    assert g.ranks() == ref.ranks()
    # the next update must grow the last core (reserve 4 observations): make that allocation fail
    r_before, last_before = g.ranks(), g.last_core()
    T.ttice_test_fail_alloc(1)
    try:
        with pytest.raises(T.TTICEError) as ei:
            g.update(Y[4:8])
        assert ei.value.code == T.TTICE_ENOMEM
    finally:
        T.ttice_test_fail_alloc(0)
    assert g.ranks() == r_before
    np.testing.assert_array_equal(g.last_core(), last_before)
    for k in range(4, 12, 4):
        s1 = ref.update(Y[k:k + 4])
        s2 = g.update(Y[k:k + 4])
        assert list(s1.ranks[:7]) == list(s2.ranks[:7])
    a, b = ref.reconstruct(0, 12).cpu().numpy(), g.reconstruct(0, 12).cpu().numpy()
    assert np.abs(a - b).max() <= 1e-10 * np.abs(a).max()
    g.close()
    ref.close()
