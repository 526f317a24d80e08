"""Host logic of the serving loop, on CPU with a stand-in handle (no kernel runs): an update that
needs a rank above its capacity grows that capacity within the memory budget and is repeated, and
the memory accounting follows what the handles hold."""
import pytest
import torch

from paper_2211_12487_gb300 import serving as S
from paper_2211_12487_gb300 import ttice as T


class FakeHandle:
    """Fails with TTICE_ECAPACITY while the capacity of rank 2 is below `needs[i]`."""

    def __init__(self, needs):
        self.caps = [1, 4, 16, 16, 3]
        self.needs = list(needs)
        self.reserved = []
        self.updates = 0

    def device_bytes(self):
        return 1000 * sum(self.caps)

    def capacities(self):
        return list(self.caps)

    def capacity_miss(self):
        return (2, self.needs[0]) if self.needs and self.needs[0] > self.caps[2] else (0, 0)

    def reserve_rank(self, k, cap):
        self.reserved.append((k, cap))
        self.caps[k] = max(self.caps[k], cap)

    def update(self, Y, stream=None):
        while self.needs and self.needs[0] <= self.caps[2]:
            self.needs.pop(0)
        if self.needs:
            raise T.TTICEError(T.TTICE_ECAPACITY, "ttice_update")
        self.updates += 1
        return "stats"


def _engine(budget):
    spec = S.StreamSpec("s", (8, 8, 8, 3), 0.1, 4)
    eng = S.ServingEngine([spec], slots=0, mem_budget=budget, device="cpu")
    return eng


def test_growth_repeats_the_update():
    eng = _engine(1 << 40)
    h = FakeHandle([40, 90])
    eng.handles["s"] = h
    eng.mem_of["s"] = h.device_bytes()
    eng.mem_used = h.device_bytes()
    assert eng._update("s", h, None, None) == "stats"
    # each growth reaches the rank needed and at least doubles the capacity
    assert h.reserved == [(2, 40), (2, 90)]
    assert h.updates == 1 and eng.grow_events == 2
    assert eng.mem_used == h.device_bytes() == eng.mem_of["s"]


def test_growth_refused_over_budget():
    h = FakeHandle([40])
    eng = _engine(h.device_bytes() + 10)
    eng.handles["s"] = h
    eng.mem_of["s"] = h.device_bytes()
    eng.mem_used = h.device_bytes()
    with pytest.raises(T.TTICEError) as ei:
        eng._update("s", h, None, None)
    assert ei.value.code == T.TTICE_ECAPACITY
    assert h.reserved == [] and eng.mem_used == h.device_bytes() and eng.grow_events == 0


def test_projection_grows_with_capacity():
    spec = S.StreamSpec("v", (20, 24, 20, 32, 3), 0.05, 32)
    caps = S.default_caps(spec)
    assert caps == [1, 20, 480, 512, 512, 512]
    base = S.projected_core_bytes(spec)
    assert base == S.projected_core_bytes(spec, caps)
    bigger = list(caps)
    bigger[3] = 1024
    assert S.projected_core_bytes(spec, bigger) > base


def test_stream_that_cannot_be_created_fails_alone():
    """Admission of a stream whose handle cannot be created (here: no GPU in the process, so the
    first device allocation fails) completes that stream's requests with the error, names the CUDA
    error behind it, and leaves the engine usable for the other streams."""
    if torch.cuda.is_available():
        pytest.skip("needs a process without a GPU")
    spec = S.StreamSpec("s", (8, 8, 8, 3), 0.1, 4)
    eng = S.ServingEngine([spec], slots=0, mem_budget=1 << 40, device="cuda")
    eng.submit(S.Request("s", None))
    eng.submit(S.Request("s", None))
    assert len(eng.completed) == 2 and "s" in eng.failed_streams and "s" not in eng.handles
    for r in eng.completed:
        assert isinstance(r.error, T.TTICEError) and r.error.code in (T.TTICE_ENOMEM, T.TTICE_ECUDA)
        assert "[cuda" in str(r.error)
    assert eng.mem_used == 0 and not any(eng.pending.values())


def test_projected_bytes_from_the_creation_code():
    """ttice_projected_bytes runs the library's creation code without allocating (no GPU here): it
    grows with the batch size and with each rank's capacity, and a capacity above what the unfolding
    allows is clipped like in ttice_create."""
    dims = (20, 24, 20, 32, 3)
    c8, c32 = T.ttice_default_capacity(), T.ttice_default_capacity()
    c8.max_batch, c32.max_batch = 8, 32
    b8, b32 = T.ttice_projected_bytes(dims, None, c8), T.ttice_projected_bytes(dims, None, c32)
    assert 0 < b8 < b32
    caps = [1, 20, 480, 512, 512, 512]
    assert T.ttice_projected_bytes(dims, None, c32, caps) == b32
    grown = list(caps)
    grown[3] = 1024
    assert T.ttice_projected_bytes(dims, None, c32, grown) > b32
    clipped = list(caps)
    clipped[1] = 10 ** 6  # r_1 <= n_1 = 20
    assert T.ttice_projected_bytes(dims, None, c32, clipped) == b32
    h = T.ttice_default_heuristics()
    h.precision = T.TTICE_FP32
    assert T.ttice_projected_bytes(dims, h, c32) != b32  # FP32 mirrors and FP32 stage buffers
    f32 = T.ttice_projected_bytes(dims, h, c32)
    h.precision = T.TTICE_TF32  # the same buffers: it differs in the products taken and the decisions
    assert T.ttice_projected_bytes(dims, h, c32) == f32
    for unbuilt in (T.TTICE_BF16, T.TTICE_SPLIT_BF16):
        h.precision = unbuilt
        with pytest.raises(T.TTICEError) as ei:
            T.ttice_projected_bytes(dims, h, c32)
        assert ei.value.code == T.TTICE_EINVAL
    with pytest.raises(T.TTICEError):
        T.ttice_projected_bytes((4, 0, 3))


def test_injected_allocation_failure_hook():
    """ttice_test_fail_alloc(1) makes the next device allocation fail as out of memory (named
    cudaErrorMemoryAllocation), once; the dry run of ttice_projected_bytes allocates nothing and
    leaves the hook armed."""
    if torch.cuda.is_available():
        pytest.skip("needs a process without a GPU")
    T.ttice_test_fail_alloc(1)
    try:
        assert T.ttice_projected_bytes((4, 4)) > 0
        with pytest.raises(T.TTICEError) as ei:
            T.ttice_create([4, 4], 0.1)
        assert ei.value.code == T.TTICE_ENOMEM and "cudaErrorMemoryAllocation" in str(ei.value)
        with pytest.raises(T.TTICEError) as ei:
            T.ttice_create([4, 4], 0.1)  # the hook fired once: now the machine's own failure
        assert "cudaErrorMemoryAllocation" not in str(ei.value)
    finally:
        T.ttice_test_fail_alloc(0)


class SlowHandle:
    """An update that runs until the test lets it finish; records whether it ever saw its handle
    closed under it."""

    def __init__(self):
        import threading

        self.started = threading.Event()
        self.go = threading.Event()
        self.closed = False
        self.closed_during_update = False
        self.updates = 0

    def update(self, Y, stream=None):
        self.started.set()
        self.go.wait(10)
        self.closed_during_update |= self.closed
        self.updates += 1
        return "stats"

    def device_bytes(self):
        return 1000

    def close(self):
        self.closed = True


def test_release_waits_for_the_update_in_flight():
    import threading
    import time

    spec = S.StreamSpec("s", (4, 4), 0.1, 1)
    eng = S.ServingEngine([spec], slots=1, mem_budget=1 << 40, device="cpu")
    h = SlowHandle()
    eng.handles["s"] = h
    eng.mem_of["s"] = h.device_bytes()
    eng.mem_used = h.device_bytes()
    eng.submit(S.Request("s", None))
    eng.submit(S.Request("s", None))  # queued behind the first
    assert h.started.wait(5)
    t = threading.Thread(target=eng.release, args=("s",))
    t.start()
    time.sleep(0.2)
    assert t.is_alive() and not h.closed  # release waits while a slot runs the stream's update
    h.go.set()
    t.join(5)
    assert not t.is_alive()
    assert h.closed and not h.closed_during_update and h.updates == 1
    assert eng.mem_used == 0 and "s" not in eng.handles
    done = sorted(eng.completed, key=lambda r: r.error is not None)
    assert len(done) == 2 and done[0].error is None and "released" in str(done[1].error)
    # the queued request was completed, so drain returns; a later submit to the name is refused
    assert eng.drain(timeout=2)
    eng.submit(S.Request("s", None))
    assert "released" in str(eng.completed[-1].error)
    eng.close()
