"""Checkpoint file of a decomposition (host code, no GPU): what the library writes is what the
header documents, reads back bit for bit, is rejected when damaged, and holds everything needed to
continue the stream (checked by resuming the oracle from it)."""
import os
import struct

import numpy as np
import pytest

from oracle import ttice_oracle as O
from paper_2211_12487_gb300 import ttice as T
from tt_streams import cp_cosine


def _oracle_state(n_inc=3):
    Y = cp_cosine(0, 4 * n_inc, dims=(6, 7, 5, 4), seed=5).numpy()
    o = O.TTICEOracle(Y.shape[1:], 0.1)
    for k in range(n_inc):
        o.update(Y[4 * k:4 * k + 4])
    last = np.zeros((len(o.last), o.ranks[-1]))
    for j, c in enumerate(o.last):
        last[j, :c.shape[0]] = c
    return Y, o, last


def _fnv1a(data: bytes) -> int:
    h = 1469598103934665603
    for byte in data:
        h ^= byte
        h = (h * 1099511628211) & 0xFFFFFFFFFFFFFFFF
    return h


def _write(path, o, last, heur=None):
    heur = heur or T.ttice_default_heuristics()
    T.ttice_checkpoint_write(str(path), o.dims, o.eps, heur, o.ranks, o.U, last)


def test_round_trip_bit_exact(tmp_path):
    _, o, last = _oracle_state()
    heur = T.ttice_default_heuristics()
    heur.skip_mode, heur.occupancy_tau, heur.precision = T.TTICE_SKIP_MEAN, 0.8, T.TTICE_FP32
    path = tmp_path / "a.ttck"
    _write(path, o, last, heur)
    ck = T.ttice_checkpoint_read(str(path))
    assert ck["dims"] == o.dims and ck["eps"] == o.eps and ck["ranks"] == o.ranks
    h = ck["heuristics"]
    assert (h.skip_mode, h.subselect, h.eps_upd_mode, h.occupancy_tau, h.precision, h.input_dtype) == \
        (heur.skip_mode, heur.subselect, heur.eps_upd_mode, heur.occupancy_tau, heur.precision, heur.input_dtype)
    for a, b in zip(ck["cores"], o.U):
        assert a.shape == b.shape and np.array_equal(a, b)
    assert np.array_equal(ck["last"], last)
    assert T.ttice_checkpoint_read_header(str(path))["n_obs"] == last.shape[0]


def test_layout_matches_the_documentation(tmp_path):
    """An independent reader of the layout documented in ttice.h, and its checksum."""
    _, o, last = _oracle_state()
    path = tmp_path / "b.ttck"
    _write(path, o, last)
    raw = path.read_bytes()
    assert raw[:8] == b"TTICECK1"
    off = 8
    version, d = struct.unpack_from("<ii", raw, off)
    off += 8
    assert version == 1 and d == len(o.dims)
    dims = list(struct.unpack_from(f"<{d}q", raw, off))
    off += 8 * d
    (eps,) = struct.unpack_from("<d", raw, off)
    off += 8
    skip, subsel, epsupd = struct.unpack_from("<iii", raw, off)
    off += 12
    (tau,) = struct.unpack_from("<d", raw, off)
    off += 8
    prec, indt = struct.unpack_from("<ii", raw, off)
    off += 8
    ranks = list(struct.unpack_from(f"<{d + 1}q", raw, off))
    off += 8 * (d + 1)
    (n_obs,) = struct.unpack_from("<q", raw, off)
    off += 8
    assert dims == o.dims and eps == o.eps and ranks == o.ranks and n_obs == last.shape[0]
    assert (skip, subsel, epsupd, tau) == (T.TTICE_SKIP_EXACT, 1, T.TTICE_EPSUPD_EXACT, 1.0)
    for i in range(d):
        n = ranks[i] * dims[i] * ranks[i + 1]
        core = np.frombuffer(raw, dtype="<f8", count=n, offset=off).reshape(ranks[i] * dims[i], ranks[i + 1])
        assert np.array_equal(core, o.U[i])
        off += 8 * n
    n = n_obs * ranks[d]
    assert np.array_equal(np.frombuffer(raw, dtype="<f8", count=n, offset=off).reshape(n_obs, ranks[d]), last)
    off += 8 * n
    (sum_,) = struct.unpack_from("<Q", raw, off)
    assert off + 8 == len(raw) and sum_ == _fnv1a(raw[:off])


@pytest.mark.parametrize("damage", ["flip", "truncate", "append", "magic"])
def test_damaged_files_are_rejected(tmp_path, damage):
    _, o, last = _oracle_state()
    path = tmp_path / "c.ttck"
    _write(path, o, last)
    raw = bytearray(path.read_bytes())
    if damage == "flip":
        raw[len(raw) // 2] ^= 0x10
    elif damage == "truncate":
        raw = raw[:-9]
    elif damage == "append":
        raw += b"\x00"
    else:
        raw[0:8] = b"TTICECK2"
    path.write_bytes(bytes(raw))
    with pytest.raises(T.TTICEError) as ei:
        T.ttice_checkpoint_read(str(path))
    assert ei.value.code == T.TTICE_EINVAL


def test_invalid_state_is_not_written(tmp_path):
    _, o, last = _oracle_state()
    bad = list(o.ranks)
    bad[1] = o.dims[0] + 1  # r_1 > r_0 n_1
    with pytest.raises(T.TTICEError):
        T.ttice_checkpoint_write(str(tmp_path / "d.ttck"), o.dims, o.eps, T.ttice_default_heuristics(), bad,
                                 o.U, last)
    with pytest.raises(T.TTICEError):
        T.ttice_checkpoint_write(str(tmp_path / "e.ttck"), o.dims, 1.5, T.ttice_default_heuristics(), o.ranks,
                                 o.U, last)
    assert not os.path.exists(tmp_path / "d.ttck")


def test_resume_continues_the_stream(tmp_path):
    """The oracle resumed from a checkpoint taken mid-stream takes the same decisions, ranks and
    reconstructions on the remaining increments as the uninterrupted run (Theorem 2: the stored
    state is all the update reads)."""
    Y, o, last = _oracle_state(n_inc=2)
    path = tmp_path / "f.ttck"
    _write(path, o, last)
    ck = T.ttice_checkpoint_read(str(path))
    r = O.TTICEOracle(ck["dims"], ck["eps"])
    r.ranks = list(ck["ranks"])
    r.U = [c.copy() for c in ck["cores"]]
    r.last = [row.copy() for row in ck["last"]]
    more = cp_cosine(8, 8, dims=(6, 7, 5, 4), seed=5).numpy()
    for k in range(2):
        s1 = o.update(more[4 * k:4 * k + 4])
        s2 = r.update(more[4 * k:4 * k + 4])
        assert s1.ranks == s2.ranks and s1.skipped == s2.skipped and s1.n_selected == s2.n_selected
    n = len(o.last)
    np.testing.assert_allclose(r.reconstruct(0, n), o.reconstruct(0, n), rtol=0, atol=1e-13)


def test_header_claiming_more_than_the_file_holds(tmp_path):
    """A header whose sizes disagree with the file's length (here n_obs set to 2^40) is rejected when
    the header is read, before any buffer is sized from it."""
    _, o, last = _oracle_state()
    path = tmp_path / "g.ttck"
    _write(path, o, last)
    raw = bytearray(path.read_bytes())
    d = len(o.dims)
    off_nobs = 8 + 4 + 4 + 8 * d + 8 + 12 + 8 + 8 + 8 * (d + 1)
    assert struct.unpack_from("<q", raw, off_nobs)[0] == last.shape[0]
    struct.pack_into("<q", raw, off_nobs, 1 << 40)
    path.write_bytes(bytes(raw))
    with pytest.raises(T.TTICEError) as ei:
        T.ttice_checkpoint_read_header(str(path))
    assert ei.value.code == T.TTICE_EINVAL


def test_header_whose_sizes_wrap_around(tmp_path):
    """A crafted header whose array sizes overflow 64 bits: d = 2, dims [2^62, 1], ranks
    [1, 2^62, 2^62].  Each core then has 2^124 elements, 2^127 bytes, and the two sum to 0 mod
    2^128, so a length check in wrapping arithmetic would accept a file that holds only a header
    and a checksum.  The reader must reject it (checked products) with TTICE_EINVAL."""
    d = 2
    body = b"TTICECK1" + struct.pack("<ii", 1, d) + struct.pack("<qq", 1 << 62, 1) + struct.pack("<d", 0.1)
    body += struct.pack("<iii", 1, 1, 0) + struct.pack("<d", 1.0) + struct.pack("<ii", 0, 0)
    body += struct.pack("<qqq", 1, 1 << 62, 1 << 62) + struct.pack("<q", 0)
    body += struct.pack("<Q", _fnv1a(body))
    path = tmp_path / "w.ttck"
    path.write_bytes(body)
    with pytest.raises(T.TTICEError) as ei:
        T.ttice_checkpoint_read_header(str(path))
    assert ei.value.code == T.TTICE_EINVAL
