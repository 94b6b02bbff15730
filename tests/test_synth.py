"""Pins of the seeded input generator (RFC 8439 vectors, sampler moments)."""
import numpy as np

from conftest import read_golden
from paper_2506_12761_gb300 import synth


def _hex(words):
    return [int(w, 16) for w in words]


def test_quarter_round_rfc8439_2_1_1():
    g = read_golden("chacha20_rfc8439.txt")
    s = [np.array([w], dtype=np.uint32) for w in _hex(g["quarter_in"])]
    with np.errstate(over="ignore"):
        synth._quarter(s, 0, 1, 2, 3)
    assert [int(x[0]) for x in s] == _hex(g["quarter_out"])


def test_block_function_rfc8439_2_3_2():
    g = read_golden("chacha20_rfc8439.txt")
    out = synth.chacha20_blocks(_hex(g["key"]), _hex(g["nonce"]), int(g["counter"][0]), 1)[0]
    assert [int(w) for w in out] == _hex(g["block"])


def test_stream_is_sequential():
    a = synth.Stream(1, 2, 3)
    w1 = np.concatenate([a.words(5), a.words(40), a.words(3)])
    w2 = synth.Stream(1, 2, 3).words(48)
    assert np.array_equal(w1, w2)
    assert not np.array_equal(w2, synth.Stream(1, 2, 4).words(48))


def test_gaussian_moments():
    e = synth.Stream(5, 1, 9).gaussian_torus((200000,), -15).view(np.int32).astype(np.float64)
    sigma = 2.0 ** 17
    assert abs(e.mean()) < 4 * sigma / np.sqrt(len(e))
    assert abs(e.std() / sigma - 1.0) < 0.01


def test_bits_and_uniform_int():
    st = synth.Stream(5, 1, 10)
    b = st.bits(10000)
    assert set(np.unique(b)) <= {0, 1} and abs(b.mean() - 0.5) < 0.03
    r = st.uniform_int(20000, 3, 11)
    assert r.min() == 3 and r.max() == 10


def test_workload_shapes():
    w = synth.idm_workload(4, 8)
    assert w["ids"][w["planted"]] == w["query"] and w["ids"].max() < 256
    w = synth.idm_workload(1000, 32, distinct=True, payload=True)
    assert len(set(int(x) for x in w["ids"])) == 1000 and w["payload"].shape == (1000,)
    w = synth.intv_workload(64)
    r = w["rects"].astype(np.int64)
    assert np.all(r[:, 0] < r[:, 1]) and np.all(r[:, 2] < r[:, 3])
    sz = synth.log_uniform_sizes(1000, 256, 16384)
    assert sz.min() >= 256 and sz.max() < 16384
