"""The seeded input generators: the C stream (workloads_gen.c) must give the
numpy stream's draws exactly, and consume it identically, so that a test
that ran with either sees the same inputs."""
import numpy as np
import pytest

from paper_1407_3383_gb300 import build as B
from paper_1407_3383_gb300 import workloads as W


@pytest.fixture(scope="module", autouse=True)
def _built():
    B.build_generator()
    W._gen = None          # reload after the build
    assert W._gen_lib() is not None


@pytest.mark.parametrize("p", [3, 17, W.P_A, W.P_B, W.P_TABLE11, W.P_TABLE12, W.P1, W.P2, W.P3,
                               (1 << 63) + 29])
def test_c_stream_equals_numpy_stream(p):
    for seed in (0, 1, W.SEED_BASE + 3, (1 << 64) - 1):
        c, py = W.SplitMix64(seed), W.SplitMix64(seed, native=False)
        for n in (0, 1, 2, 15, 16, 17, 1000, 4099):
            x, y = c.uniform_mod(p, n), py.uniform_mod(p, n)
            assert (x == y).all() and c.state == py.state
            assert (x < p).all()
            x, y = c.u64(n), py.u64(n)
            assert (x == y).all() and c.state == py.state


def test_splitmix64_published_first_outputs():
    # splitmix64 from seed 0: the first outputs of the reference generator
    # (Vigna's splitmix64.c with x = 0)
    g = W.SplitMix64(0)
    want = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    assert [int(v) for v in g.u64(3)] == want
    g = W.SplitMix64(0, native=False)
    assert [int(v) for v in g.u64(3)] == want


def test_uniform_residues_are_uniform():
    # 2^20 draws mod 7: each class within 1% of 1/7
    x = W.SplitMix64(5).uniform_mod(7, 1 << 20)
    counts = np.bincount(x.astype(np.int64), minlength=7) / x.size
    assert np.all(np.abs(counts - 1 / 7) < 0.01)
