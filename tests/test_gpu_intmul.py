"""GPU parity of the three-prime integer product (Section 5.3) with the
oracle's schoolbook product of 32-bit limbs, limb for limb; at sizes where
schoolbook is too slow, exact fingerprints modulo independent primes and the
exact low 64 bits (Python integers), plus closed forms."""
import numpy as np
import pytest

import oracle as O
import paper_1407_3383_gb300 as G
from paper_1407_3383_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def plan():
    with G.IntmulPlan(1 << 21) as p:
        yield p


def _intmul(plan, a: np.ndarray, b: np.ndarray) -> np.ndarray:
    import torch
    da = torch.from_numpy(a.astype(np.uint32)).cuda()
    db = torch.from_numpy(b.astype(np.uint32)).cuda()
    dc = torch.full((a.size + b.size,), 0xDEADBEEF, dtype=torch.uint32, device="cuda")
    nbytes = G.intmul_workspace_size(plan, a.size, b.size)
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    G.intmul_crt(plan, da, a.size, db, b.size, dc, ws)
    torch.cuda.synchronize()
    return dc.cpu().numpy()


def _to_int(limbs) -> int:
    return int.from_bytes(np.ascontiguousarray(limbs.astype(np.uint32)).tobytes(), "little")


@pytest.mark.parametrize("na,nb", [(1, 1), (1, 5), (2, 2), (3, 7), (64, 64), (100, 77),
                                   (1000, 999), (4096, 4096), (5001, 17), (1 << 14, 1 << 14)])
def test_intmul_matches_schoolbook(plan, na, nb):
    g = W.SplitMix64(na * 7919 + nb)
    a = g.limbs(na)
    b = g.limbs(nb)
    assert (_intmul(plan, a, b) == O.intmul(a, b)).all()


def test_intmul_closed_forms(plan):
    for n in [1, 33, 4096, 1 << 16]:
        a = np.full(n, 0xFFFFFFFF, dtype=np.uint32)
        c = _intmul(plan, a, a)
        assert _to_int(c) == (1 << (64 * n)) - (1 << (32 * n + 1)) + 1
    z = np.zeros(300, dtype=np.uint32)
    b = W.SplitMix64(3).limbs(200)
    assert (_intmul(plan, z, b) == 0).all()
    one = np.zeros(50, dtype=np.uint32)
    one[0] = 1
    c = _intmul(plan, one, b)
    assert (c[:200] == b).all() and (c[200:] == 0).all()


@pytest.mark.parametrize("na,nb", [(1 << 20, 1 << 20), (1 << 21, 3), (777777, 1 << 20)])
def test_intmul_large_fingerprints(plan, na, nb):
    g = W.SplitMix64(na ^ nb)
    a = g.limbs(na)
    b = g.limbs(nb)
    c = _intmul(plan, a, b)
    ia, ib, ic = _to_int(a), _to_int(b), _to_int(c)
    for q in [2305843009213693951, 4611686018427387847, 1152921504606846883, 18446744073709551557]:
        assert ic % q == (ia % q) * (ib % q) % q
    assert ic % (1 << 64) == (ia % (1 << 64)) * (ib % (1 << 64)) % (1 << 64)
    assert ic.bit_length() <= 32 * (na + nb)
    # the low m limbs of a*b depend only on a[:m] and b[:m]: schoolbook them
    m = min(4096, na, nb)
    assert (c[:m] == O.intmul(a[:m], b[:m])[:m]).all()
