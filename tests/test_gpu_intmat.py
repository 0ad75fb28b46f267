"""GPU parity of the integer matrix product by modular transforms (Section
5.3, Table 17's method): every entry against Python integers built from the
oracle's schoolbook limb products; at the paper's Table 17 shape (entries of
32 x 2^15 bits) through fingerprints modulo independent primes."""
import numpy as np
import pytest

import oracle as O
import paper_1407_3383_gb300 as G
from paper_1407_3383_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _to_int(limbs):
    return int.from_bytes(np.ascontiguousarray(limbs.astype(np.uint32)).tobytes(), "little")


def _intmat(plan, A, B):
    import torch
    n, _, na = A.shape
    nb = B.shape[2]
    dA = torch.from_numpy(A.reshape(-1)).cuda()
    dB = torch.from_numpy(B.reshape(-1)).cuda()
    dC = torch.full((n * n * (na + nb + 1),), 0xDEADBEEF, dtype=torch.uint32, device="cuda")
    ws = torch.empty(G.intmat_workspace_size(plan, n, na, nb), dtype=torch.uint8, device="cuda")
    G.intmat_mul(plan, dA, na, dB, nb, n, dC, ws)
    torch.cuda.synchronize()
    return dC.cpu().numpy().reshape(n, n, na + nb + 1)


@pytest.fixture(scope="module")
def plan():
    with G.IntmulPlan(1 << 16) as p:
        yield p


@pytest.mark.parametrize("n,na,nb", [(1, 1, 1), (2, 3, 5), (4, 64, 64), (3, 1001, 777), (8, 300, 300)])
def test_intmat_exact(plan, n, na, nb):
    g = W.SplitMix64(n * 100 + na + nb)
    A = g.limbs(n * n * na).reshape(n, n, na)
    B = g.limbs(n * n * nb).reshape(n, n, nb)
    C = _intmat(plan, A, B)
    for i in range(n):
        for j in range(n):
            want = sum(_to_int(O.intmul(A[i, l], B[l, j])) for l in range(n))
            assert _to_int(C[i, j]) == want, (i, j)


def test_intmat_table17_shape_fingerprints(plan):
    """n = 32, entries of 32 x 2^15 bits (2^15 limbs)."""
    n, na = 32, 1 << 15
    g = W.SplitMix64(1717)
    A = g.limbs(n * n * na).reshape(n, n, na)
    B = g.limbs(n * n * na).reshape(n, n, na)
    C = _intmat(plan, A, B)
    for i, j in [(0, 0), (31, 31), (7, 19)]:
        c = _to_int(C[i, j])
        for q in [2305843009213693951, 1152921504606846883]:
            want = sum((_to_int(A[i, l]) % q) * (_to_int(B[l, j]) % q) for l in range(n)) % q
            assert c % q == want
        assert c.bit_length() <= 32 * 2 * na + 5          # n = 32 products
