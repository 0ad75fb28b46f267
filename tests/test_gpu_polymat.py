"""GPU parity of the polynomial matrix product (Section 5.2): transforms of
the entries, n x n products at every frequency, inverse transforms; against
the oracle's schoolbook definition, and at the paper's Table 15 shape
(n = 32, degree < 2^15) through evaluation fingerprints."""
import numpy as np
import pytest

import oracle as O
import paper_1407_3383_gb300 as G
from paper_1407_3383_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _polymat(p, log2n, A, B):
    import torch
    n, _, d = A.shape
    with G.Plan(p, log2n) as plan:
        dt = np.uint32 if plan.word_bytes == 4 else np.uint64
        dA = torch.from_numpy(A.reshape(-1).astype(dt)).cuda()
        dB = torch.from_numpy(B.reshape(-1).astype(dt)).cuda()
        dC = torch.empty(n * n * (2 * d - 1), dtype=dA.dtype, device="cuda")
        ws = torch.empty(G.polymat_workspace_size(plan, n), dtype=torch.uint8, device="cuda")
        G.polymat_mul(plan, dA, dB, n, d, dC, ws)
        torch.cuda.synchronize()
        return dC.cpu().numpy().astype(np.uint64).reshape(n, n, 2 * d - 1)


@pytest.mark.parametrize("p,n,d,log2n", [
    (W.P_TABLE11, 1, 1, 1), (W.P_TABLE11, 3, 5, 4), (W.P_B, 4, 100, 8), (W.P_A, 8, 700, 11),
    (W.P1, 3, 37, 7), (W.P2, 5, 3000, 13), (W.P3, 2, 9000, 15), (W.P_B, 2, 20000, 16),
    (W.P_B, 16, 300, 10),          # shared-memory frequency kernel, one term per fold (p > 2^31)
    (W.P_TABLE11, 32, 100, 8),     # shared-memory frequency kernel, one fold per output
    (W.P_A, 32, 33, 7),            # 32 x 32 over 998244353 (several terms per fold)
    (W.P_TABLE11, 8, 5, 4),        # fewer frequencies than a block holds
    (W.P1, 8, 50, 7), (W.P3, 16, 20, 6), (W.P2, 32, 9, 5),   # 64-bit shared-memory kernel (128-bit sums)
])
def test_polymat_full(p, n, d, log2n):
    g = W.SplitMix64(p ^ (n * 1000 + d))
    A = g.uniform_mod(p, n * n * d).reshape(n, n, d)
    B = g.uniform_mod(p, n * n * d).reshape(n, n, d)
    assert (_polymat(p, log2n, A, B) == O.polymat_mul(p, A, B)).all()


def test_polymat_table15_shape_fingerprints():
    """n = 32, degree < 2^15 over 469762049: C_ij(x) = sum_l A_il(x) B_lj(x)."""
    p, n, d = W.P_TABLE11, 32, 1 << 15
    g = W.SplitMix64(1515)
    A = g.uniform_mod(p, n * n * d).reshape(n, n, d)
    B = g.uniform_mod(p, n * n * d).reshape(n, n, d)
    C = _polymat(p, 16, A, B)
    for i, j in [(0, 0), (31, 31), (5, 17), (20, 3)]:
        x = int(g.uniform_mod(p, 1)[0])
        want = 0
        for l in range(n):
            want = (want + O.eval_poly(p, A[i, l], x) * O.eval_poly(p, B[l, j], x)) % p
        assert O.eval_poly(p, C[i, j], x) == want
