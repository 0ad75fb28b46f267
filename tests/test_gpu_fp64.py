"""Transforms and products over doubles with Function 16 (Section 3.3,
NTT_FLAG_FP64; the paper's FMA transform of Table 12, p = 1108307720798209):
bit for bit equal to the integer plan on the same prime and to the oracle."""
import numpy as np
import pytest

import oracle as O
import paper_1407_3383_gb300 as G
from paper_1407_3383_gb300 import workloads as W

pytestmark = pytest.mark.gpu

P = W.P_TABLE12


def _dev(x, fp64):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x.astype(np.float64 if fp64 else np.uint64))).cuda()


def _host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy().astype(np.uint64)


@pytest.mark.parametrize("log2n,batch", [(1, 5), (4, 9), (8, 33), (11, 3), (13, 2), (14, 2), (16, 2), (18, 1), (20, 1)])
def test_fp64_transform_equals_integer_plan(log2n, batch):
    n = 1 << log2n
    a = W.SplitMix64(log2n * 7 + 1).uniform_mod(P, batch * n)
    with G.Plan(P, log2n, G.NTT_FLAG_FP64) as pf, G.Plan(P, log2n) as pi:
        assert pf.word_bytes == 8
        df, di = _dev(a, True), _dev(a, False)
        G.ntt_forward(pf, df, batch)
        G.ntt_forward(pi, di, batch)
        ff, fi = _host(df), _host(di)
        assert (ff == fi).all()
        if log2n <= 8:
            w = O.root_of_unity(P, log2n)
            for v in range(batch):
                assert (ff[v * n:(v + 1) * n] == O.dft(P, w, a[v * n:(v + 1) * n])).all()
        G.ntt_inverse(pf, df, batch)
        assert (_host(df) == a).all()


@pytest.mark.parametrize("log2n,na,nb,batch", [(6, 30, 35, 7), (12, 2048, 2048, 3), (14, 9000, 7000, 2),
                                               (16, 1 << 15, 1 << 15, 2), (16, 40000, 20000, 2)])
def test_fp64_products_match_oracle(log2n, na, nb, batch):
    import torch
    g = W.SplitMix64(log2n + na)
    a = g.uniform_mod(P, batch * na).reshape(batch, na)
    b = g.uniform_mod(P, batch * nb).reshape(batch, nb)
    with G.Plan(P, log2n, G.NTT_FLAG_FP64) as pf:
        dc = torch.empty(batch * (na + nb - 1), dtype=torch.float64, device="cuda")
        ws = G.alloc_workspace(pf, batch)
        G.polymul_mod_p_batch(pf, _dev(a.reshape(-1), True), na, _dev(b.reshape(-1), True), nb, batch, dc,
                              G.NTT_SCHED_FUSED, ws)
        got = _host(dc).reshape(batch, na + nb - 1)
    want = O.polymul_batch(P, a, b)
    assert (got == want).all()


def test_fp64_extreme_operands():
    """All operands p - 1: every Function 16 product sees its largest inputs."""
    import torch
    n = 4096
    a = np.full(n, P - 1, dtype=np.uint64)
    with G.Plan(P, 13, G.NTT_FLAG_FP64) as pf:
        dc = torch.empty(2 * n - 1, dtype=torch.float64, device="cuda")
        G.polymul_mod_p_batch(pf, _dev(a, True), n, _dev(a, True), n, 1, dc, G.NTT_SCHED_FUSED,
                              G.alloc_workspace(pf, 1))
        got = _host(dc)
    k = np.arange(2 * n - 1)
    terms = np.minimum(k, n - 1) - np.maximum(0, k - n + 1) + 1
    assert (got == terms.astype(np.uint64) % np.uint64(P)).all()


def test_fp64_refusals():
    import torch
    with pytest.raises(G.NttError) as e:
        G.Plan(W.P1, 10, G.NTT_FLAG_FP64)                     # p >= 2^50
    assert e.value.status == 2
    with pytest.raises(G.NttError):
        G.Plan(P, 10, G.NTT_FLAG_FP64 | G.NTT_FLAG_PLAIN)
    with G.Plan(P, 8, G.NTT_FLAG_FP64 | G.NTT_FLAG_CHECK) as pf:
        bad = torch.tensor([0.5] + [0.0] * 255, dtype=torch.float64, device="cuda")
        with pytest.raises(G.NttError) as e:
            G.ntt_forward(pf, bad, 1)                            # not an integer
        assert e.value.status == 6
