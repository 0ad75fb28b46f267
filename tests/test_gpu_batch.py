"""GPU parity of uneven, mixed-modulus batches (persistent kernel for the
one-block sizes, bucketed passes for the long products, CUDA-graph replay)
with the oracle's schoolbook products; at the full 10,000-product workload,
sampled coefficients and evaluation fingerprints."""
import numpy as np
import pytest

import oracle as O
import paper_1407_3383_gb300 as G
from paper_1407_3383_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _run_batch(primes, a_list, b_list, pidx, mode=G.NTT_BATCH_GRAPH, runs=1):
    import torch
    na = [x.size for x in a_list]
    nb = [x.size for x in b_list]
    with G.BatchPlan(primes, na, nb, pidx) as bp:
        wb = bp.word_bytes
        dt = np.uint32 if wb == 4 else np.uint64
        a = torch.from_numpy(np.concatenate(a_list).astype(dt)).cuda()
        b = torch.from_numpy(np.concatenate(b_list).astype(dt)).cuda()
        c = torch.zeros(bp.c_words, dtype=a.dtype, device="cuda")
        ws = torch.empty(bp.workspace_size(), dtype=torch.uint8, device="cuda")
        outs = []
        for _ in range(runs):
            c.zero_()
            bp.run(a, b, c, ws, mode)
            torch.cuda.synchronize()
            outs.append(c.cpu().numpy().astype(np.uint64))
        return [[o[int(bp.c_off[t]):int(bp.c_off[t] + bp.nc[t])] for t in range(len(na))] for o in outs]


def _random_batch(primes, count, lo, hi, seed):
    g = W.SplitMix64(seed)
    la = g.log_uniform_int(lo, hi, count)
    lb = np.maximum(1, (la * (0.5 + g.unit(count))).astype(np.int64))
    pidx = g.choice(len(primes), count)
    a_list = [g.uniform_mod(primes[i], int(n)) for i, n in zip(pidx, la)]
    b_list = [g.uniform_mod(primes[i], int(n)) for i, n in zip(pidx, lb)]
    return a_list, b_list, pidx


@pytest.mark.parametrize("mode", [G.NTT_BATCH_DIRECT, G.NTT_BATCH_STREAMS, G.NTT_BATCH_GRAPH])
def test_uneven_batch_u64_full(mode):
    primes = [W.P1, W.P2, W.P3]
    a_list, b_list, pidx = _random_batch(primes, 240, 1, 6000, 41)
    got = _run_batch(primes, a_list, b_list, pidx, mode, runs=2)
    want = O.polymul_ragged([primes[i] for i in pidx], a_list, b_list)
    for r in range(2):                                  # graph capture, then replay
        for t in range(len(want)):
            assert (got[r][t] == want[t]).all(), (r, t, a_list[t].size, b_list[t].size)


def test_uneven_batch_u32_full():
    primes = [W.P_A, W.P_B, W.P_TABLE11]
    a_list, b_list, pidx = _random_batch(primes, 200, 1, 12000, 42)
    got = _run_batch(primes, a_list, b_list, pidx)[0]
    want = O.polymul_ragged([primes[i] for i in pidx], a_list, b_list)
    for t in range(len(want)):
        assert (got[t] == want[t]).all(), t


@pytest.mark.parametrize("primes", [[W.P1, W.P2, W.P3], [W.P_A, W.P_B]])
def test_uneven_batch_truncated_classes(primes):
    """One product per (size 2^4 .. 2^15, class of kb blocks of n/16 output
    positions): the persistent kernel's items and the two-pass buckets
    truncate each transform to the blocks its output needs (Section 5.1);
    every word against the oracle, graph capture and replay."""
    g = W.SplitMix64(0x7B7 + len(primes))
    la, lb = [], []
    for k in range(4, 16):
        n = 1 << k
        for kb in (1, 3, 9, 12, 15, 16):
            L = max(2, kb * n // 16 - (k % 3))
            na = (L + 1) // 2 + (kb % 2)
            la.append(na)
            lb.append(L + 1 - na)
    pidx = g.choice(len(primes), len(la))
    a_list = [g.uniform_mod(primes[i], n) for i, n in zip(pidx, la)]
    b_list = [g.uniform_mod(primes[i], n) for i, n in zip(pidx, lb)]
    got = _run_batch(primes, a_list, b_list, pidx, runs=2)
    want = O.polymul_ragged([primes[i] for i in pidx], a_list, b_list)
    for r in range(2):
        for t in range(len(want)):
            assert (got[r][t] == want[t]).all(), (r, t, la[t], lb[t])


@pytest.mark.parametrize("primes", [[W.P1, W.P3], [W.P_B, W.P_A]])
def test_uneven_batch_2e16_bucket(primes):
    """Products whose transforms have 2^16 points (descriptor-driven direct
    kernels), ragged lengths on both sides of n/2."""
    g = W.SplitMix64(4242 + len(str(primes[0])))
    la = [32768, 20000, 40000, 16385, 30001]
    lb = [32768, 30000, 25000, 16000, 1]
    pidx = g.choice(len(primes), len(la))
    a_list = [g.uniform_mod(primes[i], n) for i, n in zip(pidx, la)]
    b_list = [g.uniform_mod(primes[i], n) for i, n in zip(pidx, lb)]
    got = _run_batch(primes, a_list, b_list, pidx)[0]
    want = O.polymul_ragged([primes[i] for i in pidx], a_list, b_list)
    for t in range(len(want)):
        assert (got[t] == want[t]).all(), t


@pytest.mark.parametrize("primes", [[W.P1, W.P2], [W.P_B]])
def test_uneven_batch_2e17_2e18_buckets(primes):
    """Products of 2^17 and 2^18 points in one uneven batch (descriptor-driven
    pass across 2^16-point rows): equal to the generic passes."""
    g = W.SplitMix64(1718 + len(primes))
    la = [40000, 70000, 33000, 100000, 131072]
    lb = [40000, 20000, 33000, 90000, 1]
    pidx = g.choice(len(primes), len(la))
    a_list = [g.uniform_mod(primes[i], n) for i, n in zip(pidx, la)]
    b_list = [g.uniform_mod(primes[i], n) for i, n in zip(pidx, lb)]
    G.ntt_tune_reset()
    got = _run_batch(primes, a_list, b_list, pidx)[0]
    wb = 4 if primes[0] < (1 << 32) else 8
    try:
        G.ntt_tune_import("".join(f"{wb} {k} 0 {5 if wb == 4 else 4} 4\n" for k in (17, 18)))
        padded = _run_batch(primes, a_list, b_list, pidx)[0]
    finally:
        G.ntt_tune_reset()
    for t in range(len(la)):
        assert (got[t] == padded[t]).all(), t
        p = primes[pidx[t]]
        for k in [0, got[t].size - 1, got[t].size // 3]:
            assert int(got[t][k]) == O.poly_coeff(p, a_list[t], b_list[t], k)


@pytest.mark.parametrize("primes", [[W.P1, W.P2], [W.P_B, W.P_A]])
def test_uneven_batch_truncated_rows(primes):
    """Uneven buckets of 2^17 .. 2^21 points keep each product's own row
    count lam = ceil(L / 2^16) (whole blocks of n2/16 rows past 16 rows):
    several products per bucket with different lam, equal to the padded
    generic passes and to the oracle on sampled coefficients."""
    g = W.SplitMix64(2121 + len(str(primes[0])))
    la = [40000, 70000, 130000, 100000, 150000, 250000, 200000, 600000, 1000000, 70000]
    lb = [30000, 70000, 130000, 40000, 150000, 250000, 100000, 500000, 1000000, 64000]
    pidx = [0, 0, 0, 1, 0, 0, 0, 0, 0, 1]
    a_list = [g.uniform_mod(primes[i], n) for i, n in zip(pidx, la)]
    b_list = [g.uniform_mod(primes[i], n) for i, n in zip(pidx, lb)]
    G.ntt_tune_reset()
    got = _run_batch(primes, a_list, b_list, pidx)[0]
    wb = 4 if primes[0] < (1 << 32) else 8
    try:
        G.ntt_tune_import("".join(f"{wb} {k} 0 {5 if wb == 4 else 4} 4\n" for k in (17, 18, 19, 21)))
        padded = _run_batch(primes, a_list, b_list, pidx)[0]
    finally:
        G.ntt_tune_reset()
    for t in range(len(la)):
        assert (got[t] == padded[t]).all(), t
        p = primes[pidx[t]]
        n = got[t].size
        for k in [0, n - 1, n // 3, (n * 5) // 7, 65535, 65536]:
            assert int(got[t][k]) == O.poly_coeff(p, a_list[t], b_list[t], k), (t, k)


def test_config3_full_workload_sampled():
    """10,000 products, lengths log-uniform in [2^6, 2^18], each modulo one
    of three 62-bit primes: sampled coefficients and fingerprints."""
    lengths, pidx = W.config3_shapes()
    primes_used, a_list, b_list = W.config3_operands(lengths, pidx)
    primes = [W.P1, W.P2, W.P3]
    got = _run_batch(primes, a_list, b_list, pidx)[0]
    g = W.SplitMix64(77)
    picks = list((g.u64(60) % np.uint64(len(a_list))).astype(np.int64))
    picks += [int(np.argmax(lengths)), int(np.argmin(lengths))]
    for t in picks:
        p = primes_used[t]
        n = a_list[t].size + b_list[t].size - 1
        for k in [0, n - 1, n // 2] + [int(v) for v in g.u64(3) % np.uint64(n)]:
            assert int(got[t][k]) == O.poly_coeff(p, a_list[t], b_list[t], k), (t, k)
        x = int(g.uniform_mod(p, 1)[0])
        assert O.eval_poly(p, got[t], x) == O.mulmod(O.eval_poly(p, a_list[t], x),
                                                     O.eval_poly(p, b_list[t], x), p)


def test_batch_rejects_bad_descriptors():
    with pytest.raises(G.NttError):
        G.BatchPlan([W.P1], [10, 0], [10, 5], [0, 0])           # empty operand
    with pytest.raises(G.NttError):
        G.BatchPlan([W.P1, W.P_A], [10], [10], [0])              # mixed word sizes
    with pytest.raises(G.NttError):
        G.BatchPlan([W.P1], [10], [10], [3])                     # bad modulus index


def test_autotune_keeps_results_exact():
    import torch
    p, a, b = W.config1(count=8)
    with G.Plan(p, 16) as plan:
        G.ntt_autotune(plan, 8)
        lppc, logw, lrpc = G.ntt_tune_get(4, 16)
        assert logw >= 0                        # 0: the direct 256 x 256 kernels
        da = torch.from_numpy(a.reshape(-1)).cuda()
        db = torch.from_numpy(b.reshape(-1)).cuda()
        dc = torch.empty(8 * ((1 << 16) - 1), dtype=torch.uint32, device="cuda")
        ws = G.alloc_workspace(plan, 8)
        G.polymul_mod_p_batch(plan, da, 1 << 15, db, 1 << 15, 8, dc, G.NTT_SCHED_FUSED, ws)
        torch.cuda.synchronize()
        got = dc.cpu().numpy().reshape(8, -1).astype(np.uint64)
        want = O.polymul_batch(p, a[:1].astype(np.uint64), b[:1].astype(np.uint64))
        assert (got[:1] == want).all()
