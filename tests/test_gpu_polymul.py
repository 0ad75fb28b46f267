"""GPU parity of the polynomial product over Z/pZ (Section 5.2) with the
oracle's schoolbook product, bit for bit.

Full comparisons where the schoolbook oracle finishes in seconds (sizes that
span several tiles and a ragged tail); at the full workload sizes, in the
launch configuration the benchmark times, sampled coefficients (each one an
O(L) oracle sum) plus evaluation fingerprints C(x) = A(x) B(x)."""
import numpy as np
import pytest

import oracle as O
import paper_1407_3383_gb300 as G
from paper_1407_3383_gb300 import workloads as W
from helpers import empty_dev, from_dev, to_dev

pytestmark = pytest.mark.gpu


def _polymul(p, log2n, a, b, schedule=G.NTT_SCHED_FUSED, flags=0):
    """a: (batch, na), b: (batch, nb) numpy -> (batch, na+nb-1) numpy."""
    import torch
    batch, na = a.shape
    _, nb = b.shape
    with G.Plan(p, log2n, flags) as plan:
        wb = plan.word_bytes
        da, db = to_dev(a.reshape(-1), wb), to_dev(b.reshape(-1), wb)
        dc = empty_dev(batch * (na + nb - 1), wb)
        ws = G.alloc_workspace(plan, batch, schedule)
        G.polymul_mod_p_batch(plan, da, na, db, nb, batch, dc, schedule, ws)
        torch.cuda.synchronize()
        return from_dev(dc).reshape(batch, na + nb - 1)


def test_config0_single_product_full():
    """One product mod 998244353 of two length-2048 operands through a
    size-4096 transform: all 4095 coefficients."""
    p, a, b = W.config0()
    got = _polymul(p, 12, a[None, :], b[None, :])
    assert (got[0] == O.polymul(p, a, b)).all()


@pytest.mark.parametrize("schedule", [G.NTT_SCHED_FUSED, G.NTT_SCHED_PLAIN])
@pytest.mark.parametrize("p,log2n,na,nb,batch", [
    (W.P_B, 5, 17, 16, 19),        # short vectors, many per block, ragged batch
    (W.P_A, 8, 128, 129, 33),      # one-line vectors at the 256 limit
    (W.P_B, 9, 300, 200, 5),       # first tiled size
    (W.P_B, 13, 4096, 4096, 3),    # largest one-block tile (u32)
    (W.P_B, 14, 8192, 8192, 2),    # two global passes (u32), both operands half the transform
    (W.P_B, 15, 9000, 7001, 2),    # two global passes, ragged lengths
    (W.P_A, 16, 1 << 15, 1 << 15, 2),
    (W.P_B, 16, 40000, 25535, 3),  # 2^16 points, operand a past n/2: no zero half
    (W.P_B, 16, 33000, 1, 2),      # 2^16 points, degree-0 operand b
    (W.P2, 16, 30001, 20000, 2),   # 2^16 points, 64-bit words
    (W.P1, 7, 64, 64, 21),
    (W.P2, 13, 4096, 4096, 2),     # largest one-block tile (u64)
    (W.P3, 14, 5000, 3000, 2),     # two global passes (u64)
    (W.P1, 12, 1, 1, 3),           # degree-0 operands
    (W.P_B, 6, 1, 40, 4),
])
def test_polymul_full(schedule, p, log2n, na, nb, batch):
    if schedule == G.NTT_SCHED_PLAIN and log2n < 2:
        pytest.skip()
    g = W.SplitMix64(p + log2n * 1000 + na)
    a = g.uniform_mod(p, batch * na).reshape(batch, na)
    b = g.uniform_mod(p, batch * nb).reshape(batch, nb)
    flags = G.NTT_FLAG_PLAIN if schedule == G.NTT_SCHED_PLAIN else 0
    got = _polymul(p, log2n, a, b, schedule, flags)
    want = O.polymul_batch(p, a, b)
    assert (got == want).all()


def test_extreme_residues():
    """Operands all p - 1: c_k = (number of terms) (p-1)^2 = #terms (mod p)."""
    for p, log2n, n in [(W.P_B, 16, 1 << 15), (W.P1, 14, 1 << 13), (W.P_A, 12, 2048)]:
        a = np.full((1, n), p - 1, dtype=np.uint64)
        got = _polymul(p, log2n, a, a)[0]
        k = np.arange(2 * n - 1)
        terms = np.minimum(k, n - 1) - np.maximum(0, k - n + 1) + 1
        assert (got == terms.astype(np.uint64) % np.uint64(p)).all()


def _sampled_check(p, a, b, got, samples, seed):
    batch, na = a.shape
    nb = b.shape[1]
    g = W.SplitMix64(seed)
    prods = (g.u64(samples) % np.uint64(batch)).astype(np.int64)
    ks = (g.u64(samples) % np.uint64(na + nb - 1)).astype(np.int64)
    prods = np.concatenate([prods, [0, batch - 1, batch - 1]])
    ks = np.concatenate([ks, [0, na + nb - 2, (na + nb) // 2]])
    for t, k in zip(prods, ks):
        assert int(got[t, k]) == O.poly_coeff(p, a[t], b[t], int(k)), (t, k)
    # fingerprints C(x) = A(x) B(x) at random points for several products
    for t in sorted(set(prods[:8].tolist())):
        for x in g.uniform_mod(p, 2):
            x = int(x)
            lhs = O.eval_poly(p, got[t], x)
            rhs = O.mulmod(O.eval_poly(p, a[t], x), O.eval_poly(p, b[t], x), p)
            assert lhs == rhs, (t, x)


@pytest.mark.parametrize("schedule", [G.NTT_SCHED_FUSED, G.NTT_SCHED_PLAIN])
def test_config1_full_size_sampled(schedule):
    """256 products mod 3*2^30+1 of length-2^15 operands (size-2^16
    transforms), exactly as the benchmark runs them (fused: also with the
    operand tiles brought in by TMA, the device error flag staying clear)."""
    p, a, b = W.config1()
    flags = G.NTT_FLAG_PLAIN if schedule == G.NTT_SCHED_PLAIN else 0
    got = _polymul(p, 16, a, b, schedule, flags)
    if schedule == G.NTT_SCHED_FUSED:                  # the same product with TMA operand tiles
        try:
            G.ntt_tune_import("4 16 1 0 0\n")
            assert (_polymul(p, 16, a, b, schedule, flags) == got).all()
            G.ntt_device_status()
        finally:
            G.ntt_tune_reset()
    _sampled_check(p, a.astype(np.uint64), b.astype(np.uint64), got, 64, 11)
    # eight products in full against the schoolbook oracle
    idx = [0, 1, 37, 100, 128, 201, 254, 255]
    want = O.polymul_batch(p, a[idx].astype(np.uint64), b[idx].astype(np.uint64))
    assert (got[idx] == want).all()


def test_config2_products_sampled():
    """1024 products of length 2^12 mod the 62-bit prime (size-2^13 transforms)."""
    p, a, b = W.config2_products()
    got = _polymul(p, 13, a, b)
    _sampled_check(p, a, b, got, 64, 12)
    want = O.polymul_batch(p, a[:8], b[:8])
    assert (got[:8] == want).all()


def test_fused_equals_plain_bitwise():
    p, a, b = W.config1(count=4)
    f = _polymul(p, 16, a, b, G.NTT_SCHED_FUSED)
    q = _polymul(p, 16, a, b, G.NTT_SCHED_PLAIN, G.NTT_FLAG_PLAIN)
    assert (f == q).all()


def test_errors_are_reported():
    import torch
    with G.Plan(W.P_A, 10) as plan:
        a = torch.zeros(600, dtype=torch.uint32, device="cuda")
        c = torch.zeros(2000, dtype=torch.uint32, device="cuda")
        with pytest.raises(G.NttError) as e:
            G.polymul_mod_p_batch(plan, a, 600, a, 600, 1, c)       # 1199 > 1024
        assert e.value.status == 5
        with pytest.raises(G.NttError) as e:
            G.polymul_mod_p_batch(plan, a, 100, a, 100, 1, c, G.NTT_SCHED_PLAIN)
        assert e.value.status == 1
    with G.Plan(W.P_B, 16) as plan:
        a = torch.zeros(1 << 15, dtype=torch.uint32, device="cuda")
        c = torch.zeros(1 << 16, dtype=torch.uint32, device="cuda")
        with pytest.raises(G.NttError) as e:
            G.polymul_mod_p_batch(plan, a, 1 << 15, a, 1 << 15, 1, c)   # no workspace
        assert e.value.status == 10
    with G.Plan(W.P_A, 10, G.NTT_FLAG_CHECK) as plan:
        bad = torch.full((100,), W.P_A, dtype=torch.uint32, device="cuda")
        c = torch.zeros(199, dtype=torch.uint32, device="cuda")
        with pytest.raises(G.NttError) as e:
            G.polymul_mod_p_batch(plan, bad, 100, bad, 100, 1, c)
        assert e.value.status == 6


@pytest.mark.parametrize("p", [W.P_B, W.P3])
def test_direct_kernels_equal_generic_passes(p):
    """At n = 2^16 the default shape (logw = 0) runs the direct 256 x 256
    kernels; the generic column/row passes must give the same words."""
    g = W.SplitMix64(616 + p % 1000)
    a = g.uniform_mod(p, 3 * 30000).reshape(3, 30000)
    b = g.uniform_mod(p, 3 * 27000).reshape(3, 27000)
    wb = 4 if p < (1 << 32) else 8
    G.ntt_tune_reset()
    assert G.ntt_tune_get(wb, 16)[1] == 0
    direct = _polymul(p, 16, a, b)
    try:
        G.ntt_tune_import(f"{wb} 16 0 {5 if wb == 4 else 4} 4\n")
        generic = _polymul(p, 16, a, b)
    finally:
        G.ntt_tune_reset()
    assert (direct == generic).all()
    assert (direct[1] == O.polymul(p, a[1], b[1])).all()



@pytest.mark.parametrize("p", [W.P_B, W.P1])
@pytest.mark.parametrize("beta", list(range(1, 17)))
def test_tft_products_every_length_class(p, beta):
    """n = 2^16 products whose output needs B = beta of the 16 row blocks run
    the truncated transforms (Section 5.1's TFT through Algorithm 1); they
    must equal the padded generic passes word for word and the oracle."""
    g = W.SplitMix64(0x7F7 + beta + p % 97)
    L = 4096 * beta - (1 if beta % 2 else 2047)          # both ends of the class (13+ run full-length kernels)
    na = (L + 1) // 2 + (beta % 3)                        # ragged, sometimes past n/2
    nb = L + 1 - na
    a = g.uniform_mod(p, 2 * na).reshape(2, na)
    b = g.uniform_mod(p, 2 * nb).reshape(2, nb)
    wb = 4 if p < (1 << 32) else 8
    G.ntt_tune_reset()
    tft = _polymul(p, 16, a, b)
    try:
        G.ntt_tune_import(f"{wb} 16 0 {5 if wb == 4 else 4} 4\n")
        padded = _polymul(p, 16, a, b)
    finally:
        G.ntt_tune_reset()
    assert (tft == padded).all()
    if na * nb <= 1 << 24:
        assert (tft[1] == O.polymul(p, a[1], b[1])).all()
    else:
        _sampled_check(p, a, b, tft, 24, beta)


def _tft_lengths(log2n):
    """Output lengths L <= n = 2^log2n at both ends of the classes of kb
    blocks of n/16 positions (kb = 1, 2, 7, 9, 13, 14, 15, 16)."""
    n = 1 << log2n
    blk = n // 16
    out = []
    for kb in (1, 2, 7, 9, 13, 14, 15, 16):
        out += [max(1, (kb - 1) * blk + 1), kb * blk]
    return sorted(set(out))


@pytest.mark.parametrize("p", [W.P_B, W.P1])
@pytest.mark.parametrize("log2n", list(range(4, 16)))
def test_tft_one_block_and_two_pass_sizes(p, log2n):
    """Products through n = 2^4 .. 2^15 points -- the one-block kernel and,
    above 2^13 points, the two-pass kernels --
    whose output needs kb of the 16 blocks of n/16 positions run the
    truncated transforms of Section 5.1 (kb <= 14; the rest the full ones):
    every output word against the schoolbook oracle, at both ends of each
    class, with operands on both sides of n/2."""
    g = W.SplitMix64(0x7F70 + log2n + p % 89)
    for L in _tft_lengths(log2n):
        na = max(1, min(L, (L + 1) // 2 + (L % 5) - 2))
        nb = L + 1 - na
        batch = 3 if log2n < 14 else 2
        a = g.uniform_mod(p, batch * na).reshape(batch, na)
        b = g.uniform_mod(p, batch * nb).reshape(batch, nb)
        got = _polymul(p, log2n, a, b)
        assert (got == O.polymul_batch(p, a, b)).all(), (log2n, L, na, nb)


def _generic_vs_default(p, log2n, a, b):
    wb = 4 if p < (1 << 32) else 8
    G.ntt_tune_reset()
    got = _polymul(p, log2n, a, b)
    k2 = log2n // 2
    try:
        G.ntt_tune_import(f"{wb} {log2n} 0 {5 if wb == 4 else 4} 4\n")
        padded = _polymul(p, log2n, a, b)
    finally:
        G.ntt_tune_reset()
    return got, padded


@pytest.mark.parametrize("p,log2n,L", [
    (W.P_B, 17, 65537), (W.P_B, 17, 131071),                        # n2 = 2: one row (TFT), both rows
    (W.P1, 18, 65536), (W.P1, 18, 131073), (W.P1, 18, 196608), (W.P1, 18, 262143),   # every row count
    (W.P_A, 19, 300001), (W.P2, 20, 70000), (W.P3, 20, 1048575),
    (W.P_B, 21, (1 << 20) + 5), (W.P_B, 21, 2097151),               # n2 = 32: 1 of 16 blocks (TFT), all
    (W.P1, 22, 3 << 20), (W.P_A, 23, (5 << 20) + 3), (W.P3, 24, 16777215), (W.P2, 24, 9 << 20),
])
def test_products_2e17_to_2e24(p, log2n, L):
    """n = 2^17 .. 2^24: Algorithm 1 with 2^16-point rows (a pass across the
    rows -- in registers up to 16 rows, a column kernel above -- the direct
    kernels on the rows, the inverse pass), truncated to the rows the output
    needs; equal to the padded generic passes and the oracle on sampled
    coefficients and fingerprints."""
    g = W.SplitMix64(L + log2n)
    na = (L + 1) // 2 + 17
    nb = L + 1 - na
    a = g.uniform_mod(p, na)[None, :]
    b = g.uniform_mod(p, nb)[None, :]
    got, padded = _generic_vs_default(p, log2n, a, b)
    assert (got == padded).all()
    _sampled_check(p, a, b, got, 32, L)


@pytest.mark.parametrize("p,na,nb", [(W.P_B, 256 * 100, 256 * 37), (W.P1, 256 * 128, 256), (W.P_A, 256, 256)])
def test_tma_tiles_partial_rows(p, na, nb):
    """With the TMA shape (lppc = 1), whole-row operands shorter than n/2
    take the TMA column kernel, whose copy zero-fills the rows past each
    operand; compare with the oracle and the plain-load kernels."""
    g = W.SplitMix64(na + 3 * nb)
    a = g.uniform_mod(p, 2 * na).reshape(2, na)
    b = g.uniform_mod(p, 2 * nb).reshape(2, nb)
    wb = 4 if p < (1 << 32) else 8
    G.ntt_tune_reset()
    plain = _polymul(p, 16, a, b)
    try:
        G.ntt_tune_import(f"{wb} 16 1 0 0\n")
        got = _polymul(p, 16, a, b)
        G.ntt_device_status()
    finally:
        G.ntt_tune_reset()
    assert (got == plain).all()
    assert (got == O.polymul_batch(p, a, b)).all()



@pytest.mark.parametrize("p,log2n,na,nb,batch,chunk,pinned", [
    (W.P_B, 16, 1 << 15, 1 << 15, 7, 3, True),     # ragged last chunk, three sets in flight
    (W.P_B, 16, 1 << 15, 1 << 15, 4, 1, True),     # one product per chunk
    (W.P_A, 12, 2048, 2048, 5, 64, False),          # chunk > batch, pageable host memory
    (W.P2, 13, 4096, 4000, 6, 4, True),             # 64-bit words
    (W.P_B, 15, 9000, 7001, 3, 2, True),            # two global passes with a workspace
    (W.P_A, 12, 2048, 2048, 13, 4, True),           # ramped chunks 1, 2, 4, 3, 2, 1
])
def test_polymul_host_buffers(p, log2n, na, nb, batch, chunk, pinned):
    """polymul_mod_p_batch_host (host operands, chunked copies overlapping
    the products) returns the oracle's product for every pair, twice in a row
    through the same staging buffer."""
    import torch
    a, b = W.pair_batch(p, batch, na, nb, seed=0x5EED0100 + log2n + chunk)
    dt = torch.uint32 if p < 1 << 32 else torch.uint64
    npt = np.uint32 if p < 1 << 32 else np.uint64

    def host(x):
        t = torch.from_numpy(np.ascontiguousarray(x.reshape(-1).astype(npt)))
        return t.pin_memory() if pinned else t

    ha, hb = host(a), host(b)
    nc = na + nb - 1
    with G.Plan(p, log2n) as plan:
        stage = torch.empty(G.polymul_host_stage_size(plan, na, nb, chunk), dtype=torch.uint8,
                            device="cuda")
        for rep in range(2):
            hc = torch.full((batch * nc,), 0xFFFF, dtype=dt)
            hc = hc.pin_memory() if pinned else hc
            G.polymul_mod_p_batch_host(plan, ha, na, hb, nb, batch, hc, chunk, stage)
            torch.cuda.synchronize()
            got = hc.numpy().astype(np.uint64).reshape(batch, nc)
            for t in range(batch):
                assert (got[t] == O.polymul(p, a[t], b[t])).all(), (rep, t)
        with pytest.raises(G.NttError) as e:
            G.polymul_mod_p_batch_host(plan, ha, na, hb, nb, batch, hc, chunk, stage[:256])
        assert e.value.status == 10   # NTT_ERR_WORKSPACE


def test_polymul_host_buffers_edge_cases():
    """polymul_mod_p_batch_host: an empty batch is a no-op; a zero chunk, a
    length past n and a staging buffer sized for a smaller chunk are refused
    before anything is enqueued; doubles (NTT_FLAG_FP64 plans) take the same
    path and match the integer plan's product."""
    import torch
    p = W.P_TABLE12
    a, b = W.pair_batch(p, 5, 1500, 1000, seed=0x5EED0200)
    with G.Plan(p, 12) as plan:
        stage = torch.empty(G.polymul_host_stage_size(plan, 1500, 1000, 2), dtype=torch.uint8, device="cuda")
        ha = torch.from_numpy(a.reshape(-1).astype(np.uint64)).pin_memory()
        hb = torch.from_numpy(b.reshape(-1).astype(np.uint64)).pin_memory()
        hc = torch.zeros(5 * 2499, dtype=torch.uint64).pin_memory()
        G.polymul_mod_p_batch_host(plan, ha, 1500, hb, 1000, 0, hc, 2, stage)      # empty batch
        torch.cuda.synchronize()
        assert int(hc.sum()) == 0
        for chunk, na, st, status in [(0, 1500, stage, 1), (2, 3500, stage, 5), (4, 1500, stage, 10)]:
            with pytest.raises(G.NttError) as e:
                G.polymul_mod_p_batch_host(plan, ha, na, hb, 1000, 5, hc, chunk, st)
            assert e.value.status == status, (chunk, na)
        G.polymul_mod_p_batch_host(plan, ha, 1500, hb, 1000, 5, hc, 2, stage)
        torch.cuda.synchronize()
        want = hc.numpy().copy().reshape(5, 2499)
    for t in range(5):
        assert (want[t] == O.polymul(p, a[t], b[t])).all(), t
    with G.Plan(p, 12, G.NTT_FLAG_FP64) as plan:
        stage = torch.empty(G.polymul_host_stage_size(plan, 1500, 1000, 2), dtype=torch.uint8, device="cuda")
        ha = torch.from_numpy(a.reshape(-1).astype(np.float64)).pin_memory()
        hb = torch.from_numpy(b.reshape(-1).astype(np.float64)).pin_memory()
        hc = torch.zeros(5 * 2499, dtype=torch.float64).pin_memory()
        G.polymul_mod_p_batch_host(plan, ha, 1500, hb, 1000, 5, hc, 2, stage)
        torch.cuda.synchronize()
        assert (hc.numpy().astype(np.uint64).reshape(5, 2499) == want).all()


@pytest.mark.parametrize("p", [W.P_A, W.P_B, W.P1])
@pytest.mark.parametrize("na,nb", [(2048, 2048), (3000, 1096), (1, 4095), (2047, 1), (1500, 700)])
def test_cluster_products_match_oracle_and_one_block(p, na, nb):
    """n = 4096: batches of at most 16 products run one product per
    thread-block cluster (8 CTAs exchanging rows and columns through
    distributed shared memory), larger batches the one-block kernel; both
    give the oracle's product, bit for bit, zero-half and ragged lengths."""
    g = W.SplitMix64(p ^ na ^ (nb << 20))
    a = g.uniform_mod(p, 17 * na).reshape(17, na)
    b = g.uniform_mod(p, 17 * nb).reshape(17, nb)
    one_block = _polymul(p, 12, a, b)                  # 17 products: the one-block kernel
    cluster = _polymul(p, 12, a[:16], b[:16])          # 16 products: one cluster each
    single = _polymul(p, 12, a[5:6], b[5:6])
    assert (cluster == one_block[:16]).all()
    assert (single[0] == one_block[5]).all()
    for t in (0, 7, 15):
        assert (cluster[t] == O.polymul(p, a[t], b[t])).all()
