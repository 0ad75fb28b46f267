"""The algorithmic operation counts behind the benchmark's roofline figure
(CPU only): butterflies counted by walking the radix-2 decimation-in-
frequency network, the two-pass split of Algorithm 1 checked against the
one-pass transform, and the per-launch totals of the product kernels."""
import bench


def _walk_dif(L):
    """(nontrivial, trivial) butterflies of a length-L DIF network, by
    enumerating every butterfly and its twiddle exponent."""
    nontrivial = trivial = 0
    h = L // 2
    while h >= 1:
        for s in range(0, L, 2 * h):
            for j in range(h):
                if j == 0:
                    trivial += 1          # twiddle w^0 = 1
                else:
                    nontrivial += 1
        h //= 2
    return nontrivial, trivial


def test_dif_counts_match_the_network():
    for k in range(1, 13):
        assert bench.dif_counts(1 << k) == _walk_dif(1 << k), k


def test_two_pass_split_does_the_one_pass_work():
    """n = n2 x n1: the column and row transforms have as many butterflies as
    the one-pass transform, and the step-2 twiddles that are not 1 (all but
    the first row and column of the n2 x n1 table) are exactly the twiddles
    the one-pass network applies and the split turns into trivial ones."""
    for k in range(2, 21):
        k2 = k // 2
        k1 = k - k2
        n1, n2, n = 1 << k1, 1 << k2, 1 << k
        nt_full, tr_full = bench.dif_counts(n)
        nt2, tr2 = bench.dif_counts(n2)
        nt1, tr1 = bench.dif_counts(n1)
        split_nt = n1 * nt2 + n2 * nt1
        split_tr = n1 * tr2 + n2 * tr1
        assert split_nt + split_tr == nt_full + tr_full == (n // 2) * k
        step2 = n - n1 - n2 + 1
        assert split_nt + step2 == nt_full
        assert split_tr - step2 == tr_full


def test_product_kernel_totals():
    """Per product of two length-2^15 operands at n = 2^16: the three fused
    launches together do three length-2^16 transforms, n pointwise products
    and one scaling per output word, written out from the word policy's
    instruction counts."""
    o = bench.OPS32
    log2n, na, nb, batch = 16, 1 << 15, 1 << 15, 1
    n, nc = 1 << log2n, na + nb - 1
    ops = bench.fused_kernel_ops(log2n, na, nb, batch, 14)
    nt, tr = bench.dif_counts(n)
    one_pass = nt * (o["add"] + o["sub"] + o["mulw"]) + tr * (o["add"] + o["sub"])
    total = ops["k_col_fwd_d"] + ops["k_row_polymul_d"] + ops["k_col_inv_d"]
    assert total == 3 * one_pass + n * o["mulg"] + nc * o["mulw"]
    # the TMA column kernel does the same work as the per-thread-load one
    assert ops["k_col_fwd_tma"] == ops["k_col_fwd_d"]
    # one-block sizes: everything in one launch
    small = bench.fused_kernel_ops(12, 2048, 2048, 3, 14)
    nt, tr = bench.dif_counts(1 << 12)
    per = 3 * (nt * (o["add"] + o["sub"] + o["mulw"]) + tr * (o["add"] + o["sub"]))
    assert small == {"k_tile_polymul": 3 * (per + 4096 * o["mulg"] + 4095 * o["mulw"])}


def test_algorithmic_bytes():
    assert bench.alg_bytes(1 << 15, 1 << 15, 256, 4) == 256 * ((1 << 15) * 2 + (1 << 16) - 1) * 4


def test_u64_counts():
    """The 64-bit forms: a butterfly whose difference feeds a twiddle product
    costs a sum, a lazy difference and a twiddle product; the others a sum
    and a full difference; products add three transforms, the pointwise
    products and the scaled canonical store."""
    o = bench.OPS64
    for k in range(1, 14):
        L = 1 << k
        nt, tr = bench.dif_counts(L)
        assert bench.transform_ops64(L) == nt * (o["add"] + o["sub_lazy"] + o["mulw"]) + tr * (o["add"] + o["sub"])
        assert bench.ntt64_ops(L, 3) == 3 * (bench.transform_ops64(L) + L * o["canon"])
    n, na, nb = 1 << 13, 4096, 4096
    assert bench.polymul64_ops(13, na, nb, 2) == 2 * (3 * bench.transform_ops64(n) + n * o["mulg"]
                                                      + (na + nb - 1) * (o["mulw"] + o["canon"]))
    # per radix-2 butterfly: within the 20-24 32-bit operations estimated for 64-bit words
    assert 20 <= o["add"] + o["sub_lazy"] + o["mulw"] <= 24
