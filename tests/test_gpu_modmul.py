"""GPU parity: every modular-product variant (Functions 6, 8, 13, 16 and the
transform kernels' own twiddle and pointwise products) against the oracle's
(x y) rem p, bit for bit, on random and adversarial operands."""
import numpy as np
import pytest

import oracle as O
import paper_1407_3383_gb300 as G
from paper_1407_3383_gb300 import workloads as W
from helpers import from_dev

pytestmark = pytest.mark.gpu

P32 = [W.P_A, W.P_B, W.P_TABLE11, 17, 257, 65537, (1 << 31) - 1, 4294967291]
P64 = [W.P1, W.P2, W.P3, W.P_TABLE12, 1152921504606846883]


def _operands(p: int, n: int, seed: int):
    g = W.SplitMix64(seed)
    x = g.uniform_mod(p, n)
    y = g.uniform_mod(p, n)
    special = [0, 1, 2, p - 1, p - 2, (p - 1) // 2, (p + 1) // 2]
    for v in [1 << 31, (1 << 31) - 1, 1 << 30, 1 << 61, (1 << 61) - 1, 1 << 49]:
        if v < p:
            special.append(v)
    s = np.array(special, dtype=np.uint64)
    sx = np.repeat(s, s.size)
    sy = np.tile(s, s.size)
    return np.concatenate([sx, x]), np.concatenate([sy, y])


def _run(p, kind, wb, x, y):
    import torch
    yc = None
    if kind in (G.NTT_MM_SHOUP, G.NTT_MM_MONT_FIXED):
        yc = torch.from_numpy(G.ntt_fixed_companion(p, kind, wb, y)).cuda()
    dx = torch.from_numpy(x).cuda()
    dy = torch.from_numpy(y).cuda()
    dz = torch.empty_like(dx)
    G.ntt_modmul_vec(p, kind, wb, dx, dy, yc, dz)
    torch.cuda.synchronize()
    return from_dev(dz)


KINDS32 = [G.NTT_MM_BARRETT, G.NTT_MM_SHOUP, G.NTT_MM_MONTGOMERY, G.NTT_MM_MONT_FIXED,
           G.NTT_MM_MONT_PRODUCT, G.NTT_MM_FMA, G.NTT_MM_ADD, G.NTT_MM_SUB,
           G.NTT_MM_MONT_FIXED_W, G.NTT_MM_MONT_PRODUCT_W]
KINDS64 = [G.NTT_MM_BARRETT, G.NTT_MM_SHOUP, G.NTT_MM_MONTGOMERY, G.NTT_MM_MONT_PRODUCT,
           G.NTT_MM_ADD, G.NTT_MM_SUB]


def _want(p, kind, x, y):
    if kind == G.NTT_MM_ADD:
        return np.array([O.addmod(int(a), int(b), p) for a, b in zip(x, y)], dtype=np.uint64)
    if kind == G.NTT_MM_SUB:
        return np.array([O.submod(int(a), int(b), p) for a, b in zip(x, y)], dtype=np.uint64)
    return O.mulmod_vec(p, x, y)


@pytest.mark.parametrize("p", P32)
@pytest.mark.parametrize("kind", KINDS32)
def test_modmul_u32(p, kind):
    x, y = _operands(p, 1 << 16 if kind in (G.NTT_MM_ADD, G.NTT_MM_SUB) else 1 << 18, p ^ kind)
    assert (_run(p, kind, 4, x, y) == _want(p, kind, x, y)).all()


def test_wide_forms_refuse_64_bit_words():
    import torch
    x = torch.zeros(4, dtype=torch.uint64, device="cuda")
    for kind in (G.NTT_MM_MONT_FIXED_W, G.NTT_MM_MONT_PRODUCT_W):
        with pytest.raises(G.NttError) as e:
            G.ntt_modmul_vec(W.P1, kind, 8, x, x, None, x)
        assert e.value.status == 1


@pytest.mark.parametrize("p", P64)
@pytest.mark.parametrize("kind", KINDS64 + [G.NTT_MM_FMA])
def test_modmul_u64(p, kind):
    if kind == G.NTT_MM_FMA and p >= (1 << 50):
        pytest.skip("Function 16 needs m <= 50 (Proposition 13)")
    x, y = _operands(p, 1 << 16 if kind >= G.NTT_MM_ADD else 1 << 18, p ^ (kind + 7))
    assert (_run(p, kind, 8, x, y) == _want(p, kind, x, y)).all()


@pytest.mark.parametrize("p", [17, 257, 7681])
@pytest.mark.parametrize("kind", KINDS32)
def test_modmul_exhaustive_small_primes(p, kind):
    if kind in (G.NTT_MM_ADD, G.NTT_MM_SUB) and p > 257:
        pytest.skip("sums and differences: exhaustive on the smaller primes")
    x = np.repeat(np.arange(p, dtype=np.uint64), p)
    y = np.tile(np.arange(p, dtype=np.uint64), p)
    want = _want(p, kind, x, y)
    assert (_run(p, kind, 4, x, y) == want).all()
    if kind in KINDS64:
        assert (_run(p, kind, 8, x, y) == want).all()
