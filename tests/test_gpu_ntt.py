"""GPU parity of ntt_forward / ntt_inverse with the oracle's transform by
definition (Section 5.1: position i holds A(w^[i])), bit for bit.

Small sizes are compared in full against the quadratic oracle DFT; larger
sizes (including the two-pass global schedule) on sampled outputs, each
evaluated by Horner's rule at w^[i], plus inverse(forward(a)) = a."""
import numpy as np
import pytest

import oracle as O
import paper_1407_3383_gb300 as G
from paper_1407_3383_gb300 import workloads as W
from helpers import bitrev, from_dev, to_dev

pytestmark = pytest.mark.gpu

PRIMES32 = [W.P_A, W.P_B]
PRIMES64 = [W.P1, W.P3]


def _roundtrip(plan, a, batch):
    import torch
    d = to_dev(a, plan.word_bytes)
    G.ntt_forward(plan, d, batch)
    torch.cuda.synchronize()
    fwd = from_dev(d)
    G.ntt_inverse(plan, d, batch)
    torch.cuda.synchronize()
    return fwd, from_dev(d)


@pytest.mark.parametrize("p", PRIMES32 + PRIMES64)
@pytest.mark.parametrize("log2n", [1, 2, 3, 4, 5, 7, 8, 9, 10])
def test_forward_matches_dft_small(p, log2n):
    n = 1 << log2n
    batch = 3 if log2n > 8 else 37          # ragged number of vectors per block
    a = W.SplitMix64(p + log2n).uniform_mod(p, batch * n)
    with G.Plan(p, log2n) as plan:
        assert plan.omega == O.root_of_unity(p, log2n)
        fwd, back = _roundtrip(plan, a, batch)
    for v in range(batch):
        want = O.dft(p, O.root_of_unity(p, log2n), a[v * n:(v + 1) * n])
        assert (fwd[v * n:(v + 1) * n] == want).all(), f"vector {v}"
    assert (back == a).all()


def _check_sampled(p, log2n, a, fwd, batch, samples=48, seed=1):
    n = 1 << log2n
    w = O.root_of_unity(p, log2n)
    g = W.SplitMix64(seed)
    idx = (g.u64(samples) % np.uint64(n)).astype(np.int64)
    vec = (g.u64(samples) % np.uint64(batch)).astype(np.int64)
    idx = np.concatenate([idx, [0, 1, n - 1, n // 2]])
    vec = np.concatenate([vec, [0, batch - 1, batch - 1, 0]])
    for v, i in zip(vec, idx):
        x = pow(w, bitrev(int(i), log2n), p)
        want = O.eval_poly(p, a[v * n:(v + 1) * n], x)
        assert int(fwd[v * n + i]) == want, (v, i)


@pytest.mark.parametrize("p,log2n,batch", [
    (W.P_A, 12, 2), (W.P_B, 13, 2), (W.P_B, 14, 2),      # one block per transform (u32)
    (W.P_A, 15, 2), (W.P_B, 16, 3), (W.P_A, 18, 1),      # two global passes (u32)
    (W.P1, 12, 2), (W.P3, 13, 2),                         # one block (u64)
    (W.P1, 14, 2), (W.P2, 17, 1), (W.P1, 20, 1),          # two global passes (u64)
    (W.P3, 16, 3),                                        # direct 256 x 256 kernels (u64)
    (W.P_B, 17, 2), (W.P_A, 19, 1), (W.P3, 18, 2),        # pass across 2^16-point rows + direct kernels
    (W.P_B, 21, 1), (W.P2, 22, 1), (W.P_A, 23, 1),        # column kernel across 32..128 rows
])
def test_forward_sampled_and_roundtrip(p, log2n, batch):
    n = 1 << log2n
    a = W.SplitMix64(p ^ log2n).uniform_mod(p, batch * n)
    with G.Plan(p, log2n) as plan:
        fwd, back = _roundtrip(plan, a, batch)
    _check_sampled(p, log2n, a, fwd, batch)
    assert (back == a).all()


def test_special_inputs_large():
    """delta -> all ones; constant c -> (n c, 0, ..., 0) at every size regime."""
    for p, log2n in [(W.P_B, 16), (W.P1, 15), (W.P_A, 11)]:
        n = 1 << log2n
        a = np.zeros(2 * n, dtype=np.uint64)
        a[0] = 1
        a[n:] = 77
        with G.Plan(p, log2n) as plan:
            fwd, back = _roundtrip(plan, a, 2)
        assert (fwd[:n] == 1).all()
        assert int(fwd[n]) == n * 77 % p and (fwd[n + 1:] == 0).all()
        assert (back == a).all()


@pytest.mark.parametrize("p", [W.P_B, W.P1])
def test_convolution_theorem_on_device(p):
    """forward(a * b) = forward(a) . forward(b) pointwise, with the product
    from the oracle and the transforms from the device."""
    log2n = 10
    n = 1 << log2n
    g = W.SplitMix64(p % 1000)
    a = g.uniform_mod(p, n // 2)
    b = g.uniform_mod(p, n // 2)
    c = np.concatenate([O.polymul(p, a, b), np.zeros(1, dtype=np.uint64)])
    pad = lambda v: np.concatenate([v, np.zeros(n - v.size, dtype=np.uint64)])
    with G.Plan(p, log2n) as plan:
        fa, _ = _roundtrip(plan, pad(a), 1)
        fb, _ = _roundtrip(plan, pad(b), 1)
        fc, _ = _roundtrip(plan, c, 1)
    assert (fc == O.mulmod_vec(p, fa, fb)).all()


@pytest.mark.parametrize("p", [W.P_B, W.P2])
def test_2e16_direct_and_unaligned_generic_agree(p):
    """2^16-point transforms of 16-byte-aligned data run the direct kernels;
    data that is only word-aligned takes the generic passes.  Both must give
    the oracle's values and the same words."""
    import torch
    log2n, batch = 16, 2
    n = 1 << log2n
    a = W.SplitMix64(p ^ 0x16).uniform_mod(p, batch * n)
    with G.Plan(p, log2n) as plan:
        G.ntt_tune_reset()
        aligned = to_dev(a, plan.word_bytes)
        G.ntt_forward(plan, aligned, batch)
        buf = to_dev(np.zeros(batch * n + 1, dtype=np.uint64), plan.word_bytes)
        shifted = buf[1:]                                  # one word off a 16-byte boundary
        shifted.copy_(to_dev(a, plan.word_bytes))
        G.ntt_forward(plan, shifted, batch)
        torch.cuda.synchronize()
        f1, f2 = from_dev(aligned), from_dev(shifted)
        assert (f1 == f2).all()
        _check_sampled(p, log2n, a, f1, batch)
        G.ntt_inverse(plan, aligned, batch)
        G.ntt_inverse(plan, shifted, batch)
        torch.cuda.synchronize()
        assert (from_dev(aligned) == a).all() and (from_dev(shifted) == a).all()

