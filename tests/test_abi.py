"""The C-ABI library: it loads, exports every symbol include/gbntt.h declares,
and its host-only planning calls agree with the oracle.  CPU only (no call
here launches device work)."""
import ctypes

import numpy as np
import pytest

import oracle as O
import paper_1407_3383_gb300 as G
from paper_1407_3383_gb300 import workloads as W


def test_library_exports_every_declared_symbol():
    lib = G.lib()
    names = G.header_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
    assert lib.ntt_version().startswith(b"gbntt")


def test_status_strings():
    lib = G.lib()
    assert lib.ntt_status_str(0) == b"NTT_OK"
    assert lib.ntt_status_str(4) == b"NTT_ERR_NO_ROOT"
    assert lib.ntt_status_str(999) == b"NTT_ERR_UNKNOWN"


def test_find_prime_matches_oracle():
    for bits, l in [(62, 40), (31, 20), (40, 30), (32, 30)]:
        for i in range(3):
            try:
                want = O.find_prime(bits, l, i)
            except ValueError:
                with pytest.raises(G.NttError):
                    G.ntt_find_prime(bits, l, i)
                continue
            assert G.ntt_find_prime(bits, l, i) == want
    assert [G.ntt_find_prime(62, 40, i) for i in range(3)] == [W.P1, W.P2, W.P3]


@pytest.mark.parametrize("p", [W.P_A, W.P_B, W.P_TABLE11, W.P_TABLE12, W.P1, W.P2, W.P3])
def test_root_of_unity_matches_oracle(p):
    v2 = (p - 1 & -(p - 1)).bit_length() - 1
    for log2n in sorted({1, 4, 12, 16, min(v2, 24), v2}):
        g, w = G.ntt_root_of_unity(p, log2n)
        assert g == O.least_generator(p)
        assert w == O.root_of_unity(p, log2n)
    with pytest.raises(G.NttError) as e:
        G.ntt_root_of_unity(p, v2 + 1)
    assert e.value.status == 4


def test_fixed_companions():
    """psi = floor(2^n y / p) (Function 8) and the Remark 8 companion, checked
    through the identities they must satisfy."""
    for p in [W.P_A, W.P_B, 17]:
        y = W.SplitMix64(p).uniform_mod(p, 200)
        psi = G.ntt_fixed_companion(p, G.NTT_MM_SHOUP, 4, y)
        for yi, si in zip(y.tolist(), psi.tolist()):
            assert si * p <= (yi << 32) < (si + 1) * p
        phi = G.ntt_fixed_companion(p, G.NTT_MM_MONT_FIXED, 4, y)
        for yi, fi in zip(y.tolist(), phi.tolist()):
            wm = (yi << 32) % p
            assert (fi * p - wm) % (1 << 32) == 0      # phi = wm p^-1 (mod 2^32)
    for p in [W.P1, W.P3, 17]:
        y = W.SplitMix64(p).uniform_mod(p, 200)
        psi = G.ntt_fixed_companion(p, G.NTT_MM_SHOUP, 8, y)
        for yi, si in zip(y.tolist(), psi.tolist()):
            assert si * p <= (yi << 64) < (si + 1) * p


@pytest.mark.parametrize("p,log2n,status", [
    (998244355, 10, 3),            # composite
    (998244354, 10, 2),            # even
    (W.P_A, 24, 4),                # 2^24 does not divide p - 1
    ((1 << 62) + 135, 10, 2),      # >= 2^62
    (W.P_A, 0, 1),                 # n = 1 not supported
    (W.P_A, 25, 5),                # beyond the largest plan
    (7, 1, 2),                     # 16 does not divide p - 1
])
def test_plan_create_rejects_bad_arguments(p, log2n, status):
    """Argument errors are found on the host before any device call."""
    h = ctypes.c_void_p()
    rc = G.lib().ntt_plan_create(p, log2n, 0, ctypes.byref(h))
    assert rc == status
    assert not h.value


def test_polymul_rejects_null_plan():
    assert G.lib().polymul_mod_p_batch(None, None, 1, None, 1, 1, None, 0, None, 0, None) == 1
    assert G.lib().polymul_workspace_size(None, 4, 0) == 0
