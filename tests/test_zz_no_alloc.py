"""polymul_mod_p_batch_static: the product entry point that allocates nothing.

It exists for callers that cannot allocate device memory when they need a
product: hosts that own all device memory through their own allocator or a
fixed budget, and latency-critical loops that cannot take an allocation's
implicit synchronisation.  It must give exactly what polymul_mod_p_batch
gives with a caller-allocated workspace, on two calls in a row, and a call
after the first must leave the device's free memory unchanged.  This file is
collected last so a failure here cannot hide failures elsewhere; it also
passes when run alone in a fresh process (the first call performs the
one-time scratch set-up)."""
import numpy as np
import pytest

import paper_1407_3383_gb300 as G
from paper_1407_3383_gb300 import workloads as W
from helpers import empty_dev, from_dev, to_dev

pytestmark = pytest.mark.gpu


def _inputs(p, batch, na, nb, seed):
    g = W.SplitMix64(seed)
    return (g.uniform_mod(p, batch * na).reshape(batch, na),
            g.uniform_mod(p, batch * nb).reshape(batch, nb))


@pytest.mark.parametrize("p,log2n,na,nb,batch", [
    (W.P_B, 16, 1 << 15, 1 << 15, 8),     # two-pass transforms: uses the fixed scratch
    (W.P1, 15, 9000, 7000, 4),            # 64-bit words, ragged lengths
    (W.P_A, 12, 2048, 2048, 3),           # one-block transforms: no scratch needed
])
def test_static_scratch_matches_workspace_entry(p, log2n, na, nb, batch):
    import torch
    with G.Plan(p, log2n) as plan:
        wb = plan.word_bytes
        ws = G.alloc_workspace(plan, batch)
        for call in range(2):                       # two calls in a row
            a, b = _inputs(p, batch, na, nb, seed=1000 * call + log2n)
            da, db = to_dev(a.reshape(-1), wb), to_dev(b.reshape(-1), wb)
            c_ref = empty_dev(batch * (na + nb - 1), wb)
            c_static = empty_dev(batch * (na + nb - 1), wb)
            G.polymul_mod_p_batch(plan, da, na, db, nb, batch, c_ref, G.NTT_SCHED_FUSED, ws)
            torch.cuda.synchronize()
            free_before = torch.cuda.mem_get_info()[0]
            G.polymul_mod_p_batch_static(plan, da, na, db, nb, batch, c_static)
            torch.cuda.synchronize()
            if call:                                # after the first call's set-up
                assert torch.cuda.mem_get_info()[0] == free_before, "the call allocated device memory"
            ref = from_dev(c_ref)
            got = from_dev(c_static)
            assert (got == ref).all(), f"call {call}"


def test_static_scratch_rejects_oversized_batches():
    import torch
    with G.Plan(W.P_B, 16) as plan:
        # 2 * 2^16 * 4 bytes per product: 65 products exceed the 32 MiB array
        a = torch.zeros(65 << 15, dtype=torch.uint32, device="cuda")
        c = torch.zeros(65 * ((1 << 16) - 1), dtype=torch.uint32, device="cuda")
        with pytest.raises(G.NttError) as e:
            G.polymul_mod_p_batch_static(plan, a, 1 << 15, a, 1 << 15, 65, c)
        assert e.value.status == 10
        assert "scratch" in str(e.value)
