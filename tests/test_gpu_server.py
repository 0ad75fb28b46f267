"""The serving loop: every result is the same when a request runs alone and
when it runs in a mix of concurrently admitted requests (bit for bit), and
matches the oracle; admission waits for arena memory instead of failing."""
import numpy as np
import pytest

import oracle as O
import paper_1407_3383_gb300 as G
from paper_1407_3383_gb300 import workloads as W

pytestmark = pytest.mark.gpu

PRIMES = [W.P1, W.P2, W.P3]


def _requests(count, seed, lo=1 << 9, hi=1 << 17):
    import torch
    g = W.SplitMix64(seed)
    sizes = g.log_uniform_int(lo, hi, count)
    reqs = []
    for t, n in enumerate(sizes):
        n = int(n)
        if t % 5 == 4:                                    # polynomial product mod P_i
            pi = int(g.choice(3, 1)[0])
            a = g.uniform_mod(PRIMES[pi], n)
            b = g.uniform_mod(PRIMES[pi], max(1, n // 2))
            ta = torch.from_numpy(a).pin_memory()
            tb = torch.from_numpy(b).pin_memory()
            tc = torch.zeros(a.size + b.size - 1, dtype=torch.uint64).pin_memory()
            reqs.append((G.NTT_REQ_POLYMUL, pi, a, b, ta, tb, tc))
        else:                                             # integer product
            a = g.limbs(n)
            b = g.limbs(max(1, n - 7))
            ta = torch.from_numpy(a).pin_memory()
            tb = torch.from_numpy(b).pin_memory()
            tc = torch.zeros(a.size + b.size, dtype=torch.uint32).pin_memory()
            reqs.append((G.NTT_REQ_INTMUL, 0, a, b, ta, tb, tc))
    return reqs


def _to_int(limbs):
    return int.from_bytes(np.ascontiguousarray(limbs.astype(np.uint32)).tobytes(), "little")


def _check_oracle(kind, pi, a, b, c):
    if kind == G.NTT_REQ_POLYMUL:
        p = PRIMES[pi]
        if a.size * b.size <= (1 << 24):
            assert (c.astype(np.uint64) == O.polymul(p, a, b)).all()
        else:
            x = 123456789
            assert O.eval_poly(p, c, x) == O.mulmod(O.eval_poly(p, a, x), O.eval_poly(p, b, x), p)
    else:
        if a.size * b.size <= (1 << 24):
            assert (c == O.intmul(a, b)).all()
        else:
            ia, ib, ic = _to_int(a), _to_int(b), _to_int(c)
            for q in [2305843009213693951, 1152921504606846883]:
                assert ic % q == (ia % q) * (ib % q) % q


def test_same_result_alone_and_in_the_mix():
    reqs = _requests(30, 5)
    with G.Server(max_limbs=1 << 17, mem_bytes=2 << 30, slots=4) as srv:
        alone = []
        for kind, pi, a, b, ta, tb, tc in reqs:
            rid = srv.submit(kind, ta, tb, tc, prime=pi)
            srv.wait(rid)
            srv.release(rid)
            alone.append(tc.numpy().copy())
            tc.zero_()
        ids = [srv.submit(kind, ta, tb, tc, prime=pi) for kind, pi, a, b, ta, tb, tc in reqs]
        lat = [srv.wait(rid) for rid in ids]
        stats = srv.stats()
        for rid in ids:
            srv.release(rid)
    assert stats["completed"] == 2 * len(reqs)
    assert stats["peak_inflight"] > 1                      # requests overlapped on the device
    assert all(x > 0 for x in lat)
    for (kind, pi, a, b, ta, tb, tc), one in zip(reqs, alone):
        mix = tc.numpy()
        assert (mix == one).all()
        _check_oracle(kind, pi, a, b, mix)


def test_memory_admission_queues_requests():
    """An arena that holds one large request at a time: everything still
    completes, strictly one request in flight."""
    import torch
    g = W.SplitMix64(9)
    n = 1 << 16
    pairs = [(g.limbs(n), g.limbs(n)) for _ in range(4)]
    ws_probe = G.IntmulPlan(n)
    need = G.intmul_workspace_size(ws_probe, n, n) + 4 * (4 * n) + 4096
    ws_probe.close()
    with G.Server(max_limbs=n, mem_bytes=need + need // 2, slots=4) as srv:
        bufs = [(torch.from_numpy(a).pin_memory(), torch.from_numpy(b).pin_memory(),
                 torch.zeros(2 * n, dtype=torch.uint32).pin_memory()) for a, b in pairs]
        ids = [srv.submit(G.NTT_REQ_INTMUL, ta, tb, tc) for ta, tb, tc in bufs]
        for rid in ids:
            srv.wait(rid)
        assert srv.stats()["peak_inflight"] == 1
        for (a, b), (ta, tb, tc) in zip(pairs, bufs):
            ia, ib, ic = _to_int(a), _to_int(b), _to_int(tc.numpy())
            assert ic % 2305843009213693951 == (ia * ib) % 2305843009213693951


def test_oversized_request_is_rejected():
    import torch
    with G.Server(max_limbs=1 << 10, mem_bytes=64 << 20, slots=2) as srv:
        a = torch.zeros(1 << 12, dtype=torch.uint32).pin_memory()
        c = torch.zeros(1 << 13, dtype=torch.uint32).pin_memory()
        with pytest.raises(G.NttError) as e:
            srv.submit(G.NTT_REQ_INTMUL, a, a, c)
        assert e.value.status == 5


def test_wait_times_out_on_a_pending_request():
    """ntt_server_wait with a time limit shorter than the request returns
    NTT_ERR_TIMEOUT (a host-side wait: nothing on the GPU is made to hang);
    the request still completes correctly afterwards, and a request that is
    not finished cannot be released."""
    import torch
    g = W.SplitMix64(17)
    n = 1 << 21
    bufs = [(torch.from_numpy(g.limbs(n)).pin_memory(), torch.from_numpy(g.limbs(n)).pin_memory(),
             torch.zeros(2 * n, dtype=torch.uint32).pin_memory()) for _ in range(3)]
    with G.Server(max_limbs=n, mem_bytes=4 << 30, slots=1) as srv:
        ids = [srv.submit(G.NTT_REQ_INTMUL, ta, tb, tc) for ta, tb, tc in bufs]
        with pytest.raises(G.NttError) as e:      # the last one queues behind two others
            srv.wait(ids[-1], 0)
        assert e.value.status == 8                # NTT_ERR_TIMEOUT
        with pytest.raises(G.NttError) as e:
            srv.release(ids[-1])
        assert e.value.status == 1                # NTT_ERR_ARG: still pending or running
        for rid in ids:
            srv.wait(rid, 600000)
            srv.release(rid)
    for ta, tb, tc in bufs:
        ia, ib, ic = _to_int(ta.numpy()), _to_int(tb.numpy()), _to_int(tc.numpy())
        assert ic % 2305843009213693951 == (ia * ib) % 2305843009213693951
