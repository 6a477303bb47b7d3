"""The repair server: continuous batching keeps every result identical to the
same program repaired alone, for requests of uneven sizes and both modes
arriving while others run; its capacity and ticket errors are reported."""
import time

import pytest

import oracle
from paper_2011_08373_gb300 import synth

pytestmark = pytest.mark.gpu

KEYS = ("status", "mask", "weight", "added", "removed", "iters", "traj", "clauses", "forbidden",
        "access_pairs")


@pytest.fixture(scope="module")
def gb():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2011_08373_gb300.build import build
    from paper_2011_08373_gb300 import binding

    build()
    binding.lib()
    return binding


def _mix(n_small, n_large):
    progs = synth.generate("uneven4096_mixed", n_small, start=5000)
    progs += synth.generate("large_128x1024_s24", n_large)
    # interleave the large ones
    out = []
    step = max(1, len(progs) // max(1, n_large))
    small, large = progs[:n_small], progs[n_small:]
    for i, p in enumerate(small):
        out.append(p)
        if large and i % step == step // 2:
            out.append(large.pop())
    return out + large


def test_results_same_alone_and_in_the_mix(gb):
    progs = _mix(300, 3)
    alone = [gb.repair(p) for p in progs]  # each program repaired on its own
    gaps = synth.poisson_arrivals(4000.0, len(progs), seed=7)
    with gb.Server(mem_budget_bytes=1 << 30, n_slots=3) as srv:
        tickets = []
        t0 = time.perf_counter()
        for p, t in zip(progs, gaps):
            while time.perf_counter() - t0 < t:
                pass
            tickets.append(srv.submit(p))
        assert srv.drain(120000)
        got = {}
        for tk in tickets:
            r = srv.poll(tk)
            assert r is not None
            got[tk] = r
        assert srv.stats()["launches"] > 1  # work arrived while other launches ran
    for p, tk, want in zip(progs, tickets, alone):
        res, lat = got[tk]
        assert lat > 0
        for k in KEYS:
            assert res[k] == want[k], k


def test_small_programs_match_oracle_through_server(gb):
    progs = synth.generate("uneven4096_mixed", 300, start=9000)
    progs = [p for p in progs if p.blocks * p.threads <= 600][:20]
    with gb.Server(mem_budget_bytes=256 << 20, n_slots=2) as srv:
        tickets = [srv.submit(p) for p in progs]
        assert srv.drain(60000)
        for p, tk in zip(progs, tickets):
            res, _ = srv.poll(tk)
            want = oracle.repair(p)
            for k in KEYS:
                assert res[k] == want[k], k


def test_server_rejects_oversized_and_unknown(gb):
    # 4 statements x 2,048 blocks x 1,024 threads: 16 MiB of traces, more than
    # an 8 MiB slot
    big = synth.make_program([{"op": "W"}, {"op": "R", "b": 1}, {"op": "W", "b": 2}, {"op": "R"}],
                             blocks=2048, threads=1024, m_shared=4096)
    with gb.Server(mem_budget_bytes=16 << 20, n_slots=2) as srv:
        with pytest.raises(gb.GrError) as e:
            srv.submit(big)
        assert e.value.code == gb.ECAPACITY
        with pytest.raises(gb.GrError):
            srv.poll(12345)


def test_wide_lane_requests_match_oracle(gb):
    """Programs with many blocks that differ take the server's wide lane;
    interleaved with small ones, every result equals the oracle's."""
    wide = synth.generate("interblock256_64x256_s16", 6, blocks=40, threads=16, m_words=2048)
    for p in wide:  # one statement's block offset differs: blocks see different patterns
        p.c[0] = p.c[0] + 1
    small = [p for p in synth.generate("uneven4096_mixed", 200, start=500) if p.blocks * p.threads <= 400][:12]
    progs = [x for pair in zip(small, wide) for x in pair] + small[len(wide):]
    with gb.Server(mem_budget_bytes=512 << 20, n_slots=3) as srv:
        tickets = [srv.submit(p) for p in progs]
        assert srv.drain(60000)
        for p, tk in zip(progs, tickets):
            res, _ = srv.poll(tk)
            want = oracle.repair(p)
            for k in KEYS:
                assert res[k] == want[k], (p.blocks, k)
