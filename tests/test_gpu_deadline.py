"""The loop's time limit (gr_options.deadline_us): the paper runs every kernel
under a per-kernel timeout (Section 5, experimental setup); a program whose
loop runs past it stops with GR_TIMEOUT after a Solve, before checking the
next proposal.  Against the oracle, which has no deadline: a timed-out
program's checked masks are a prefix of the oracle's trajectory, every other
program's result is the oracle's, and a deadline nothing reaches changes
nothing."""
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


@pytest.fixture(scope="module")
def batch():
    progs = synth.generate("batch1024_4x256_s24", 48, blocks=2, threads=64, m_words=256)
    # uneven programs small enough for the oracle's all-pairs enumeration
    progs += [p for p in synth.generate("uneven4096_mixed", 200) if p.blocks * p.threads <= 1024][:48]
    return progs, oracle.repair_batch(progs, n_threads=8)


def _timed_out_is_prefix(gb, got, want):
    n_to = 0
    for g, w in zip(got, want):
        if g["status"] == gb.TIMEOUT:
            n_to += 1
            assert g["mask"] == 0 and g["weight"] == 0 and g["removed"] == 0
            # it stopped with a next proposal in hand, which the oracle checks
            assert 1 <= g["iters"] < w["iters"]
            assert g["traj"] == w["traj"][:g["iters"]]
        else:
            for k in KEYS:
                assert g[k] == w[k], (k, g[k], w[k])
    return n_to


def test_one_microsecond_deadline_batch(gb, batch):
    progs, want = batch
    for strategy in (0, 1):
        w = want if strategy == 0 else oracle.repair_batch(progs, n_threads=8, strategy=1)
        got = gb.repair_batch(progs, deadline_us=1, strategy=strategy)
        n_to = _timed_out_is_prefix(gb, got, w)
        # every program whose loop continues past its first Solve times out there
        assert n_to == sum(1 for r in w if r["iters"] >= 2) > 0


def test_one_microsecond_deadline_plain_and_wide(gb, batch):
    import numpy as np
    import torch

    progs, want = batch
    sub = progs[:12]
    got = [gb.repair_plain(p, deadline_us=1) for p in sub]
    assert _timed_out_is_prefix(gb, got, want[:12]) > 0
    db = gb.DeviceBatch(sub, deadline_us=1)
    db.run_wide()
    torch.cuda.synchronize()
    assert _timed_out_is_prefix(gb, db.results(), want[:12]) > 0
    assert np.all(db.results_raw()["status"] <= gb.TIMEOUT)


def test_unreached_deadline_changes_nothing(gb, batch):
    progs, want = batch
    for g, w in zip(gb.repair_batch(progs, deadline_us=10 ** 9), want):
        for k in KEYS:
            assert g[k] == w[k], (k, g[k], w[k])
