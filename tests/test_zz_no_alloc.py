"""gr_repair_packed_noalloc: the batched repair for callers that cannot
allocate device memory where they run it (allocation-free host paths,
plug-ins whose host forbids allocation after start-up, real-time loops that
must not pay cudaMalloc's implicit synchronisation).  Its scratch is a fixed
64 MiB device array inside the library.  The test calls it through the C ABI
twice in a row and compares every result with gr_repair_packed, which takes a
caller-provided scratch buffer; both are exact integer computations, so the
comparison is bit-exact.  It also checks the capacity error.  Collected last
so that a failure here stops a -x run only after every other test."""
import ctypes as C

import numpy as np
import pytest

from paper_2011_08373_gb300 import synth

pytestmark = pytest.mark.gpu

KEYS = ("status", "mask", "weight", "added", "removed", "iters", "n_clauses", "clauses", "traj",
        "forbidden", "access_pairs")


@pytest.fixture(scope="module")
def env():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2011_08373_gb300.build import build
    from paper_2011_08373_gb300 import binding

    build()
    binding.lib()
    return torch, binding


def _results(torch, binding, out, off, n):
    torch.cuda.synchronize()
    raw = out[off:off + n * binding.RESULT_DTYPE.itemsize].cpu().numpy()
    return raw.view(binding.RESULT_DTYPE).copy()


def test_noalloc_matches_packed_twice(env):
    torch, binding = env
    L = binding.lib()
    progs = synth.generate("batch1024_4x256_s24", 192) + synth.generate("uneven4096_mixed", 96)
    ref = binding.DeviceBatch(progs)
    ref.run()
    want = ref.results_raw()
    n = len(progs)
    out = torch.empty(n * binding.RESULT_DTYPE.itemsize + 256, dtype=torch.uint8, device="cuda")
    off = (-out.data_ptr()) % 256
    opts = binding._options(True, 64)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        out.fill_(0xAB)  # stale output must not survive a call
        rc = L.gr_repair_packed_noalloc(C.c_void_p(ref._arena_ptr), n, C.byref(opts),
                                        C.c_void_p(out.data_ptr() + off), C.c_void_p(stream))
        assert rc == binding.OK, binding.last_error()
        got = _results(torch, binding, out, off, n)
        for k in KEYS:
            assert np.array_equal(got[k], want[k]), (call, k)


def test_noalloc_rejects_batch_beyond_its_scratch(env):
    torch, binding = env
    L = binding.lib()
    big = synth.generate("large_128x1024_s24", 11)  # about 69 MB of traces
    host, scratch_bytes = binding.pack(big)
    assert scratch_bytes > 64 << 20
    arena = torch.empty(host.nbytes + 256, dtype=torch.uint8, device="cuda")
    off = (-arena.data_ptr()) % 256
    arena[off:off + host.nbytes].copy_(torch.from_numpy(host))
    out = torch.empty(len(big) * binding.RESULT_DTYPE.itemsize + 256, dtype=torch.uint8, device="cuda")
    oo = (-out.data_ptr()) % 256
    rc = L.gr_repair_packed_noalloc(C.c_void_p(arena.data_ptr() + off), len(big), None,
                                    C.c_void_p(out.data_ptr() + oo),
                                    C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == binding.ECAPACITY
    assert "scratch" in binding.last_error()
