"""The allocation-free field entry point (sg_sk_fields_noalloc) agrees with the regular path.

Callers that cannot allocate device memory -- a host that fixes the library's memory budget, or
a plugin whose process owns all device allocations -- use sg_sk_fields_noalloc, which keeps its
tensor-core operand images in a fixed static device array instead of a workspace.  Its fields
h = J s must reproduce what the regular handle computes: for every replica, one half of
sum_i s_i h_i equals the energy count that sg_measure reports for the same spins (bit-exact, as
everywhere in this suite), and h equals the exact integer product J s.  Two calls in a row (the
array keeps the previous call's contents) must both agree.  The sizes cover the array's limits
(n = 2048 with 128 replicas fills it), the smallest replica count (16), sizes that are and are
not multiples of the 128-spin tile, and every replica tile width of the field kernel.
This file is collected last on purpose.
"""
import numpy as np
import pytest

import sg_inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1906_11195_gb300 import _build
    _build.build()
    import paper_1906_11195_gb300 as m
    return m


def fields_noalloc(sg, J, spins):
    R, n = spins.shape
    Jd = torch.from_numpy(np.ascontiguousarray(J, dtype=np.int8)).cuda()
    sd = torch.from_numpy(np.ascontiguousarray(spins, dtype=np.int8)).cuda()
    hd = torch.full((R, n), 12345, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    sg.sg_sk_fields_noalloc(Jd.data_ptr(), sd.data_ptr(), n, R, hd.data_ptr(), stream.cuda_stream)
    return hd.cpu().numpy().astype(np.int64)


@pytest.mark.parametrize("n,R", [(1000, 32), (2048, 128), (128, 16), (1500, 64)])
def test_noalloc_fields_match_regular_path_twice(sg, n, R):
    J = sg_inputs.sk_couplings(n, 77 + n)
    temps = [0.4] * R
    run = sg.SKRun(J, temps, 5, kernel=sg.SG_SK_BLOCKED, block=128, tw=[0], tm=[])
    Jl = J.astype(np.int64)
    for step in range(2):  # two calls in a row, on different spin configurations
        if step:
            run.sweep(7)
        spins = run.spins()
        _, _, E = run.measure()
        h = fields_noalloc(sg, J, spins)
        assert np.array_equal(h, spins.astype(np.int64) @ Jl.T)
        half = (spins.astype(np.int64) * h).sum(axis=1) // 2
        assert np.array_equal(half, E[0, :, 0])
    run.close()


def test_noalloc_rejects_sizes_beyond_the_limit(sg):
    t = torch.zeros(16, dtype=torch.int8, device="cuda")
    h = torch.zeros(16, dtype=torch.int32, device="cuda")
    with pytest.raises(sg.SGError) as e:
        sg.sg_sk_fields_noalloc(t.data_ptr(), t.data_ptr(), 4096, 16, h.data_ptr(), 0)
    assert e.value.code == sg.SG_EINVAL and "2048" in str(e.value)
