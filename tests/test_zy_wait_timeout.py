"""The timeout path of the bounded device waits, without a GPU fault.  Colour kernel (VB): with the waits
shortened to nothing (SG_TEST_STAGE_WAIT_NS=0), a consumer gives up on the first stage that has
not landed yet, the kernel drains its copies in flight (with the normal bound), flags the
handle's status word and exits; sg_synchronize then reports SG_ETIMEOUT and the context stays
usable: a fresh handle afterwards runs and matches the oracle."""
import numpy as np
import pytest

import oracle
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


@pytest.mark.parametrize("fused", ["0", "1"])
def test_shortened_waits_report_timeout_and_leave_the_context_usable(sg, monkeypatch, fused):
    rp, col, eid = sg_inputs.poisson_graph(200_000, 4.0, 3)
    jb = sg_inputs.vb_lane_couplings(eid, eid.max() + 1, 3)
    g = dict(row_ptr=rp, col=col, jbits=jb, seed=2, temps=[1.0, 1.0])
    monkeypatch.setenv("SG_VB_COLOUR_VARIANT", "1")  # pinned: no autotuner sweeps at attach
    monkeypatch.setenv("SG_VB_FUSED", fused)
    monkeypatch.setenv("SG_TEST_STAGE_WAIT_NS", "0")
    run = sg.VBRun([g], 64, 2, sg.SG_VB_PACKED)
    run.sweep(2)
    with pytest.raises(sg.SGError) as e:
        run.synchronize()
    assert e.value.code == sg.SG_ETIMEOUT
    run.close()
    monkeypatch.delenv("SG_TEST_STAGE_WAIT_NS")
    tw, tm = np.array([0], dtype=np.int64), np.array([0, 3], dtype=np.int64)
    ok = sg.VBRun([g], 4, 2, sg.SG_VB_PACKED, tw=tw, tm=tm)
    ok.sweep(3)
    ok.synchronize()
    C, q, E = ok.results()
    ok.close()
    ref = oracle.vb_run(rp, col, jb, 4, g["temps"], g["seed"], 3, tw, tm)
    assert np.array_equal(C[0][:, :4], ref["C"]) and np.array_equal(E[0][:, :4], ref["E"])


@pytest.mark.parametrize("block", [64, 128, 512])
def test_sk_shortened_waits_report_timeout_and_leave_the_context_usable(sg, monkeypatch, block):
    """The same for the SK sweep: with every bounded wait of a sweep shortened to one test, the
    field kernel (and the in-block kernel, when its coupling copy has not landed) gives up, waits
    for its copies and tensor-core work in flight with the normal bound, frees its tensor memory,
    flags the status word and exits; sg_synchronize reports SG_ETIMEOUT, and a fresh handle
    afterwards matches the oracle."""
    n, R = 1024, 32
    J = sg_inputs.sk_couplings(n, 5)
    temps = [0.4] * R
    monkeypatch.setenv("SG_TEST_STAGE_WAIT_NS", "0")
    run = sg.SKRun(J, temps, 3, kernel=sg.SG_SK_BLOCKED, block=block)
    run.sweep(2)
    with pytest.raises(sg.SGError) as e:
        run.synchronize()
    assert e.value.code == sg.SG_ETIMEOUT
    run.close()
    monkeypatch.delenv("SG_TEST_STAGE_WAIT_NS")
    tw, tm = [0], [0, 3]
    ok = sg.SKRun(J, temps, 3, kernel=sg.SG_SK_BLOCKED, block=block, tw=tw, tm=tm)
    ok.sweep(3)
    ok.synchronize()
    C, q, E = ok.results()
    spins = ok.spins()
    ok.close()
    ref = oracle.sk_run(J, temps, 3, 3, tw, tm)
    assert np.array_equal(spins, ref["spins"])
    assert np.array_equal(C[0, :, 0], ref["C"]) and np.array_equal(E[0, :, 0], ref["E"])
