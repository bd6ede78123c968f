"""Window-averaged measurement on the GPU against the oracle (bit-exact integer sums).

Every sweep tau inside window m (bounds[m] <= tau < bounds[m+1]) is measured and added into
window m; the oracle measures the same taus one by one (a point schedule holding every tau) and
the test sums them.  Geometric windows with ratio 2^(1/4) (VB, main text) and tritone lumps (SK,
SI section 1); the point schedule runs beside the windows unchanged.
"""
import numpy as np
import pytest

import oracle
import sg_inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

sg = None


@pytest.fixture(scope="module", autouse=True)
def _lib():
    global sg
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1906_11195_gb300 import _build
    _build.build()
    import paper_1906_11195_gb300 as m
    sg = m


def window_sums(bounds, tw, taus, C, q, E):
    """Sum oracle point values (columns = taus) into the windows; counts as the library's."""
    nb = len(bounds) - 1
    Cs = np.zeros(C.shape[:-1] + (nb,), dtype=np.int64)
    qs = np.zeros(q.shape[:-1] + (nb,), dtype=np.int64)
    Es = np.zeros(E.shape[:-1] + (nb,), dtype=np.int64)
    n = np.zeros((len(tw) + 1, nb), dtype=np.int64)
    for u, t in enumerate(taus):
        m = np.searchsorted(bounds, t, side="right") - 1
        if m < 0 or m >= nb:
            continue
        Cs[..., m] += C[..., u]
        qs[..., m] += q[..., u]
        Es[..., m] += E[..., u]
        for w, t0 in enumerate(tw):
            n[w, m] += t >= t0
        n[-1, m] += 1
    return Cs, qs, Es, n


@pytest.mark.parametrize("kernel,L", [("packed", 64), ("plain", 8)])
def test_vb_geometric_windows_match_oracle(kernel, L):
    rp, col, eid = sg_inputs.poisson_graph(3000, 4.0, 31)
    jb = sg_inputs.vb_lane_couplings(eid, eid.max() + 1, 31)
    g = dict(row_ptr=rp, col=col, jbits=jb, seed=9, temps=[1.0, 0.6])
    tw, tm = np.array([0, 4, 16], dtype=np.int64), np.array([0, 8, 64], dtype=np.int64)
    bounds = sg_inputs.geometric_windows(2, 150)
    sweeps = int(bounds[-1]) + 5  # past the last window: later sweeps add nothing
    k = sg.SG_VB_PACKED if kernel == "packed" else sg.SG_VB_PLAIN
    run = sg.VBRun([g], n_lanes=L, n_replicas=2, kernel=k, tw=tw, tm=tm, windows=bounds)
    run.sweep(sweeps)
    run.synchronize()
    C, q, E, n = run.windows()
    Cp, qp, Ep = run.results()
    run.close()
    taus = np.arange(0, sweeps + 1, dtype=np.int64)
    ref = oracle.vb_run(rp, col, jb, L, g["temps"], g["seed"], sweeps, tw, taus)
    Cs, qs, Es, ns = window_sums(bounds, tw, taus, ref["C"], ref["q"], ref["E"])
    assert np.array_equal(n, ns)
    assert np.array_equal(C[0][:, :L], Cs[:, :L]) and np.array_equal(E[0][:, :L], Es[:, :L])
    assert np.array_equal(q[0][:, :L], qs[:, :L])
    # the point schedule is untouched by the windows
    pts = [int(np.flatnonzero(taus == t)[0]) for t in tm]
    assert np.array_equal(Cp[0][:, :L], ref["C"][:, :L][..., pts])


def test_vb_windows_partial_and_resumed():
    """Reading mid-window counts only the sweeps done; a checkpoint taken mid-window resumes
    with the window sums intact."""
    rp, col, eid = sg_inputs.poisson_graph(2000, 4.0, 8)
    jb = sg_inputs.vb_lane_couplings(eid, eid.max() + 1, 8)
    g = dict(row_ptr=rp, col=col, jbits=jb, seed=4, temps=[0.8, 0.8])
    tw, tm = np.array([0, 3], dtype=np.int64), np.array([10], dtype=np.int64)
    bounds = sg_inputs.geometric_windows(1, 90)
    straight = sg.VBRun([g], 64, 2, sg.SG_VB_PACKED, tw=tw, tm=tm, windows=bounds)
    straight.sweep(37)
    C37, _, _, n37 = straight.windows()
    straight.sweep(60)
    want = straight.windows()
    straight.close()
    taus = np.arange(0, 98, dtype=np.int64)
    ref = oracle.vb_run(rp, col, jb, 64, g["temps"], g["seed"], 97, tw, taus)
    Cs, _, _, ns = window_sums(bounds, tw, taus[:38], ref["C"][..., :38], ref["q"][..., :38],
                               ref["E"][..., :38])
    assert np.array_equal(n37, ns) and np.array_equal(C37[0], Cs)
    a = sg.VBRun([g], 64, 2, sg.SG_VB_PACKED, tw=tw, tm=tm, windows=bounds)
    a.sweep(37)
    blob = a.save_state()
    a.close()
    b = sg.VBRun([g], 64, 2, sg.SG_VB_PACKED, tw=tw, tm=tm, windows=bounds)
    b.load_state(blob)
    b.sweep(60)
    got = b.windows()
    b.close()
    for x, y in zip(got, want):
        assert np.array_equal(x, y)


def test_sk_tritone_lumps_match_oracle():
    n, R = 320, 16
    J = sg_inputs.sk_couplings(n, 17)
    temps = [0.4] * 8 + [0.7] * 8
    tw, tm = np.array([0, 4], dtype=np.int64), np.array([4, 32], dtype=np.int64)
    bounds = sg_inputs.tritone_windows(60)
    sweeps = int(bounds[-1])
    run = sg.SKRun(J, temps, 12, kernel=sg.SG_SK_BLOCKED, block=64, tw=tw, tm=tm, windows=bounds)
    run.sweep(sweeps)
    run.synchronize()
    C, q, E, nn = run.windows()
    run.close()
    taus = np.arange(0, sweeps + 1, dtype=np.int64)
    ref = oracle.sk_run(J, temps, 12, sweeps, tw, taus)
    Cs, qs, Es, ns = window_sums(bounds, tw, taus, ref["C"], ref["q"], ref["E"])
    assert np.array_equal(nn, ns)
    assert np.array_equal(C[0, :, 0], Cs) and np.array_equal(E[0, :, 0], Es)
    assert np.array_equal(q[0, :, 0], qs)


def test_sk_batch_windows_match_oracle():
    sizes = [200, 333]
    R = 16
    samples = [dict(J=sg_inputs.sk_couplings(nn, 70 + k), seed=3 + k, temps=[0.5] * R)
               for k, nn in enumerate(sizes)]
    tw = np.array([0, 2], dtype=np.int64)
    bounds = sg_inputs.tritone_windows(40)
    sweeps = int(bounds[-1])
    run = sg.SKBatchRun(samples, R, kernel=sg.SG_SK_BLOCKED, block=0, tw=tw, tm=[5],
                        windows=bounds)
    run.sweep(sweeps)
    C, q, E, nn = run.windows()
    run.close()
    taus = np.arange(0, sweeps + 1, dtype=np.int64)
    for b, x in enumerate(samples):
        ref = oracle.sk_run(x["J"], x["temps"], x["seed"], sweeps, tw, taus)
        Cs, qs, Es, ns = window_sums(bounds, tw, taus, ref["C"], ref["q"], ref["E"])
        assert np.array_equal(nn, ns)
        assert np.array_equal(C[b, :, 0], Cs) and np.array_equal(E[b, :, 0], Es)
        assert np.array_equal(q[b, :, 0], qs)
