"""Host logic of workflow.BatchAdvancer on CPU, with stand-ins for the two
GPU paths: chunking, the move of a replica that leaves the crystal runner's
range (its state restored from before the chunk, the chunk rerun on the
multi-kernel path, later chunks there, alongside the crystal runner for the
others), and the gather/scatter of uneven replicas.  The stand-in runner keeps
the runner's contract: a replica that raises an error keeps its state of the
chunk's first step."""
import types

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2201_04622_gb300 import ne  # noqa: E402
from paper_2201_04622_gb300 import workflow as WF  # noqa: E402


def test_advancer_moves_a_failing_replica_and_keeps_the_others(monkeypatch):
    offs = [0, 4, 10, 15]                  # three replicas of 4, 6 and 5 atoms
    mds = [types.SimpleNamespace(replica=r) for r in range(3)]
    crystals = [("c", r) for r in range(3)]
    x0 = torch.tensor(np.random.default_rng(1).normal(size=(15, 3)), dtype=torch.float64)
    x, v = x0.clone(), torch.zeros_like(x0)
    W = torch.zeros((3, 2), dtype=torch.float64)
    calls, last = [], {}

    def rows(o, q):
        return slice(o[q], o[q + 1])

    def crystal(ctx, batch, crs, xs, vs, Ws, s0, ns, stream=None):
        md = batch.mds
        assert crs is None
        ids = [m.replica for m in md]
        calls.append(("crystal", ids, s0, ns))
        last["ids"] = ids
        o = [0]
        for m in md:
            o.append(o[-1] + offs[m.replica + 1] - offs[m.replica])
        fail = s0 == 20 and 1 in ids       # replica 1 leaves the range in the third chunk
        for q, m in enumerate(md):
            if fail and m.replica == 1:
                continue                   # a replica that failed is not written back
            xs[rows(o, q)] += ns * 1e-3 * (m.replica + 1)
            Ws[q, 0] += ns * (m.replica + 1)
        if fail:
            raise ne.NeError(ne.NE_ERANGE, "ne_crystal_run_segment", "stand-in")

    def general(ctx, md, o, xs, vs, x0s, boxes, Ws, s0, ns, stream=None):
        calls.append(("general", [m.replica for m in md], s0, ns))
        for q, m in enumerate(md):
            xs[rows(o, q)] += ns * 2e-3 * (m.replica + 1)
            Ws[q, 1] += ns * (m.replica + 1)

    def status(ctx, n):
        return np.array([ne.NE_ERANGE if r == 1 else ne.NE_OK for r in last["ids"]][:n], dtype=np.int32)

    monkeypatch.setattr(ne, "CrystalBatch", lambda mds, crs: types.SimpleNamespace(mds=mds))
    monkeypatch.setattr(ne, "ne_crystal_run_segment", crystal)
    monkeypatch.setattr(ne, "ne_switch_run_segment", general)
    monkeypatch.setattr(ne, "ne_ctx_replica_status", status)
    monkeypatch.setattr(ne, "ne_ctx_clone", lambda ctx, n, r: "ctx2")
    monkeypatch.setattr(ne, "ne_ctx_destroy", lambda ctx: None)

    adv = WF.BatchAdvancer("ctx", mds, crystals, offs, [None] * 3, x0, chunk=10)
    with pytest.warns(UserWarning):
        adv.advance(x, v, W, 0, 40)
    adv.close()
    assert adv.moved == [1]
    assert [c for c in calls if c[0] == "crystal"] == [
        ("crystal", [0, 1, 2], 0, 10), ("crystal", [0, 1, 2], 10, 10), ("crystal", [0, 1, 2], 20, 10),
        ("crystal", [0, 2], 30, 10)]
    assert sorted(c for c in calls if c[0] == "general") == [("general", [1], 20, 10), ("general", [1], 30, 10)]
    # replicas 0 and 2: 40 crystal steps; replica 1: 20 crystal steps, then 20 on the other path
    for r, (nc, ng) in enumerate([(40, 0), (20, 20), (40, 0)]):
        want = x0[offs[r]:offs[r + 1]] + nc * 1e-3 * (r + 1) + ng * 2e-3 * (r + 1)
        assert torch.allclose(x[offs[r]:offs[r + 1]], want, rtol=0, atol=1e-12)
        assert float(W[r, 0]) == nc * (r + 1) and float(W[r, 1]) == ng * (r + 1)


def test_transition_temperatures_locate_every_crossing():
    """Sec. IV: the temperature where G_a(T) = G_b(T), and which phase wins above it."""
    from paper_2201_04622_gb300.workflow import transition_temperatures as tt
    T = np.arange(100.0, 1001.0, 10.0)
    # straight lines crossing at 487 K, b stable below and a above: found to rounding
    got = tt(T, -1e-4 * T, -1e-4 * T + 2e-7 * (T - 487.0))
    assert len(got) == 1 and abs(got[0][0] - 487.0) < 1e-9 and got[0][1] == 0
    # three crossings of a sine, alternating winners, each within the grid's interpolation error
    got = tt(T, 0 * T, 1e-3 * np.sin(T / 100.0))
    want = [100 * np.pi, 200 * np.pi, 300 * np.pi]
    assert [g[1] for g in got] == [1, 0, 1]
    assert np.allclose([g[0] for g in got], want, atol=0.1)
    # exact zeros on the grid count once; a touch without a sign change counts not at all
    assert tt([1.0, 2.0, 3.0, 4.0], [1, 0, 0, -1], [0, 0, 0, 0]) == [(2.5, 0)]
    assert tt([1.0, 2.0, 3.0], [1, 0, 1], [0, 0, 0]) == []
    assert tt([1.0, 2.0], [0, 0], [0, 0]) == []
    with pytest.raises(ValueError):
        tt([2.0, 1.0], [0, 1], [1, 0])
