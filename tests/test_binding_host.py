"""The Python binding's argument checks, without a GPU.

Every device buffer is checked for its length before its device, so the
sizes each wrapper requires can be read on the CPU: a stand-in library
records nothing, a recording _dev collects the minimum sizes each wrapper
asks for, and those are compared with what the C ABI reads and writes.
"""
import ctypes as C
import types

import numpy as np
import pytest
import torch

import oracle as O
from paper_2201_04622_gb300 import ne


def test_dev_checks_the_size_before_the_device():
    t = torch.zeros(5, dtype=torch.float64)
    with pytest.raises(ne.NeError, match="too small"):
        ne._dev(t, 6)
    with pytest.raises(ne.NeError, match="CUDA"):
        ne._dev(t, 5)
    with pytest.raises(ne.NeError, match="CUDA"):
        ne._dev(t)
    with pytest.raises(ne.NeError, match="CUDA"):
        ne._dev(np.zeros(5), 1)
    assert ne._dev(None, 10) is None


@pytest.fixture
def recorded(monkeypatch):
    """Run a wrapper against a stand-in library; return the (numel, required)
    pairs of its device buffers in argument order."""
    def run(fn, *args, **kw):
        calls = []
        monkeypatch.setattr(ne, "_dev", lambda t, n=None: calls.append((None if t is None else t.numel(), n)))
        monkeypatch.setattr(ne, "_stream", lambda s: None)
        fake = types.SimpleNamespace(**{name: (lambda *a: 0) for name in ne.SYMBOLS})
        monkeypatch.setattr(ne, "load", lambda *a, **k: fake)
        fn(*args, **kw)
        return calls
    return run


def _z(*shape):
    return torch.zeros(shape, dtype=torch.float64)


def test_single_replica_runs_require_their_work_and_trace_lengths(recorded):
    md = ne.md_params(t_eq=3, t_s=5)
    n = 10
    rows = (2 * 3 + 2 * 5 - 1) // 4 + 1
    got = recorded(ne.ne_switch_run, None, md, _z(n, 3), _z(n, 3), _z(n, 3), [1.0] * 3, _z(1), _z(1),
                   _z(6), _z(6), _z(rows, 8), 4)
    assert [r for _, r in got] == [3 * n, 3 * n, 3 * n, 1, 1, 6, 6, 8 * rows]
    assert all(numel >= req for numel, req in got)
    got = recorded(ne.ne_rs_run, None, md, 0.5, _z(n, 3), _z(n, 3), _z(n, 3), [1.0] * 3, _z(6), _z(6))
    assert [r for _, r in got] == [3 * n, 3 * n, 3 * n, 6, 6]


def test_trace_rows_match_the_rows_the_oracle_writes():
    """ne_switch_run's trace holds one row every trace_stride steps of the
    2 t_eq + 2 t_s steps; the oracle (an independent implementation of the
    same schedule) fills exactly that many rows."""
    x0, box = O.create_crystal(O.BCC, 2.87, 3, 3, 3)
    for t_eq, t_s, stride in [(3, 5, 4), (0, 7, 7), (2, 4, 1), (5, 6, 3)]:
        m = O.md(T=100.0, h0=O.H0_HARMONIC, k_h0=5.0, k_spring=5.0, t_eq=t_eq, t_s=t_s, seed=2)
        r = O.switch_run(None, np.zeros((3, 2, 2)), m, x0, O.init_velocities(m, len(x0)), x0, box,
                         trace_stride=stride)
        steps = r["trace"][:, 0]
        written = 1 + int(np.count_nonzero(steps[1:]))  # row 0 is step 0
        assert written == ne._trace_rows(ne.md_params(t_eq=t_eq, t_s=t_s), stride)


def test_batched_runs_require_the_atoms_their_offsets_name(recorded):
    mds = [ne.md_params(), ne.md_params()]
    offs, boxes = [0, 16, 40], [[10.0] * 3, [12.0] * 3]
    x = _z(40, 3)
    got = recorded(ne.ne_switch_run_batched, None, mds, offs, x, x, x, boxes, _z(2), _z(2))
    assert [r for _, r in got] == [120, 120, 120, 2, 2]
    got = recorded(ne.ne_switch_run_segment, None, mds, offs, x, x, x, boxes, _z(2, 2), 0, 10)
    assert [r for _, r in got] == [120, 120, 120, 4]
    got = recorded(ne.ne_profile_segment, None, mds, offs, x, x, x, boxes, _z(2, 2), 0, 10)
    assert [r for _, r in got] == [120, 120, 120, 4]
    ctx = C.c_void_p(0x5150)
    ne._CTX_EAM[ctx.value] = (7, 5.3)
    try:
        got = recorded(ne.ne_switch_run_segment_grad, ctx, mds, offs, x, x, x, boxes, _z(2, 2), 0, 10, _z(11),
                       _z(42))
        assert [r for _, r in got] == [120, 120, 120, 4, 11, 42]
    finally:
        ne._CTX_EAM.pop(ctx.value)
    for bad_offs in ([0, 16], [1, 16, 40], [0, 16, 16], [0, 20, 16]):
        with pytest.raises(ne.NeError, match="offsets"):
            recorded(ne.ne_switch_run_segment, None, mds, bad_offs, x, x, x, boxes, _z(2, 2), 0, 10)
    with pytest.raises(ne.NeError, match="box"):
        recorded(ne.ne_switch_run_segment, None, mds, offs, x, x, x, boxes[:1], _z(2, 2), 0, 10)


def test_crystal_runner_requires_the_atoms_of_its_cells(recorded):
    """bcc 2 atoms per cubic cell, fcc and hcp (orthohexagonal cell) 4: the
    same counts as the crystal builder's."""
    crystals = [(ne.NE_BCC, 2.87, 2, 2, 2), (ne.NE_FCC, 3.65, 2, 3, 2), (ne.NE_HCP, 2.58, 2, 3, 2, 1.6)]
    n_atoms = sum(len(ne.ne_create_crystal(c[0], c[1], c[2], c[3], c[4])[0]) for c in crystals)
    assert n_atoms == ne._crystal_atoms(crystals)
    mds = [ne.md_params(t_s=5) for _ in crystals]
    x = _z(n_atoms, 3)
    got = recorded(ne.ne_crystal_run_segment, None, mds, crystals, x, x, _z(3, 2), 0, 10)
    assert [r for _, r in got] == [3 * n_atoms, 3 * n_atoms, 6]
    got = recorded(ne.ne_crystal_run_segment_cum, None, mds, crystals, x, x, _z(3, 2), _z(3 * 2 * 6), 0, 10)
    assert [r for _, r in got] == [3 * n_atoms, 3 * n_atoms, 6, 36]


def test_theta_buffers_require_the_context_knots(recorded):
    ctx = C.c_void_p(0x6160)
    ne._CTX_EAM[ctx.value] = (9, 5.3)
    try:
        for fn in (ne.ne_ctx_set_theta, ne.ne_ctx_get_theta):
            assert recorded(fn, ctx, _z(54)) == [(54, 54)]
        got = recorded(ne.ne_eam_backward, ctx, ne.NE_FP64, _z(4, 3), [9.0] * 3, 1.0, _z(4, 3), _z(54))
        assert [r for _, r in got] == [12, 12, 54]
        got = recorded(ne.ne_eam_backward_acc, ctx, ne.NE_FP64, _z(4, 3), [9.0] * 3, 1.0, _z(54))
        assert [r for _, r in got] == [12, 54]
    finally:
        ne._CTX_EAM.pop(ctx.value)
    # a context the binding did not create: no knot count, no check
    assert recorded(ne.ne_ctx_set_theta, C.c_void_p(0x7170), _z(3)) == [(3, None)]


def test_autotuner_refuses_a_box_no_candidate_fits(monkeypatch):
    """Candidates whose list range 2 (r_c + skin) reaches the box are skipped
    (r_c of the context's own potential); with none left the tuner says so
    before any device work, and the caller's skins are left as they were."""
    from paper_2201_04622_gb300 import autotune

    def no_device_work(*a, **k):
        raise AssertionError("the tuner reached the library")

    monkeypatch.setattr(ne, "ne_ctx_set_tuning", no_device_work)
    monkeypatch.setattr(ne, "ne_profile_segment", no_device_work)
    ctx = C.c_void_p(0x8180)
    ne._CTX_EAM[ctx.value] = (5000, 5.3)
    try:
        mds = [ne.md_params(skin=0.7)]
        x = _z(128, 3)
        # bcc 4^3 is 11.48 A wide: 2 (5.3 + 0.5) = 11.6 and 2 (5.3 + 0.7) = 12 do not fit
        with pytest.raises(ValueError, match="no candidate"):
            autotune.tune(ctx, mds, [0, 128], x, x.clone(), x.clone(), [[11.48] * 3], _z(1, 2),
                          skins=[0.5, 0.7])
        assert mds[0].skin == 0.7
    finally:
        ne._CTX_EAM.pop(ctx.value)
    with pytest.raises(ValueError, match="not created"):
        autotune.tune(C.c_void_p(0x9190), [ne.md_params()], [0, 128], x, x, x, [[20.0] * 3], _z(1, 2))


def test_crystal_plan_wrapper_reads_the_four_integers(monkeypatch):
    """ne_ctx_crystal_plan: runner 1 is the cluster runner, 2 the brick
    runner; the four integers come back in the dict the bench reports."""
    def plan(r, t, n, c):
        def fake(ctx, pr, pt, pn, pc):
            pr._obj.value, pt._obj.value, pn._obj.value, pc._obj.value = r, t, n, c
            return 0
        return fake
    for args, want in (((1, 2, 120, 6), {"runner": "cluster", "threads_per_atom": 2, "ctas": 120, "cluster_ctas": 6}),
                       ((2, 3, 128, 0), {"runner": "brick", "threads_per_atom": 3, "ctas": 128, "cluster_ctas": 0})):
        monkeypatch.setattr(ne, "load", lambda *a, f=plan(*args), **k: types.SimpleNamespace(ne_ctx_crystal_plan=f))
        assert ne.ne_ctx_crystal_plan(None) == want
