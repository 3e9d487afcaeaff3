"""Launch-shape tuning never changes a result: batches (2D tile shapes, 1D
work modes), single 1D solvers and the server tuned on its live mix give the
same bits as untuned runs."""
import numpy as np
import pytest

from paper_1111_6583_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()


def _batch_run(specs, prec, shape):
    import torch
    from paper_1111_6583_gb300 import claw
    b = claw.Batch(specs, prec)
    chosen = b.tune() if shape == "auto" else (b.tune(*shape) if shape else None)
    infos = b.evolve()
    torch.cuda.synchronize()
    q = [t.double().cpu().numpy() for t in b.sync()]
    b.close()
    return q, [i["steps"] for i in infos], chosen


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_batch_2d_shapes_bitwise(prec):
    specs = [wl.sw_humps_2d(n, [(0.4, 0.1, 0.4, 0.6), (0.2, 0.2, 0.7, 0.3)], t)
             for n, t in ((40, 0.3), (97, 0.2), (64, 0.25), (150, 0.1))]
    ref, steps, _ = _batch_run(specs, prec, None)
    for shape in ("auto", (64, 8), (128, 41), (64, 128)):
        q, st, chosen = _batch_run(specs, prec, shape)
        assert st == steps, shape
        for a, b in zip(q, ref):
            assert np.array_equal(a, b), (shape, chosen)


def test_batch_1d_work_modes_bitwise():
    ens = wl.elasticity_ensemble(48, lo_exp=10, hi_exp=13)
    specs = [wl.elasticity_member(e["n"], e["amp"], e["width"], t_end=3.0) for e in ens]
    ref, steps, _ = _batch_run(specs, "fp32", None)
    for shape in ("auto", (0, 1), (0, 2)):
        q, st, chosen = _batch_run(specs, "fp32", shape)
        assert st == steps, shape
        assert chosen[1] in (1, 2)
        for a, b in zip(q, ref):
            assert np.array_equal(a, b), shape


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_solver_1d_work_modes_bitwise(prec):
    import torch
    from paper_1111_6583_gb300 import claw
    spec = wl.acoustics_1d(n=20000, t_end=0.05)
    out = []
    for shape in (None, "auto", (0, 1), (0, 2)):
        s = claw.Solver(spec, prec)
        if shape == "auto":
            assert s.tune()[1] in (1, 2)
        elif shape:
            s.tune(*shape)
        s.evolve(0.05)
        torch.cuda.synchronize()
        out.append(s.q.double().cpu().numpy())
        s.close()
    for q in out[1:]:
        assert np.array_equal(q, out[0])


def _serve(specs, tune_at):
    from paper_1111_6583_gb300 import claw
    sv = claw.Server(specs[0], "fp32", budget_bytes=1 << 30, max_slots=16)
    tickets = [sv.submit(sp) for sp in specs]
    done, pumps, chosen = {}, 0, None
    while len(done) < len(tickets):
        sv.pump(2)
        pumps += 1
        if pumps == tune_at:
            chosen = sv.tune()
        for t in sv.take_done():
            done[t] = sv.poll(t)
        assert pumps < 100000
    sv.close()
    return [done[t] for t in tickets], chosen


def test_server_tuned_on_live_mix_bitwise():
    """Tuning a few pumps into the stream (requests in flight) changes no
    request's steps or state; each still equals its single solve."""
    import torch
    from paper_1111_6583_gb300 import claw
    specs = [wl.sw_humps_2d(n, [(0.3, 0.15, 0.5, 0.5)], t)
             for n, t in ((48, 0.3), (130, 0.2), (77, 0.25), (200, 0.15), (64, 0.3))]
    ref, _ = _serve(specs, tune_at=-1)
    got, chosen = _serve(specs, tune_at=3)
    assert chosen is not None and chosen[0] in (64, 128)
    for a, b, sp in zip(got, ref, specs):
        assert a["steps"] == b["steps"]
        assert np.array_equal(a["q"], b["q"])
        s = claw.Solver(sp, "fp32")
        s.evolve(sp["t_end"])
        torch.cuda.synchronize()
        assert np.array_equal(s.q.cpu().numpy(), a["q"])
        s.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_sharpclaw_2d_tiles_bitwise(prec):
    """Every SharpClaw 2D tile (WENO5, characteristic-wise Euler) gives the
    default tile's bits; the autotuner's pick is one of them; shapes the
    method does not have are refused."""
    import torch
    from paper_1111_6583_gb300 import claw
    spec = wl.shock_bubble_2d(nx=100, ny=52)  # ragged in both directions
    out, chosen = {}, None
    for shape in (None, "auto", (32, 4), (32, 8), (16, 16)):
        s = claw.Solver(spec, prec)
        if shape == "auto":
            chosen = s.tune()
        elif shape:
            assert tuple(s.tune(*shape)) == shape
        info = s.evolve(0.02, max_steps=6)
        torch.cuda.synchronize()
        out[shape] = (info["steps"], s.q.double().cpu().numpy())
        s.close()
    ref = out[None]
    for shape, (st, q) in out.items():
        assert st == ref[0], shape
        assert np.array_equal(q, ref[1]), (shape, chosen)
    assert tuple(chosen) in ((16, 8), (32, 4), (32, 8), (16, 16))
    s = claw.Solver(spec, prec)
    for bad in ((64, 21), (8, 16)):
        with pytest.raises(RuntimeError):
            s.tune(*bad)
    s.close()
    sp7 = dict(spec, weno_order=7)
    s = claw.Solver(sp7, prec)
    with pytest.raises(RuntimeError):
        s.tune(32, 4)  # higher orders keep the default tile
    assert tuple(s.tune()) == (16, 8)
    s.close()


def test_sharpclaw_batch_and_server_tiles_bitwise():
    """A SharpClaw batch and a SharpClaw server tuned (auto and by hand) give
    their untuned bits."""
    import torch
    from paper_1111_6583_gb300 import claw
    specs = [wl.shock_bubble_2d(nx=nx, ny=ny) for nx, ny in ((64, 32), (100, 52), (48, 40))]
    for sp in specs:
        sp["t_end"] = 0.01
    ref, steps, _ = _batch_run(specs, "fp32", None)
    for shape in ("auto", (32, 4), (16, 16)):
        q, st, chosen = _batch_run(specs, "fp32", shape)
        assert st == steps, shape
        for a, b in zip(q, ref):
            assert np.array_equal(a, b), (shape, chosen)
    sv = claw.Server(specs[0], "fp32", budget_bytes=1 << 30, max_slots=8)
    tickets = [sv.submit(sp) for sp in specs]
    sv.pump(1)
    assert tuple(sv.tune()) in ((16, 8), (32, 4), (32, 8), (16, 16))
    done, pumps = {}, 0
    while len(done) < len(tickets):
        sv.pump(2)
        pumps += 1
        for t in sv.take_done():
            done[t] = sv.poll(t)
        assert pumps < 100000
    sv.close()
    for t, b in zip(tickets, ref):
        assert np.array_equal(done[t]["q"], b)
    torch.cuda.synchronize()
