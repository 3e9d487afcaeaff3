"""The staged FP32 1D step (interior units delivered to shared memory by bulk
asynchronous copies) against its direct-load form: the same bits.  A state
or aux buffer that starts 4 bytes off a 16-byte boundary cannot be copied in
bulk, so every unit of a step that reads it takes the direct loads; the
aligned run stages its interior units.  Also the bounded barrier wait's
self-test: a wait that nothing completes gives up within its limit, and a
bulk copy completes with the right bytes."""
import numpy as np
import pytest

from paper_1111_6583_gb300 import workloads as wl
from tests.gpu_util import FP32_SHOCK_L1_TOL, rel_l1

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()


def _offset_copy(a, dtype):
    """a as a CUDA tensor of `dtype` whose data start 4 bytes past a 16-byte
    boundary (contiguous, same shape)."""
    import torch
    a = np.asarray(a)
    flat = torch.empty(a.size + 4, dtype=dtype, device="cuda")
    base = flat.data_ptr()
    off = ((16 - base % 16) % 16) // 4 + 1  # elements to the first misaligned start
    v = flat[off:off + a.size].view(a.shape)
    assert v.data_ptr() % 16 == 4
    v.copy_(torch.as_tensor(a, dtype=dtype))
    return v


def _run(spec, t_end, q=None, aux=None):
    import torch
    from paper_1111_6583_gb300 import claw
    s = claw.Solver(spec, "fp32", q=q, aux=aux)
    info = s.evolve(t_end)
    torch.cuda.synchronize()
    out = s.sync().double().cpu().numpy().copy()
    s.close()
    return out, info["steps"]


@pytest.mark.parametrize("n", [20000, 4 * 4099])
def test_acoustics_staged_equals_direct(n):
    import torch
    spec = wl.acoustics_1d(n=n, t_end=0.05)
    ref, st = _run(spec, 0.05)
    got, st2 = _run(spec, 0.05, q=_offset_copy(spec["q0"], torch.float32))
    assert st == st2 and st > 5
    assert np.array_equal(ref, got)


def test_elasticity_staged_equals_direct():
    import torch
    spec = wl.elasticity_member(12000, 0.3, 0.05, t_end=2.0)
    ref, st = _run(spec, 2.0)
    got, st2 = _run(spec, 2.0, aux=_offset_copy(spec["aux"], torch.float32))
    assert st == st2 and st > 5
    assert np.array_equal(ref, got)


def test_staged_batch_against_oracle():
    """A batch whose members mix staged interiors and direct-load edges
    (sizes below, at and above one unit's footprint) against the oracle."""
    import torch
    import oracle
    from paper_1111_6583_gb300 import claw
    specs = [wl.acoustics_1d(n=n, t_end=0.02) for n in (40, 256, 257, 964, 2000, 9999)]
    b = claw.Batch(specs, "fp32")
    infos = b.evolve()
    torch.cuda.synchronize()
    qs = [t.double().cpu().numpy() for t in b.sync()]
    b.close()
    for sp, q, inf in zip(specs, qs, infos):
        qo, _ = oracle.evolve(oracle.make_problem(sp), sp["q0"], t_end=sp["t_end"])
        assert inf["t"] == pytest.approx(sp["t_end"], abs=0.0)
        assert rel_l1(q, qo) <= FP32_SHOCK_L1_TOL, sp["q0"].shape


def test_bounded_wait_self_test():
    from paper_1111_6583_gb300 import claw
    gave_up, copied, waited = claw.async_wait_probe(20000)
    assert gave_up and copied
    assert 20000.0 <= waited < 2e6


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_sharpclaw_staged_rows_equal_loaded_cells(prec):
    """SharpClaw stages the halo rows of interior tiles by bulk copies when
    the state is 16-byte aligned, and loads cell by cell otherwise: a state
    that starts 4 (FP32) or 8 (FP64) bytes off the boundary gives the same
    bits (2D Euler, WENO5-char; 2D p-system with aux fields)."""
    import torch
    dt = torch.float32 if prec == "fp32" else torch.float64
    for spec, t_end in ((wl.shock_bubble_2d(nx=128, ny=64), 0.02),
                        (wl.psystem_checkerboard_2d(periods=2, cells_per_period=32), 0.05)):
        ref, st = _run_prec(spec, prec, t_end)
        got, st2 = _run_prec(spec, prec, t_end, q=_offset_copy_dt(spec["q0"], dt))
        assert st == st2 and st > 2
        assert np.array_equal(ref, got)


def _offset_copy_dt(a, dtype):
    """a as a contiguous CUDA tensor of `dtype` starting one element past a
    16-byte boundary."""
    import torch
    a = np.asarray(a)
    es = torch.empty(0, dtype=dtype).element_size()
    flat = torch.empty(a.size + 16, dtype=dtype, device="cuda")
    base = flat.data_ptr()
    off = ((16 - base % 16) % 16) // es + 1
    v = flat[off:off + a.size].view(a.shape)
    assert v.data_ptr() % 16 != 0
    v.copy_(torch.as_tensor(a, dtype=dtype))
    return v


def _run_prec(spec, prec, t_end, q=None):
    import torch
    from paper_1111_6583_gb300 import claw
    s = claw.Solver(spec, prec, q=q)
    info = s.evolve(t_end)
    torch.cuda.synchronize()
    out = s.sync().double().cpu().numpy().copy()
    s.close()
    return out, info["steps"]
