"""Helpers shared by the GPU tests: run the same seeded input through the CUDA
library (C ABI via the binding) and through the CPU oracle, and compare."""
import numpy as np

FP64_TOL = 1e-12      # max-norm relative, FP64 GPU vs FP64 oracle
FP32_SMOOTH_TOL = 1e-5
FP32_SHOCK_L1_TOL = 1e-4


def rel_maxnorm(q, ref):
    """Per field max|q - ref| / max|ref| (fields that are zero in ref use the
    largest field's scale), maximised over fields."""
    q = np.asarray(q, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    m = ref.shape[0]
    big = np.abs(ref).max()
    worst = 0.0
    for k in range(m):
        den = np.abs(ref[k]).max()
        if den < 1e-12 * big:
            den = big
        worst = max(worst, np.abs(q[k] - ref[k]).max() / den)
    return worst


def rel_l1(q, ref):
    """L1 norm of the difference over all fields and cells relative to the L1
    norm of the reference (a field that the reference holds near zero, such as
    the residual velocity of a pulse that has returned to rest, is measured
    against the whole state rather than against itself)."""
    q = np.asarray(q, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return np.abs(q - ref).sum() / np.abs(ref).sum()


def gpu_fixed_steps(spec, prec, dt, nsteps):
    import torch
    from paper_1111_6583_gb300 import claw
    s = claw.Solver(spec, prec)
    cfls = []
    for _ in range(nsteps):
        info = s.step(dt)
        cfls.append(info["cfl"])
    s.sync()
    torch.cuda.synchronize()
    q = s.q.double().cpu().numpy()
    s.close()
    return q, cfls


def oracle_fixed_steps(orc, spec, dt, nsteps):
    P = orc.make_problem(spec)
    q = spec["q0"].copy()
    cfls = []
    for _ in range(nsteps):
        q, cfl = orc.step(P, q, spec.get("aux"), dt)
        cfls.append(cfl)
    return q, cfls


def gpu_evolve(spec, prec, t_end, max_steps=0, use_graph=True, tune=None):
    import torch
    from paper_1111_6583_gb300 import claw
    s = claw.Solver(spec, prec)
    if tune is not None:
        s.tune(*tune)
    info = s.evolve(t_end, max_steps=max_steps, use_graph=use_graph)
    torch.cuda.synchronize()
    q = s.q.double().cpu().numpy()
    s.close()
    return q, info


def oracle_evolve(orc, spec, t_end, max_steps=10 ** 9):
    P = orc.make_problem(spec)
    return orc.evolve(P, spec["q0"], spec.get("aux"), t_end=t_end, max_steps=max_steps)
