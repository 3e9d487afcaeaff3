"""Seeded synthetic workloads shaped like the paper's examples.

This module holds problem descriptions and initial data only -- none of the
finite-volume method's arithmetic.  Both the CUDA path (through the binding)
and the CPU oracle consume what it returns, so it imports neither.

A workload spec is a plain dict:

    ndim, n, lower, upper            grid (cell counts, domain box)
    rp, scheme, lim, order,          method (Riemann solver, classic/SharpClaw,
    transverse, char_decomp,          limiter, order, transverse mode, WENO
    entropy_fix, weno_eps             projection, Harten-Hyman fix, epsilon)
    bc_lower, bc_upper, inflow       boundary conditions per direction
    params                           solver constants (rho,K | g | gamma | u,v)
    cfl_desired, cfl_max,            CFL controller
    dt_initial, dt_max, max_retries
    t_end                            final time
    q0, aux                          float64 arrays [m][ny][nx] ([m][nx] in 1D)

Seeds: base 6583, numpy PCG64.
"""
from __future__ import annotations

import math

import numpy as np

SEED = 6583


def _centers(lo, hi, n):
    dx = (hi - lo) / n
    return lo + (np.arange(n) + 0.5) * dx


def _base(ndim, n, lower, upper, rp, **kw):
    spec = dict(ndim=ndim, n=list(n), lower=list(lower), upper=list(upper), rp=rp,
                scheme="classic", lim="mc", order=2, transverse=2, char_decomp=0,
                entropy_fix=1, weno_eps=1e-6, bc_lower=["periodic"] * ndim,
                bc_upper=["periodic"] * ndim, inflow=[], params=[], cfl_desired=0.9,
                cfl_max=1.0, dt_initial=0.0, dt_max=1e30, max_retries=8)
    spec.update(kw)
    return spec


# --------------------------------------------------------------------------
# 1D linear acoustics pulse (Table 1 system, 1D form)
# --------------------------------------------------------------------------
def acoustics_1d(n=2000, t_end=2.0, lim="mc"):
    """x in [-1,1], periodic, rho=1, K=4 (c=2), p0 = exp(-100 x^2) + 1 on
    [0.3,0.5], u0 = 0; at t=2 both pulses are back at their start."""
    x = _centers(-1.0, 1.0, n)
    p = np.exp(-100.0 * x * x) + ((x >= 0.3) & (x <= 0.5)).astype(np.float64)
    q0 = np.stack([p, np.zeros_like(p)])
    spec = _base(1, [n], [-1.0], [1.0], "acoustics", lim=lim, params=[1.0, 4.0],
                 bc_lower=["periodic"], bc_upper=["periodic"])
    spec.update(q0=np.ascontiguousarray(q0), aux=None, t_end=t_end)
    return spec


# --------------------------------------------------------------------------
# 2D and 3D linear acoustics, constant medium (Table 1 acoustics workload)
# --------------------------------------------------------------------------
def acoustics_2d(n=1024, t_end=0.5, lim="mc"):
    """[-1,1]^2, rho = 1, K = 4 (c = 2), p0 = exp(-100 r^2) + 1 on the square
    [0.3,0.5]^2, u0 = v0 = 0, walls, MC limiter, full transverse corrections,
    CFL 0.9."""
    x = _centers(-1.0, 1.0, n)
    X, Y = np.meshgrid(x, x, indexing="xy")
    sq = ((X >= 0.3) & (X <= 0.5) & (Y >= 0.3) & (Y <= 0.5)).astype(np.float64)
    p = np.exp(-100.0 * (X * X + Y * Y)) + sq
    z = np.zeros_like(p)
    spec = _base(2, [n, n], [-1.0, -1.0], [1.0, 1.0], "acoustics", lim=lim, params=[1.0, 4.0],
                 bc_lower=["wall", "wall"], bc_upper=["wall", "wall"])
    spec.update(q0=np.ascontiguousarray(np.stack([p, z, z])), aux=None, t_end=t_end)
    return spec


def acoustics_3d(n=256, t_end=0.25, lim="mc"):
    """The 3D form on [-1,1]^3: same medium, p0 = exp(-100 r^2) + 1 on the
    cube [0.3,0.5]^3, zero velocity, walls, MC, transverse and
    double-transverse corrections, CFL 0.9."""
    x = _centers(-1.0, 1.0, n)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    cube = ((X >= 0.3) & (X <= 0.5) & (Y >= 0.3) & (Y <= 0.5) & (Z >= 0.3) &
            (Z <= 0.5)).astype(np.float64)
    p = np.exp(-100.0 * (X * X + Y * Y + Z * Z)) + cube
    z = np.zeros_like(p)
    spec = _base(3, [n, n, n], [-1.0] * 3, [1.0] * 3, "acoustics", lim=lim, params=[1.0, 4.0],
                 bc_lower=["wall"] * 3, bc_upper=["wall"] * 3)
    spec.update(q0=np.ascontiguousarray(np.stack([p, z, z, z])), aux=None, t_end=t_end)
    return spec


# --------------------------------------------------------------------------
# 2D shallow-water radial dam break (Table 1 shallow-water workload)
# --------------------------------------------------------------------------
def sw_dambreak_2d(n=1024, t_end=1.5, transverse=2, lim="mc"):
    """[-2.5,2.5]^2, h = 2 for r < 0.5 else 1, hu = hv = 0, g = 1, walls,
    Roe + Harten-Hyman, MC limiter, CFL 0.9."""
    x = _centers(-2.5, 2.5, n)
    X, Y = np.meshgrid(x, x, indexing="xy")  # [ny][nx]
    r = np.sqrt(X * X + Y * Y)
    h = np.where(r < 0.5, 2.0, 1.0)
    q0 = np.stack([h, np.zeros_like(h), np.zeros_like(h)])
    spec = _base(2, [n, n], [-2.5, -2.5], [2.5, 2.5], "sw_roe", lim=lim, transverse=transverse,
                 params=[1.0], bc_lower=["wall", "wall"], bc_upper=["wall", "wall"])
    spec.update(q0=np.ascontiguousarray(q0), aux=None, t_end=t_end)
    return spec


# --------------------------------------------------------------------------
# 2D Euler shock-bubble (Sec. 7.2, planar form)
# --------------------------------------------------------------------------
def post_shock_state(mach=2.0, gamma=1.4, rho1=1.0, p1=1.0):
    """Rankine-Hugoniot state behind a shock of the given Mach number moving
    into gas at rest (rho1, p1): returns (rho2, u2, p2)."""
    c1 = math.sqrt(gamma * p1 / rho1)
    m2 = mach * mach
    p2 = p1 * (1.0 + 2.0 * gamma / (gamma + 1.0) * (m2 - 1.0))
    rho2 = rho1 * (gamma + 1.0) * m2 / ((gamma - 1.0) * m2 + 2.0)
    u2 = mach * c1 * (1.0 - rho1 / rho2)
    return rho2, u2, p2


def shock_bubble_2d(nx=2048, ny=1024, t_end=0.2, scheme="sharpclaw", gamma=1.4,
                    sub=16, char_decomp=1):
    """[0,2]x[0,1]; Mach-2 planar shock at x = 0.2 moving into rho = p = 1;
    bubble rho = 0.1, p = 1, radius 0.2 at (0.5, 0.5), cell-averaged by a
    sub x sub sample of the inside fraction; inflow (post-shock) left, extrap
    right, walls top/bottom; SharpClaw WENO5 + SSP-RK3 by default."""
    x = _centers(0.0, 2.0, nx)
    y = _centers(0.0, 1.0, ny)
    dx, dy = 2.0 / nx, 1.0 / ny
    # inside fraction of the bubble per cell from a sub x sub point sample
    off = (np.arange(sub) + 0.5) / sub - 0.5
    frac = np.zeros((ny, nx))
    X, Y = np.meshgrid(x, y, indexing="xy")
    for a in off:
        for b in off:
            xs = X + a * dx
            ys = Y + b * dy
            frac += ((xs - 0.5) ** 2 + (ys - 0.5) ** 2 < 0.04)
    frac /= sub * sub
    rho = frac * 0.1 + (1.0 - frac) * 1.0
    E_amb = 1.0 / (gamma - 1.0)
    E = np.full_like(rho, E_amb)
    rho2, u2, p2 = post_shock_state(2.0, gamma)
    E2 = p2 / (gamma - 1.0) + 0.5 * rho2 * u2 * u2
    left = X < 0.2
    rho = np.where(left, rho2, rho)
    mx = np.where(left, rho2 * u2, 0.0)
    my = np.zeros_like(rho)
    E = np.where(left, E2, E)
    q0 = np.stack([rho, mx, my, E])
    spec = _base(2, [nx, ny], [0.0, 0.0], [2.0, 1.0], "euler_roe", scheme=scheme,
                 char_decomp=char_decomp, params=[gamma],
                 bc_lower=["inflow", "wall"], bc_upper=["extrap", "wall"],
                 inflow=[rho2, rho2 * u2, 0.0, E2],
                 cfl_desired=0.5 if scheme == "sharpclaw" else 0.8,
                 cfl_max=0.6 if scheme == "sharpclaw" else 1.0)
    spec.update(q0=np.ascontiguousarray(q0), aux=None, t_end=t_end)
    return spec


def post_shock_state_from_pressure(p2, gamma=1.4, rho1=1.0, p1=1.0):
    """Rankine-Hugoniot state behind the shock whose post-shock pressure is
    p2 (gas at rest ahead): Mach^2 = 1 + (gamma+1)/(2 gamma) (p2/p1 - 1)."""
    mach = math.sqrt(1.0 + (gamma + 1.0) / (2.0 * gamma) * (p2 / p1 - 1.0))
    return post_shock_state(mach, gamma, rho1, p1)


def shock_bubble_axisym(nx=1280, ny=320, t_end=0.6, scheme="classic", gamma=1.4, sub=16,
                        dim_split=0, cfl=(0.8, 1.0), source_split="godunov"):
    """The shock-bubble interaction of Sec. 7.2 in its axisymmetric form:
    (z, r) = (x, y) on [0, 2] x [0, 0.5], Euler with a passive tracer and the
    geometric source -(1/r)(rho v, rho u v, rho v^2, (E + p) v) by Godunov
    (or Strang) splitting.  Ahead of the shock rho = p = 1 at rest; a sphere of rho = 0.1
    (p = 1), radius 0.2, centred on the axis at z = 0.5, carries tracer 1
    (cell fractions from a sub x sub point sample); the shock at z = 0.2 has
    the paper's post-shock pressure 5 (rho and u by Rankine-Hugoniot, about
    2.82 and 1.61), which also enters at the left.  Reflecting axis r = 0,
    extrapolation at r = 0.5 and z = 2.  Classic unsplit with full
    transverse corrections, MC limiter, CFL 0.8."""
    x = _centers(0.0, 2.0, nx)
    y = _centers(0.0, 0.5, ny)
    dx, dy = 2.0 / nx, 0.5 / ny
    off = (np.arange(sub) + 0.5) / sub - 0.5
    frac = np.zeros((ny, nx))
    X, Y = np.meshgrid(x, y, indexing="xy")
    for a in off:
        for b in off:
            frac += ((X + a * dx - 0.5) ** 2 + (Y + b * dy) ** 2 < 0.04)
    frac /= sub * sub
    rho = frac * 0.1 + (1.0 - frac) * 1.0
    E = np.full_like(rho, 1.0 / (gamma - 1.0))
    rho2, u2, p2 = post_shock_state_from_pressure(5.0, gamma)
    E2 = p2 / (gamma - 1.0) + 0.5 * rho2 * u2 * u2
    left = X < 0.2
    rho = np.where(left, rho2, rho)
    mx = np.where(left, rho2 * u2, 0.0)
    E = np.where(left, E2, E)
    tracer = np.where(left, 0.0, frac)
    q0 = np.stack([rho, mx, np.zeros_like(rho), E, tracer])
    spec = _base(2, [nx, ny], [0.0, 0.0], [2.0, 0.5], "euler_tracer", scheme=scheme,
                 params=[gamma], source="axisymmetric", source_split=source_split,
                 dim_split=dim_split,
                 bc_lower=["inflow", "wall"], bc_upper=["extrap", "extrap"],
                 inflow=[rho2, rho2 * u2, 0.0, E2, 0.0], cfl_desired=cfl[0], cfl_max=cfl[1])
    spec.update(q0=np.ascontiguousarray(q0), aux=None, t_end=t_end)
    return spec


# --------------------------------------------------------------------------
# Listing 1: 2D Euler Riemann problem (Lax-Liu case 6), the paper's hello world
# --------------------------------------------------------------------------
def euler_quadrants_2d(n=100, t_end=0.3, gamma=1.4):
    """Unit square, extrapolation BCs, gamma 1.4; the four-quadrant initial
    data of the paper's first listing."""
    x = _centers(0.0, 1.0, n)
    X, Y = np.meshgrid(x, x, indexing="xy")
    l = (X < 0.5).astype(float); r = (X >= 0.5).astype(float)
    b = (Y < 0.5).astype(float); t = (Y >= 0.5).astype(float)
    rho = 2.0 * l * t + 1.0 * l * b + 1.0 * r * t + 3.0 * r * b
    mx = 0.75 * t - 0.75 * b
    my = 0.5 * l - 0.5 * r
    E = 0.5 * rho * (mx ** 2 + my ** 2) + 1.0 / (gamma - 1.0)
    q0 = np.stack([rho, mx, my, E])
    spec = _base(2, [n, n], [0.0, 0.0], [1.0, 1.0], "euler_roe", params=[gamma],
                 bc_lower=["extrap", "extrap"], bc_upper=["extrap", "extrap"])
    spec.update(q0=np.ascontiguousarray(q0), aux=None, t_end=t_end)
    return spec


# --------------------------------------------------------------------------
# 1D nonlinear elasticity in a layered medium (Sec. 7.3, 1D analogue)
# --------------------------------------------------------------------------
def layered_medium(x, width=0.5):
    """(rho, K) = (1, 1) on even layers [2k w, (2k+1) w), (4, 4) on odd ones."""
    odd = (np.floor(x / width).astype(np.int64) % 2) == 1
    rho = np.where(odd, 4.0, 1.0)
    K = np.where(odd, 4.0, 1.0)
    return rho, K


def elasticity_member(n, amp, width, dx=1.0 / 32.0, t_end=50.0):
    L = n * dx
    x = _centers(0.0, L, n)
    rho, K = layered_medium(x)
    sig0 = amp * np.exp(-((x - 0.5 * L) / width) ** 2)
    eps0 = np.log1p(sig0) / K
    q0 = np.stack([eps0, np.zeros_like(eps0)])
    aux = np.stack([rho, K])
    spec = _base(1, [n], [0.0], [L], "elasticity_fwave", num_aux=2,
                 bc_lower=["periodic"], bc_upper=["periodic"])
    spec.update(q0=np.ascontiguousarray(q0), aux=np.ascontiguousarray(aux), t_end=t_end)
    return spec


def elasticity_ensemble(members=4096, seed=SEED, lo_exp=12, hi_exp=16, t_end=50.0):
    """Uneven 1D elasticity ensemble: N_k = round(2^(lo + (hi-lo) u)), amplitude
    U(0.1, 0.5), width U(1, 5), dx = 1/32 (16 cells per layer), periodic."""
    rng = np.random.Generator(np.random.PCG64(seed))
    u = rng.random(members)
    amp = rng.uniform(0.1, 0.5, members)
    width = rng.uniform(1.0, 5.0, members)
    sizes = np.rint(2.0 ** (lo_exp + (hi_exp - lo_exp) * u)).astype(np.int64)
    return [dict(n=int(sizes[k]), amp=float(amp[k]), width=float(width[k]), t_end=t_end)
            for k in range(members)]


# --------------------------------------------------------------------------
# serving stream: 2D shallow-water humps
# --------------------------------------------------------------------------
def checkerboard_medium(x, y, k_hi=5.0, rho_hi=5.0):
    """(rho, K) of the checkerboard crystal of Sec. 7.3: (1, 1) where
    (x - floor(x) - 1/2)(y - floor(y) - 1/2) < 0, (rho_hi, k_hi) where > 0
    (lengths in material periods)."""
    s = (x - np.floor(x) - 0.5) * (y - np.floor(y) - 0.5)
    hi = s > 0
    return np.where(hi, rho_hi, 1.0), np.where(hi, k_hi, 1.0)


def psystem_checkerboard_2d(periods=32, cells_per_period=64, amp=5.0, var=5.0, t_end=20.0,
                            weno_order=5, integrator="ssp104", cfl=(1.0, 1.2)):
    """2D p-system in the checkerboard medium (Sec. 7.3) at reduced size:
    the positive quadrant [0, periods]^2, walls at x = 0 and y = 0 (the
    problem's mirror symmetry), zero-order extrapolation at the far sides,
    Gaussian stress pulse sigma_0 = amp exp(-(x^2 + y^2) / (2 var)) at the
    origin, zero velocity; eps_0 = ln(1 + sigma_0) / K.  Cell centres never lie
    on a material edge when cells_per_period is even, so the centre values
    are the cell averages of (rho, K).  SharpClaw WENO, component-wise."""
    assert cells_per_period % 2 == 0
    n = periods * cells_per_period
    c = _centers(0.0, float(periods), n)
    Y, X = np.meshgrid(c, c, indexing="ij")
    rho, K = checkerboard_medium(X, Y)
    sig0 = amp * np.exp(-(X * X + Y * Y) / (2.0 * var))
    eps0 = np.log1p(sig0) / K
    q0 = np.stack([eps0, np.zeros_like(eps0), np.zeros_like(eps0)])
    aux = np.stack([rho, K])
    spec = _base(2, [n, n], [0.0, 0.0], [float(periods)] * 2, "elasticity_fwave",
                 scheme="sharpclaw", char_decomp=0, weno_order=weno_order,
                 time_integrator=integrator, cfl_desired=cfl[0], cfl_max=cfl[1], num_aux=2,
                 bc_lower=["wall", "wall"], bc_upper=["extrap", "extrap"])
    spec.update(q0=np.ascontiguousarray(q0), aux=np.ascontiguousarray(aux), t_end=t_end)
    return spec


def acoustics_vc_2d(n=1024, t_end=0.6, capacity=True, cfl=(0.9, 1.0)):
    """2D acoustics in a heterogeneous medium (the Table 1 acoustics system
    with spatially varying coefficients): [-1, 1]^2, (rho, c) = (1, 1) for
    x < 0.3 and (4, 0.5) beyond (an impedance jump of 2), a circular pressure
    pulse p = exp(-80 r^2) at (-0.4, 0), at rest, walls; with capacity, the
    medium sits on a grid stretched in x (x = xi + 0.1 sin(pi xi)), entering
    as kappa = dx/dxi = 1 + 0.1 pi cos(pi xi) on the uniform xi grid.  Classic,
    MC, full transverse corrections, CFL 0.9."""
    xi = _centers(-1.0, 1.0, n)
    XI, Y = np.meshgrid(xi, xi, indexing="xy")
    X = XI + 0.1 * np.sin(np.pi * XI) if capacity else XI
    rho = np.where(X < 0.3, 1.0, 4.0)
    c = np.where(X < 0.3, 1.0, 0.5)
    p = np.exp(-80.0 * ((X + 0.4) ** 2 + Y ** 2))
    q0 = np.stack([p, np.zeros_like(p), np.zeros_like(p)])
    auxl = [rho, c]
    kw = {}
    if capacity:
        auxl.append(1.0 + 0.1 * np.pi * np.cos(np.pi * XI))
        kw["capa_index"] = 2
    aux = np.stack(auxl)
    spec = _base(2, [n, n], [-1.0, -1.0], [1.0, 1.0], "acoustics_vc", num_aux=len(auxl),
                 bc_lower=["wall", "wall"], bc_upper=["wall", "wall"], cfl_desired=cfl[0],
                 cfl_max=cfl[1], **kw)
    spec.update(q0=np.ascontiguousarray(q0), aux=np.ascontiguousarray(aux), t_end=t_end)
    return spec


def sw_humps_2d(n, humps, t_end):
    """[0,1]^2, depth 1 plus Gaussian humps (a, w, cx, cy), walls, g = 1."""
    x = _centers(0.0, 1.0, n)
    X, Y = np.meshgrid(x, x, indexing="xy")
    h = np.ones((n, n))
    for (a, w, cx, cy) in humps:
        r2 = (X - cx) ** 2 + (Y - cy) ** 2
        h = h + a * np.exp(-r2 / (w * w))
    q0 = np.stack([h, np.zeros_like(h), np.zeros_like(h)])
    spec = _base(2, [n, n], [0.0, 0.0], [1.0, 1.0], "sw_roe", params=[1.0],
                 bc_lower=["wall", "wall"], bc_upper=["wall", "wall"])
    spec.update(q0=np.ascontiguousarray(q0), aux=None, t_end=t_end)
    return spec


def serving_stream(requests=2000, rate=200.0, seed=SEED + 5, lo_exp=6, hi_exp=10):
    """Poisson arrivals (exponential gaps of mean 1/rate); n = round(2^(6+4u));
    1-3 humps of height U(0.1,1), width U(0.05,0.3), centres U(0.15,0.85)^2;
    t_end U(0.5, 2)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = rng.exponential(1.0 / rate, requests)
    arrivals = np.cumsum(gaps)
    out = []
    for k in range(requests):
        u = rng.random()
        n = int(round(2.0 ** (lo_exp + (hi_exp - lo_exp) * u)))
        nh = int(rng.integers(1, 4))
        humps = [(float(rng.uniform(0.1, 1.0)), float(rng.uniform(0.05, 0.3)),
                  float(rng.uniform(0.15, 0.85)), float(rng.uniform(0.15, 0.85)))
                 for _ in range(nh)]
        out.append(dict(arrival=float(arrivals[k]), n=n, humps=humps,
                        t_end=float(rng.uniform(0.5, 2.0))))
    return out


# --------------------------------------------------------------------------
# small generic cases for parity tests
# --------------------------------------------------------------------------
def random_smooth_2d(rp, nx, ny, seed=SEED, params=None, bc="periodic", **kw):
    """Smooth positive random field (a few Fourier modes) for the given system."""
    rng = np.random.Generator(np.random.PCG64(seed))
    x = _centers(0.0, 1.0, nx)
    y = _centers(0.0, 1.0, ny)
    X, Y = np.meshgrid(x, y, indexing="xy")

    def field(amp):
        f = np.zeros_like(X)
        for _ in range(3):
            kx, ky = rng.integers(1, 4, 2)
            ph = rng.uniform(0, 2 * np.pi)
            f += amp * rng.uniform(0.3, 1.0) * np.sin(2 * np.pi * (kx * X + ky * Y) + ph)
        return f

    if rp == "sw_roe":
        q0 = np.stack([1.0 + field(0.1), field(0.1), field(0.1)])
        params = params or [1.0]
    elif rp in ("euler_roe", "euler_hlle", "euler_tracer"):
        rho = 1.0 + field(0.1)
        mx, my = field(0.2), field(0.2)
        p = 1.0 + field(0.1)
        E = p / 0.4 + 0.5 * (mx * mx + my * my) / rho
        q0 = np.stack([rho, mx, my, E])
        if rp == "euler_tracer":
            q0 = np.concatenate([q0, (0.5 + field(0.5))[None]])
        params = params or [1.4]
    elif rp == "acoustics":
        q0 = np.stack([field(0.5), field(0.5), field(0.5)])
        params = params or [1.0, 4.0]
    elif rp == "advection":
        q0 = np.stack([field(1.0)])
        params = params or [1.0, 0.5]
    elif rp == "acoustics_vc":
        # layered medium (rho, c) with a smooth capacity field as a third aux
        rho = np.where(X < 0.5, 1.0, 2.5) * (1.0 + 0.2 * np.sin(2 * np.pi * Y))
        c = np.where(X < 0.5, 1.0, 0.6) * (1.0 + 0.1 * np.cos(2 * np.pi * Y))
        kap = 1.0 + 0.3 * np.sin(2 * np.pi * X) * np.sin(2 * np.pi * Y)
        q0 = np.stack([field(0.5), field(0.5), field(0.5)])
        aux = np.stack([rho, c, kap])
        params = []
    elif rp == "elasticity_fwave":
        # checkerboard medium of period 1/4 (material edges on cell edges when
        # 8 divides nx and ny; otherwise cells take the centre's material)
        rho, K = checkerboard_medium(4.0 * X, 4.0 * Y, k_hi=3.0, rho_hi=2.0)
        sig = 0.3 + field(0.1)
        q0 = np.stack([np.log1p(sig) / K, field(0.2), field(0.2)])
        aux = np.stack([rho, K])
        params = []
    else:
        raise ValueError(rp)
    if rp == "elasticity_fwave":
        kw.setdefault("scheme", "sharpclaw")
        kw.setdefault("char_decomp", 0)
        kw.setdefault("num_aux", 2)
    elif rp == "acoustics_vc":
        kw.setdefault("num_aux", 3)
        kw.setdefault("char_decomp", 0)
    else:
        aux = None
    spec = _base(2, [nx, ny], [0.0, 0.0], [1.0, 1.0], rp, params=params,
                 bc_lower=[bc, bc], bc_upper=[bc, bc], **kw)
    spec.update(q0=np.ascontiguousarray(q0),
                aux=np.ascontiguousarray(aux) if aux is not None else None,
                t_end=kw.get("t_end", 0.1))
    return spec


def random_1d(rp, n, seed=SEED, bc=("periodic", "periodic"), jump=True, **kw):
    """Smooth random 1D data (a few Fourier modes) plus, when jump, a step in
    the middle; physical states for SW/Euler/elasticity."""
    rng = np.random.Generator(np.random.PCG64(seed))
    x = _centers(0.0, 1.0, n)

    def field(amp):
        f = np.zeros_like(x)
        for _ in range(3):
            k = rng.integers(1, 5)
            f += amp * rng.uniform(0.3, 1.0) * np.sin(2 * np.pi * k * x + rng.uniform(0, 6.3))
        if jump:
            f += amp * np.where(x > 0.5, 1.0, 0.0)
        return f

    aux = None
    if rp == "sw_roe":
        q0 = np.stack([1.5 + field(0.2), field(0.3)])
        params = [1.0]
    elif rp in ("euler_roe", "euler_hlle", "euler_tracer"):
        rho = 1.5 + field(0.2)
        m = field(0.3)
        p = 1.5 + field(0.2)
        q0 = np.stack([rho, m, p / 0.4 + 0.5 * m * m / rho])
        if rp == "euler_tracer":
            q0 = np.concatenate([q0, (0.5 + field(0.5))[None]])
        params = [1.4]
    elif rp == "acoustics":
        q0 = np.stack([field(0.5), field(0.5)])
        params = [1.3, 2.5]
    elif rp == "advection":
        q0 = np.stack([field(1.0)])
        params = [0.8]
    elif rp == "elasticity_fwave":
        rho, K = layered_medium(x * 8.0)
        sig = 0.2 + field(0.1)
        q0 = np.stack([np.log1p(sig) / K, field(0.3)])
        aux = np.stack([rho, K])
        params = []
    elif rp == "acoustics_vc":
        rho = np.where(x < 0.5, 1.0, 2.5)
        c = np.where(x < 0.5, 1.0, 0.6)
        kap = 1.0 + 0.3 * np.sin(2 * np.pi * x)
        q0 = np.stack([field(0.5), field(0.5)])
        aux = np.stack([rho, c, kap])
        params = []
    else:
        raise ValueError(rp)
    if rp == "acoustics_vc":
        kw.setdefault("char_decomp", 0)
    spec = _base(1, [n], [0.0], [1.0], rp, params=kw.pop("params", params),
                 bc_lower=[bc[0]], bc_upper=[bc[1]],
                 num_aux=kw.pop("num_aux", 2 if rp == "elasticity_fwave" else
                                (3 if rp == "acoustics_vc" else 0)), **kw)
    spec.update(q0=np.ascontiguousarray(q0),
                aux=np.ascontiguousarray(aux) if aux is not None else None,
                t_end=kw.get("t_end", 0.1))
    return spec


def random_3d(rp, nx, ny, nz, seed=SEED, bc="periodic", **kw):
    """Smooth random 3D data for advection (u, v, w) or acoustics (p, u, v, w)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    z = _centers(0.0, 1.0, nz)
    y = _centers(0.0, 1.0, ny)
    x = _centers(0.0, 1.0, nx)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")

    def field(amp):
        f = np.zeros_like(X)
        for _ in range(3):
            k = rng.integers(1, 3, 3)
            f += amp * rng.uniform(0.3, 1.0) * np.sin(
                2 * np.pi * (k[0] * X + k[1] * Y + k[2] * Z) + rng.uniform(0, 6.3))
        return f

    if rp == "advection":
        q0 = np.stack([field(1.0)])
        params = kw.pop("params", [0.7, -0.5, 0.4])
    elif rp == "acoustics":
        q0 = np.stack([field(0.5), field(0.5), field(0.5), field(0.5)])
        params = kw.pop("params", [1.3, 2.5])
    else:
        raise ValueError(rp)
    spec = _base(3, [nx, ny, nz], [0.0, 0.0, 0.0], [1.0, 1.0, 1.0], rp, params=params,
                 bc_lower=[bc] * 3, bc_upper=[bc] * 3, **kw)
    spec.update(q0=np.ascontiguousarray(q0), aux=None, t_end=kw.get("t_end", 0.1))
    return spec
