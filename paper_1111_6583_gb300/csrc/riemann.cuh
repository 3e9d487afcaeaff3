// riemann.cuh -- pointwise Riemann solvers, transverse solvers, limiters and
// characteristic projections for the device kernels.
//
// Each solver is a policy struct templated on the working precision R and the
// dimension ND, with compile-time direction DIR (0 = x, 1 = y):
//   solve<DIR>(C, ql, qr, al, ar, W, s, am, ap, ctx)   normal solve: waves W^p,
//       speeds s^p, fluctuations A^-dQ, A^+dQ (Sec. 2, fluctuation form) and a
//       linearisation ctx kept for the transverse solve;
//   trans<DIR>(C, ctx, a, bm, bp)   split a normal fluctuation a into the
//       down-/up-going transverse fluctuations B^-a, B^+a (Sec. 2.1);
//   to_char / from_char   characteristic projection for SharpClaw.
// Formulas: LeVeque, Finite Volume Methods for Hyperbolic Problems (acoustics,
// shallow-water and Euler Roe solvers, Harten-Hyman entropy fix, transverse
// solvers); Einfeldt (HLLE); Bale-LeVeque-Mitran-Rossmanith (f-waves).
#pragma once

#include "claw_common.cuh"

namespace claw {

template <int ND, int DIR>
struct Dirs {
  static constexpr int n = (ND == 1) ? 1 : 1 + DIR;   // normal momentum / velocity
  static constexpr int t = (ND == 1) ? -1 : 2 - DIR;  // tangential component
};

// Precision traits.  FP64 uses IEEE division and square root (parity with
// the FP64 oracle to 1e-12); FP32 uses the hardware approximations (relative
// error ~1e-7, well inside the FP32 tolerance of 1e-5).
template <typename R>
struct FM;
template <>
struct FM<double> {
  __device__ static __forceinline__ double div(double a, double b) { return a / b; }
  __device__ static __forceinline__ double rcp(double a) { return 1.0 / a; }
  __device__ static __forceinline__ double sqrt(double a) { return ::sqrt(a); }
  __device__ static __forceinline__ double rsqrt(double a) { return ::rsqrt(a); }
  __device__ static __forceinline__ double exp(double a) { return ::exp(a); }
};
// FP32 reciprocal: the hardware approximation (PTX rcp.approx.ftz.f32,
// relative error about 2^-23; subnormal inputs and results flush to zero)
__device__ __forceinline__ float rcp_approx(float a) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
  return r;
}
template <>
struct FM<float> {
  // a * (1/b) from the approximate reciprocal: two roundings, no range
  // handling (a zero b gives an infinity, as a zero wave norm does in the
  // limiter, where the zero-wave test decides)
  __device__ static __forceinline__ float div(float a, float b) { return a * rcp_approx(b); }
  __device__ static __forceinline__ float rcp(float a) { return rcp_approx(a); }
  // a rsqrt(a) for a > 0; sqrt(+-0) = +-0 and NaN below zero by selects (no branch)
  __device__ static __forceinline__ float sqrt(float a) {
    const float y = a * rsqrtf(a);
    return a > 0.f ? y : (a == 0.f ? a : __int_as_float(0x7fffffff));
  }
  __device__ static __forceinline__ float rsqrt(float a) { return rsqrtf(a); }
  __device__ static __forceinline__ float exp(float a) { return __expf(a); }
};

template <typename R>
__device__ __forceinline__ R rsq(R x) { return FM<R>::rsqrt(x); }

// Sign tests and maxima on the bit patterns (integer pipe; the FP64 pipe is
// the scarce unit).  gt0(x) == (x > 0) and lt0(x) == (x < 0) for every
// non-NaN x (+0 and -0 are neither); a NaN counts by its sign bit.
__device__ __forceinline__ long long fbits(double x) { return __double_as_longlong(x); }
__device__ __forceinline__ int fbits(float x) { return __float_as_int(x); }
template <typename R>
__device__ __forceinline__ bool gt0(R x) { return fbits(x) > 0; }
template <typename R>
__device__ __forceinline__ bool lt0(R x) {
  return fbits(x) < 0 && (fbits(x) << 1) != 0;
}
// FP32: one float compare each (the FP32 pipes are not scarce); a NaN is
// neither positive nor negative here
__device__ __forceinline__ bool gt0(float x) { return x > 0.f; }
__device__ __forceinline__ bool lt0(float x) { return x < 0.f; }
// x is +0 or -0
__device__ __forceinline__ bool zero_mag(double x) {
  return (fbits(x) & 0x7fffffffffffffffLL) == 0;
}
__device__ __forceinline__ bool zero_mag(float x) { return x == 0.f; }
// larger of two non-negative values (or NaNs with clear sign bit, which win:
// their bit patterns lie above +inf)
template <typename R>
__device__ __forceinline__ R max_nonneg(R a, R b) { return fbits(b) > fbits(a) ? b : a; }
// x is a positive normal finite number
__device__ __forceinline__ bool pos_normal(double x) {
  const long long b = fbits(x);
  return b >= 0x0010000000000000LL && b < 0x7ff0000000000000LL;
}
__device__ __forceinline__ bool pos_normal(float x) {
  const int b = fbits(x);
  return b >= 0x00800000 && b < 0x7f800000;
}

// A^- dQ = sum_p min(s^p,0) W^p,  A^+ dQ = sum_p max(s^p,0) W^p.  NZ(p, k)
// tells which wave components can be non-zero (the rest are structural
// zeros of the solver and are skipped).
struct AllNZ {
  __device__ static constexpr bool f(int, int) { return true; }
};
template <int M, int MW, typename R, class NZ = AllNZ>
__device__ __forceinline__ void split_waves(const R (&W)[MW][M], const R (&s)[MW], R (&am)[M],
                                            R (&ap)[M]) {
#pragma unroll
  for (int k = 0; k < M; ++k) {
    am[k] = R(0);
    ap[k] = R(0);
  }
  if (sizeof(R) == 8 && lt0(s[0]) && gt0(s[MW - 1])) {
    // first family left-going, last right-going (every subsonic state; FP64
    // skips the products with zero, FP32 takes the select form below)
#pragma unroll
    for (int k = 0; k < M; ++k) {
      if (NZ::f(0, k)) am[k] = s[0] * W[0][k];
      if (NZ::f(MW - 1, k)) ap[k] = s[MW - 1] * W[MW - 1][k];
    }
#pragma unroll
    for (int p = 1; p < MW - 1; ++p) {
      const bool neg = lt0(s[p]);
      const R sm = neg ? s[p] : R(0), sp = neg ? R(0) : s[p];
#pragma unroll
      for (int k = 0; k < M; ++k) {
        if (!NZ::f(p, k)) continue;
        am[k] += sm * W[p][k];
        ap[k] += sp * W[p][k];
      }
    }
    return;
  }
#pragma unroll
  for (int p = 0; p < MW; ++p) {
    const R sm = fmin(s[p], R(0)), sp = fmax(s[p], R(0));
#pragma unroll
    for (int k = 0; k < M; ++k) {
      if (!NZ::f(p, k)) continue;
      am[k] += sm * W[p][k];
      ap[k] += sp * W[p][k];
    }
  }
}

// ---------------------------------------------------------------------------
// scalar advection q_t + u q_x + v q_y = 0
// ---------------------------------------------------------------------------
template <typename R, int ND>
struct RpAdvection {
  static constexpr int M = 1, MW = 1, MA = 0, NCTX = 1, NPC = 0;
  template <int DIR>
  struct NZ : AllNZ {};
  static constexpr bool FWAVE = false;
  static constexpr int WALL_X = -1, WALL_Y = -1;
  // the wave is the jump itself: its one component is its strength
  template <int DIR>
  __host__ __device__ static constexpr int strength() { return 0; }
  template <int DIR>
  __device__ static __forceinline__ void wave_of(const MConsts<R>&, int, R al, R (&w)[M]) {
    w[0] = al;
  }
  template <int DIR>
  __device__ static __forceinline__ void solve(const MConsts<R>& C, const R (&ql)[M],
                                               const R (&qr)[M], const R*, const R*,
                                               R (&W)[MW][M], R (&s)[MW], R (&am)[M],
                                               R (&ap)[M], R (&ctx)[NCTX]) {
    const R u = C.p[DIR];
    W[0][0] = qr[0] - ql[0];
    s[0] = u;
    am[0] = fmin(u, R(0)) * W[0][0];
    ap[0] = fmax(u, R(0)) * W[0][0];
    ctx[0] = R(0);
  }
  // physical flux in direction DIR (A^-dQ + A^+dQ of every solve equals the
  // flux jump, so the in-cell total fluctuation is a flux difference)
  template <int DIR>
  __device__ static __forceinline__ void flux(const MConsts<R>& C, const R (&q)[M], const R*,
                                              R (&f)[M]) {
    f[0] = C.p[DIR] * q[0];
  }
  template <int DIR>
  __device__ static __forceinline__ void trans(const MConsts<R>& C, const R (&)[NCTX],
                                               const R (&a)[M], R (&bm)[M], R (&bp)[M]) {
    const R v = C.p[1 - DIR];
    bm[0] = fmin(v, R(0)) * a[0];
    bp[0] = fmax(v, R(0)) * a[0];
  }
  template <int DIR>
  __device__ static __forceinline__ void char_ctx(const MConsts<R>&, const R (&)[M],
                                                  const R (&)[M], R (&ctx)[NCTX]) {
    ctx[0] = R(0);
  }
  template <int DIR>
  __device__ static __forceinline__ void to_char(const MConsts<R>&, const R (&)[NCTX],
                                                 const R (&q)[M], R (&w)[M]) {
    w[0] = q[0];
  }
  template <int DIR>
  __device__ static __forceinline__ void from_char(const MConsts<R>&, const R (&)[NCTX],
                                                   const R (&w)[M], R (&q)[M]) {
    q[0] = w[0];
  }
};

// ---------------------------------------------------------------------------
// linear acoustics (p, u[, v]), constant rho, K: the paper's Table-1 system
// ---------------------------------------------------------------------------
template <typename R, int ND>
struct RpAcoustics {
  static constexpr int M = ND + 1, MW = 2, MA = 0, NCTX = 1, NPC = 0;
  // waves live in the pressure and normal-velocity components
  template <int DIR>
  struct NZ {
    __device__ static constexpr bool f(int, int k) { return k == 0 || k == 1 + DIR; }
  };
  static constexpr bool FWAVE = false;
  // speeds -c < 0 < c (rho, K > 0 are checked on the host)
  static constexpr bool SIGNED_WAVES = true;
  static constexpr int WALL_X = 1, WALL_Y = (ND == 2) ? 2 : -1;
  // W^1 = a1 (-Z, 1), W^2 = a2 (Z, 1) in (p, u_n): the normal velocity
  // component of each wave is its strength
  template <int DIR>
  __host__ __device__ static constexpr int strength() { return Dirs<ND, DIR>::n; }
  // the wave of family p with strength al (normal velocity al)
  template <int DIR>
  __device__ static __forceinline__ void wave_of(const MConsts<R>& C, int p, R al, R (&w)[M]) {
    constexpr int n = Dirs<ND, DIR>::n;
#pragma unroll
    for (int k = 0; k < M; ++k) w[k] = R(0);
    w[0] = (p == 0 ? -C.aco_Z : C.aco_Z) * al;
    w[n] = al;
  }
  template <int DIR>
  __device__ static __forceinline__ void solve(const MConsts<R>& C, const R (&ql)[M],
                                               const R (&qr)[M], const R*, const R*,
                                               R (&W)[MW][M], R (&s)[MW], R (&am)[M],
                                               R (&ap)[M], R (&ctx)[NCTX]) {
    constexpr int n = Dirs<ND, DIR>::n;
    const R Z = C.aco_Z, c = C.aco_c, h = C.aco_h;
    const R dp = qr[0] - ql[0], du = qr[n] - ql[n];
    const R a1 = (Z * du - dp) * h;
    const R a2 = (Z * du + dp) * h;
#pragma unroll
    for (int k = 0; k < M; ++k) {
      W[0][k] = R(0);
      W[1][k] = R(0);
    }
    W[0][0] = -Z * a1;
    W[0][n] = a1;
    W[1][0] = Z * a2;
    W[1][n] = a2;
    s[0] = -c;
    s[1] = c;
#pragma unroll
    for (int k = 0; k < M; ++k) {
      am[k] = -c * W[0][k];
      ap[k] = c * W[1][k];
    }
    ctx[0] = R(0);
  }
  template <int DIR>
  __device__ static __forceinline__ void flux(const MConsts<R>& C, const R (&q)[M], const R*,
                                              R (&f)[M]) {
    constexpr int n = Dirs<ND, DIR>::n;
#pragma unroll
    for (int k = 0; k < M; ++k) f[k] = R(0);
    f[0] = C.p[1] * q[n];
    f[n] = FM<R>::div(q[0], C.p[0]);
  }
  template <int DIR>
  __device__ static __forceinline__ void trans(const MConsts<R>& C, const R (&)[NCTX],
                                               const R (&a)[M], R (&bm)[M], R (&bp)[M]) {
    constexpr int n = Dirs<ND, DIR>::n, t = Dirs<ND, DIR>::t;
    const R Z = C.aco_Z, c = C.aco_c, h = C.aco_h;
    const R b1 = (Z * a[t] - a[0]) * h;
    const R b2 = (Z * a[t] + a[0]) * h;
    bm[0] = c * Z * b1;
    bm[n] = R(0);
    bm[t] = -c * b1;
    bp[0] = c * Z * b2;
    bp[n] = R(0);
    bp[t] = c * b2;
  }
  template <int DIR>
  __device__ static __forceinline__ void char_ctx(const MConsts<R>&, const R (&)[M],
                                                  const R (&)[M], R (&ctx)[NCTX]) {
    ctx[0] = R(0);
  }
  template <int DIR>
  __device__ static __forceinline__ void to_char(const MConsts<R>& C, const R (&)[NCTX],
                                                 const R (&q)[M], R (&w)[M]) {
    constexpr int n = Dirs<ND, DIR>::n, t = Dirs<ND, DIR>::t;
    const R Z = C.aco_Z, h = C.aco_h;
    w[0] = (Z * q[n] - q[0]) * h;
    w[1] = (Z * q[n] + q[0]) * h;
    if (ND == 2) w[ND] = q[t < 0 ? 0 : t];
  }
  template <int DIR>
  __device__ static __forceinline__ void from_char(const MConsts<R>& C, const R (&)[NCTX],
                                                   const R (&w)[M], R (&q)[M]) {
    constexpr int n = Dirs<ND, DIR>::n, t = Dirs<ND, DIR>::t;
    const R Z = C.aco_Z;
    q[0] = Z * (w[1] - w[0]);
    q[n] = w[0] + w[1];
    if (ND == 2) q[t < 0 ? 0 : t] = w[ND];
  }
};

// ---------------------------------------------------------------------------
// shallow water (h, hu[, hv]) with the Roe solver and Harten-Hyman fix
// ---------------------------------------------------------------------------
template <typename R, int ND>
struct RpSW {
  static constexpr int M = ND + 1, MW = ND + 1, MA = 0, NCTX = 4;  // ctx: un, ut, c, 1/(2c)
  static constexpr int NPC = 2;  // per-cell prep: 1/sqrt(h), g h^3
  static constexpr bool FWAVE = false;
  static constexpr int WALL_X = 1, WALL_Y = (ND == 2) ? 2 : -1;
  // the shear wave (2D) has only the tangential component
  template <int DIR>
  struct NZ {
    __device__ static constexpr bool f(int p, int k) {
      return ND == 1 || p != 1 || k == 2 - DIR;
    }
  };
  __device__ static __forceinline__ void cell_pc(const MConsts<R>& C, const R (&q)[M],
                                                 R (&pc)[NPC]) {
    pc[0] = rsq(q[0]);
    pc[1] = C.g * (q[0] * q[0] * q[0]);
  }

  // Roe averages from the cells' 1/sqrt(h): u^ = (hu_l/sqrt(h_l) +
  // hu_r/sqrt(h_r)) / (sqrt(h_l) + sqrt(h_r)); c^ = sqrt(g h^) and 1/(2 c^)
  // from one reciprocal square root.
  template <int DIR>
  __device__ static __forceinline__ void roe_pc(const MConsts<R>& C, const R (&ql)[M],
                                                const R (&qr)[M], R il, R ir, R (&x)[NCTX]) {
    constexpr int n = Dirs<ND, DIR>::n, t = Dirs<ND, DIR>::t;
    const R hl = ql[0], hr = qr[0];
    const R iden = FM<R>::rcp(hl * il + hr * ir);   // 1/(sqrt(hl)+sqrt(hr))
    x[0] = (ql[n] * il + qr[n] * ir) * iden;     // sqrt(h) u = hu/sqrt(h)
    x[1] = (t >= 0) ? (ql[t < 0 ? 0 : t] * il + qr[t < 0 ? 0 : t] * ir) * iden : R(0);
    const R gh = C.g * (R(0.5) * (hl + hr));
    const R rc = rsq(gh);
    x[2] = gh * rc;
    x[3] = R(0.5) * rc;
  }
  template <int DIR>
  __device__ static __forceinline__ void roe(const MConsts<R>& C, const R (&ql)[M],
                                             const R (&qr)[M], R (&x)[NCTX]) {
    roe_pc<DIR>(C, ql, qr, rsq(ql[0]), rsq(qr[0]), x);
  }
  // the sign tests below with g h^3 given (gh3 = C.g * (h * h * h)); the
  // comparisons of non-negative values run on their bit patterns
  __device__ static __forceinline__ bool minus_neg_c(R h, R hu, R gh3) {
    return gt0(h) && (lt0(hu) || fbits(hu * hu) < fbits(gh3));
  }
  __device__ static __forceinline__ bool plus_pos_c(R h, R hu, R gh3) {
    return gt0(h) && (gt0(hu) || fbits(hu * hu) < fbits(gh3));
  }

  // eigen-coefficients of d in the frame (normal a, tangential b) at (un, ut, c)
  template <int A, int B>
  __device__ static __forceinline__ void coef(R un, R ut, R c, R i2c, const R (&d)[M],
                                              R (&al)[MW]) {
    al[0] = ((un + c) * d[0] - d[A]) * i2c;
    al[MW - 1] = (d[A] - (un - c) * d[0]) * i2c;
    if (B >= 0) al[1] = d[B < 0 ? 0 : B] - ut * d[0];
  }
  // sum_p k_p r_p in the frame (normal a, tangential b)
  template <int A, int B>
  __device__ static __forceinline__ void assemble(R un, R ut, R c, const R (&k)[MW], R (&o)[M]) {
    const R k0 = k[0], kl = k[MW - 1];
    o[0] = k0 + kl;
    o[A] = k0 * (un - c) + kl * (un + c);
    if (B >= 0) o[B < 0 ? 0 : B] = (k0 + kl) * ut + k[1];
  }

  template <int DIR>
  __device__ static __forceinline__ R sonic(const MConsts<R>& C, R h, R hu, int plus) {
    const R c = FM<R>::sqrt(C.g * h);
    const R u = FM<R>::div(hu, h);
    return plus ? u + c : u - c;
  }
  // Signs of u -/+ c for a state (h, hu) without square roots or divisions:
  // with h > 0, u - c < 0  <=>  hu < 0 or hu^2 < g h^3, and u + c > 0  <=>
  // hu > 0 or hu^2 < g h^3.  A state with h <= 0 satisfies none of them.
  __device__ static __forceinline__ bool minus_neg(const MConsts<R>& C, R h, R hu) {
    return h > R(0) && (hu < R(0) || hu * hu < C.g * (h * h * h));
  }
  __device__ static __forceinline__ bool minus_pos(const MConsts<R>& C, R h, R hu) {
    return gt0(h) && gt0(hu) && fbits(hu * hu) > fbits(C.g * (h * h * h));
  }
  __device__ static __forceinline__ bool plus_neg(const MConsts<R>& C, R h, R hu) {
    return gt0(h) && lt0(hu) && fbits(hu * hu) > fbits(C.g * (h * h * h));
  }
  __device__ static __forceinline__ bool plus_pos(const MConsts<R>& C, R h, R hu) {
    return h > R(0) && (hu > R(0) || hu * hu < C.g * (h * h * h));
  }

  template <int DIR>
  __device__ static __forceinline__ void solve(const MConsts<R>& C, const R (&ql)[M],
                                               const R (&qr)[M], const R* al, const R* ar,
                                               R (&W)[MW][M], R (&s)[MW], R (&am)[M],
                                               R (&ap)[M], R (&x)[NCTX]) {
    R pl[NPC], pr[NPC];
    cell_pc(C, ql, pl);
    cell_pc(C, qr, pr);
    solve_pc<DIR>(C, ql, qr, pl, pr, W, s, am, ap, x);
  }
  // the normal solve with the cells' prep (1/sqrt(h), g h^3) given
  template <int DIR>
  __device__ static __forceinline__ void solve_pc(const MConsts<R>& C, const R (&ql)[M],
                                                  const R (&qr)[M], const R (&pl)[NPC],
                                                  const R (&pr)[NPC], R (&W)[MW][M], R (&s)[MW],
                                                  R (&am)[M], R (&ap)[M], R (&x)[NCTX]) {
    constexpr int n = Dirs<ND, DIR>::n, t = Dirs<ND, DIR>::t;
    roe_pc<DIR>(C, ql, qr, pl[0], pr[0], x);
    const R un = x[0], ut = x[1], c = x[2];
    const R i2c = x[3];
    R d[M], al[MW];
#pragma unroll
    for (int k = 0; k < M; ++k) d[k] = qr[k] - ql[k];
    coef<n, t>(un, ut, c, i2c, d, al);
#pragma unroll
    for (int p = 0; p < MW; ++p)
#pragma unroll
      for (int k = 0; k < M; ++k) W[p][k] = R(0);
    W[0][0] = al[0];
    W[0][n] = al[0] * (un - c);
    W[MW - 1][0] = al[MW - 1];
    W[MW - 1][n] = al[MW - 1] * (un + c);
    if (t >= 0) {
      W[0][t < 0 ? 0 : t] = al[0] * ut;
      W[1][t < 0 ? 0 : t] = al[1];
      W[MW - 1][t < 0 ? 0 : t] = al[MW - 1] * ut;
      s[1] = un;
    }
    s[0] = un - c;
    s[MW - 1] = un + c;
    if (C.entropy_fix) {
      // first family: transonic when u-c < 0 at Q_l and > 0 at Q_l + W^1
      const R hm = ql[0] + W[0][0], hum = ql[n] + W[0][n];
      if (minus_neg_c(ql[0], ql[n], pl[1]) && minus_pos(C, hm, hum)) {
        const R lamL = sonic<DIR>(C, ql[0], ql[n], 0);
        const R lamR = sonic<DIR>(C, hm, hum, 0);
        if (lamL < R(0) && lamR > R(0)) {
          const R beta = FM<R>::div(lamR - s[0], lamR - lamL);
#pragma unroll
          for (int k = 0; k < M; ++k) {
            R tot = R(0);
#pragma unroll
            for (int p = 0; p < MW; ++p) tot += s[p] * W[p][k];
            am[k] = beta * lamL * W[0][k];
            ap[k] = tot - am[k];
          }
          return;
        }
      }
      // last family: u+c < 0 at Q_r - W^last and > 0 at Q_r
      const R hm2 = qr[0] - W[MW - 1][0], hum2 = qr[n] - W[MW - 1][n];
      if (plus_pos_c(qr[0], qr[n], pr[1]) && plus_neg(C, hm2, hum2)) {
        const R muL = sonic<DIR>(C, hm2, hum2, 1);
        const R muR = sonic<DIR>(C, qr[0], qr[n], 1);
        if (muL < R(0) && muR > R(0)) {
          const R beta = FM<R>::div(muR - s[MW - 1], muR - muL);
#pragma unroll
          for (int k = 0; k < M; ++k) {
            R tot = R(0);
#pragma unroll
            for (int p = 0; p < MW; ++p) tot += s[p] * W[p][k];
            ap[k] = (R(1) - beta) * muR * W[MW - 1][k];
            am[k] = tot - ap[k];
          }
          return;
        }
      }
    }
    split_waves<M, MW, R, NZ<DIR>>(W, s, am, ap);
  }

  template <int DIR>
  __device__ static __forceinline__ void flux(const MConsts<R>& C, const R (&q)[M], const R*,
                                              R (&f)[M]) {
    constexpr int n = Dirs<ND, DIR>::n, t = Dirs<ND, DIR>::t;
    const R u = FM<R>::div(q[n], q[0]);
    f[0] = q[n];
    f[n] = q[n] * u + R(0.5) * C.g * (q[0] * q[0]);
    if (t >= 0) f[t < 0 ? 0 : t] = q[t < 0 ? 0 : t] * u;
  }
  template <int DIR>
  __device__ static __forceinline__ void trans(const MConsts<R>& C, const R (&x)[NCTX],
                                               const R (&a)[M], R (&bm)[M], R (&bp)[M]) {
    constexpr int n = Dirs<ND, DIR>::n, t = Dirs<ND, DIR>::t;
    // transverse frame: normal = t (speed ut), tangential = n (speed un)
    const R un = x[0], ut = x[1], c = x[2];
    const R i2c = x[3];
    R be[MW], km[MW], kp[MW];
    coef<t, n>(ut, un, c, i2c, a, be);
    const R lm = ut - c, lp = ut + c;
    if (ND == 2 && lt0(lm) && gt0(lp)) {
      // subsonic in the transverse direction: the first family goes down,
      // the last up, the shear wave by the sign of ut
      const R k0 = lm * be[0], k2 = lp * be[MW - 1];
      const R k1 = ut * be[1];
      const bool neg = lt0(ut);
      constexpr int tt = t < 0 ? 0 : t;
      bm[0] = k0;
      bm[tt] = k0 * lm;
      bm[n] = k0 * un + (neg ? k1 : R(0));
      bp[0] = k2;
      bp[tt] = k2 * lp;
      bp[n] = k2 * un + (neg ? R(0) : k1);
      return;
    }
    const R lam[3] = {lm, ut, lp};
#pragma unroll
    for (int p = 0; p < MW; ++p) {
      km[p] = fmin(lam[p == MW - 1 ? 2 : p], R(0)) * be[p];
      kp[p] = fmax(lam[p == MW - 1 ? 2 : p], R(0)) * be[p];
    }
    assemble<t, n>(ut, un, c, km, bm);
    assemble<t, n>(ut, un, c, kp, bp);
  }

  template <int DIR>
  __device__ static __forceinline__ void char_ctx(const MConsts<R>& C, const R (&ql)[M],
                                                  const R (&qr)[M], R (&x)[NCTX]) {
    roe<DIR>(C, ql, qr, x);
  }
  template <int DIR>
  __device__ static __forceinline__ void to_char(const MConsts<R>&, const R (&x)[NCTX],
                                                 const R (&q)[M], R (&w)[M]) {
    constexpr int n = Dirs<ND, DIR>::n, t = Dirs<ND, DIR>::t;
    coef<n, t>(x[0], x[1], x[2], x[3], q, w);
  }
  template <int DIR>
  __device__ static __forceinline__ void from_char(const MConsts<R>&, const R (&x)[NCTX],
                                                   const R (&w)[M], R (&q)[M]) {
    constexpr int n = Dirs<ND, DIR>::n, t = Dirs<ND, DIR>::t;
    assemble<n, t>(x[0], x[1], x[2], w, q);
  }
};

// ---------------------------------------------------------------------------
// Euler equations (rho, rho u[, rho v], E), ideal gas; Roe and HLLE solvers
// ---------------------------------------------------------------------------
template <typename R, int ND>
struct EulerBase {
  static constexpr int M = ND + 2, E = ND + 1, NCTX = 6;  // ctx: un, ut, H, c, 1/c^2, 1/(2c)

  template <int DIR>
  __device__ static __forceinline__ R pressure(const MConsts<R>& C, const R (&q)[M], R irho) {
    constexpr int n = Dirs<ND, DIR>::n, t = Dirs<ND, DIR>::t;
    const R ke = (t >= 0) ? q[n] * q[n] + q[t < 0 ? 0 : t] * q[t < 0 ? 0 : t] : q[n] * q[n];
    return C.gm1 * (q[E] - R(0.5) * ke * irho);
  }

  // Roe averages; also returns the two pressures
  template <int DIR>
  __device__ static __forceinline__ void roe(const MConsts<R>& C, const R (&ql)[M],
                                             const R (&qr)[M], R (&x)[NCTX], R& pl, R& pr) {
    constexpr int n = Dirs<ND, DIR>::n, t = Dirs<ND, DIR>::t;
    const R il = rsq(ql[0]), ir = rsq(qr[0]);  // 1/sqrt(rho)
    const R irl = il * il, irr = ir * ir;      // 1/rho
    pl = pressure<DIR>(C, ql, irl);
    pr = pressure<DIR>(C, qr, irr);
    const R sl = ql[0] * il, sr = qr[0] * ir;  // sqrt(rho)
    const R iden = FM<R>::rcp(sl + sr);
    x[0] = (ql[n] * il + qr[n] * ir) * iden;
    x[1] = (t >= 0) ? (ql[t < 0 ? 0 : t] * il + qr[t < 0 ? 0 : t] * ir) * iden : R(0);
    x[2] = ((ql[E] + pl) * il + (qr[E] + pr) * ir) * iden;  // sqrt(rho) H = (E+p)/sqrt(rho)
    const R c2 = C.gm1 * (x[2] - R(0.5) * (x[0] * x[0] + x[1] * x[1]));
    // c, 1/c^2 and 1/(2c) from one reciprocal square root
    const R rc = rsq(c2);
    x[3] = c2 * rc;
    x[4] = rc * rc;
    x[5] = R(0.5) * rc;
  }

  // eigen-coefficients of d in the frame (normal a, tangential b)
  template <int A, int B>
  __device__ static __forceinline__ void coef(const MConsts<R>& C, R un, R ut, R H, R c, R ic2,
                                              R i2c, const R (&d)[M], R (&al)[M]) {
    const R ash = (B >= 0) ? d[B < 0 ? 0 : B] - ut * d[0] : R(0);
    const R a2 = C.gm1 * ((H - un * un) * d[0] + un * d[A] - d[E] + ut * ash) * ic2;
    const R a4 = (d[A] + (c - un) * d[0] - c * a2) * i2c;
    al[0] = d[0] - a2 - a4;
    al[1] = a2;
    if (B >= 0) al[2] = ash;
    al[M - 1] = a4;
  }
  // sum_p k_p r_p in the frame (normal a, tangential b)
  template <int A, int B>
  __device__ static __forceinline__ void assemble(R un, R ut, R H, R c, const R (&k)[M],
                                                  R (&o)[M]) {
    const R k0 = k[0], k1 = k[1], kl = k[M - 1];
    const R ksh = (B >= 0) ? k[2] : R(0);
    const R s3 = k0 + k1 + kl;
    o[0] = s3;
    o[A] = k0 * (un - c) + k1 * un + kl * (un + c);
    if (B >= 0) o[B < 0 ? 0 : B] = s3 * ut + ksh;
    o[E] = k0 * (H - un * c) + k1 * (R(0.5) * (un * un + ut * ut)) + ksh * ut + kl * (H + un * c);
  }

  template <int DIR>
  __device__ static __forceinline__ void flux(const MConsts<R>& C, const R (&q)[M], const R*,
                                              R (&f)[M]) {
    constexpr int n = Dirs<ND, DIR>::n, t = Dirs<ND, DIR>::t;
    const R ir = FM<R>::rcp(q[0]);
    const R p = pressure<DIR>(C, q, ir);
    const R u = q[n] * ir;
    f[0] = q[n];
    f[n] = q[n] * u + p;
    if (t >= 0) f[t < 0 ? 0 : t] = q[t < 0 ? 0 : t] * u;
    f[E] = u * (q[E] + p);
  }
  template <int DIR>
  __device__ static __forceinline__ void trans(const MConsts<R>& C, const R (&x)[NCTX],
                                               const R (&a)[M], R (&bm)[M], R (&bp)[M]) {
    constexpr int n = Dirs<ND, DIR>::n, t = Dirs<ND, DIR>::t;
    const R un = x[0], ut = x[1], H = x[2], c = x[3];
    R be[M], km[M], kp[M];
    coef<t, n>(C, ut, un, H, c, x[4], x[5], a, be);
#pragma unroll
    for (int p = 0; p < M; ++p) {
      const R lam = (p == 0) ? ut - c : (p == M - 1 ? ut + c : ut);
      km[p] = fmin(lam, R(0)) * be[p];
      kp[p] = fmax(lam, R(0)) * be[p];
    }
    assemble<t, n>(ut, un, H, c, km, bm);
    assemble<t, n>(ut, un, H, c, kp, bp);
  }

  template <int DIR>
  __device__ static __forceinline__ void char_ctx(const MConsts<R>& C, const R (&ql)[M],
                                                  const R (&qr)[M], R (&x)[NCTX]) {
    R pl, pr;
    roe<DIR>(C, ql, qr, x, pl, pr);
  }
  template <int DIR>
  __device__ static __forceinline__ void to_char(const MConsts<R>& C, const R (&x)[NCTX],
                                                 const R (&q)[M], R (&w)[M]) {
    constexpr int n = Dirs<ND, DIR>::n, t = Dirs<ND, DIR>::t;
    coef<n, t>(C, x[0], x[1], x[2], x[3], x[4], x[5], q, w);
  }
  template <int DIR>
  __device__ static __forceinline__ void from_char(const MConsts<R>&, const R (&x)[NCTX],
                                                   const R (&w)[M], R (&q)[M]) {
    constexpr int n = Dirs<ND, DIR>::n, t = Dirs<ND, DIR>::t;
    assemble<n, t>(x[0], x[1], x[2], x[3], w, q);
  }
};

template <typename R, int ND>
struct RpEulerRoe : EulerBase<R, ND> {
  using B = EulerBase<R, ND>;
  static constexpr int M = B::M, MW = B::M, MA = 0, NCTX = B::NCTX, E = B::E, NPC = 0;
  // the shear wave (2D) lives in the tangential momentum and the energy
  template <int DIR>
  struct NZ {
    __device__ static constexpr bool f(int p, int k) {
      return ND == 1 || p != 2 || k == 2 - DIR || k == E;
    }
  };
  static constexpr bool FWAVE = false;
  static constexpr int WALL_X = 1, WALL_Y = (ND == 2) ? 2 : -1;

  // Signs of u -/+ c without square roots or divisions: with rho > 0 and
  // X = rho E - (m_n^2 + m_t^2)/2 > 0 (so p > 0), rho^2 c^2 = gamma (gamma-1) X
  // and u - c < 0 <=> m_n < 0 or m_n^2 < gamma (gamma-1) X.
  template <int DIR>
  __device__ static __forceinline__ void sign_terms(const MConsts<R>& C, const R (&q)[M], R& mn,
                                                    R& rc2, bool& phys) {
    constexpr int n = Dirs<ND, DIR>::n, t = Dirs<ND, DIR>::t;
    const R ke = (t >= 0) ? q[n] * q[n] + q[t < 0 ? 0 : t] * q[t < 0 ? 0 : t] : q[n] * q[n];
    const R X = q[0] * q[E] - R(0.5) * ke;
    mn = q[n];
    rc2 = C.gamma * C.gm1 * X;
    phys = gt0(q[0]) && gt0(X);
  }
  // (comparisons of the non-negative m^2 and rho^2 c^2 on their bit patterns)
  template <int DIR>
  __device__ static __forceinline__ bool minus_neg(const MConsts<R>& C, const R (&q)[M]) {
    R m, r;
    bool ph;
    sign_terms<DIR>(C, q, m, r, ph);
    return ph && (lt0(m) || fbits(m * m) < fbits(r));
  }
  template <int DIR>
  __device__ static __forceinline__ bool minus_pos(const MConsts<R>& C, const R (&q)[M]) {
    R m, r;
    bool ph;
    sign_terms<DIR>(C, q, m, r, ph);
    return ph && gt0(m) && fbits(m * m) > fbits(r);
  }
  template <int DIR>
  __device__ static __forceinline__ bool plus_neg(const MConsts<R>& C, const R (&q)[M]) {
    R m, r;
    bool ph;
    sign_terms<DIR>(C, q, m, r, ph);
    return ph && lt0(m) && fbits(m * m) > fbits(r);
  }
  template <int DIR>
  __device__ static __forceinline__ bool plus_pos(const MConsts<R>& C, const R (&q)[M]) {
    R m, r;
    bool ph;
    sign_terms<DIR>(C, q, m, r, ph);
    return ph && (gt0(m) || fbits(m * m) < fbits(r));
  }

  template <int DIR>
  __device__ static __forceinline__ R sonic(const MConsts<R>& C, const R (&q)[M], int plus) {
    constexpr int n = Dirs<ND, DIR>::n;
    const R ir = FM<R>::rcp(q[0]);
    const R p = B::template pressure<DIR>(C, q, ir);
    const R c = FM<R>::sqrt(C.gamma * p * ir);
    const R u = q[n] * ir;
    return plus ? u + c : u - c;
  }

  template <int DIR>
  __device__ static __forceinline__ void solve(const MConsts<R>& C, const R (&ql)[M],
                                               const R (&qr)[M], const R*, const R*,
                                               R (&W)[MW][M], R (&s)[MW], R (&am)[M],
                                               R (&ap)[M], R (&x)[NCTX]) {
    constexpr int n = Dirs<ND, DIR>::n, t = Dirs<ND, DIR>::t;
    R pl, pr;
    B::template roe<DIR>(C, ql, qr, x, pl, pr);
    const R un = x[0], ut = x[1], H = x[2], c = x[3];
    R d[M], al[M];
#pragma unroll
    for (int k = 0; k < M; ++k) d[k] = qr[k] - ql[k];
    B::template coef<n, t>(C, un, ut, H, c, x[4], x[5], d, al);
#pragma unroll
    for (int p = 0; p < MW; ++p)
#pragma unroll
      for (int k = 0; k < M; ++k) W[p][k] = R(0);
    // (un - c), entropy, [shear], (un + c)
    W[0][0] = al[0];
    W[0][n] = al[0] * (un - c);
    W[0][E] = al[0] * (H - un * c);
    W[1][0] = al[1];
    W[1][n] = al[1] * un;
    W[1][E] = al[1] * (R(0.5) * (un * un + ut * ut));
    W[M - 1][0] = al[M - 1];
    W[M - 1][n] = al[M - 1] * (un + c);
    W[M - 1][E] = al[M - 1] * (H + un * c);
    if (t >= 0) {
      constexpr int tt = t < 0 ? 0 : t;
      W[0][tt] = al[0] * ut;
      W[1][tt] = al[1] * ut;
      W[2][tt] = al[2];
      W[2][E] = al[2] * ut;
      W[M - 1][tt] = al[M - 1] * ut;
      s[2] = un;
    }
    s[0] = un - c;
    s[1] = un;
    s[M - 1] = un + c;
    if (C.entropy_fix) {
      R qm[M];
#pragma unroll
      for (int k = 0; k < M; ++k) qm[k] = ql[k] + W[0][k];
      if (minus_neg<DIR>(C, ql) && minus_pos<DIR>(C, qm)) {
        const R lamL = sonic<DIR>(C, ql, 0);
        const R lamR = sonic<DIR>(C, qm, 0);
        if (lamL < R(0) && lamR > R(0)) {
          const R beta = FM<R>::div(lamR - s[0], lamR - lamL);
#pragma unroll
          for (int k = 0; k < M; ++k) {
            R tot = R(0);
#pragma unroll
            for (int p = 0; p < MW; ++p) tot += s[p] * W[p][k];
            am[k] = beta * lamL * W[0][k];
            ap[k] = tot - am[k];
          }
          return;
        }
      }
#pragma unroll
      for (int k = 0; k < M; ++k) qm[k] = qr[k] - W[M - 1][k];
      if (plus_neg<DIR>(C, qm) && plus_pos<DIR>(C, qr)) {
        const R muL = sonic<DIR>(C, qm, 1);
        const R muR = sonic<DIR>(C, qr, 1);
        if (muL < R(0) && muR > R(0)) {
          const R beta = FM<R>::div(muR - s[M - 1], muR - muL);
#pragma unroll
          for (int k = 0; k < M; ++k) {
            R tot = R(0);
#pragma unroll
            for (int p = 0; p < MW; ++p) tot += s[p] * W[p][k];
            ap[k] = (R(1) - beta) * muR * W[M - 1][k];
            am[k] = tot - ap[k];
          }
          return;
        }
      }
    }
    split_waves<M, MW, R, NZ<DIR>>(W, s, am, ap);
  }
};

template <typename R, int ND>
struct RpEulerHLLE : EulerBase<R, ND> {
  using B = EulerBase<R, ND>;
  static constexpr int M = B::M, MW = 2, MA = 0, NCTX = B::NCTX, E = B::E, NPC = 0;
  template <int DIR>
  struct NZ : AllNZ {};
  static constexpr bool FWAVE = false;
  static constexpr int WALL_X = 1, WALL_Y = (ND == 2) ? 2 : -1;

  template <int DIR>
  __device__ static __forceinline__ void flux_p(const R (&q)[M], R p, R (&f)[M]) {
    constexpr int n = Dirs<ND, DIR>::n, t = Dirs<ND, DIR>::t;
    const R u = FM<R>::div(q[n], q[0]);
    f[0] = q[n];
    f[n] = q[n] * u + p;
    if (t >= 0) f[t < 0 ? 0 : t] = q[t < 0 ? 0 : t] * u;
    f[E] = u * (q[E] + p);
  }

  template <int DIR>
  __device__ static __forceinline__ void solve(const MConsts<R>& C, const R (&ql)[M],
                                               const R (&qr)[M], const R*, const R*,
                                               R (&W)[MW][M], R (&s)[MW], R (&am)[M],
                                               R (&ap)[M], R (&x)[NCTX]) {
    constexpr int n = Dirs<ND, DIR>::n;
    R pl, pr;
    B::template roe<DIR>(C, ql, qr, x, pl, pr);
    const R cl = FM<R>::sqrt(C.gamma * FM<R>::div(pl, ql[0])),
            cr = FM<R>::sqrt(C.gamma * FM<R>::div(pr, qr[0]));
    const R s1 = fmin(FM<R>::div(ql[n], ql[0]) - cl, x[0] - x[3]);
    const R s2 = fmax(FM<R>::div(qr[n], qr[0]) + cr, x[0] + x[3]);
    R fl[M], fr[M];
    flux_p<DIR>(ql, pl, fl);
    flux_p<DIR>(qr, pr, fr);
    const R iden = FM<R>::rcp(s1 - s2);
#pragma unroll
    for (int k = 0; k < M; ++k) {
      const R qs = (fr[k] - fl[k] - s2 * qr[k] + s1 * ql[k]) * iden;
      W[0][k] = qs - ql[k];
      W[1][k] = qr[k] - qs;
    }
    s[0] = s1;
    s[1] = s2;
    split_waves<M, MW, R>(W, s, am, ap);
  }
};

// ---------------------------------------------------------------------------
// nonlinear elasticity / p-system (eps, rho u) with f-waves, aux (rho, K),
// sigma(eps) = exp(K eps) - 1 (Sec. 7.3 constitutive law, shifted to sigma(0)=0)
// ---------------------------------------------------------------------------
// Nonlinear elasticity / p-system with f-waves (Sec. 7.3; Bale-LeVeque-
// Mitran-Rossmanith f-wave splitting): q = (eps, m_x[, m_y]), aux (rho, K) per
// cell, sigma = exp(K eps) - 1, normal flux (-m_n/rho, -sigma) in the
// (eps, m_n) components and none in the tangential momentum.  Each side uses
// its own impedance Z = rho c, c = sqrt(K exp(K eps) / rho).  In 2D only the
// normal solves exist (SharpClaw), so there is no transverse solver.
template <typename R, int ND>
struct RpElasticity {
  static constexpr int M = ND + 1, MW = 2, MA = 2, NCTX = 1, NPC = 0;
  // f-waves live in the strain and normal-momentum components
  template <int DIR>
  struct NZ {
    __device__ static constexpr bool f(int, int k) { return k == 0 || k == (ND == 1 ? 1 : 1 + DIR); }
  };
  static constexpr bool FWAVE = true;
  // s^1 = -c_l < 0 < c_r = s^2 for every state (c = sqrt(K e^(K eps) / rho) > 0)
  static constexpr bool SIGNED_WAVES = true;
  static constexpr int WALL_X = 1, WALL_Y = (ND == 2) ? 2 : -1;
  template <int DIR>
  __device__ static __forceinline__ void solve(const MConsts<R>&, const R (&ql)[M],
                                               const R (&qr)[M], const R* al, const R* ar,
                                               R (&W)[MW][M], R (&s)[MW], R (&am)[M],
                                               R (&ap)[M], R (&ctx)[NCTX]) {
    constexpr int n = (ND == 1) ? 1 : 1 + DIR;
    const R rl = al[0], Kl = al[1], rr = ar[0], Kr = ar[1];
    const R el = FM<R>::exp(Kl * ql[0]), er = FM<R>::exp(Kr * qr[0]);
    const R irl = FM<R>::rcp(rl), irr = FM<R>::rcp(rr);
    const R cl = FM<R>::sqrt(Kl * el * irl), cr = FM<R>::sqrt(Kr * er * irr);
    const R Zl = rl * cl, Zr = rr * cr;
    const R d1 = ql[n] * irl - qr[n] * irr;  // jump of -u_n
    const R d2 = el - er;                    // jump of -sigma
    const R iz = FM<R>::rcp(Zl + Zr);
    const R b1 = (Zr * d1 + d2) * iz;
    const R b2 = (Zl * d1 - d2) * iz;
#pragma unroll
    for (int p = 0; p < MW; ++p)
#pragma unroll
      for (int k = 0; k < M; ++k) W[p][k] = R(0);
    W[0][0] = b1;
    W[0][n] = b1 * Zl;
    W[1][0] = b2;
    W[1][n] = -b2 * Zr;
    s[0] = -cl;
    s[1] = cr;
    // f-wave split by the sign of the speed (c > 0 on both sides)
#pragma unroll
    for (int k = 0; k < M; ++k) {
      am[k] = R(0);
      ap[k] = R(0);
    }
#pragma unroll
    for (int p = 0; p < MW; ++p)
#pragma unroll
      for (int k = 0; k < M; ++k) {
        if (s[p] < R(0)) am[k] += W[p][k];
        else if (s[p] > R(0)) ap[k] += W[p][k];
        else {
          am[k] += R(0.5) * W[p][k];
          ap[k] += R(0.5) * W[p][k];
        }
      }
    ctx[0] = R(0);
  }
  template <int DIR>
  __device__ static __forceinline__ void flux(const MConsts<R>&, const R (&q)[M], const R* a,
                                              R (&f)[M]) {
    constexpr int n = (ND == 1) ? 1 : 1 + DIR;
#pragma unroll
    for (int k = 0; k < M; ++k) f[k] = R(0);
    f[0] = -FM<R>::div(q[n], a[0]);
    f[n] = R(1) - FM<R>::exp(a[1] * q[0]);
  }
  template <int DIR>
  __device__ static __forceinline__ void trans(const MConsts<R>&, const R (&)[NCTX],
                                               const R (&)[M], R (&bm)[M], R (&bp)[M]) {
#pragma unroll
    for (int k = 0; k < M; ++k) bm[k] = bp[k] = R(0);
  }
  template <int DIR>
  __device__ static __forceinline__ void char_ctx(const MConsts<R>&, const R (&)[M],
                                                  const R (&)[M], R (&ctx)[NCTX]) {
    ctx[0] = R(0);
  }
  template <int DIR>
  __device__ static __forceinline__ void to_char(const MConsts<R>&, const R (&)[NCTX],
                                                 const R (&q)[M], R (&w)[M]) {
#pragma unroll
    for (int k = 0; k < M; ++k) w[k] = q[k];
  }
  template <int DIR>
  __device__ static __forceinline__ void from_char(const MConsts<R>&, const R (&)[NCTX],
                                                   const R (&w)[M], R (&q)[M]) {
#pragma unroll
    for (int k = 0; k < M; ++k) q[k] = w[k];
  }
};

// ---------------------------------------------------------------------------
// linear acoustics in a varying medium: aux (rho, c) per cell (LeVeque FVM
// book, heterogeneous media).  The left-going wave carries the left cell's
// impedance and speed, the right-going one the right cell's; the transverse
// split of a fluctuation held by a cell solves the transverse Riemann
// problems with its neighbours below and above (TRANS_AUX: it needs their
// media, so 2D classic steps with this solver run the per-face path).
// ---------------------------------------------------------------------------
template <typename R, int ND>
struct RpAcousticsVC {
  static constexpr int M = ND + 1, MW = 2, MA = 2, NCTX = 1, NPC = 0;
  static constexpr bool FWAVE = false, TRANS_AUX = true;
  static constexpr int WALL_X = 1, WALL_Y = (ND == 2) ? 2 : -1;
  template <int DIR>
  struct NZ {
    __device__ static constexpr bool f(int, int k) { return k == 0 || k == 1 + DIR; }
  };
  template <int DIR>
  __device__ static __forceinline__ void solve(const MConsts<R>&, const R (&ql)[M],
                                               const R (&qr)[M], const R* al, const R* ar,
                                               R (&W)[MW][M], R (&s)[MW], R (&am)[M],
                                               R (&ap)[M], R (&ctx)[NCTX]) {
    constexpr int n = Dirs<ND, DIR>::n;
    const R Zl = al[0] * al[1], Zr = ar[0] * ar[1];
    const R dp = qr[0] - ql[0], du = qr[n] - ql[n];
    const R iz = FM<R>::rcp(Zl + Zr);
    const R a1 = (-dp + Zr * du) * iz;
    const R a2 = (dp + Zl * du) * iz;
#pragma unroll
    for (int k = 0; k < M; ++k) W[0][k] = W[1][k] = R(0);
    W[0][0] = -a1 * Zl;
    W[0][n] = a1;
    W[1][0] = a2 * Zr;
    W[1][n] = a2;
    s[0] = -al[1];
    s[1] = ar[1];
#pragma unroll
    for (int k = 0; k < M; ++k) {
      am[k] = s[0] * W[0][k];
      ap[k] = s[1] * W[1][k];
    }
    ctx[0] = R(0);
  }
  // flux (rho c^2 u_n, p / rho) in the (p, u_n) components with one cell's medium
  template <int DIR>
  __device__ static __forceinline__ void flux(const MConsts<R>&, const R (&q)[M], const R* a,
                                              R (&f)[M]) {
    constexpr int n = Dirs<ND, DIR>::n;
#pragma unroll
    for (int k = 0; k < M; ++k) f[k] = R(0);
    f[0] = a[0] * a[1] * a[1] * q[n];
    f[n] = FM<R>::div(q[0], a[0]);
  }
  template <int DIR>
  __device__ static __forceinline__ void trans(const MConsts<R>&, const R (&)[NCTX],
                                               const R (&)[M], R (&bm)[M], R (&bp)[M]) {
#pragma unroll
    for (int k = 0; k < M; ++k) bm[k] = bp[k] = R(0);
  }
  // B^- a: down-going wave between the cell below (am_) and the cell (ac);
  // B^+ a: up-going wave between the cell and the one above (ap_)
  template <int DIR>
  __device__ static __forceinline__ void trans_aux(const MConsts<R>&, const R* am_, const R* ac,
                                                   const R* ap_, const R (&a)[M], R (&bm)[M],
                                                   R (&bp)[M]) {
    constexpr int t = Dirs<ND, DIR>::t < 0 ? 0 : Dirs<ND, DIR>::t;
    const R Zm = am_[0] * am_[1], Zc = ac[0] * ac[1], Zp = ap_[0] * ap_[1];
#pragma unroll
    for (int k = 0; k < M; ++k) bm[k] = bp[k] = R(0);
    // one reciprocal for both impedance sums (positive, of the media's scale,
    // so their product stays in range)
    const R sm = Zm + Zc, sp = Zc + Zp;
    const R inv = FM<R>::rcp(sm * sp);
    const R b1 = (-a[0] + Zc * a[t]) * (sp * inv);
    const R b2 = (a[0] + Zc * a[t]) * (sm * inv);
    bm[0] = am_[1] * b1 * Zm;
    bm[t] = -am_[1] * b1;
    bp[0] = ap_[1] * b2 * Zp;
    bp[t] = ap_[1] * b2;
  }
  template <int DIR>
  __device__ static __forceinline__ void char_ctx(const MConsts<R>&, const R (&)[M],
                                                  const R (&)[M], R (&ctx)[NCTX]) {
    ctx[0] = R(0);
  }
  template <int DIR>
  __device__ static __forceinline__ void to_char(const MConsts<R>&, const R (&)[NCTX],
                                                 const R (&q)[M], R (&w)[M]) {
#pragma unroll
    for (int k = 0; k < M; ++k) w[k] = q[k];
  }
  template <int DIR>
  __device__ static __forceinline__ void from_char(const MConsts<R>&, const R (&)[NCTX],
                                                   const R (&w)[M], R (&q)[M]) {
#pragma unroll
    for (int k = 0; k < M; ++k) q[k] = w[k];
  }
};

template <class RP, class = void>
struct trans_aux_rp {
  static constexpr bool value = false;
};
template <class RP>
struct trans_aux_rp<RP, decltype((void)RP::TRANS_AUX, void())> {
  static constexpr bool value = RP::TRANS_AUX;
};

// ---------------------------------------------------------------------------
// Euler with a passive tracer phi (phi_t + u . grad phi = 0; Sec. 7.2): the
// Euler Roe solver on the first ND + 2 components and a tracer wave (the jump
// of phi alone) moving with the normal Roe velocity, placed before the u + c
// wave.  The tracer equation is not in conservation form, so SharpClaw's
// in-cell fluctuation comes from a Riemann solve (INCELL_SOLVE), not from a
// flux difference.
// ---------------------------------------------------------------------------
template <typename R, int ND>
struct RpEulerTracer {
  using EU = RpEulerRoe<R, ND>;
  static constexpr int ME = EU::M;                 // Euler components
  static constexpr int M = ME + 1, MW = ME + 1, MA = 0, NCTX = EU::NCTX, NPC = 0;
  static constexpr int TR = ME;                    // tracer component
  static constexpr int E = EU::E;                  // energy component
  static constexpr bool FWAVE = false, INCELL_SOLVE = true;
  static constexpr int WALL_X = 1, WALL_Y = (ND == 2) ? 2 : -1;
  template <int DIR>
  struct NZ {
    // Euler waves carry no tracer; the tracer wave carries nothing else
    __device__ static constexpr bool f(int p, int k) {
      return (p == ME - 1) ? k == TR : k != TR;
    }
  };
  // wave slot of Euler wave e (the last Euler wave moves one slot up)
  __device__ static constexpr int slot(int e) { return e == ME - 1 ? ME : e; }

  template <int DIR>
  __device__ static __forceinline__ void solve(const MConsts<R>& C, const R (&ql)[M],
                                               const R (&qr)[M], const R*, const R*,
                                               R (&W)[MW][M], R (&s)[MW], R (&am)[M],
                                               R (&ap)[M], R (&x)[NCTX]) {
    R el[ME], er[ME], We[ME][ME], se[ME], ame[ME], ape[ME];
#pragma unroll
    for (int k = 0; k < ME; ++k) {
      el[k] = ql[k];
      er[k] = qr[k];
    }
    EU::template solve<DIR>(C, el, er, nullptr, nullptr, We, se, ame, ape, x);
#pragma unroll
    for (int e = 0; e < ME; ++e) {
#pragma unroll
      for (int k = 0; k < ME; ++k) W[slot(e)][k] = We[e][k];
      W[slot(e)][TR] = R(0);
      s[slot(e)] = se[e];
    }
    const R dphi = qr[TR] - ql[TR];
    const R un = x[0];
#pragma unroll
    for (int k = 0; k < ME; ++k) W[ME - 1][k] = R(0);
    W[ME - 1][TR] = dphi;
    s[ME - 1] = un;
#pragma unroll
    for (int k = 0; k < ME; ++k) {
      am[k] = ame[k];
      ap[k] = ape[k];
    }
    am[TR] = fmin(un, R(0)) * dphi;
    ap[TR] = fmax(un, R(0)) * dphi;
  }
  template <int DIR>
  __device__ static __forceinline__ void flux(const MConsts<R>& C, const R (&q)[M], const R*,
                                              R (&f)[M]) {
    // the conservative part only (the tracer has no flux); SharpClaw uses
    // the Riemann solve for the in-cell fluctuation of this system
    R e[ME], fe[ME];
#pragma unroll
    for (int k = 0; k < ME; ++k) e[k] = q[k];
    EU::template flux<DIR>(C, e, nullptr, fe);
#pragma unroll
    for (int k = 0; k < ME; ++k) f[k] = fe[k];
    f[TR] = R(0);
  }
  template <int DIR>
  __device__ static __forceinline__ void trans(const MConsts<R>& C, const R (&x)[NCTX],
                                               const R (&a)[M], R (&bm)[M], R (&bp)[M]) {
    R ae[ME], bme[ME], bpe[ME];
#pragma unroll
    for (int k = 0; k < ME; ++k) ae[k] = a[k];
    EU::template trans<DIR>(C, x, ae, bme, bpe);
#pragma unroll
    for (int k = 0; k < ME; ++k) {
      bm[k] = bme[k];
      bp[k] = bpe[k];
    }
    const R ut = x[1];  // transverse Roe velocity carries the tracer
    bm[TR] = fmin(ut, R(0)) * a[TR];
    bp[TR] = fmax(ut, R(0)) * a[TR];
  }
  template <int DIR>
  __device__ static __forceinline__ void char_ctx(const MConsts<R>& C, const R (&ql)[M],
                                                  const R (&qr)[M], R (&x)[NCTX]) {
    R el[ME], er[ME];
#pragma unroll
    for (int k = 0; k < ME; ++k) {
      el[k] = ql[k];
      er[k] = qr[k];
    }
    EU::template char_ctx<DIR>(C, el, er, x);
  }
  template <int DIR>
  __device__ static __forceinline__ void to_char(const MConsts<R>& C, const R (&x)[NCTX],
                                                 const R (&q)[M], R (&w)[M]) {
    R e[ME], we[ME];
#pragma unroll
    for (int k = 0; k < ME; ++k) e[k] = q[k];
    EU::template to_char<DIR>(C, x, e, we);
#pragma unroll
    for (int k = 0; k < ME; ++k) w[k] = we[k];
    w[TR] = q[TR];
  }
  template <int DIR>
  __device__ static __forceinline__ void from_char(const MConsts<R>& C, const R (&x)[NCTX],
                                                   const R (&w)[M], R (&q)[M]) {
    R we[ME], e[ME];
#pragma unroll
    for (int k = 0; k < ME; ++k) we[k] = w[k];
    EU::template from_char<DIR>(C, x, we, e);
#pragma unroll
    for (int k = 0; k < ME; ++k) q[k] = e[k];
    q[TR] = w[TR];
  }
};

// policy traits with defaults: Euler-family systems (axisymmetric source),
// and systems whose SharpClaw in-cell fluctuation needs a Riemann solve
template <class RP, class = void>
struct is_euler_rp {
  static constexpr bool value = false;
};
template <class RP>
struct is_euler_rp<RP, decltype((void)RP::E, void())> {
  static constexpr bool value = true;
};
template <class RP, class = void>
struct incell_solve {
  static constexpr bool value = false;
};
template <class RP>
struct incell_solve<RP, decltype((void)RP::INCELL_SOLVE, void())> {
  static constexpr bool value = RP::INCELL_SOLVE;
};

// solvers of two waves whose first always moves left and second right
// (RP::SIGNED_WAVES): the upwind side and the sign of each wave are known
// without looking at the speeds
template <class RP, class = void>
struct signed_waves {
  static constexpr bool value = false;
};
template <class RP>
struct signed_waves<RP, decltype((void)RP::SIGNED_WAVES, void())> {
  static constexpr bool value = RP::SIGNED_WAVES && RP::MW == 2;
};
// Systems whose waves of each family are multiples of one fixed vector
// (constant-coefficient advection and acoustics): W^p = alpha_p r^p, so the
// limiter's ratio (W^p_up . W^p) / (W^p . W^p) is alpha_p,up / alpha_p, the
// ratio of any one component that r^p does not zero.  RP::strength<DIR>()
// names such a component; the kernels then hand `correction` that component
// of the upwind wave and of the wave itself in place of the dot product and
// the norm (a signed value, zero exactly when the wave is).  Other solvers
// give -1.
template <class RP, class = void>
struct has_strength {
  static constexpr bool value = false;
};
template <class RP>
struct has_strength<RP, decltype((void)RP::template strength<0>(), void())> {
  static constexpr bool value = true;
};
template <class RP, int DIR>
__host__ __device__ constexpr int strength_k() {
  if constexpr (has_strength<RP>::value) return RP::template strength<DIR>();
  else return -1;
}

// sign of wave p's speed: -1, 0 or 1
template <class RP, typename R>
__device__ __forceinline__ R wave_sign(int p, R s) {
  if constexpr (signed_waves<RP>::value) return p == 0 ? R(-1) : R(1);
  else return s > R(0) ? R(1) : (s < R(0) ? R(-1) : R(0));
}

// ---------------------------------------------------------------------------
// wave limiters (LeVeque FVM book, high-resolution methods)
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ R limiter(int lim, R th) {
  switch (lim) {
    case CLAW_LIM_MINMOD: return fmax(R(0), fmin(R(1), th));
    case CLAW_LIM_SUPERBEE: return fmax(R(0), fmax(fmin(R(1), R(2) * th), fmin(R(2), th)));
    case CLAW_LIM_VANLEER: {
      const R a = fabs(th);
      return FM<R>::div(th + a, R(1) + a);
    }
    case CLAW_LIM_MC: return fmax(R(0), fmin(R(0.5) * (R(1) + th), fmin(R(2), R(2) * th)));
    default: return R(1);
  }
}

// MC limiter max(0, min((1+th)/2, 2, 2 th)) with the branch chosen on the bit
// pattern of th (2 th below th = 1/3, (1+th)/2 up to th = 3, then 2).
template <typename R>
__device__ __forceinline__ R limiter_mc(R th) {
  if (!gt0(th)) return R(0);
  const R two_th = R(2) * th, mid = R(0.5) * (R(1) + th);
  const auto b = fbits(th);
  return b < fbits(R(1) / R(3)) ? two_th : (b <= fbits(R(3)) ? mid : R(2));
}
// FP32: max(0, min((1+th)/2, 2, 2 th)) by min/max (no branch)
template <>
__device__ __forceinline__ float limiter_mc<float>(float th) {
  return fmaxf(0.f, fminf(fminf(0.5f * (1.f + th), 2.f), 2.f * th));
}
// the same as one fused multiply-add, a th + b with (a, b) chosen by the
// branch: (2, 0), (1/2, 1/2) or (0, 2); the middle branch rounds once
template <typename R>
__device__ __forceinline__ R limiter_mc_fma(R th) {
  const auto b = fbits(th);
  const bool pos = gt0(th), lo = b < fbits(R(1) / R(3)), mid = b <= fbits(R(3));
  const R a = !pos ? R(0) : (lo ? R(2) : (mid ? R(0.5) : R(0)));
  const R c = !pos ? R(0) : (lo ? R(0) : (mid ? R(0.5) : R(2)));
  return a * th + c;
}

// phi(theta) a for theta = u / a without the division: phi vanishes for
// theta <= 0, and for same-signed u and a each limiter's phi(u/a) a is
// sgn(a) g(|u|, |a|) (identities of the limiter functions; the rounding
// differs from forming theta first):
//   minmod   min(|u|, |a|)
//   superbee max(min(2|u|, |a|), min(|u|, 2|a|))
//   MC       min(|a + u| / 2, 2|a|, 2|u|)
//   van Leer 2 |u| |a| / (|u| + |a|)
//   none     a
template <typename R>
__device__ __forceinline__ R limited_strength(int lim, R u, R a) {
  if (lim == CLAW_LIM_NONE) return a;
  const bool same = (gt0(u) && gt0(a)) || (lt0(u) && lt0(a));
  const R au = fabs(u), aa = fabs(a);
  R g;
  switch (lim) {
    case CLAW_LIM_MINMOD: g = fmin(au, aa); break;
    case CLAW_LIM_SUPERBEE: g = fmax(fmin(R(2) * au, aa), fmin(au, R(2) * aa)); break;
    case CLAW_LIM_VANLEER: g = FM<R>::div(R(2) * au * aa, au + aa); break;
    default: g = fmin(R(0.5) * fabs(a + u), fmin(R(2) * aa, R(2) * au)); break;  // MC
  }
  g = same ? g : R(0);
  return lt0(a) ? -g : g;
}

// Second-order correction at one interface (Eq. (lwflux) with limited waves):
//   F = 1/2 sum_p c_p phi(theta_p) W^p,  c_p = |s|(1 - dt/dx |s|)   (waves)
//                                          = sgn(s)(1 - dt/dx |s|) (f-waves)
// dot_up[p] = W^p_upwind . W^p, nrm[p] = W^p . W^p (zero wave -> no correction);
// for the solvers with wave strengths (strength_k >= 0) the strength
// component of W^p_upwind and of W^p (same ratio, nrm[p] signed).
// theta_p = dot_up[p] / nrm[p]; with three or more waves, when every partial
// product of the norms is a normal number, the reciprocals come from one
// division (1/n_p = prod_{q != p} n_q / prod_q n_q).  DIR selects the
// solver's structural zeros.
// LIMC >= 0 fixes the limiter at compile time (else C.lim).  FP32 takes
// every wave's ratio by selects, without branches.
template <class RP, typename R, int DIR = 0, int LIMC = -1>
__device__ __forceinline__ void correction(const MConsts<R>& C, const R (&W)[RP::MW][RP::M],
                                           const R (&s)[RP::MW], const R (&dot_up)[RP::MW],
                                           const R (&nrm)[RP::MW], R dtdn, R (&F)[RP::M]) {
  using NZ = typename RP::template NZ<DIR>;
  constexpr int MW = RP::MW;
  static_assert(strength_k<RP, DIR>() < 0 || MW <= 2, "signed strengths: no batched reciprocal");
  const int lim = LIMC >= 0 ? LIMC : C.lim;
#pragma unroll
  for (int k = 0; k < RP::M; ++k) F[k] = R(0);
  if constexpr (strength_k<RP, DIR>() >= 0 && !RP::FWAVE && sizeof(R) == 8) {
    // FP64 wave strengths: the limited strength phi_p a_p by the
    // division-free forms (no IEEE division on the FP64 pipe), then its wave
    // phi_p W^p from the solver's eigenvector.  FP32 keeps theta = u / a:
    // its division is one approximate reciprocal, cheaper than the selects.
#pragma unroll
    for (int p = 0; p < MW; ++p) {
      const R al = limited_strength<R>(lim, dot_up[p], nrm[p]);
      const R a = fabs(s[p]);
      const R cf = R(0.5) * a * (R(1) - dtdn * a);
      R w[RP::M];
      RP::template wave_of<DIR>(C, p, al, w);
#pragma unroll
      for (int k = 0; k < RP::M; ++k)
        if (NZ::f(p, k)) F[k] += cf * w[k];
    }
    return;
  }
  if constexpr (sizeof(R) == 4) {
    const R hd = R(0.5) * dtdn;
#pragma unroll
    for (int p = 0; p < MW; ++p) {
      const R th = FM<R>::div(dot_up[p], nrm[p]);
      R phi = lim == CLAW_LIM_MC ? limiter_mc<R>(th) : limiter<R>(lim, th);
      phi = lim == CLAW_LIM_NONE ? R(1) : phi;
      phi = nrm[p] == R(0) ? R(0) : phi;  // a zero wave gets no correction
      const R a = fabsf(s[p]);
      R cf;
      if (MW >= 3 && !RP::FWAVE) {
        cf = (R(0.5) - hd * a) * a * phi;
      } else {
        const R sg = RP::FWAVE ? wave_sign<RP, R>(p, s[p]) : a;
        cf = R(0.5) * sg * (R(1) - dtdn * a) * phi;
      }
#pragma unroll
      for (int k = 0; k < RP::M; ++k)
        if (NZ::f(p, k)) F[k] += cf * W[p][k];
    }
    return;
  }
  R inv[MW];
  bool batched = false;
  if (MW >= 3 && lim != CLAW_LIM_NONE) {
    // every partial product must be a normal number: a subnormal one (a tiny
    // wave next to large ones) would lose precision in the reciprocals
    R pre[MW];
    R prod = nrm[0];
    bool normal = pos_normal(prod);
    pre[0] = R(1);
#pragma unroll
    for (int p = 1; p < MW; ++p) {
      pre[p] = prod;
      prod = prod * nrm[p];
      normal = normal && pos_normal(prod);
    }
    if (normal) {
      const R r = FM<R>::rcp(prod);
      R suf = r;
#pragma unroll
      for (int p = MW - 1; p >= 0; --p) {
        inv[p] = p == 0 ? suf : suf * pre[p];
        suf = suf * nrm[p];
      }
      batched = true;
    }
  }
  const R hd = R(0.5) * dtdn;
#pragma unroll
  for (int p = 0; p < MW; ++p) {
    R phi;
    // a norm is never -0; a signed strength may be
    if (strength_k<RP, DIR>() >= 0 ? zero_mag(nrm[p]) : fbits(nrm[p]) == 0) phi = R(0);
    else if (lim == CLAW_LIM_NONE) phi = R(1);
    else {
      const R th = batched ? dot_up[p] * inv[p] : FM<R>::div(dot_up[p], nrm[p]);
      // systems of three or more waves take the fused forms (one rounding
      // less per wave; the long linear runs of two-wave systems keep the
      // oracle's order)
      phi = lim == CLAW_LIM_MC ? (MW >= 3 ? limiter_mc_fma<R>(th) : limiter_mc<R>(th))
                               : limiter<R>(lim, th);
    }
    const R a = fabs(s[p]);
    R cf;
    if (MW >= 3 && !RP::FWAVE) {
      cf = (R(0.5) - hd * a) * a * phi;  // 1/2 |s| (1 - dt/dx |s|) phi
    } else {
      const R sg = RP::FWAVE ? (signed_waves<RP>::value ? (p == 0 ? R(-1) : R(1))
                                                       : (gt0(s[p]) ? R(1) : (lt0(s[p]) ? R(-1) : R(0))))
                             : a;
      cf = R(0.5) * sg * (R(1) - dtdn * a) * phi;
    }
#pragma unroll
    for (int k = 0; k < RP::M; ++k)
      if (NZ::f(p, k)) F[k] += cf * W[p][k];
  }
}

}  // namespace claw
