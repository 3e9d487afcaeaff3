/*
 * oracle.c -- plain FP64 CPU oracle for the finite-volume time step of
 * Clawpack-classic and SharpClaw (PyClaw, Ketcheson et al.).
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).  Written for readability against
 * the paper and the published methods it cites, not for speed: every step is
 * a separate pass over whole arrays, in the order the method states it.
 * OpenMP pragmas only split independent rows/columns; per-cell arithmetic and
 * every reduction order are fixed, so results do not depend on thread count.
 *
 * Compiled with -O2 -ffp-contract=off (no FMA contraction).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include "oracle.h"

#define MAXM 8
#define MAXW 8

/* ------------------------------------------------------------------------ */
/* problem shape                                                             */
/* ------------------------------------------------------------------------ */

int orc_num_eqn(int rp, int ndim) {
  switch (rp) {
    case ORC_RP_ADVECTION: return 1;
    case ORC_RP_ACOUSTICS: return ndim + 1;
    case ORC_RP_SW_ROE: return ndim == 1 ? 2 : (ndim == 2 ? 3 : 0);
    case ORC_RP_EULER_ROE:
    case ORC_RP_EULER_HLLE: return ndim <= 2 ? ndim + 2 : 0;
    case ORC_RP_ELASTICITY_FWAVE: return ndim == 1 ? 2 : (ndim == 2 ? 3 : 0);
    case ORC_RP_EULER_TRACER: return ndim <= 2 ? ndim + 3 : 0;
    case ORC_RP_ACOUSTICS_VC: return ndim <= 2 ? ndim + 1 : 0;
  }
  return 0;
}

int orc_num_waves(int rp, int ndim) {
  switch (rp) {
    case ORC_RP_ADVECTION: return 1;
    case ORC_RP_ACOUSTICS: return 2;
    case ORC_RP_SW_ROE: return ndim == 1 ? 2 : 3;
    case ORC_RP_EULER_ROE: return ndim == 1 ? 3 : 4;
    case ORC_RP_EULER_HLLE: return 2;
    case ORC_RP_ELASTICITY_FWAVE: return 2;
    case ORC_RP_EULER_TRACER: return ndim == 1 ? 4 : 5;
    case ORC_RP_ACOUSTICS_VC: return 2;
  }
  return 0;
}

int orc_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* index of the momentum / velocity component normal to direction dir */
static int comp_n(const orc_prob* P, int dir) { return P->ndim == 1 ? 1 : 1 + dir; }
/* index of the tangential component (-1 in 1D) */
static int comp_t(const orc_prob* P, int dir) { return P->ndim == 1 ? -1 : 2 - dir; }
/* index of the energy component of the Euler equations */
static int comp_e(const orc_prob* P) { return P->ndim == 1 ? 2 : 3; }
static int is_fwave(const orc_prob* P) { return P->rp == ORC_RP_ELASTICITY_FWAVE; }
/* index of the tracer of the Euler-with-tracer system (last component) */
static int comp_tr(const orc_prob* P) { return P->ndim + 2; }
static int is_euler(const orc_prob* P) {
  return P->rp == ORC_RP_EULER_ROE || P->rp == ORC_RP_EULER_HLLE || P->rp == ORC_RP_EULER_TRACER;
}

/* ------------------------------------------------------------------------ */
/* eigen-decompositions (LeVeque FVM book: acoustics, shallow water, Euler)  */
/* Each helper works in a frame whose "normal" component is a and tangential */
/* component b (b < 0: no tangential component).  Given a jump d it returns   */
/* the eigen-coefficients alpha, eigenvectors r[p*m+k] and speeds lam[p].    */
/* ------------------------------------------------------------------------ */

/* Linear acoustics with constant rho, K: c = sqrt(K/rho), Z = rho c.
 * r1 = (-Z, 1) speed -c, r2 = (Z, 1) speed +c on (p, u_a); when with_shear,
 * a third zero-speed eigenvector (0, 0, 1) carries the tangential velocity. */
static int acoustics_eig(const orc_prob* P, int a, int b, int with_shear, const double* d,
                         double* alpha, double* r, double* lam) {
  int m = P->num_eqn;
  double rho = P->params[0], K = P->params[1];
  double c = sqrt(K / rho);
  double Z = rho * c;
  int nw = (with_shear && b >= 0) ? 3 : 2;
  memset(r, 0, sizeof(double) * nw * m);
  alpha[0] = (-d[0] + Z * d[a]) / (2.0 * Z);
  alpha[1] = (d[0] + Z * d[a]) / (2.0 * Z);
  r[0 * m + 0] = -Z; r[0 * m + a] = 1.0; lam[0] = -c;
  r[1 * m + 0] = Z;  r[1 * m + a] = 1.0; lam[1] = c;
  if (nw == 3) { alpha[2] = d[b]; r[2 * m + b] = 1.0; lam[2] = 0.0; }
  return nw;
}

/* Shallow water at a Roe state (un, ut, c = sqrt(g hbar)).  Waves ordered
 * (un - c, [shear un], un + c). */
static int sw_eig(const orc_prob* P, int a, int b, double un, double ut, double c,
                  const double* d, double* alpha, double* r, double* lam) {
  int m = P->num_eqn;
  int nw = (b >= 0) ? 3 : 2;
  int last = nw - 1;
  memset(r, 0, sizeof(double) * nw * m);
  alpha[0] = ((un + c) * d[0] - d[a]) / (2.0 * c);
  alpha[last] = (d[a] - (un - c) * d[0]) / (2.0 * c);
  r[0 * m + 0] = 1.0; r[0 * m + a] = un - c; lam[0] = un - c;
  r[last * m + 0] = 1.0; r[last * m + a] = un + c; lam[last] = un + c;
  if (b >= 0) {
    alpha[1] = d[b] - ut * d[0];
    r[0 * m + b] = ut;
    r[1 * m + b] = 1.0; lam[1] = un;
    r[last * m + b] = ut;
  }
  return nw;
}

/* Euler (ideal gas) at a Roe state (un, ut, H, c, c2 = c*c).  Waves ordered
 * (un - c, entropy un, [shear un], un + c). */
static int euler_eig(const orc_prob* P, int a, int b, double un, double ut, double H,
                     double c, double c2, const double* d, double* alpha, double* r,
                     double* lam) {
  int m = P->num_eqn;
  int e = comp_e(P);
  double gm1 = P->params[0] - 1.0;
  int nw = (b >= 0) ? 4 : 3;
  int last = nw - 1;
  double ash = (b >= 0) ? d[b] - ut * d[0] : 0.0;
  double a2 = gm1 * ((H - un * un) * d[0] + un * d[a] - d[e] + ut * ash) / c2;
  double a4 = (d[a] + (c - un) * d[0] - c * a2) / (2.0 * c);
  double a1 = d[0] - a2 - a4;
  memset(r, 0, sizeof(double) * nw * m);
  alpha[0] = a1;
  r[0 * m + 0] = 1.0; r[0 * m + a] = un - c; r[0 * m + e] = H - un * c; lam[0] = un - c;
  alpha[1] = a2;
  r[1 * m + 0] = 1.0; r[1 * m + a] = un; r[1 * m + e] = 0.5 * (un * un + ut * ut); lam[1] = un;
  if (b >= 0) {
    r[0 * m + b] = ut;
    r[1 * m + b] = ut;
    alpha[2] = ash;
    r[2 * m + b] = 1.0; r[2 * m + e] = ut; lam[2] = un;
    r[last * m + b] = ut;
  }
  alpha[last] = a4;
  r[last * m + 0] = 1.0; r[last * m + a] = un + c; r[last * m + e] = H + un * c;
  lam[last] = un + c;
  return nw;
}

/* Euler with a passive tracer phi (phi_t + u . grad phi = 0, Sec. 7.2): the
 * Euler waves with a zero tracer component, and a tracer wave (jump of phi
 * alone) moving with the normal velocity, placed before the u + c wave so
 * that the first and last waves stay the acoustic ones. */
static int euler_tracer_eig(const orc_prob* P, int a, int b, double un, double ut, double H,
                            double c, double c2, const double* d, double* alpha, double* r,
                            double* lam) {
  int m = P->num_eqn, tr = comp_tr(P);
  int nwe = euler_eig(P, a, b, un, ut, H, c, c2, d, alpha, r, lam);
  int last = nwe;  /* acoustic u + c wave moves one slot up */
  alpha[last] = alpha[nwe - 1];
  lam[last] = lam[nwe - 1];
  for (int k = 0; k < m; ++k) r[last * m + k] = r[(nwe - 1) * m + k];
  alpha[nwe - 1] = d[tr];
  lam[nwe - 1] = un;
  for (int k = 0; k < m; ++k) r[(nwe - 1) * m + k] = (k == tr) ? 1.0 : 0.0;
  return nwe + 1;
}

/* ------------------------------------------------------------------------ */
/* Roe averages                                                              */
/* ------------------------------------------------------------------------ */

/* shallow water: hbar = (hl+hr)/2, sqrt(h)-weighted velocities, c = sqrt(g hbar) */
static void sw_roe_avg(const orc_prob* P, int dir, const double* ql, const double* qr,
                       double* un, double* ut, double* c) {
  int n = comp_n(P, dir), t = comp_t(P, dir);
  double g = P->params[0];
  double hl = ql[0], hr = qr[0];
  double sl = sqrt(hl), sr = sqrt(hr);
  double ul = ql[n] / hl, ur = qr[n] / hr;
  double hbar = 0.5 * (hl + hr);
  *un = (sl * ul + sr * ur) / (sl + sr);
  if (t >= 0) {
    double vl = ql[t] / hl, vr = qr[t] / hr;
    *ut = (sl * vl + sr * vr) / (sl + sr);
  } else {
    *ut = 0.0;
  }
  *c = sqrt(g * hbar);
}

/* Euler pressure p = (gamma-1)(E - (mn^2 + mt^2)/(2 rho)) */
static double euler_pressure(const orc_prob* P, const double* q) {
  int e = comp_e(P);
  double gm1 = P->params[0] - 1.0;
  double ke = q[1] * q[1];
  if (P->ndim == 2) ke = q[1] * q[1] + q[2] * q[2];
  return gm1 * (q[e] - 0.5 * ke / q[0]);
}

/* Euler Roe averages: sqrt(rho)-weighted un, ut, H; c2 = (gamma-1)(H - (un^2+ut^2)/2) */
static void euler_roe_avg(const orc_prob* P, int dir, const double* ql, const double* qr,
                          double* un, double* ut, double* H, double* c, double* c2) {
  int n = comp_n(P, dir), t = comp_t(P, dir), e = comp_e(P);
  double gm1 = P->params[0] - 1.0;
  double rl = ql[0], rr = qr[0];
  double pl = euler_pressure(P, ql), pr = euler_pressure(P, qr);
  double ul = ql[n] / rl, ur = qr[n] / rr;
  double vl = 0.0, vr = 0.0;
  if (t >= 0) { vl = ql[t] / rl; vr = qr[t] / rr; }
  double Hl = (ql[e] + pl) / rl, Hr = (qr[e] + pr) / rr;
  double sl = sqrt(rl), sr = sqrt(rr);
  double den = sl + sr;
  *un = (sl * ul + sr * ur) / den;
  *ut = (sl * vl + sr * vr) / den;
  *H = (sl * Hl + sr * Hr) / den;
  *c2 = gm1 * (*H - 0.5 * (*un * *un + *ut * *ut));
  *c = sqrt(*c2);
}

/* characteristic speeds u - c (which = 0) or u + c (which = 1) of one state */
static double state_speed(const orc_prob* P, int dir, const double* q, int which) {
  int n = comp_n(P, dir);
  double u = q[n] / q[0];
  double c;
  if (P->rp == ORC_RP_SW_ROE) {
    c = sqrt(P->params[0] * q[0]);
  } else {
    double p = euler_pressure(P, q);
    c = sqrt(P->params[0] * p / q[0]);
  }
  return which == 0 ? u - c : u + c;
}

/* Euler flux in direction dir */
static void euler_flux(const orc_prob* P, int dir, const double* q, double* f) {
  int n = comp_n(P, dir), t = comp_t(P, dir), e = comp_e(P);
  double p = euler_pressure(P, q);
  double u = q[n] / q[0];
  f[0] = q[n];
  f[n] = q[n] * u + p;
  if (t >= 0) f[t] = q[t] * u;
  f[e] = u * (q[e] + p);
}

/* ------------------------------------------------------------------------ */
/* Riemann solvers (normal)                                                  */
/* ------------------------------------------------------------------------ */

static void split_by_speed(int m, int nw, const double* W, const double* s, double* amdq,
                           double* apdq) {
  for (int k = 0; k < m; ++k) { amdq[k] = 0.0; apdq[k] = 0.0; }
  for (int p = 0; p < nw; ++p)
    for (int k = 0; k < m; ++k) {
      amdq[k] += fmin(s[p], 0.0) * W[p * m + k];
      apdq[k] += fmax(s[p], 0.0) * W[p * m + k];
    }
}

/* f-waves: A^-dQ = sum_{s<0} Z, A^+dQ = sum_{s>0} Z, s = 0 split half/half */
static void split_fwaves(int m, int nw, const double* Z, const double* s, double* amdq,
                         double* apdq) {
  for (int k = 0; k < m; ++k) { amdq[k] = 0.0; apdq[k] = 0.0; }
  for (int p = 0; p < nw; ++p)
    for (int k = 0; k < m; ++k) {
      if (s[p] < 0.0) amdq[k] += Z[p * m + k];
      else if (s[p] > 0.0) apdq[k] += Z[p * m + k];
      else { amdq[k] += 0.5 * Z[p * m + k]; apdq[k] += 0.5 * Z[p * m + k]; }
    }
}

/* Harten-Hyman entropy fix for the first (u-c) and last (u+c) families.
 * Returns 1 and writes amdq/apdq when a transonic rarefaction is found. */
static int harten_hyman(const orc_prob* P, int dir, int m, int nw, const double* ql,
                        const double* qr, const double* W, const double* s, double* amdq,
                        double* apdq) {
  double total[MAXM];
  double qm[MAXM] = {0};
  int last = nw - 1;
  for (int k = 0; k < m; ++k) {
    total[k] = 0.0;
    for (int p = 0; p < nw; ++p) total[k] += s[p] * W[p * m + k];
  }
  /* family 1: middle state Q_l + W^1 */
  for (int k = 0; k < m; ++k) qm[k] = ql[k] + W[0 * m + k];
  {
    double lamL = state_speed(P, dir, ql, 0);
    double lamR = state_speed(P, dir, qm, 0);
    if (lamL < 0.0 && lamR > 0.0) {
      double beta = (lamR - s[0]) / (lamR - lamL);
      for (int k = 0; k < m; ++k) {
        amdq[k] = beta * lamL * W[0 * m + k];
        apdq[k] = total[k] - amdq[k];
      }
      return 1;
    }
  }
  /* last family: middle state Q_r - W^last */
  for (int k = 0; k < m; ++k) qm[k] = qr[k] - W[last * m + k];
  {
    double lamL = state_speed(P, dir, qm, 1);
    double lamR = state_speed(P, dir, qr, 1);
    if (lamL < 0.0 && lamR > 0.0) {
      double beta = (lamR - s[last]) / (lamR - lamL);
      for (int k = 0; k < m; ++k) {
        apdq[k] = (1.0 - beta) * lamR * W[last * m + k];
        amdq[k] = total[k] - apdq[k];
      }
      return 1;
    }
  }
  return 0;
}

void orc_riemann(const orc_prob* P, int dir, const double* ql, const double* qr,
                 const double* auxl, const double* auxr, double* wave, double* s,
                 double* amdq, double* apdq) {
  int m = P->num_eqn;
  int nw = orc_num_waves(P->rp, P->ndim);
  int n = comp_n(P, dir), t = comp_t(P, dir);
  double d[MAXM], alpha[MAXW], r[MAXW * MAXM];
  for (int k = 0; k < m; ++k) d[k] = qr[k] - ql[k];
  switch (P->rp) {
    case ORC_RP_ADVECTION: {
      wave[0] = d[0];
      s[0] = P->params[dir];
      break;
    }
    case ORC_RP_ACOUSTICS: {
      acoustics_eig(P, n, t, 0, d, alpha, r, s);
      for (int p = 0; p < nw; ++p)
        for (int k = 0; k < m; ++k) wave[p * m + k] = alpha[p] * r[p * m + k];
      break;
    }
    case ORC_RP_SW_ROE: {
      double un, ut, c;
      sw_roe_avg(P, dir, ql, qr, &un, &ut, &c);
      sw_eig(P, n, t, un, ut, c, d, alpha, r, s);
      for (int p = 0; p < nw; ++p)
        for (int k = 0; k < m; ++k) wave[p * m + k] = alpha[p] * r[p * m + k];
      break;
    }
    case ORC_RP_EULER_ROE: {
      double un, ut, H, c, c2;
      euler_roe_avg(P, dir, ql, qr, &un, &ut, &H, &c, &c2);
      euler_eig(P, n, t, un, ut, H, c, c2, d, alpha, r, s);
      for (int p = 0; p < nw; ++p)
        for (int k = 0; k < m; ++k) wave[p * m + k] = alpha[p] * r[p * m + k];
      break;
    }
    case ORC_RP_EULER_TRACER: {
      double un, ut, H, c, c2;
      euler_roe_avg(P, dir, ql, qr, &un, &ut, &H, &c, &c2);
      euler_tracer_eig(P, n, t, un, ut, H, c, c2, d, alpha, r, s);
      for (int p = 0; p < nw; ++p)
        for (int k = 0; k < m; ++k) wave[p * m + k] = alpha[p] * r[p * m + k];
      break;
    }
    case ORC_RP_ACOUSTICS_VC: {
      /* linear acoustics in a varying medium, aux (rho, c) per cell: the
       * left-going wave carries the left impedance, the right-going the
       * right one (LeVeque FVM book, heterogeneous media) */
      double Zl = auxl[0] * auxl[1], Zr = auxr[0] * auxr[1];
      double a1 = (-d[0] + Zr * d[n]) / (Zl + Zr);
      double a2 = (d[0] + Zl * d[n]) / (Zl + Zr);
      for (int k = 0; k < 2 * m; ++k) wave[k] = 0.0;
      wave[0] = -a1 * Zl; wave[n] = a1; s[0] = -auxl[1];
      wave[m] = a2 * Zr; wave[m + n] = a2; s[1] = auxr[1];
      break;
    }
    case ORC_RP_EULER_HLLE: {
      double un, ut, H, c, c2;
      double fl[MAXM], fr[MAXM], qs[MAXM];
      euler_roe_avg(P, dir, ql, qr, &un, &ut, &H, &c, &c2);
      double sl = fmin(state_speed(P, dir, ql, 0), un - c);
      double sr = fmax(state_speed(P, dir, qr, 1), un + c);
      euler_flux(P, dir, ql, fl);
      euler_flux(P, dir, qr, fr);
      for (int k = 0; k < m; ++k)
        qs[k] = (fr[k] - fl[k] - sr * qr[k] + sl * ql[k]) / (sl - sr);
      for (int k = 0; k < m; ++k) {
        wave[0 * m + k] = qs[k] - ql[k];
        wave[1 * m + k] = qr[k] - qs[k];
      }
      s[0] = sl;
      s[1] = sr;
      break;
    }
    case ORC_RP_ELASTICITY_FWAVE: {
      /* p-system (Sec. 7.3): sigma(eps) = exp(K eps) - 1, normal velocity
       * u_n = m_n / rho, normal flux (-u_n, -sigma) in the (eps, m_n)
       * components; the tangential momentum has no normal flux (2D) */
      int n = comp_n(P, dir), t = comp_t(P, dir);
      double rl = auxl[0], Kl = auxl[1], rr = auxr[0], Kr = auxr[1];
      double el = exp(Kl * ql[0]), er = exp(Kr * qr[0]);
      double sigl = el - 1.0, sigr = er - 1.0;
      double ul = ql[n] / rl, ur = qr[n] / rr;
      double cl = sqrt(Kl * el / rl), cr = sqrt(Kr * er / rr);
      double Zl = rl * cl, Zr = rr * cr;
      double d1 = ul - ur;       /* (-u_r) - (-u_l) */
      double d2 = sigl - sigr;   /* (-sigma_r) - (-sigma_l) */
      double b1 = (Zr * d1 + d2) / (Zl + Zr);
      double b2 = (Zl * d1 - d2) / (Zl + Zr);
      for (int k = 0; k < 2 * m; ++k) wave[k] = 0.0;
      wave[0] = b1; wave[n] = b1 * Zl; s[0] = -cl;
      wave[m] = b2; wave[m + n] = -b2 * Zr; s[1] = cr;
      (void)t;
      break;
    }
  }
  if (is_fwave(P)) {
    split_fwaves(m, nw, wave, s, amdq, apdq);
    return;
  }
  if (P->entropy_fix &&
      (P->rp == ORC_RP_SW_ROE || P->rp == ORC_RP_EULER_ROE || P->rp == ORC_RP_EULER_TRACER)) {
    if (harten_hyman(P, dir, m, nw, ql, qr, wave, s, amdq, apdq)) return;
  }
  split_by_speed(m, nw, wave, s, amdq, apdq);
}

/* ------------------------------------------------------------------------ */
/* transverse solvers (2D)                                                   */
/* ------------------------------------------------------------------------ */

/* Transverse split of asdq in a varying acoustic medium: the down-going part
 * is the left-going wave of the transverse Riemann problem between the cell
 * below (aux a_m) and the cell holding the fluctuation (a_c); the up-going
 * part the right-going wave between a_c and the cell above (a_p). */
void orc_transverse_vc(const orc_prob* P, int dir, const double* a_m, const double* a_c,
                       const double* a_p, const double* asdq, double* bm, double* bp) {
  int m = P->num_eqn, t = comp_t(P, dir);
  double Zm = a_m[0] * a_m[1], Zc = a_c[0] * a_c[1], Zp = a_p[0] * a_p[1];
  for (int k = 0; k < m; ++k) { bm[k] = 0.0; bp[k] = 0.0; }
  double b1 = (-asdq[0] + Zc * asdq[t]) / (Zm + Zc);
  double b2 = (asdq[0] + Zc * asdq[t]) / (Zc + Zp);
  bm[0] = a_m[1] * b1 * Zm;
  bm[t] = -a_m[1] * b1;
  bp[0] = a_p[1] * b2 * Zp;
  bp[t] = a_p[1] * b2;
}

void orc_transverse(const orc_prob* P, int dir, const double* ql, const double* qr,
                    const double* auxl, const double* auxr, const double* asdq,
                    double* bmasdq, double* bpasdq) {
  (void)auxl; (void)auxr;
  int m = P->num_eqn;
  int n = comp_n(P, dir), t = comp_t(P, dir);
  int tdir = 1 - dir;
  double beta[MAXW], r[MAXW * MAXM], lam[MAXW];
  int nw = 0;
  for (int k = 0; k < m; ++k) { bmasdq[k] = 0.0; bpasdq[k] = 0.0; }
  switch (P->rp) {
    case ORC_RP_ADVECTION: {
      double v = P->params[tdir];
      bmasdq[0] = fmin(v, 0.0) * asdq[0];
      bpasdq[0] = fmax(v, 0.0) * asdq[0];
      return;
    }
    case ORC_RP_ACOUSTICS:
      /* eigenvectors of the transverse direction: frame normal = t */
      nw = acoustics_eig(P, t, n, 0, asdq, beta, r, lam);
      break;
    case ORC_RP_SW_ROE: {
      double un, ut, c;
      sw_roe_avg(P, dir, ql, qr, &un, &ut, &c);
      nw = sw_eig(P, t, n, ut, un, c, asdq, beta, r, lam);
      break;
    }
    case ORC_RP_EULER_ROE:
    case ORC_RP_EULER_HLLE: {
      double un, ut, H, c, c2;
      euler_roe_avg(P, dir, ql, qr, &un, &ut, &H, &c, &c2);
      nw = euler_eig(P, t, n, ut, un, H, c, c2, asdq, beta, r, lam);
      break;
    }
    case ORC_RP_EULER_TRACER: {
      double un, ut, H, c, c2;
      euler_roe_avg(P, dir, ql, qr, &un, &ut, &H, &c, &c2);
      nw = euler_tracer_eig(P, t, n, ut, un, H, c, c2, asdq, beta, r, lam);
      break;
    }
    default:
      return;
  }
  for (int p = 0; p < nw; ++p)
    for (int k = 0; k < m; ++k) {
      bmasdq[k] += fmin(lam[p], 0.0) * beta[p] * r[p * m + k];
      bpasdq[k] += fmax(lam[p], 0.0) * beta[p] * r[p * m + k];
    }
}

/* ------------------------------------------------------------------------ */
/* characteristic matrices for SharpClaw (Roe state of the interface)        */
/* ------------------------------------------------------------------------ */

int orc_char_matrices(const orc_prob* P, int dir, const double* ql, const double* qr,
                      double* Lmat, double* Rmat) {
  int m = P->num_eqn;
  int n = comp_n(P, dir), t = comp_t(P, dir);
  double e[MAXM], alpha[MAXW], r[MAXW * MAXM], lam[MAXW];
  double un = 0, ut = 0, H = 0, c = 0, c2 = 0;
  if (P->rp == ORC_RP_ELASTICITY_FWAVE) return ORC_EINVAL;
  if (P->rp == ORC_RP_SW_ROE) sw_roe_avg(P, dir, ql, qr, &un, &ut, &c);
  if (is_euler(P)) euler_roe_avg(P, dir, ql, qr, &un, &ut, &H, &c, &c2);
  for (int col = 0; col < m; ++col) {
    for (int k = 0; k < m; ++k) e[k] = (k == col) ? 1.0 : 0.0;
    switch (P->rp) {
      case ORC_RP_ADVECTION: alpha[0] = e[0]; r[0] = 1.0; break;
      case ORC_RP_ACOUSTICS: acoustics_eig(P, n, t, 1, e, alpha, r, lam); break;
      case ORC_RP_SW_ROE: sw_eig(P, n, t, un, ut, c, e, alpha, r, lam); break;
      case ORC_RP_EULER_TRACER: euler_tracer_eig(P, n, t, un, ut, H, c, c2, e, alpha, r, lam); break;
      default: euler_eig(P, n, t, un, ut, H, c, c2, e, alpha, r, lam); break;
    }
    /* column col of L is L e_col = alpha */
    for (int p = 0; p < m; ++p) Lmat[p * m + col] = alpha[p];
  }
  /* R[k][p] = r_p[k] */
  for (int p = 0; p < m; ++p)
    for (int k = 0; k < m; ++k) Rmat[k * m + p] = r[p * m + k];
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* limiters (LeVeque FVM book, Sec. 6.9)                                     */
/* ------------------------------------------------------------------------ */

double orc_phi(int lim, double th) {
  switch (lim) {
    case ORC_LIM_MINMOD: return fmax(0.0, fmin(1.0, th));
    case ORC_LIM_SUPERBEE: return fmax(0.0, fmax(fmin(1.0, 2.0 * th), fmin(2.0, th)));
    case ORC_LIM_VANLEER: return (th + fabs(th)) / (1.0 + fabs(th));
    case ORC_LIM_MC: return fmax(0.0, fmin((1.0 + th) / 2.0, fmin(2.0, 2.0 * th)));
    default: return 1.0;
  }
}

/* Second-order correction flux at one interface (Eq. (lwflux), LeVeque 1997):
 * F = 1/2 sum_p c_p Wlim^p, c_p = |s|(1 - dt/dx |s|) (waves) or
 * sign(s)(1 - dt/dx |s|) (f-waves).  Wlim^p = phi(theta) W^p with
 * theta = (W^p_up . W^p)/(W^p . W^p), upwind side by the sign of s^p
 * (s > 0: left neighbour, otherwise right); a zero wave stays zero. */
static void correction_flux(const orc_prob* P, int m, int nw, const double* Wl,
                            const double* W, const double* Wr, const double* s, double dtdx,
                            double* F) {
  double Wt[MAXW * MAXM];
  for (int p = 0; p < nw; ++p) {
    double nrm = 0.0;
    for (int k = 0; k < m; ++k) nrm += W[p * m + k] * W[p * m + k];
    double phi = 1.0;
    if (nrm == 0.0) {
      phi = 0.0;
    } else if (P->lim != ORC_LIM_NONE) {
      const double* Wu = (s[p] > 0.0) ? Wl : Wr;
      double dot = 0.0;
      for (int k = 0; k < m; ++k) dot += Wu[p * m + k] * W[p * m + k];
      phi = orc_phi(P->lim, dot / nrm);
    }
    for (int k = 0; k < m; ++k) Wt[p * m + k] = phi * W[p * m + k];
  }
  for (int k = 0; k < m; ++k) {
    double acc = 0.0;
    for (int p = 0; p < nw; ++p) {
      double a = fabs(s[p]);
      double sg = is_fwave(P) ? (s[p] > 0.0 ? 1.0 : (s[p] < 0.0 ? -1.0 : 0.0)) : a;
      acc += sg * (1.0 - dtdx * a) * Wt[p * m + k];
    }
    F[k] = 0.5 * acc;
  }
}

/* ------------------------------------------------------------------------ */
/* ghost cells (Sec. 4: periodic, reflecting, outflow, inflow)               */
/* ------------------------------------------------------------------------ */

static int wall_comp(const orc_prob* P, int dir) {
  if (P->rp == ORC_RP_ADVECTION) return -1;
  return comp_n(P, dir);
}

/* value of ghost cell index i (outside 0..n-1) along one direction */
static void ghost_source(int bc, int n, int i, int* src, int* mirror) {
  *mirror = 0;
  if (i < 0) {
    int k = -i; /* 1..g */
    if (bc == ORC_BC_PERIODIC) *src = n - k;
    else if (bc == ORC_BC_WALL) { *src = k - 1; *mirror = 1; }
    else *src = 0;
  } else {
    int k = i - (n - 1);
    if (bc == ORC_BC_PERIODIC) *src = k - 1;
    else if (bc == ORC_BC_WALL) { *src = n - k; *mirror = 1; }
    else *src = n - 1;
  }
}

void orc_fill_ghost(const orc_prob* P, const double* q, int ncomp, int g, int is_aux,
                    double* qg) {
  int nx = P->nx, ny = (P->ndim == 2) ? P->ny : 1;
  int gy = (P->ndim == 2) ? g : 0;
  int NX = nx + 2 * g, NY = ny + 2 * gy;
  size_t plane = (size_t)NX * NY;
  for (int c = 0; c < ncomp; ++c)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i)
        qg[c * plane + (size_t)(j + gy) * NX + (i + g)] = q[(size_t)c * nx * ny + (size_t)j * nx + i];
  /* x ghosts on interior rows */
  for (int j = 0; j < ny; ++j)
    for (int side = 0; side < 2; ++side)
      for (int k = 1; k <= g; ++k) {
        int i = side == 0 ? -k : nx - 1 + k;
        int bc = side == 0 ? P->bc_lo[0] : P->bc_hi[0];
        int src, mir;
        ghost_source(bc, nx, i, &src, &mir);
        for (int c = 0; c < ncomp; ++c) {
          double v = qg[c * plane + (size_t)(j + gy) * NX + (src + g)];
          if (!is_aux) {
            if (bc == ORC_BC_INFLOW) v = P->inflow[c];
            else if (mir && c == wall_comp(P, 0)) v = -v;
          }
          qg[c * plane + (size_t)(j + gy) * NX + (i + g)] = v;
        }
      }
  if (P->ndim < 2) return;
  /* y ghosts on all columns, including the x ghosts (defines the corners) */
  for (int i = -g; i < nx + g; ++i)
    for (int side = 0; side < 2; ++side)
      for (int k = 1; k <= g; ++k) {
        int j = side == 0 ? -k : ny - 1 + k;
        int bc = side == 0 ? P->bc_lo[1] : P->bc_hi[1];
        int src, mir;
        ghost_source(bc, ny, j, &src, &mir);
        for (int c = 0; c < ncomp; ++c) {
          double v = qg[c * plane + (size_t)(src + gy) * NX + (i + g)];
          if (!is_aux) {
            if (bc == ORC_BC_INFLOW) v = P->inflow[c];
            else if (mir && c == wall_comp(P, 1)) v = -v;
          }
          qg[c * plane + (size_t)(j + gy) * NX + (i + g)] = v;
        }
      }
}

/* ------------------------------------------------------------------------ */
/* helpers to read one cell of a ghosted array                               */
/* ------------------------------------------------------------------------ */

typedef struct {
  const double* a;
  int ncomp, NX, NY, g, gy;
} garr;

static void gcell(const garr* G, int i, int j, double* out) {
  size_t plane = (size_t)G->NX * G->NY;
  size_t off = (size_t)(j + G->gy) * G->NX + (i + G->g);
  for (int c = 0; c < G->ncomp; ++c) out[c] = G->a[c * plane + off];
}

static double* ghosted(const orc_prob* P, const double* q, int ncomp, int g, int is_aux,
                       garr* G) {
  int ny = (P->ndim == 2) ? P->ny : 1;
  int gy = (P->ndim == 2) ? g : 0;
  G->ncomp = ncomp; G->g = g; G->gy = gy;
  G->NX = P->nx + 2 * g; G->NY = ny + 2 * gy;
  double* buf = (double*)malloc(sizeof(double) * (size_t)ncomp * G->NX * G->NY + 8);
  if (ncomp > 0) orc_fill_ghost(P, q, ncomp, g, is_aux, buf);
  G->a = buf;
  return buf;
}

/* ------------------------------------------------------------------------ */
/* classic 1D step (Eq. (fluxdiff) with Eq. (lwflux) in fluctuation form)   */
/* ------------------------------------------------------------------------ */

static int classic1d(const orc_prob* P, double* q, const double* aux, double dt, double* cfl) {
  int N = P->nx, m = P->num_eqn, ma = P->num_aux;
  int nw = orc_num_waves(P->rp, 1);
  double dtdx = dt / P->dx;
  garr Q, A;
  double* qb = ghosted(P, q, m, 2, 0, &Q);
  double* ab = ghosted(P, aux, ma, 2, 1, &A);
  int nint = N + 3; /* interfaces i = -1 .. N+1, stored at i+1 */
  double* W = (double*)malloc(sizeof(double) * nint * nw * m);
  double* S = (double*)malloc(sizeof(double) * nint * nw);
  double* AM = (double*)malloc(sizeof(double) * nint * m);
  double* AP = (double*)malloc(sizeof(double) * nint * m);
  double* F = (double*)calloc((size_t)(N + 1) * m, sizeof(double));
  double smax = 0.0;
  const int capa = P->capa_index;
  for (int i = -1; i <= N + 1; ++i) {
    double ql[MAXM], qr[MAXM], al[MAXM] = {0}, ar[MAXM] = {0};
    gcell(&Q, i - 1, 0, ql);
    gcell(&Q, i, 0, qr);
    if (ma) { gcell(&A, i - 1, 0, al); gcell(&A, i, 0, ar); }
    int ii = i + 1;
    orc_riemann(P, 0, ql, qr, al, ar, W + ii * nw * m, S + ii * nw, AM + ii * m, AP + ii * m);
    if (i >= 0 && i <= N)
      for (int p = 0; p < nw; ++p) {
        double sp = S[ii * nw + p];
        /* with a capacity the Courant number of a wave uses the capacity of
         * the cell it moves into */
        double a = capa < 0 ? fabs(sp)
                            : (sp > 0.0 ? sp / ar[capa] : (sp < 0.0 ? -sp / al[capa] : 0.0));
        if (!(a <= smax)) smax = a; /* NaN propagates */
      }
  }
  if (P->order == 2)
    for (int i = 0; i <= N; ++i) {
      int ii = i + 1;
      double dtc = dtdx;
      if (capa >= 0) {
        double al[MAXM], ar[MAXM];
        gcell(&A, i - 1, 0, al); gcell(&A, i, 0, ar);
        dtc = 0.5 * (dtdx / al[capa] + dtdx / ar[capa]);
      }
      correction_flux(P, m, nw, W + (ii - 1) * nw * m, W + ii * nw * m, W + (ii + 1) * nw * m,
                      S + ii * nw, dtc, F + i * m);
    }
  for (int i = 0; i < N; ++i) {
    double dti = dtdx;
    if (capa >= 0) {
      double ac[MAXM];
      gcell(&A, i, 0, ac);
      dti = dtdx / ac[capa];
    }
    for (int k = 0; k < m; ++k) {
      double* qk = q + (size_t)k * N + i;
      *qk = *qk - dti * (AP[(i + 1) * m + k] + AM[(i + 2) * m + k]) -
            dti * (F[(i + 1) * m + k] - F[i * m + k]);
    }
  }
  *cfl = dt * smax / P->dx;
  free(qb); free(ab); free(W); free(S); free(AM); free(AP); free(F);
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* classic 2D unsplit step with transverse propagation (LeVeque 1997)        */
/* ------------------------------------------------------------------------ */

/* per x-interface (or y-interface) record */
typedef struct {
  double amdq[MAXM], apdq[MAXM], F[MAXM];
  double bm_ap[MAXM], bp_ap[MAXM], bm_am[MAXM], bp_am[MAXM];
} iface_rec;

/* One sweep in direction dir over lines; fills recs for interfaces 0..n of
 * lines -1..nl (line index l stored at l+1) and the per-line max speed. */
static void sweep(const orc_prob* P, int dir, const garr* Q, const garr* A, double dtdn,
                  iface_rec* recs, double* line_smax) {
  int m = P->num_eqn, ma = P->num_aux;
  int nw = orc_num_waves(P->rp, 2);
  int n = dir == 0 ? P->nx : P->ny;   /* cells along the line */
  int nl = dir == 0 ? P->ny : P->nx;  /* number of interior lines */
  #pragma omp parallel for schedule(static)
  for (int l = -1; l <= nl; ++l) {
    int nint = n + 3;
    double* W = (double*)malloc(sizeof(double) * nint * nw * m);
    double* S = (double*)malloc(sizeof(double) * nint * nw);
    double* AM = (double*)malloc(sizeof(double) * nint * m);
    double* AP = (double*)malloc(sizeof(double) * nint * m);
    double smax = 0.0;
    for (int i = -1; i <= n + 1; ++i) {
      double ql[MAXM], qr[MAXM], al[MAXM] = {0}, ar[MAXM] = {0};
      if (dir == 0) { gcell(Q, i - 1, l, ql); gcell(Q, i, l, qr); }
      else { gcell(Q, l, i - 1, ql); gcell(Q, l, i, qr); }
      if (ma) {
        if (dir == 0) { gcell(A, i - 1, l, al); gcell(A, i, l, ar); }
        else { gcell(A, l, i - 1, al); gcell(A, l, i, ar); }
      }
      int ii = i + 1;
      orc_riemann(P, dir, ql, qr, al, ar, W + ii * nw * m, S + ii * nw, AM + ii * m, AP + ii * m);
      if (i >= 0 && i <= n && l >= 0 && l < nl)
        for (int p = 0; p < nw; ++p) {
          double sp = S[ii * nw + p];
          double a = P->capa_index < 0
                         ? fabs(sp)
                         : (sp > 0.0 ? sp / ar[P->capa_index]
                                     : (sp < 0.0 ? -sp / al[P->capa_index] : 0.0));
          if (!(a <= smax)) smax = a;
        }
    }
    line_smax[l + 1] = smax;
    for (int i = 0; i <= n; ++i) {
      int ii = i + 1;
      iface_rec* R = recs + (size_t)(l + 1) * (n + 1) + i;
      for (int k = 0; k < m; ++k) {
        R->amdq[k] = AM[ii * m + k];
        R->apdq[k] = AP[ii * m + k];
        R->F[k] = 0.0;
      }
      double kl = 1.0, kr = 1.0;  /* capacities of the two cells */
      if (P->capa_index >= 0) {
        double al[MAXM], ar[MAXM];
        if (dir == 0) { gcell(A, i - 1, l, al); gcell(A, i, l, ar); }
        else { gcell(A, l, i - 1, al); gcell(A, l, i, ar); }
        kl = al[P->capa_index];
        kr = ar[P->capa_index];
      }
      if (P->order == 2)
        correction_flux(P, m, nw, W + (ii - 1) * nw * m, W + ii * nw * m,
                        W + (ii + 1) * nw * m, S + ii * nw,
                        P->capa_index < 0 ? dtdn : 0.5 * (dtdn / kl + dtdn / kr), R->F);
      if (P->transverse) {
        double ql[MAXM], qr[MAXM], al[MAXM] = {0}, ar[MAXM] = {0};
        double ap[MAXM], am[MAXM];
        if (dir == 0) { gcell(Q, i - 1, l, ql); gcell(Q, i, l, qr); }
        else { gcell(Q, l, i - 1, ql); gcell(Q, l, i, qr); }
        if (ma) {
          if (dir == 0) { gcell(A, i - 1, l, al); gcell(A, i, l, ar); }
          else { gcell(A, l, i - 1, al); gcell(A, l, i, ar); }
        }
        for (int k = 0; k < m; ++k) {
          if (P->transverse == 2) {
            ap[k] = R->apdq[k] - R->F[k];
            am[k] = R->amdq[k] + R->F[k];
          } else {
            ap[k] = R->apdq[k];
            am[k] = R->amdq[k];
          }
        }
        if (P->rp == ORC_RP_ACOUSTICS_VC) {
          /* the transverse neighbours of the cell each fluctuation enters */
          double m_r[MAXM], p_r[MAXM], m_l[MAXM], p_l[MAXM];
          if (dir == 0) {
            gcell(A, i, l - 1, m_r); gcell(A, i, l + 1, p_r);
            gcell(A, i - 1, l - 1, m_l); gcell(A, i - 1, l + 1, p_l);
          } else {
            gcell(A, l - 1, i, m_r); gcell(A, l + 1, i, p_r);
            gcell(A, l - 1, i - 1, m_l); gcell(A, l + 1, i - 1, p_l);
          }
          orc_transverse_vc(P, dir, m_r, ar, p_r, ap, R->bm_ap, R->bp_ap);
          orc_transverse_vc(P, dir, m_l, al, p_l, am, R->bm_am, R->bp_am);
        } else {
          orc_transverse(P, dir, ql, qr, al, ar, ap, R->bm_ap, R->bp_ap);
          orc_transverse(P, dir, ql, qr, al, ar, am, R->bm_am, R->bp_am);
        }
        if (P->capa_index >= 0)
          /* transverse parts scaled by the capacity of the cell their
           * fluctuation enters (right cell for A^+, left for A^-) */
          for (int k = 0; k < m; ++k) {
            R->bm_ap[k] /= kr; R->bp_ap[k] /= kr;
            R->bm_am[k] /= kl; R->bp_am[k] /= kl;
          }
      } else {
        for (int k = 0; k < m; ++k) {
          R->bm_ap[k] = 0.0; R->bp_ap[k] = 0.0; R->bm_am[k] = 0.0; R->bp_am[k] = 0.0;
        }
      }
    }
    free(W); free(S); free(AM); free(AP);
  }
}

/* mask: 1 x-interfaces only, 2 y-interfaces only (one sweep of the
 * dimensionally split method, no transverse terms), 3 the unsplit step */
static int classic2d(const orc_prob* P, double* q, const double* aux, double dt, double* cfl,
                     int mask) {
  int nx = P->nx, ny = P->ny, m = P->num_eqn, ma = P->num_aux;
  double dtdx = (mask & 1) ? dt / P->dx : 0.0, dtdy = (mask & 2) ? dt / P->dy : 0.0;
  garr Q, A;
  double* qb = ghosted(P, q, m, 2, 0, &Q);
  double* ab = ghosted(P, aux, ma, 2, 1, &A);
  /* x-interfaces: i = 0..nx on rows -1..ny ; y-interfaces: j = 0..ny on columns -1..nx */
  iface_rec* X = (iface_rec*)malloc(sizeof(iface_rec) * (size_t)(ny + 2) * (nx + 1));
  iface_rec* Y = (iface_rec*)malloc(sizeof(iface_rec) * (size_t)(nx + 2) * (ny + 1));
  double* smx = (double*)malloc(sizeof(double) * (ny + 2));
  double* smy = (double*)malloc(sizeof(double) * (nx + 2));
  orc_prob Ps = *P;
  if (mask != 3) Ps.transverse = 0;
  sweep(&Ps, 0, &Q, &A, dtdx, X, smx);
  sweep(&Ps, 1, &Q, &A, dtdy, Y, smy);
#define XR(i, j) (X + (size_t)((j) + 1) * (nx + 1) + (i))
#define YR(i, j) (Y + (size_t)((i) + 1) * (ny + 1) + (j))
  /* total correction fluxes: normal part plus transverse contributions */
  double* Ft = (double*)malloc(sizeof(double) * (size_t)ny * (nx + 1) * m);
  double* Gt = (double*)malloc(sizeof(double) * (size_t)nx * (ny + 1) * m);
  #pragma omp parallel for schedule(static)
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i <= nx; ++i)
      for (int k = 0; k < m; ++k) {
        /* x-interface (i,j) receives A^+ b^+ of y-interface (i-1, j), A^- b^+ of (i, j),
           A^+ b^- of (i-1, j+1) and A^- b^- of (i, j+1) */
        double tr = YR(i - 1, j)->bp_ap[k] + YR(i, j)->bm_ap[k] + YR(i - 1, j + 1)->bp_am[k] +
                    YR(i, j + 1)->bm_am[k];
        Ft[((size_t)j * (nx + 1) + i) * m + k] = XR(i, j)->F[k] - 0.5 * dtdy * tr;
      }
  #pragma omp parallel for schedule(static)
  for (int i = 0; i < nx; ++i)
    for (int j = 0; j <= ny; ++j)
      for (int k = 0; k < m; ++k) {
        /* y-interface (i,j) receives B^+ a^+ of x-interface (i, j-1), B^- a^+ of (i, j),
           B^+ a^- of (i+1, j-1) and B^- a^- of (i+1, j) */
        double tr = XR(i, j - 1)->bp_ap[k] + XR(i, j)->bm_ap[k] + XR(i + 1, j - 1)->bp_am[k] +
                    XR(i + 1, j)->bm_am[k];
        Gt[((size_t)i * (ny + 1) + j) * m + k] = YR(i, j)->F[k] - 0.5 * dtdx * tr;
      }
  #pragma omp parallel for schedule(static)
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      /* capacity-form differencing: the cell's updates divided by its kappa */
      double cx = dtdx, cy = dtdy;
      if (P->capa_index >= 0) {
        double ac[MAXM];
        gcell(&A, i, j, ac);
        cx = dtdx / ac[P->capa_index];
        cy = dtdy / ac[P->capa_index];
      }
      for (int k = 0; k < m; ++k) {
        double* qk = q + (size_t)k * nx * ny + (size_t)j * nx + i;
        double fl = Ft[((size_t)j * (nx + 1) + i) * m + k];
        double fr = Ft[((size_t)j * (nx + 1) + i + 1) * m + k];
        double gb = Gt[((size_t)i * (ny + 1) + j) * m + k];
        double gtp = Gt[((size_t)i * (ny + 1) + j + 1) * m + k];
        *qk = *qk - cx * (XR(i, j)->apdq[k] + XR(i + 1, j)->amdq[k]) -
              cy * (YR(i, j)->apdq[k] + YR(i, j + 1)->amdq[k]) - cx * (fr - fl) -
              cy * (gtp - gb);
      }
    }
#undef XR
#undef YR
  double sx = 0.0, sy = 0.0;
  for (int l = 0; l < ny + 2; ++l) if (!(smx[l] <= sx)) sx = smx[l];
  for (int l = 0; l < nx + 2; ++l) if (!(smy[l] <= sy)) sy = smy[l];
  double nx_ = (mask & 1) ? dt * sx / P->dx : 0.0, ny_ = (mask & 2) ? dt * sy / P->dy : 0.0;
  *cfl = (nx_ >= ny_ || isnan(nx_)) ? nx_ : ny_;
  free(qb); free(ab); free(X); free(Y); free(smx); free(smy); free(Ft); free(Gt);
  return ORC_OK;
}

static int classic3d(const orc_prob* P, double* q, double dt, double* cfl);

/* ------------------------------------------------------------------------ */
/* source terms by fractional steps (Sec. 2, Eq. (conslaw) right-hand side;  */
/* Sec. 7.2 axisymmetric Euler)                                              */
/* ------------------------------------------------------------------------ */

/* axisymmetric geometric source of the Euler equations in (z, r) = (x, y):
 * psi = -(1/r) (rho v, rho u v, rho v^2, (E + p) v) with v the radial
 * velocity; the tracer has none */
static void axisym_source(const orc_prob* P, const double* q, double r, double* f) {
  int m = P->num_eqn;
  double rho = q[0], u = q[1] / rho, v = q[2] / rho;
  double p = euler_pressure(P, q);
  for (int k = 0; k < m; ++k) f[k] = 0.0;
  f[0] = -(rho * v) / r;
  f[1] = -(rho * u * v) / r;
  f[2] = -(rho * v * v) / r;
  f[3] = -((q[3] + p) * v) / r;
}

/* the source ODE q' = psi(q) over dt in every cell by the two-stage
 * second-order Runge-Kutta method (Heun): q1 = q + dt psi(q),
 * q <- (q + q1 + dt psi(q1)) / 2 */
void orc_source_step(const orc_prob* P, double* q, double dt) {
  if (P->source != 1) return;
  int nx = P->nx, ny = P->ny, m = P->num_eqn;
  size_t plane = (size_t)nx * ny;
  #pragma omp parallel for schedule(static)
  for (int j = 0; j < ny; ++j) {
    double r = P->lower[1] + (j + 0.5) * P->dy;
    for (int i = 0; i < nx; ++i) {
      double q0[MAXM], q1[MAXM], f0[MAXM], f1[MAXM];
      size_t off = (size_t)j * nx + i;
      for (int k = 0; k < m; ++k) q0[k] = q[k * plane + off];
      axisym_source(P, q0, r, f0);
      for (int k = 0; k < m; ++k) q1[k] = q0[k] + dt * f0[k];
      axisym_source(P, q1, r, f1);
      for (int k = 0; k < m; ++k) q[k * plane + off] = 0.5 * (q0[k] + (q1[k] + dt * f1[k]));
    }
  }
}

/* the source before the hyperbolic step: a half step for Strang splitting,
 * nothing for Godunov */
static void source_before(const orc_prob* P, double* q, double dt) {
  if (P->ndim == 2 && P->source_split == 2) orc_source_step(P, q, 0.5 * dt);
}
/* the source after an accepted hyperbolic step: the other Strang half step,
 * or the whole step for Godunov */
static void source_after(const orc_prob* P, double* q, double dt) {
  if (P->ndim == 2) orc_source_step(P, q, P->source_split == 2 ? 0.5 * dt : dt);
}

int orc_classic_step(const orc_prob* P, double* q, const double* aux, double dt, double* cfl) {
  if (P->ndim == 1) return classic1d(P, q, aux, dt, cfl);
  /* the 2D p-system is solved with SharpClaw only (normal solves, Sec. 7.3) */
  if (P->ndim == 2 && P->rp == ORC_RP_ELASTICITY_FWAVE) return ORC_EINVAL;
  if (P->ndim == 3) return classic3d(P, q, dt, cfl);
  int st;
  source_before(P, q, dt);
  if (P->dim_split) {
    /* Godunov dimensional splitting: x sweeps over dt, then y sweeps over dt */
    double c1 = 0.0, c2 = 0.0;
    st = classic2d(P, q, aux, dt, &c1, 1);
    if (st == ORC_OK) st = classic2d(P, q, aux, dt, &c2, 2);
    *cfl = (c1 >= c2 || isnan(c1)) ? c1 : c2;
  } else {
    st = classic2d(P, q, aux, dt, cfl, 3);
  }
  if (st == ORC_OK) source_after(P, q, dt);
  return st;
}


/* ------------------------------------------------------------------------ */
/* classic 3D unsplit step with transverse and double-transverse propagation */
/* (LeVeque 1997): advection and linear acoustics                            */
/* ------------------------------------------------------------------------ */

/* cell (i,j,k) of a ghosted 3D array with ghost width 2, ncomp fields */
typedef struct {
  const double* a;
  int m, NX, NY, NZ;
} g3arr;

static void g3cell(const g3arr* G, int i, int j, int k, double* out) {
  size_t plane = (size_t)G->NX * G->NY * G->NZ;
  size_t off = ((size_t)(k + 2) * G->NY + (j + 2)) * G->NX + (i + 2);
  for (int c = 0; c < G->m; ++c) out[c] = G->a[c * plane + off];
}

/* ghost cells of a 3D array: x ghosts on interior (y,z) rows, then y ghosts on
 * all x for interior z, then z ghosts everywhere */
static void fill_ghost3(const orc_prob* P, const double* q, double* qg) {
  const int nx = P->nx, ny = P->ny, nz = P->nz, m = P->num_eqn, g = 2;
  const int NX = nx + 2 * g, NY = ny + 2 * g, NZ = nz + 2 * g;
  const size_t plane = (size_t)NX * NY * NZ;
#define QG(c, i, j, k) qg[(c) * plane + ((size_t)((k) + g) * NY + ((j) + g)) * NX + ((i) + g)]
  for (int c = 0; c < m; ++c)
    for (int k = 0; k < nz; ++k)
      for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i)
          QG(c, i, j, k) = q[(size_t)c * nx * ny * nz + ((size_t)k * ny + j) * nx + i];
  const int n3[3] = {nx, ny, nz};
  for (int d = 0; d < 3; ++d) {
    /* ranges: directions before d include ghosts, after d interior only */
    int lo[3], hi[3];
    for (int e = 0; e < 3; ++e) {
      lo[e] = e < d ? -g : 0;
      hi[e] = e < d ? n3[e] + g : n3[e];
    }
    for (int side = 0; side < 2; ++side)
      for (int kk = 1; kk <= g; ++kk) {
        int gi = side == 0 ? -kk : n3[d] - 1 + kk;
        int bc = side == 0 ? P->bc_lo[d] : P->bc_hi[d];
        int src, mir;
        ghost_source(bc, n3[d], gi, &src, &mir);
        int wall = wall_comp(P, d);
        for (int a = lo[(d + 1) % 3]; a < hi[(d + 1) % 3]; ++a)
          for (int b = lo[(d + 2) % 3]; b < hi[(d + 2) % 3]; ++b) {
            int idx[3], sidx[3];
            idx[d] = gi;
            idx[(d + 1) % 3] = a;
            idx[(d + 2) % 3] = b;
            sidx[0] = idx[0]; sidx[1] = idx[1]; sidx[2] = idx[2];
            sidx[d] = src;
            for (int c = 0; c < m; ++c) {
              double v = QG(c, sidx[0], sidx[1], sidx[2]);
              if (bc == ORC_BC_INFLOW) v = P->inflow[c];
              else if (mir && c == wall) v = -v;
              QG(c, idx[0], idx[1], idx[2]) = v;
            }
          }
      }
  }
#undef QG
}

/* normal solve of a 3D problem in direction d */
static void rp3(const orc_prob* P, int d, const double* ql, const double* qr, double* W,
                double* s, double* amdq, double* apdq) {
  int m = P->num_eqn;
  if (P->rp == ORC_RP_ADVECTION) {
    W[0] = qr[0] - ql[0];
    s[0] = P->params[d];
  } else {
    /* acoustics (p, u, v, w): the two waves of the normal velocity 1+d */
    double alpha[MAXW], r[MAXW * MAXM], d_[MAXM] = {0};
    int n = 1 + d;
    for (int k = 0; k < m; ++k) d_[k] = qr[k] - ql[k];
    acoustics_eig(P, n, -1, 0, d_, alpha, r, s);
    for (int p = 0; p < 2; ++p)
      for (int k = 0; k < m; ++k) W[p * m + k] = alpha[p] * r[p * m + k];
  }
  split_by_speed(m, orc_num_waves(P->rp, 3), W, s, amdq, apdq);
}

/* split a (a fluctuation of a d-normal solve) in direction e */
static void trans3(const orc_prob* P, int e, const double* a, double* em, double* ep) {
  int m = P->num_eqn;
  for (int k = 0; k < m; ++k) { em[k] = 0.0; ep[k] = 0.0; }
  if (P->rp == ORC_RP_ADVECTION) {
    double v = P->params[e];
    em[0] = fmin(v, 0.0) * a[0];
    ep[0] = fmax(v, 0.0) * a[0];
    return;
  }
  double beta[MAXW], r[MAXW * MAXM], lam[MAXW];
  acoustics_eig(P, 1 + e, -1, 0, a, beta, r, lam);
  for (int p = 0; p < 2; ++p)
    for (int k = 0; k < m; ++k) {
      em[k] += fmin(lam[p], 0.0) * beta[p] * r[p * m + k];
      ep[k] += fmax(lam[p], 0.0) * beta[p] * r[p * m + k];
    }
}

/* add coef*v to the flux correction of the face (f0,f1,f2) in direction e
 * when that face bounds an interior cell */
static void add_face(const orc_prob* P, double* Fe, int e, const int* f, double coef,
                     const double* v) {
  const int n3[3] = {P->nx, P->ny, P->nz};
  for (int d = 0; d < 3; ++d) {
    int hi = (d == e) ? n3[d] : n3[d] - 1;
    if (f[d] < 0 || f[d] > hi) return;
  }
  const int NXF = P->nx + (e == 0), NYF = P->ny + (e == 1);
  size_t off = (((size_t)f[2] * NYF + f[1]) * NXF + f[0]) * P->num_eqn;
  for (int k = 0; k < P->num_eqn; ++k) Fe[off + k] += coef * v[k];
}

static int classic3d(const orc_prob* P, double* q, double dt, double* cfl) {
  const int nx = P->nx, ny = P->ny, nz = P->nz, m = P->num_eqn;
  const int nw = orc_num_waves(P->rp, 3);
  const double dxs[3] = {P->dx, P->dy, P->dz};
  const int n3[3] = {nx, ny, nz};
  g3arr Q;
  Q.m = m; Q.NX = nx + 4; Q.NY = ny + 4; Q.NZ = nz + 4;
  double* qb = (double*)malloc(sizeof(double) * (size_t)m * Q.NX * Q.NY * Q.NZ);
  fill_ghost3(P, q, qb);
  Q.a = qb;
  /* per direction: fluctuations and total flux corrections on interior faces */
  double* AM[3];
  double* AP[3];
  double* FC[3];
  for (int e = 0; e < 3; ++e) {
    size_t nf = (size_t)(nx + (e == 0)) * (ny + (e == 1)) * (nz + (e == 2)) * m;
    AM[e] = (double*)calloc(nf, sizeof(double));
    AP[e] = (double*)calloc(nf, sizeof(double));
    FC[e] = (double*)calloc(nf, sizeof(double));
  }
  double smax[3] = {0.0, 0.0, 0.0};
  for (int d = 0; d < 3; ++d) {
    const int e1 = (d + 1) % 3, e2 = (d + 2) % 3;
    const double dtdn = dt / dxs[d];
    const int n = n3[d];
    double* W = (double*)malloc(sizeof(double) * (n + 3) * nw * m);
    double* S = (double*)malloc(sizeof(double) * (n + 3) * nw);
    double* AMl = (double*)malloc(sizeof(double) * (n + 3) * m);
    double* APl = (double*)malloc(sizeof(double) * (n + 3) * m);
    /* lines along d, one ghost layer in each transverse direction */
    for (int a = -1; a <= n3[e1]; ++a)
      for (int b = -1; b <= n3[e2]; ++b) {
        const int interior_line = a >= 0 && a < n3[e1] && b >= 0 && b < n3[e2];
        for (int i = -1; i <= n + 1; ++i) {
          int il[3], ir[3];
          il[d] = i - 1; ir[d] = i;
          il[e1] = ir[e1] = a;
          il[e2] = ir[e2] = b;
          double ql[MAXM], qr[MAXM];
          g3cell(&Q, il[0], il[1], il[2], ql);
          g3cell(&Q, ir[0], ir[1], ir[2], qr);
          int ii = i + 1;
          rp3(P, d, ql, qr, W + ii * nw * m, S + ii * nw, AMl + ii * m, APl + ii * m);
          if (interior_line && i >= 0 && i <= n)
            for (int p = 0; p < nw; ++p) {
              double v = fabs(S[ii * nw + p]);
              if (!(v <= smax[d])) smax[d] = v;
            }
        }
        for (int i = 0; i <= n; ++i) {
          int ii = i + 1;
          double F[MAXM] = {0};
          if (P->order == 2)
            correction_flux(P, m, nw, W + (ii - 1) * nw * m, W + ii * nw * m,
                            W + (ii + 1) * nw * m, S + ii * nw, dtdn, F);
          int f[3];
          f[d] = i; f[e1] = a; f[e2] = b;
          /* normal fluctuations and correction on this face */
          add_face(P, AM[d], d, f, 1.0, AMl + ii * m);
          add_face(P, AP[d], d, f, 1.0, APl + ii * m);
          add_face(P, FC[d], d, f, 1.0, F);
          if (!P->transverse) continue;
          double apq[MAXM], amq[MAXM];
          for (int k = 0; k < m; ++k) {
            apq[k] = APl[ii * m + k] - (P->transverse == 2 ? F[k] : 0.0);
            amq[k] = AMl[ii * m + k] + (P->transverse == 2 ? F[k] : 0.0);
          }
          for (int side = 0; side < 2; ++side) {
            /* a+ goes into the cell at d-index i, a- into the cell at i-1 */
            const double* av = side == 0 ? apq : amq;
            int c[3];
            c[d] = side == 0 ? i : i - 1; c[e1] = a; c[e2] = b;
            for (int t = 0; t < 2; ++t) {
              const int e = t == 0 ? e1 : e2, g2 = t == 0 ? e2 : e1;
              double em[MAXM], ep[MAXM];
              trans3(P, e, av, em, ep);
              /* transverse: faces of cell c in direction e */
              int fu[3] = {c[0], c[1], c[2]};
              fu[e] = c[e] + 1;
              add_face(P, FC[e], e, fu, -0.5 * dtdn, ep);
              add_face(P, FC[e], e, c, -0.5 * dtdn, em);
              /* double transverse: the part E^+-a of the fluctuation has moved on
                 into cell c +- 1 in e, so its share of the third-direction (g2)
                 transverse flux moves from the g2-faces of c to those of c +- 1:
                 +1/6 (dt/dx_d)(dt/dx_e) G^+-E^+-a at c's faces, -1/6 at the
                 shifted cell's faces (six orderings of the three directions
                 make the corner-transport-upwind triple term) */
              const double dte = dt / dxs[e];
              for (int sgn = 0; sgn < 2; ++sgn) {
                /* E^+ a moves up in e (positive speeds), E^- a down (negative
                   speeds, so the moved amount is -E^- a) */
                const double* bv = sgn == 0 ? ep : em;
                const double k6 = (sgn == 0 ? 1.0 : -1.0) * dtdn * dte / 6.0;
                int c2[3] = {c[0], c[1], c[2]};
                c2[e] += sgn == 0 ? 1 : -1;
                double gm[MAXM], gp[MAXM];
                trans3(P, g2, bv, gm, gp);
                int fu1[3] = {c[0], c[1], c[2]};
                fu1[g2] = c[g2] + 1;
                add_face(P, FC[g2], g2, fu1, k6, gp);
                add_face(P, FC[g2], g2, c, k6, gm);
                int fu2[3] = {c2[0], c2[1], c2[2]};
                fu2[g2] = c2[g2] + 1;
                add_face(P, FC[g2], g2, fu2, -k6, gp);
                add_face(P, FC[g2], g2, c2, -k6, gm);
              }
            }
          }
        }
      }
    free(W); free(S); free(AMl); free(APl);
  }
  /* conservative update */
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i)
        for (int c = 0; c < m; ++c) {
          double* qc = q + (size_t)c * nx * ny * nz + ((size_t)k * ny + j) * nx + i;
          double upd = *qc;
          for (int d = 0; d < 3; ++d) {
            const int NXF = nx + (d == 0), NYF = ny + (d == 1);
            int lo[3] = {i, j, k}, hi[3] = {i, j, k};
            hi[d] += 1;
            size_t ol = (((size_t)lo[2] * NYF + lo[1]) * NXF + lo[0]) * m + c;
            size_t oh = (((size_t)hi[2] * NYF + hi[1]) * NXF + hi[0]) * m + c;
            const double dtdn = dt / dxs[d];
            upd = upd - dtdn * (AP[d][ol] + AM[d][oh]) - dtdn * (FC[d][oh] - FC[d][ol]);
          }
          *qc = upd;
        }
  double nu = 0.0;
  for (int d = 0; d < 3; ++d) {
    double v = dt * smax[d] / dxs[d];
    if (!(v <= nu)) nu = v;
  }
  *cfl = nu;
  free(qb);
  for (int e = 0; e < 3; ++e) { free(AM[e]); free(AP[e]); free(FC[e]); }
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* SharpClaw: WENO5 reconstruction + fluctuations + SSP-RK3                  */
/* ------------------------------------------------------------------------ */

/* Jiang-Shu WENO5, left-biased value at x_{i+1/2} from v_{i-2..i+2} */
double orc_weno5(const double* v, double eps) {
  double a = v[0], b = v[1], c = v[2], d = v[3], e = v[4];
  double q0 = (2.0 * a - 7.0 * b + 11.0 * c) / 6.0;
  double q1 = (-b + 5.0 * c + 2.0 * d) / 6.0;
  double q2 = (2.0 * c + 5.0 * d - e) / 6.0;
  double t0 = a - 2.0 * b + c, u0 = a - 4.0 * b + 3.0 * c;
  double t1 = b - 2.0 * c + d, u1 = b - d;
  double t2 = c - 2.0 * d + e, u2 = 3.0 * c - 4.0 * d + e;
  double b0 = 13.0 / 12.0 * (t0 * t0) + 0.25 * (u0 * u0);
  double b1 = 13.0 / 12.0 * (t1 * t1) + 0.25 * (u1 * u1);
  double b2 = 13.0 / 12.0 * (t2 * t2) + 0.25 * (u2 * u2);
  double e0 = eps + b0, e1 = eps + b1, e2 = eps + b2;
  double a0 = 0.1 / (e0 * e0), a1 = 0.6 / (e1 * e1), a2 = 0.3 / (e2 * e2);
  double sum = a0 + a1 + a2;
  return (a0 * q0 + a1 * q1 + a2 * q2) / sum;
}

/* WENO of order 2r-1 (Jiang-Shu weights d_k / (eps + beta_k)^2 normalised to
 * sum 1): candidate values q_k = sum_j c[k][j] v[k+j], smoothness beta_k =
 * v_k^T B[k] v_k over the stencil's r cells.  beta measures derivatives only,
 * so it is unchanged when a constant is subtracted from the data; the form is
 * evaluated on v - v[k] to keep its rounding relative to the variation. */
/* Error-free transformations: a + b = s + e exactly (Knuth's TwoSum) and
 * a b = p + e exactly (by one fused multiply-add). */
static void two_sum(double a, double b, double* s, double* e) {
  *s = a + b;
  const double z = *s - a;
  *e = (a - (*s - z)) + (b - z);
}
static void two_prod(double a, double b, double* p, double* e) {
  *p = a * b;
  *e = fma(a, b, -*p);
}

/* The smoothness indicator beta = sum_a sum_b B_ab dv_a dv_b on the
 * differences dv_j = v_j - v_0 (Sec. 3.3: the form of sum_l int (p^(l))^2).
 * Its terms grow with the order (coefficients in the thousands at orders 15
 * and 17) while beta itself stays of the size of dv^2, so a plain running sum
 * would carry rounding errors far above beta's own; the products and the sum
 * are therefore evaluated by error-free transformations with compensation
 * (Ogita, Rump and Oishi, "Accurate sum and dot product", 2005), which
 * returns the form's value to about one rounding. */
static double smoothness_form(int r, const double* Bk, const double* v) {
  double hi = 0.0, lo = 0.0;
  for (int a = 0; a < r; ++a) {
    const double da = v[a] - v[0];
    for (int b = 0; b < r; ++b) {
      const double db = v[b] - v[0];
      double x, xe, y, ye, se;
      two_prod(Bk[a * r + b], da, &x, &xe);  /* B da = x + xe */
      two_prod(x, db, &y, &ye);              /* x db = y + ye */
      two_sum(hi, y, &hi, &se);
      lo += se + ye + xe * db;
    }
  }
  return hi + lo;
}

double orc_weno_r(int r, const double* c, const double* d, const double* B, const double* v,
                  double eps) {
  double qk[9], alpha[9], sum = 0.0;
  for (int k = 0; k < r; ++k) {
    double q = 0.0;
    for (int j = 0; j < r; ++j) q += c[k * r + j] * v[k + j];
    const double beta = smoothness_form(r, B + k * r * r, v + k);
    qk[k] = q;
    alpha[k] = d[k] / ((eps + beta) * (eps + beta));
    sum += alpha[k];
  }
  double out = 0.0;
  for (int k = 0; k < r; ++k) out += (alpha[k] / sum) * qk[k];
  return out;
}

/* left-biased edge value of the problem's WENO order from v[0..2r-2] */
static double weno_edge(const orc_prob* P, int r, const double* v) {
  if (r == 3) return orc_weno5(v, P->weno_eps);
  return orc_weno_r(r, P->weno_c, P->weno_d, P->weno_b, v, P->weno_eps);
}

int orc_sharp_L(const orc_prob* P, const double* q, const double* aux, double* L, double* smax) {
  int m = P->num_eqn, ma = P->num_aux;
  int nx = P->nx, ny = (P->ndim == 2) ? P->ny : 1;
  size_t ncell = (size_t)nx * ny;
  const int r = P->weno_r > 3 ? P->weno_r : 3;  /* ghost width and stencil half-width */
  if (r > 9) return ORC_EINVAL;
  garr Q, A;
  double* qb = ghosted(P, q, m, r, 0, &Q);
  double* ab = ghosted(P, aux, ma, r, 1, &A);
  if (P->char_decomp && P->rp == ORC_RP_ELASTICITY_FWAVE) { free(qb); free(ab); return ORC_EINVAL; }
  for (size_t c = 0; c < ncell * m; ++c) L[c] = 0.0;
  smax[0] = 0.0; smax[1] = 0.0;
  for (int dir = 0; dir < P->ndim; ++dir) {
    int n = dir == 0 ? nx : ny;
    int nl = dir == 0 ? ny : nx;
    double dn = dir == 0 ? P->dx : P->dy;
    double* lmax = (double*)calloc(nl, sizeof(double));
    #pragma omp parallel for schedule(static)
    for (int l = 0; l < nl; ++l) {
      double* qL = (double*)malloc(sizeof(double) * (n + 1) * m);  /* left edge of cell i   */
      double* qR = (double*)malloc(sizeof(double) * (n + 1) * m);  /* right edge of cell i-1 */
      double* AM = (double*)malloc(sizeof(double) * (n + 1) * m);
      double* AP = (double*)malloc(sizeof(double) * (n + 1) * m);
      double sm = 0.0;
      /* reconstruction at every interface i - 1/2, i = 0..n */
      for (int i = 0; i <= n; ++i) {
        /* the 2r cells i-r .. i+r-1 around interface i - 1/2 */
        double cells[18][MAXM], w[18][MAXM];
        double Lm[MAXM * MAXM], Rm[MAXM * MAXM];
        for (int k6 = 0; k6 < 2 * r; ++k6) {
          int ci = i - r + k6;
          if (dir == 0) gcell(&Q, ci, l, cells[k6]); else gcell(&Q, l, ci, cells[k6]);
        }
        if (P->char_decomp) {
          orc_char_matrices(P, dir, cells[r - 1], cells[r], Lm, Rm);
          for (int k6 = 0; k6 < 2 * r; ++k6)
            for (int p = 0; p < m; ++p) {
              double acc = 0.0;
              for (int k = 0; k < m; ++k) acc += Lm[p * m + k] * cells[k6][k];
              w[k6][p] = acc;
            }
        } else {
          for (int k6 = 0; k6 < 2 * r; ++k6)
            for (int p = 0; p < m; ++p) w[k6][p] = cells[k6][p];
        }
        double wm[MAXM], wp[MAXM];
        for (int p = 0; p < m; ++p) {
          double v[17];
          for (int k = 0; k < 2 * r - 1; ++k) v[k] = w[k][p];          /* cells i-r..i+r-2 */
          wm[p] = weno_edge(P, r, v);                                   /* right edge of cell i-1 */
          for (int k = 0; k < 2 * r - 1; ++k) v[k] = w[2 * r - 1 - k][p]; /* cells i+r-1..i-r+1 */
          wp[p] = weno_edge(P, r, v);                                   /* left edge of cell i */
        }
        for (int k = 0; k < m; ++k) {
          if (P->char_decomp) {
            double am = 0.0, ap = 0.0;
            for (int p = 0; p < m; ++p) { am += Rm[k * m + p] * wm[p]; ap += Rm[k * m + p] * wp[p]; }
            qR[i * m + k] = am;
            qL[i * m + k] = ap;
          } else {
            qR[i * m + k] = wm[k];
            qL[i * m + k] = wp[k];
          }
        }
      }
      /* interface Riemann problems (q^R_{i-1}, q^L_i) */
      for (int i = 0; i <= n; ++i) {
        double al[MAXM] = {0}, ar[MAXM] = {0};
        double W[MAXW * MAXM], S[MAXW];
        if (ma) {
          if (dir == 0) { gcell(&A, i - 1, l, al); gcell(&A, i, l, ar); }
          else { gcell(&A, l, i - 1, al); gcell(&A, l, i, ar); }
        }
        orc_riemann(P, dir, qR + i * m, qL + i * m, al, ar, W, S, AM + i * m, AP + i * m);
        for (int p = 0; p < orc_num_waves(P->rp, P->ndim); ++p) {
          double sp = S[p];
          double a = P->capa_index < 0
                         ? fabs(sp)
                         : (sp > 0.0 ? sp / ar[P->capa_index]
                                     : (sp < 0.0 ? -sp / al[P->capa_index] : 0.0));
          if (!(a <= sm)) sm = a;
        }
      }
      /* total fluctuation inside each cell: Riemann problem (q^L_i, q^R_i) */
      for (int i = 0; i < n; ++i) {
        double al[MAXM] = {0};
        double W[MAXW * MAXM], S[MAXW], am[MAXM], ap[MAXM];
        if (ma) { if (dir == 0) gcell(&A, i, l, al); else gcell(&A, l, i, al); }
        orc_riemann(P, dir, qL + i * m, qR + (i + 1) * m, al, al, W, S, am, ap);
        size_t cell = dir == 0 ? (size_t)l * nx + i : (size_t)i * nx + l;
        /* with a capacity: -(1/(kappa_i dx)) (...) */
        double dnk = P->capa_index < 0 ? dn : dn * al[P->capa_index];
        for (int k = 0; k < m; ++k) {
          double adq = am[k] + ap[k];
          L[(size_t)k * ncell + cell] =
              L[(size_t)k * ncell + cell] - (AP[i * m + k] + AM[(i + 1) * m + k] + adq) / dnk;
        }
      }
      lmax[l] = sm;
      free(qL); free(qR); free(AM); free(AP);
    }
    for (int l = 0; l < nl; ++l) if (!(lmax[l] <= smax[dir])) smax[dir] = lmax[l];
    free(lmax);
  }
  free(qb); free(ab);
  return ORC_OK;
}

/* Shu-Osher SSP-RK3 stage: out = a_k Q^n + b_k (Q^(k) + dt L(Q^(k))) */
static double rk3_stage(int stage, double qn, double qk, double Lk, double dt) {
  if (stage == 0) return qk + dt * Lk;
  if (stage == 1) return 0.75 * qn + 0.25 * (qk + dt * Lk);
  return (1.0 / 3.0) * qn + (2.0 / 3.0) * (qk + dt * Lk);
}

double orc_ssp_rk3_linear(double lambda, double dt, double q0) {
  double q1 = rk3_stage(0, q0, q0, lambda * q0, dt);
  double q2 = rk3_stage(1, q0, q1, lambda * q1, dt);
  return rk3_stage(2, q0, q2, lambda * q2, dt);
}

/* Ketcheson's ten-stage fourth-order SSP method in its low-storage form:
 * five forward-Euler steps of size dt/6 on q1, then q2 = q2/25 + 9 q1/25,
 * q1 = 15 q2 - 5 q1, four more dt/6 steps on q1, and finally
 * q1 = q2 + 3/5 q1 + dt/10 L(q1).  Lfun evaluates L into its third argument
 * and returns the largest Courant number it saw (or NaN). */
typedef double (*lfun_t)(const void* ctx, const double* q, double* L);

static double ssp104(lfun_t Lf, const void* ctx, size_t n, double* q, double dt) {
  double* q1 = (double*)malloc(sizeof(double) * n);
  double* q2 = (double*)malloc(sizeof(double) * n);
  double* L = (double*)malloc(sizeof(double) * n);
  double nu = 0.0;
  memcpy(q1, q, sizeof(double) * n);
  memcpy(q2, q, sizeof(double) * n);
  for (int st = 0; st < 9; ++st) {
    double v = Lf(ctx, q1, L);
    if (!(v <= nu)) nu = v;
    for (size_t c = 0; c < n; ++c) q1[c] = q1[c] + dt / 6.0 * L[c];
    if (st == 4) {
      for (size_t c = 0; c < n; ++c) {
        q2[c] = q2[c] / 25.0 + 9.0 * q1[c] / 25.0;
        q1[c] = 15.0 * q2[c] - 5.0 * q1[c];
      }
    }
  }
  double v = Lf(ctx, q1, L);
  if (!(v <= nu)) nu = v;
  for (size_t c = 0; c < n; ++c) q[c] = q2[c] + 3.0 / 5.0 * q1[c] + dt / 10.0 * L[c];
  free(q1); free(q2); free(L);
  return nu;
}

static double lin_L(const void* ctx, const double* q, double* L) {
  L[0] = *(const double*)ctx * q[0];
  return 0.0;
}

double orc_ssp104_linear(double lambda, double dt, double q0) {
  double q = q0;
  ssp104(lin_L, &lambda, 1, &q, dt);
  return q;
}

typedef struct {
  const orc_prob* P;
  const double* aux;
  double dt;
  int status;
} sharp_ctx;

static double sharp_L_fn(const void* vctx, const double* q, double* L) {
  sharp_ctx* c = (sharp_ctx*)vctx;
  double smax[2];
  if (orc_sharp_L(c->P, q, c->aux, L, smax) != ORC_OK) c->status = ORC_EINVAL;
  double nu = 0.0;
  for (int d = 0; d < c->P->ndim; ++d) {
    double v = c->dt * smax[d] / (d == 0 ? c->P->dx : c->P->dy);
    if (!(v <= nu)) nu = v;
  }
  return nu;
}

int orc_sharp_step(const orc_prob* P, double* q, const double* aux, double dt, double* cfl) {
  source_before(P, q, dt);
  if (P->time_integrator == 1) {
    int ny1 = (P->ndim == 2) ? P->ny : 1;
    sharp_ctx c = {P, aux, dt, ORC_OK};
    *cfl = ssp104(sharp_L_fn, &c, (size_t)P->nx * ny1 * P->num_eqn, q, dt);
    if (c.status == ORC_OK) source_after(P, q, dt);
    return c.status;
  }
  int ny = (P->ndim == 2) ? P->ny : 1;
  size_t ntot = (size_t)P->nx * ny * P->num_eqn;
  double* qn = (double*)malloc(sizeof(double) * ntot);
  double* qk = (double*)malloc(sizeof(double) * ntot);
  double* L = (double*)malloc(sizeof(double) * ntot);
  memcpy(qn, q, sizeof(double) * ntot);
  memcpy(qk, q, sizeof(double) * ntot);
  double nu = 0.0;
  int st = ORC_OK;
  for (int stage = 0; stage < 3; ++stage) {
    double smax[2];
    st = orc_sharp_L(P, qk, aux, L, smax);
    if (st != ORC_OK) break;
    for (int d = 0; d < P->ndim; ++d) {
      double v = dt * smax[d] / (d == 0 ? P->dx : P->dy);
      if (!(v <= nu)) nu = v;
    }
    for (size_t c = 0; c < ntot; ++c) qk[c] = rk3_stage(stage, qn[c], qk[c], L[c], dt);
  }
  memcpy(q, qk, sizeof(double) * ntot);
  *cfl = nu;
  free(qn); free(qk); free(L);
  if (st == ORC_OK) source_after(P, q, dt);
  return st;
}

/* ------------------------------------------------------------------------ */
/* CFL control (Sec. 4: check the Courant number, choose the next step)      */
/* ------------------------------------------------------------------------ */

static void max_speeds3(const orc_prob* P, const double* q, double* smax) {
  const int nx = P->nx, ny = P->ny, nz = P->nz, m = P->num_eqn, nw = orc_num_waves(P->rp, 3);
  const int n3[3] = {nx, ny, nz};
  g3arr Q;
  Q.m = m; Q.NX = nx + 4; Q.NY = ny + 4; Q.NZ = nz + 4;
  double* qb = (double*)malloc(sizeof(double) * (size_t)m * Q.NX * Q.NY * Q.NZ);
  fill_ghost3(P, q, qb);
  Q.a = qb;
  for (int d = 0; d < 3; ++d) {
    smax[d] = 0.0;
    const int e1 = (d + 1) % 3, e2 = (d + 2) % 3;
    for (int a = 0; a < n3[e1]; ++a)
      for (int b = 0; b < n3[e2]; ++b)
        for (int i = 0; i <= n3[d]; ++i) {
          int il[3], ir[3];
          il[d] = i - 1; ir[d] = i;
          il[e1] = ir[e1] = a;
          il[e2] = ir[e2] = b;
          double ql[MAXM], qr[MAXM], W[MAXW * MAXM], S[MAXW], am[MAXM], ap[MAXM];
          g3cell(&Q, il[0], il[1], il[2], ql);
          g3cell(&Q, ir[0], ir[1], ir[2], qr);
          rp3(P, d, ql, qr, W, S, am, ap);
          for (int p = 0; p < nw; ++p) {
            double v = fabs(S[p]);
            if (!(v <= smax[d])) smax[d] = v;
          }
        }
  }
  free(qb);
}

void orc_max_speeds(const orc_prob* P, const double* q, const double* aux, double* smax) {
  if (P->ndim == 3) { max_speeds3(P, q, smax); return; }
  int m = P->num_eqn, ma = P->num_aux, nw = orc_num_waves(P->rp, P->ndim);
  int nx = P->nx, ny = (P->ndim == 2) ? P->ny : 1;
  garr Q, A;
  double* qb = ghosted(P, q, m, 2, 0, &Q);
  double* ab = ghosted(P, aux, ma, 2, 1, &A);
  smax[0] = 0.0; smax[1] = 0.0;
  for (int dir = 0; dir < P->ndim; ++dir) {
    int n = dir == 0 ? nx : ny, nl = dir == 0 ? ny : nx;
    for (int l = 0; l < nl; ++l)
      for (int i = 0; i <= n; ++i) {
        double ql[MAXM], qr[MAXM], al[MAXM] = {0}, ar[MAXM] = {0};
        double W[MAXW * MAXM], S[MAXW], am[MAXM], ap[MAXM];
        if (dir == 0) { gcell(&Q, i - 1, l, ql); gcell(&Q, i, l, qr); }
        else { gcell(&Q, l, i - 1, ql); gcell(&Q, l, i, qr); }
        if (ma) {
          if (dir == 0) { gcell(&A, i - 1, l, al); gcell(&A, i, l, ar); }
          else { gcell(&A, l, i - 1, al); gcell(&A, l, i, ar); }
        }
        orc_riemann(P, dir, ql, qr, al, ar, W, S, am, ap);
        for (int p = 0; p < nw; ++p) {
          double sp = S[p];
          double a = P->capa_index < 0
                         ? fabs(sp)
                         : (sp > 0.0 ? sp / ar[P->capa_index]
                                     : (sp < 0.0 ? -sp / al[P->capa_index] : 0.0));
          if (!(a <= smax[dir])) smax[dir] = a;
        }
      }
  }
  free(qb); free(ab);
}

/* final-time clipping: the step that would pass t_end is shortened to reach it */
static int clip_dt(double t, double t_end, double* dt) {
  if (t + *dt >= t_end) { *dt = t_end - t; return 1; }
  return 0;
}

static int all_finite(const double* q, size_t n) {
  for (size_t i = 0; i < n; ++i) if (!isfinite(q[i])) return 0;
  return 1;
}

int orc_evolve(const orc_prob* P, double* q, const double* aux, double t0, double t_end,
               int max_steps, orc_run_info* info) {
  int ny = (P->ndim >= 2) ? P->ny : 1;
  int nz = (P->ndim == 3) ? P->nz : 1;
  size_t ntot = (size_t)P->nx * ny * nz * P->num_eqn;
  double* qold = (double*)malloc(sizeof(double) * ntot);
  double t = t0, dt;
  int steps = 0, rejects = 0, retries = 0, status = ORC_OK;
  double cfl_last = 0.0, cfl_seen = 0.0;
  if (P->dt_initial > 0.0) {
    dt = P->dt_initial;
  } else {
    double smax[3], rate = 0.0;
    const double dxs[3] = {P->dx, P->dy, P->dz};
    orc_max_speeds(P, q, aux, smax);
    for (int d = 0; d < P->ndim; ++d) {
      double v = smax[d] / dxs[d];
      if (v > rate) rate = v;
    }
    dt = rate > 0.0 ? P->cfl_desired / rate : P->dt_max;
  }
  if (dt > P->dt_max) dt = P->dt_max;
  int final = clip_dt(t, t_end, &dt);
  while (t < t_end && steps < max_steps) {
    double nu;
    memcpy(qold, q, sizeof(double) * ntot);
    if (P->scheme == ORC_SHARPCLAW) status = orc_sharp_step(P, q, aux, dt, &nu);
    else status = orc_classic_step(P, q, aux, dt, &nu);
    if (status != ORC_OK) break;
    if (isnan(nu) || !all_finite(q, ntot)) {
      memcpy(q, qold, sizeof(double) * ntot);
      status = ORC_ENONPHYSICAL;
      break;
    }
    if (nu > P->cfl_max) {
      ++rejects;
      ++retries;
      memcpy(q, qold, sizeof(double) * ntot);
      if (retries > P->max_retries) { status = ORC_ECFL; break; }
      dt = dt * P->cfl_desired / nu;
      if (dt > P->dt_max) dt = P->dt_max;
      final = clip_dt(t, t_end, &dt);
      continue;
    }
    t = final ? t_end : t + dt;
    ++steps;
    retries = 0;
    cfl_last = nu;
    if (nu > cfl_seen) cfl_seen = nu;
    dt = nu > 0.0 ? dt * P->cfl_desired / nu : P->dt_max;
    if (dt > P->dt_max) dt = P->dt_max;
    final = clip_dt(t, t_end, &dt);
  }
  if (info) {
    info->t = t; info->dt_next = dt; info->cfl_last = cfl_last; info->cfl_max_seen = cfl_seen;
    info->steps = steps; info->rejects = rejects; info->status = status;
  }
  free(qold);
  return status;
}

/* ------------------------------------------------------------------------ */
/* conserved totals: (sum_i Q_i) dV per field, Neumaier compensated sum      */
/* ------------------------------------------------------------------------ */

void orc_totals(const orc_prob* P, const double* q, double* out) {
  int ny = (P->ndim >= 2) ? P->ny : 1;
  int nz = (P->ndim == 3) ? P->nz : 1;
  size_t n = (size_t)P->nx * ny * nz;
  double dV = (P->ndim == 3) ? P->dx * P->dy * P->dz
                             : ((P->ndim == 2) ? P->dx * P->dy : P->dx);
  for (int k = 0; k < P->num_eqn; ++k) {
    double s = 0.0, c = 0.0;
    for (size_t i = 0; i < n; ++i) {
      double x = q[(size_t)k * n + i];
      double t = s + x;
      if (fabs(s) >= fabs(x)) c += (s - t) + x;
      else c += (x - t) + s;
      s = t;
    }
    out[k] = (s + c) * dV;
  }
}
