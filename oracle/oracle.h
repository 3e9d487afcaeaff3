/*
 * oracle.h -- plain, slow FP64 CPU oracle for the finite-volume time step of
 * Clawpack-classic and SharpClaw (PyClaw, Ketcheson et al.).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link or
 * call this code: only the tests, the smoke check and the benchmark's CPU
 * baseline leg use it.  It shares no header, helper, table or constant with the
 * CUDA library; the two sides are written independently from the paper
 * (Sec. 2: Eq. (conslaw), Eq. (fluxdiff), Eq. (lwflux); Sec. 2.1) and from the
 * published methods the paper cites (LeVeque 1997 wave propagation; LeVeque's
 * FVM book for limiters, Roe/transverse solvers and the Harten-Hyman entropy
 * fix; Ketcheson-Parsani-LeVeque for SharpClaw; Jiang-Shu WENO5; Shu-Osher
 * SSP-RK3; Einfeldt HLLE; Bale-LeVeque-Mitran-Rossmanith f-waves).
 *
 * Layout: q is field-major, interior cells only: q[m][nz][ny][nx] (x fastest),
 * matching PyClaw's q[m,i,j] field-major arrays (Sec. 3.2).  1D uses ny = 1.
 */
#ifndef CLAW_ORACLE_H
#define CLAW_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* Riemann solver ids */
enum { ORC_RP_ADVECTION = 0, ORC_RP_ACOUSTICS = 1, ORC_RP_SW_ROE = 2,
       ORC_RP_EULER_ROE = 3, ORC_RP_EULER_HLLE = 4, ORC_RP_ELASTICITY_FWAVE = 5,
       ORC_RP_EULER_TRACER = 6, ORC_RP_ACOUSTICS_VC = 7 };
/* wave limiters */
enum { ORC_LIM_NONE = 0, ORC_LIM_MINMOD = 1, ORC_LIM_SUPERBEE = 2,
       ORC_LIM_VANLEER = 3, ORC_LIM_MC = 4 };
/* boundary conditions */
enum { ORC_BC_PERIODIC = 0, ORC_BC_WALL = 1, ORC_BC_EXTRAP = 2, ORC_BC_INFLOW = 3 };
/* schemes */
enum { ORC_CLASSIC = 0, ORC_SHARPCLAW = 1 };
/* status */
enum { ORC_OK = 0, ORC_EINVAL = 1, ORC_ECFL = 5, ORC_ENONPHYSICAL = 6 };

typedef struct {
  int ndim;             /* 1, 2 or 3 (3D: classic, advection and acoustics) */
  int nx, ny;           /* interior cells (ny = 1 in 1D) */
  double dx, dy;        /* cell widths */
  int rp;               /* ORC_RP_* */
  int scheme;           /* ORC_CLASSIC / ORC_SHARPCLAW */
  int lim;              /* ORC_LIM_* */
  int order;            /* classic: 1 Godunov, 2 Lax-Wendroff + limiter */
  int transverse;       /* classic 2D: 0 none, 1 fluctuations, 2 fluctuations+corrections */
  int char_decomp;      /* SharpClaw: 0 component-wise, 1 characteristic-wise */
  int entropy_fix;      /* Harten-Hyman on Roe solvers */
  int num_eqn, num_aux, num_waves;
  int bc_lo[3], bc_hi[3];
  double inflow[8];     /* fixed ghost state for ORC_BC_INFLOW */
  double params[8];     /* advection: u,v | acoustics: rho,K | SW: g | Euler: gamma */
  double cfl_desired, cfl_max, dt_initial, dt_max;
  int max_retries;
  double weno_eps;      /* WENO5 epsilon (Jiang-Shu) */
  int nz;               /* 3D: cells in z (1 otherwise) */
  double dz;            /* 3D: cell width in z */
  int time_integrator;  /* SharpClaw: 0 SSP-RK3 (Shu-Osher), 1 SSP(10,4) (Ketcheson 2008) */
  int weno_r;           /* SharpClaw: WENO order 2r-1; 0 or 3 = WENO5 (Jiang-Shu) */
  /* for weno_r > 3: coefficients from their definitions (oracle/weno_coeffs.py):
   * weno_c[k*r+j] reconstruction, weno_d[k] optimal weights,
   * weno_b[(k*r+a)*r+b] smoothness quadratic forms */
  double weno_c[81], weno_d[9], weno_b[729];
  int source;           /* 0 none; 1 axisymmetric Euler geometric source about y = 0
                           (r = y; Sec. 7.2), by fractional steps (source_split) */
  int dim_split;        /* classic 2D: 0 unsplit; 1 dimensional splitting (x sweeps,
                           then y sweeps, Godunov) */
  double lower[2];      /* lower corner of the grid (cell centres for the source) */
  int capa_index;       /* aux field holding the capacity kappa (Eq. (conslaw)); -1 none */
  int source_split;     /* fractional steps for the source (Sec. 2; Sec. 7.1 uses Strang):
                           1 Godunov, S(dt) after the step; 2 Strang, S(dt/2) before
                           and after it */
} orc_prob;

typedef struct {
  double t;             /* time reached */
  double dt_next;       /* next step size the controller chose */
  double cfl_last;      /* Courant number of the last accepted step */
  double cfl_max_seen;  /* largest accepted Courant number */
  int steps;            /* accepted steps */
  int rejects;          /* rejected attempts */
  int status;           /* ORC_OK / ORC_ECFL / ORC_ENONPHYSICAL */
} orc_run_info;

int orc_num_eqn(int rp, int ndim);
int orc_num_waves(int rp, int ndim);

/* One Riemann solve in direction dir (0 = x, 1 = y) of a problem of P->ndim
 * dimensions.  Outputs wave[p*meqn+m], s[p], amdq[m], apdq[m].  The waves of
 * the f-wave solver are flux-difference waves Z^p. */
void orc_riemann(const orc_prob* P, int dir, const double* ql, const double* qr,
                 const double* auxl, const double* auxr,
                 double* wave, double* s, double* amdq, double* apdq);
/* Transverse split of asdq at the interface (ql, qr) of a dir-normal solve into
 * the two transverse-direction fluctuations bmasdq (down-going), bpasdq (up-going). */
void orc_transverse(const orc_prob* P, int dir, const double* ql, const double* qr,
                    const double* auxl, const double* auxr, const double* asdq,
                    double* bmasdq, double* bpasdq);
/* Varying-medium acoustics (aux rho, c): transverse split of asdq held by the
 * cell with aux a_c between its neighbours a_m (below) and a_p (above). */
void orc_transverse_vc(const orc_prob* P, int dir, const double* a_m, const double* a_c,
                       const double* a_p, const double* asdq, double* bm, double* bp);
/* limiter function phi(theta) */
double orc_phi(int lim, double theta);
/* WENO5 left-biased value at x_{i+1/2} from v[0..4] = v_{i-2..i+2} */
double orc_weno5(const double* v, double eps);
/* WENO of order 2r-1: left-biased value at x_{i+1/2} from v[0..2r-2] =
 * v_{i-r+1..i+r-1}, with the coefficient layout of orc_prob */
double orc_weno_r(int r, const double* c, const double* d, const double* B, const double* v,
                  double eps);
/* characteristic matrices at the interface (ql, qr): Lmat (meqn x meqn,
 * rows = left eigenvectors), Rmat (columns = right eigenvectors), row-major. */
int orc_char_matrices(const orc_prob* P, int dir, const double* ql, const double* qr,
                      double* Lmat, double* Rmat);

/* Fill a ghosted copy qg[m][ny+2g][nx+2g] (1D: [m][nx+2g]) from interior q. */
void orc_fill_ghost(const orc_prob* P, const double* q, int ncomp, int g, int is_aux,
                    double* qg);

/* One classic step in place with the given dt; *cfl receives the Courant
 * number (max over directions of dt*max|s|/dx).  Returns ORC_OK. */
int orc_classic_step(const orc_prob* P, double* q, const double* aux, double dt, double* cfl);
/* SharpClaw semi-discrete operator L(Q) (per cell, field-major) and the
 * largest interface wave speed per direction (smax[0] x, smax[1] y). */
int orc_sharp_L(const orc_prob* P, const double* q, const double* aux, double* L, double* smax);
/* One SharpClaw SSP-RK3 step in place; *cfl as in orc_classic_step. */
int orc_sharp_step(const orc_prob* P, double* q, const double* aux, double dt, double* cfl);
/* One SSP-RK3 step of the scalar linear ODE q' = lambda q (same stage code). */
double orc_ssp_rk3_linear(double lambda, double dt, double q0);
/* One SSP(10,4) step of q' = lambda q (same stage code as orc_sharp_step). */
double orc_ssp104_linear(double lambda, double dt, double q0);
/* Apply the source step of the problem (P->source) for time dt to q in place. */
void orc_source_step(const orc_prob* P, double* q, double dt);
/* Largest first-order interface wave speed per direction on Q (used for dt0). */
void orc_max_speeds(const orc_prob* P, const double* q, const double* aux, double* smax);

/* Evolve from t0 to t_end with the CFL controller (accept / reject / clip). */
int orc_evolve(const orc_prob* P, double* q, const double* aux, double t0, double t_end,
               int max_steps, orc_run_info* info);
/* Conserved totals sum_i Q_i dV per field (Neumaier compensated), out[m]. */
void orc_totals(const orc_prob* P, const double* q, double* out);
/* number of OpenMP threads the oracle uses (1 without OpenMP) */
int orc_threads(void);

#ifdef __cplusplus
}
#endif
#endif
