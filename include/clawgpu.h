/*
 * clawgpu.h -- C ABI of the GB300 (sm_103a) finite-volume library for
 * hyperbolic conservation laws, after PyClaw (Ketcheson, Mandli, Ahmadia,
 * Alghamdi, Quezada de Luna, Parsani, Knepley, Emmett: "PyClaw: Accessible,
 * Extensible, Scalable Tools for Wave Propagation Problems").
 *
 * The library advances  kappa q_t + div f(q, x) = s(q, x)  (Sec. 2,
 * Eq. (conslaw); kappa = 1 unless a capacity field is named by capa_index,
 * s = 0 unless claw_method.source names a source term) on uniform Cartesian
 * grids with
 *   - Clawpack-classic: Godunov update in fluctuation form (Eq. (fluxdiff))
 *     plus limited second-order corrections (Eq. (lwflux)) and, in 2D,
 *     transverse corrections (Sec. 2.1, "transverse Riemann solver");
 *   - SharpClaw: WENO5 reconstruction of interface values, fluctuations from
 *     interface and in-cell Riemann problems, SSP-RK3 in time (Sec. 2 method
 *     of lines, Sec. 2.1);
 * each step ending with the CFL check and choice of the next step (Sec. 4).
 *
 * Conventions
 *   - Every call returns claw_status (0 = CLAW_OK).  No call throws.
 *   - Device memory for the state belongs to the caller; the library borrows
 *     it for the life of the handle.  The library allocates its own work
 *     buffers (a second/third copy of the state, a control block) at
 *     claw_bind_state and frees them at destroy.
 *   - State layout: field-major, interior cells only, x fastest:
 *       q[m][nz][ny][nx] (3D), q[m][ny][nx] (2D), q[m][nx] (1D) -- PyClaw's
 *       field-major q[m, i, j] (Sec. 3.2).  3D adds double-transverse terms.
 *     aux has the same layout with num_aux fields.
 *   - CLAW_FP64: q/aux are double.  CLAW_FP32: q/aux are float and the
 *     Riemann/limiter/WENO arithmetic is float; time, dt, the CFL number and
 *     the conserved totals stay double.
 *   - A handle is used from one host thread at a time and enqueues its work
 *     on the stream given at creation (cudaStream_t passed as void*).  With
 *     NULL (the legacy default stream) a single-grid solver runs on a private
 *     stream ordered after and before the caller's work by events.
 */
#ifndef CLAWGPU_H
#define CLAWGPU_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int claw_status;
enum {
  CLAW_OK = 0,
  CLAW_EINVAL = 1,        /* bad argument or unsupported combination        */
  CLAW_ENOMEM = 2,        /* a device or host allocation failed             */
  CLAW_EBUDGET = 3,       /* request exceeds the server's HBM budget        */
  CLAW_ECUDA = 4,         /* a CUDA runtime call failed                     */
  CLAW_ECFL = 5,          /* Courant number above cfl_max after max_retries */
  CLAW_ENONPHYSICAL = 6,  /* NaN/Inf in speeds or state (e.g. h <= 0)       */
  CLAW_ETIMEOUT = 7,      /* a bounded wait gave up                         */
  CLAW_EBUSY = 8          /* result not ready yet (server poll)             */
};

enum { CLAW_FP64 = 0, CLAW_FP32 = 1 };
enum { CLAW_CLASSIC = 0, CLAW_SHARPCLAW = 1 };
enum { CLAW_RP_ADVECTION = 0, CLAW_RP_ACOUSTICS = 1, CLAW_RP_SW_ROE = 2,
       CLAW_RP_EULER_ROE = 3, CLAW_RP_EULER_HLLE = 4, CLAW_RP_ELASTICITY_FWAVE = 5,
       CLAW_RP_EULER_TRACER = 6, CLAW_RP_ACOUSTICS_VC = 7 };
/* Source terms (Eq. (conslaw) right-hand side) by fractional steps (Sec. 2;
 * Sec. 7.1 uses Strang's splitting): CLAW_SOURCE_AXISYMMETRIC is the
 * geometric source of the Euler equations in cylindrical symmetry about
 * y = 0 (Sec. 7.2: (z, r) = (x, y); -(1/r)(rho v, rho u v, rho v^2,
 * (E + p) v), tracer none), integrated over each fractional step by a
 * two-stage second-order Runge-Kutta method.  CLAW_SPLIT_GODUNOV: the source
 * over dt after every accepted step; CLAW_SPLIT_STRANG: over dt/2 before the
 * step (into an extra state buffer, so a rejected attempt leaves Q^n as it
 * was) and over dt/2 after every accepted step. */
enum { CLAW_SOURCE_NONE = 0, CLAW_SOURCE_AXISYMMETRIC = 1 };
enum { CLAW_SPLIT_GODUNOV = 1, CLAW_SPLIT_STRANG = 2 };
enum { CLAW_LIM_NONE = 0, CLAW_LIM_MINMOD = 1, CLAW_LIM_SUPERBEE = 2, CLAW_LIM_VANLEER = 3,
       CLAW_LIM_MC = 4 };
enum { CLAW_BC_PERIODIC = 0, CLAW_BC_WALL = 1, CLAW_BC_EXTRAP = 2, CLAW_BC_INFLOW = 3 };
/* SharpClaw time integrators (Sec. 2.1): Shu-Osher three-stage SSP-RK3, and
 * Ketcheson's ten-stage fourth-order SSP(10,4) in its two-register low-storage
 * form (SSP coefficient 6, so the CFL limit is about six times that of one
 * forward-Euler stage spread over ten stages). */
enum { CLAW_SSP_RK3 = 0, CLAW_SSP104 = 1 };

/* Domain (Sec. 3.2: tensor product of equispaced 1D grids).  n[d] cells on
 * [lower[d], upper[d]]; entries beyond ndim are ignored. */
typedef struct {
  int ndim;            /* 1, 2 or 3 (3D: classic scheme, advection and acoustics) */
  int64_t n[3];
  double lower[3], upper[3];
} claw_grid;

/* Solver description (Sec. 3.2 Solver; Listing 1 and the SharpClaw listing). */
typedef struct {
  int scheme;          /* CLAW_CLASSIC | CLAW_SHARPCLAW                          */
  int rp;              /* CLAW_RP_* Riemann solver                               */
  int lim;             /* CLAW_LIM_* wave limiter (classic)                       */
  int prec;            /* CLAW_FP64 | CLAW_FP32                                   */
  int order;           /* classic: 1 Godunov, 2 with limited corrections          */
  int transverse;      /* classic 2D: 0 none, 1 fluctuations, 2 with corrections  */
  int weno_order;      /* SharpClaw: 5 (default), 7, 9, ..., 17 (Sec. 3.3, PyWENO orders) */
  int char_decomp;     /* SharpClaw: 0 component-wise, 1 characteristic-wise      */
  int entropy_fix;     /* Harten-Hyman fix in the Roe solvers (SW, Euler)         */
  int max_retries;     /* rejected attempts allowed per step                      */
  double cfl_desired;  /* target Courant number for the next step                 */
  double cfl_max;      /* a step above this Courant number is rejected            */
  double dt_initial;   /* first dt; <= 0: from the wave speeds of the initial data */
  double dt_max;       /* upper bound on dt                                       */
  double weno_eps;     /* WENO5 epsilon (Jiang-Shu), default 1e-6                 */
  int bc_lower[3];     /* CLAW_BC_* per direction                                 */
  int bc_upper[3];
  double inflow[8];    /* ghost state for CLAW_BC_INFLOW                          */
  double params[8];    /* advection u,v | acoustics rho,K | SW g | Euler gamma    */
  int num_eqn;         /* filled in by claw_method_init / validated by create     */
  int num_aux;         /* elasticity: 2 (rho, K); acoustics_vc: 2 (rho, c); others
                          0; one more when a capacity field follows them           */
  int time_integrator; /* SharpClaw: CLAW_SSP_RK3 (default) | CLAW_SSP104          */
  int source;          /* CLAW_SOURCE_*; axisymmetric: 2D Euler systems, y >= 0    */
  int dim_split;       /* classic 2D: 0 unsplit (default); 1 dimensional splitting
                          (x sweeps then y sweeps over dt, no transverse terms)    */
  int capa_index;      /* -1 (default): no capacity; else the aux field holding the
                          capacity kappa of Eq. (conslaw), which must be the field
                          after the solver's own (num_aux = solver's + 1); 1D/2D   */
  int source_split;    /* CLAW_SPLIT_GODUNOV (default) | CLAW_SPLIT_STRANG        */
} claw_method;

typedef struct {
  double t;            /* time after the call                                      */
  double dt_used;      /* dt of the last accepted step                             */
  double dt_next;      /* dt the controller chose next                             */
  double cfl;          /* Courant number of the last accepted step                 */
  double cfl_max_seen; /* largest accepted Courant number since bind               */
  int64_t steps;       /* accepted steps since bind                                */
  int64_t rejects;     /* rejected attempts since bind                             */
  int accepted;        /* claw_step: 1 if the last attempt was accepted            */
  int status;          /* CLAW_OK, CLAW_ECFL or CLAW_ENONPHYSICAL                   */
} claw_step_info;

typedef struct claw_solver claw_solver;
typedef struct claw_batch claw_batch;
typedef struct claw_server claw_server;
/* server schedules (claw_server_schedule) */
enum { CLAW_SCHED_ALL = 0, CLAW_SCHED_SRW = 1 };

/* Fill *m with the defaults for a Riemann solver in ndim dimensions:
 * classic, MC limiter, order 2, transverse 2, FP64, CFL 0.9/1.0, walls...
 * (periodic BCs), WENO5 char-wise, entropy fix on.  Returns CLAW_EINVAL for
 * an unknown solver or dimension. */
claw_status claw_method_init(claw_method* m, int rp, int ndim);

/* Create a solver for one grid.  stream: cudaStream_t (may be NULL).  Fails
 * with CLAW_EINVAL on an unsupported combination (e.g. SharpClaw
 * characteristic projection with the f-wave solver, 2D elasticity). */
claw_status claw_solver_create(const claw_method* m, const claw_grid* g, void* stream,
                               claw_solver** out);

/* Bind the caller's device state q_dev (and aux_dev, NULL if num_aux == 0) at
 * time t0; allocates the work buffers and computes the first dt (Sec. 4).
 * Data are read from q_dev on the stream; the caller must not write q_dev
 * while the handle runs.  Rebinding replaces the previous state. */
claw_status claw_bind_state(claw_solver* s, void* q_dev, const void* aux_dev, double t0);

/* One step.  dt > 0: take exactly that step (no rejection; the Courant
 * number is still reported).  dt <= 0: controller step -- attempt with the
 * chosen dt, reject and retry while the Courant number exceeds cfl_max (up
 * to max_retries), then accept.  Synchronises the stream; fills *info.  The
 * new state lives in the current buffer (claw_current_state); call
 * claw_sync_state to have it in q_dev. */
claw_status claw_step(claw_solver* s, double dt, claw_step_info* info);

/* Launch shape of the step: mode 0 runs the autotuner (times the candidate
 * shapes on the bound state without changing it) and returns the choice in
 * *bw, *h; mode 1 sets them (CLAW_EINVAL for a shape the method does not
 * have).  Classic 2D: *bw (64 or 128 threads = strip width + 4) and *h (rows
 * per block).  Classic 1D: *h is how warps take work (1: a whole tile of 4
 * warp units, 2: one unit; *bw is ignored).  SharpClaw 2D: the tile of cells
 * a block reconstructs, *bw x *h = 16 x 8, 32 x 4, 32 x 8 or 16 x 16 with
 * fifth-order WENO (timed on the first stage), 16 x 8 with the higher
 * orders; SharpClaw 1D: 128 x 1.  Every shape gives the same result bit for
 * bit.  3D grids and the per-face classic path ignore the shape. */
claw_status claw_solver_tune(claw_solver* s, int mode, int* bw, int* h);

/* Enqueue n controller step attempts on the stream without synchronising
 * (rejected attempts count).  Attempts after t_end or after an error do no
 * work.  Set t_end first with claw_set_t_end (default: +inf). */
claw_status claw_advance(claw_solver* s, int n);
claw_status claw_set_t_end(claw_solver* s, double t_end, int64_t max_steps);

/* Advance to t_end (final step clipped to land on it, Sec. 4) or max_steps
 * accepted steps (<= 0: no limit).  use_graph != 0 replays a captured CUDA
 * graph of attempts.  The result is in q_dev on return. */
claw_status claw_evolve_to_time(claw_solver* s, double t_end, int64_t max_steps, int use_graph,
                                claw_step_info* info);

/* Read the controller state (synchronises the stream). */
claw_status claw_get_info(claw_solver* s, claw_step_info* info);
/* Device pointer of the buffer that holds the current state. */
claw_status claw_current_state(claw_solver* s, void** q_cur);
/* Copy the current state into q_dev if it lives in a work buffer. */
claw_status claw_sync_state(claw_solver* s);

/* Conserved totals (sum_i kappa_i Q_i) * dV per field (kappa = 1 without a
 * capacity field), FP64 with compensated summation, into host
 * out[num_eqn] (synchronises). */
claw_status claw_conserved_totals(claw_solver* s, double* out);

/* Checkpoint: state + controller into a host buffer.  With host_buf NULL,
 * *bytes receives the size needed.  Restore puts both back. */
claw_status claw_checkpoint(claw_solver* s, void* host_buf, size_t* bytes);
claw_status claw_restore(claw_solver* s, const void* host_buf, size_t bytes);

/* End-to-end step from host memory: copy q_host_in (pinned or pageable) to the
 * device state, take n controller attempts, copy the state back to
 * q_host_out.  Synchronises. */
claw_status claw_step_host(claw_solver* s, const void* q_host_in, void* q_host_out, int n);

claw_status claw_solver_destroy(claw_solver* s);

/* ---------------------------------------------------------------------- */
/* Batched solves: many grids of one method advanced together, one fused   */
/* launch per step over a table of tiles (each grid keeps its own t, dt).  */
/* ---------------------------------------------------------------------- */

/* grids[n]: one per member (same ndim and method; 1D, 2D or 3D).  Row-kernel
 * methods run one fused launch per step over all members' tiles; methods on
 * the per-face classic path (a capacity field, or 2D varying-medium
 * acoustics) and 3D grids (the face sweeps and update of Sec. 2's 3D
 * algorithm) run their kernels member by member inside each attempt. */
claw_status claw_batch_create(const claw_method* m, const claw_grid* grids, int n, void* stream,
                              claw_batch** out);
/* q[k], aux[k]: device pointers of member k (caller-owned); t_end[k]. */
claw_status claw_batch_bind(claw_batch* b, void* const* q, const void* const* aux,
                            const double* t_end);
/* Run until every member reaches its t_end (or fails).  use_graph != 0
 * replays captured CUDA graphs.  info[k] per member (may be NULL). */
claw_status claw_batch_evolve(claw_batch* b, int use_graph, int64_t max_steps,
                              claw_step_info* info);
/* Enqueue n fused step attempts for all unfinished members (no sync). */
claw_status claw_batch_advance(claw_batch* b, int n);
claw_status claw_batch_info(claw_batch* b, claw_step_info* info);
/* Launch shape of the batch's fused step (classic or SharpClaw), as
 * claw_solver_tune: mode 0 times the candidates on all bound members at once
 * (dry attempts: no member's state, t or dt changes) and keeps the fastest;
 * mode 1 sets *bw, *h.  Results do not depend on the shape.  Call after
 * claw_batch_bind; per-face and 3D batches keep their fixed launches. */
claw_status claw_batch_tune(claw_batch* b, int mode, int* bw, int* h);
claw_status claw_batch_sync_state(claw_batch* b);
claw_status claw_batch_destroy(claw_batch* b);

/* ---------------------------------------------------------------------- */
/* Serving: continuous batching of independent solves that arrive over time */
/* ---------------------------------------------------------------------- */

typedef struct {
  int status;          /* CLAW_OK, CLAW_EBUSY (queued/running), or an error       */
  int64_t steps;       /* accepted steps                                           */
  double t;            /* time reached                                             */
  double t_submit;     /* seconds (server clock) at submit                         */
  double t_admit;      /* seconds at admission to the device                       */
  double t_done;       /* seconds at completion                                    */
} claw_req_info;

/* hbm_budget_bytes bounds the device memory of admitted requests (state,
 * work buffers, aux, control blocks; with a Strang-split source one more
 * state buffer; on the per-face classic path its face arrays).  max_slots
 * bounds concurrent requests.  Classic 1D/2D and SharpClaw methods, with or
 * without a source term; on the per-face path (a capacity field, or 2D
 * varying-medium acoustics) the kernels run request by request. */
claw_status claw_server_create(const claw_method* m, size_t hbm_budget_bytes, int max_slots,
                               void* stream, claw_server** out);
/* The same for grids of ndim dimensions (1, 2 or 3; claw_server_create takes
 * 2 when num_eqn is the 2D system's field count, else 1).  3D requests run
 * the classic face sweeps and update request by request (Sec. 2's 3D
 * algorithm with transverse and double-transverse terms). */
claw_status claw_server_create_nd(const claw_method* m, int ndim, size_t hbm_budget_bytes,
                                  int max_slots, void* stream, claw_server** out);
/* Submit one solve: grid, initial state (host memory, the method's precision
 * and layout), aux (host, may be NULL), t_end.  Returns a ticket.  Fails with
 * CLAW_EBUDGET when the request alone exceeds the budget. */
claw_status claw_server_submit(claw_server* sv, const claw_grid* g, const void* q0_host,
                               const void* aux_host, double t_end, uint64_t* ticket);
/* Drive the server: take `steps` fused step attempts over the requests the
 * schedule picks (below), retire the requests found finished, admit queued
 * requests that fit (first come, first served).  The pump is pipelined: it
 * enqueues its attempts first and does the bookkeeping of the previous
 * pump's attempts (statuses gathered on the device) while the GPU runs them,
 * so a request is stepped from the pump after the one that admitted it and
 * retired by the pump after the one whose attempts finished it; the
 * arithmetic of every request is unchanged.  Returns the number of running
 * and queued requests in *running and *queued (either may be NULL). */
claw_status claw_server_pump(claw_server* sv, int steps, int* running, int* queued);
/* Which running requests a pump steps.  CLAW_SCHED_ALL: every running request
 * in every attempt.  CLAW_SCHED_SRW (the default, min_cells = 2^23): shortest
 * remaining work first -- requests not yet stepped, then any left out of 16
 * pumps in a row, then the rest by estimated remaining cell updates (cells x
 * (t_end - t) / dt from the last pump), until the picked requests hold
 * min_cells cells.  The schedule changes only when a request advances, never
 * its arithmetic: each result is the same under either policy. */
claw_status claw_server_schedule(claw_server* sv, int policy, int64_t min_cells);
/* Launch shape of the server's fused step, as claw_batch_tune: mode 0
 * times the candidates on the requests running now (the live mix; dry
 * attempts change none of them; CLAW_EINVAL when none is running), mode 1
 * sets *bw, *h.  Running requests take the shape from their next attempt;
 * results do not depend on it. */
claw_status claw_server_tune(claw_server* sv, int mode, int* bw, int* h);
/* Tickets of the requests that finished since the last call, oldest first,
 * at most cap of them (the rest stay for the next call); *n = how many were
 * written.  A client polls these instead of every ticket it holds. */
claw_status claw_server_take_done(claw_server* sv, uint64_t* tickets, int cap, int* n);
/* Poll a ticket; when done, copies the final state to q_host_out (may be
 * NULL) and releases it.  CLAW_EBUSY while queued or running. */
claw_status claw_server_poll(claw_server* sv, uint64_t ticket, void* q_host_out,
                             claw_req_info* info);
claw_status claw_server_destroy(claw_server* sv);

/* ---------------------------------------------------------------------- */
/* Allocation-free step                                                     */
/* ---------------------------------------------------------------------- */

/* One SharpClaw SSP-RK3 step of size dt from q_in to q_out (caller device
 * memory, layout as above; aux may be NULL when num_aux == 0), for callers
 * that cannot let the library allocate device memory -- applications whose
 * device memory is owned by their own allocator or fixed arena, or paths
 * where cudaMalloc would synchronise the device or is not allowed.  The paper
 * has no counterpart: it is a service of this library.  The two intermediate
 * stage states, the control block and the grid descriptors live in one
 * static device array of 8 MiB that every GPU loading the library keeps until
 * exit; a grid whose two stage states do not fit (with 1 KiB of control
 * data) is rejected with CLAW_EINVAL and a message from claw_last_error.  The
 * first call on a device (that device current) looks up the array's address;
 * make it before any stream capture.  Every call reuses the array, rewriting
 * the control block first; calls that overlap on the GPU race.  Runs on
 * stream (cudaStream_t, may be NULL) and synchronises it; *cfl (may be NULL)
 * receives the Courant number.  Returns CLAW_ENONPHYSICAL on non-finite
 * results. */
claw_status claw_sharp_step_noalloc(const claw_method* m, const claw_grid* g, const void* q_in,
                                    void* q_out, const void* aux, double dt, void* stream,
                                    double* cfl);

/* ---------------------------------------------------------------------- */
/* Diagnostics                                                              */
/* ---------------------------------------------------------------------- */

/* Measured FMA throughput of the current device in TFLOP/s (one FMA = 2
 * FLOPs), for the ALU roofline of the FP64-bound kernels: a probe kernel with
 * eight independent FMA chains per thread, as many blocks as fit at once on
 * every SM, the best of six timed launches (after two warm-up launches) on
 * stream (cudaStream_t, may be NULL; synchronised).  *sm_mhz (may be NULL)
 * receives the SM clock that launch ran at (SM cycles over global-timer time
 * of one block), so the rate per clock is *tflops / *sm_mhz.  prec:
 * CLAW_FP64 or CLAW_FP32.  Takes about 0.1-0.3 s.  Not part of the paper's
 * method. */
claw_status claw_fma_peak(int prec, void* stream, double* tflops, double* sm_mhz);

/* Self-test of the bounded wait on the shared-memory barriers that complete
 * the bulk asynchronous copies of the staged 1D kernels.  One thread waits
 * limit_us microseconds (1 .. 1e6) on a barrier that nothing arrives at and
 * must give up (*gave_up = 1, *waited_us = the time it waited); it then
 * copies 256 bytes from global to shared memory in bulk, waits for that copy
 * and compares it word by word (*copied = 1 when it completed and matched).
 * Runs on stream (cudaStream_t, may be NULL; synchronised).  The kernels
 * report such a timeout as CLAW_ETIMEOUT on the grid's status.  Not part of
 * the paper's method. */
claw_status claw_async_wait_probe(int limit_us, void* stream, int* gave_up, int* copied,
                                  double* waited_us);

/* Seconds on the server's clock (monotonic). */
double claw_clock(void);

/* Static description of the last error on a handle (or the last global
 * error when handle is NULL).  Never NULL. */
const char* claw_last_error(const void* handle);

/* Library version string. */
const char* claw_version(void);

#ifdef __cplusplus
}
#endif
#endif
