/*
 * dbm.h - C ABI of the GB300 (sm_103a) polar-coordinate discrete-Boltzmann
 * detonation update of Lin, Xu, Zhang and Li, "Polar coordinate lattice
 * Boltzmann kinetic modeling of detonation phenomena" (arXiv:1308.0653).
 *
 * One time step advances every grid site (i_r, i_theta) and each of the 33
 * discrete velocities of the D2V33 set (Sec. II.B): moments -> equilibrium
 * f^eq (Eq. feq) -> BGK relaxation integrated exactly + chemical term M
 * (Eq. LB_evolution_equation, Sec. II.B) -> first-order upwind streaming in r
 * and theta -> reaction progress lambda by the exact solution of Cochran's
 * rate law plus upwind transport (Eq. Cochran, Eq. Eqlambda).
 *
 * Conventions shared by every entry point:
 *   grid      r_j = r_in + (j + 1/2) dr, dr = (r_out - r_in) / nr, j = 0..nr-1;
 *             theta_m = m dtheta, dtheta = span / ntheta, m = 0..ntheta-1, with
 *             span = 2 pi, or pi/4 for a sector (dbm_params.sector).
 *   fields    host or device arrays of double, row-major [ntheta][nr]
 *             (index m * nr + j); velocities in polar components u_r, u_theta.
 *   velocity  index v = 0 for the rest particle, v = 1 + 8 (k - 1) + i for
 *             speed v_k (k = 1..4) in Cartesian direction i pi / 4 (i = 0..7).
 *   streams   `stream` arguments are cudaStream_t values passed as void*;
 *             NULL means the legacy default stream.
 *   status    every function returns a DBM_* status and never aborts or
 *             exits; dbm_strerror() names it.  Errors raised by work already
 *             queued on the GPU surface at the next call that synchronises
 *             (dbm_moments, dbm_status, dbm_poll).
 *   memory    device memory is supplied by the caller (for example a PyTorch
 *             tensor) and only borrowed by the library until the matching
 *             destroy call; host arrays are caller-owned and only read or
 *             written during the call (or, for dbm_submit, copied).
 *
 * Readings of the paper taken where it is garbled or silent (all documented
 * in the library's design notes): the last term of F_k has a minus sign; the
 * lambda-update denominator is (a + b lam) E + b (1 - lam); the streaming
 * terms are subtracted (upwind); radial boundaries are zero-gradient ghosts;
 * f starts at f^eq of the initial fields; lambda is kept in [0, 1].
 */
#ifndef DBM_H
#define DBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
#define DBM_OK          0  /* success                                              */
#define DBM_EINVAL      1  /* invalid argument (NULL pointer, size, parameter)     */
#define DBM_ECFL        2  /* max |C_r| + |C_theta| > 1: first-order upwind unstable */
#define DBM_ENOMEM      3  /* caller buffer too small / server pool exhausted      */
#define DBM_EBUSY       4  /* server queue full                                    */
#define DBM_ENOTREADY   5  /* request still queued or running                      */
#define DBM_ETIMEOUT    6  /* a bounded wait (host or device) gave up              */
#define DBM_ENONFINITE  7  /* a moment came out NaN or infinite                    */
#define DBM_ECUDA       8  /* a CUDA runtime call failed                           */
#define DBM_ECANCELLED  9  /* request cancelled before it finished                 */
#define DBM_ENOTFOUND  10  /* unknown ticket                                       */
#define DBM_EDEVICE    11  /* a device-side self-check failed: shared-memory layout,
                              or (DBM_DEBUG builds) a copy or store out of bounds   */

#define DBM_NV 33          /* D2V33: 1 rest + 4 rings x 8 directions (Sec. II.B)  */

/* precision of f and of the per-step arithmetic */
#define DBM_FP32 0
#define DBM_FP64 1

/* radial boundary rules (Sec. II.D) */
#define DBM_BC_OUTFLOW 0   /* zero-gradient ghost: f(-1) = f(0), f(nr) = f(nr-1)  */
                           /* (the paper defers annulus boundaries; reading)      */
#define DBM_BC_CENTRE  1   /* disc centre, inner boundary only, needs r_in = 0.    */
                           /* In a sector: f(-1, theta, k, i) = f(0, theta, k, i+4) */
                           /* (the paper's rule); on a full 2 pi grid (ntheta even) */
                           /* the point across the centre, f(-1, theta_m, k, i) =  */
                           /* f(0, theta_{m + ntheta/2}, k, i), lambda likewise     */

/* heat put into f by M (Sec. II.B) */
#define DBM_R_EXPLICIT   0 /* R(lambda^t, P^t) of Eq. (Cochran): the paper's form */
#define DBM_R_CONSISTENT 1 /* R = (lambda_react - lambda^t) / dt: heat = rho Q dlam */

/* ---- parameters of one simulation --------------------------------------- */
typedef struct dbm_params {
    int32_t nr, ntheta;        /* grid size, both >= 1                            */
    int32_t precision;         /* DBM_FP32 or DBM_FP64                            */
    int32_t reaction_energy;   /* DBM_R_EXPLICIT (default) or DBM_R_CONSISTENT     */
    int32_t r_bc_inner;        /* DBM_BC_OUTFLOW or DBM_BC_CENTRE (r_in = 0)      */
    int32_t r_bc_outer;        /* DBM_BC_OUTFLOW                                  */
    int32_t rows_per_item;     /* theta rows per CTA work item; 0 = automatic     */
    int32_t variant;           /* step-kernel variant 1..dbm_num_variants();      */
                               /* 0 = autotuned choice for the size class, else   */
                               /* the library default                             */
    int32_t sector;            /* 0: full 2 pi grid; 1: pi/4 sector whose theta   */
                               /* wrap rotates velocities (i -> i+1 below row 0,  */
                               /* i -> i-1 above the last row), Sec. II.D, Fig. 1 */
    int32_t reserved;          /* must be 0                                       */
    double r_in, r_out;        /* radii, 0 < r_in < r_out (r_in = 0: disc centre) */
    double dt, tau;            /* time step and BGK relaxation time (Sec. II.C)   */
    double Q;                  /* heat release per unit mass (Sec. II.A)          */
    double omega1, omega2;     /* Cochran rate constants, >= 0 (Eq. Cochran)      */
    double m, n;               /* Cochran pressure exponents (paper: 1, 1)        */
    double T_th;               /* ignition temperature (paper: 1.1)               */
    double v[4];               /* ring speeds v_1..v_4 (paper: 1.5 3.5 7.5 12.5)  */
} dbm_params;

typedef struct dbm_s dbm_t;    /* one simulation bound to a caller device buffer */

/* Library version string (static storage). */
const char *dbm_version(void);

/* Static text naming a status code. */
const char *dbm_strerror(int status);

/* Text of the last CUDA failure reported as DBM_ECUDA on this thread
 * (thread-local static storage; empty if none). */
const char *dbm_last_error(void);

/* Fill *p with the paper's constants (Sec. II.B, III.A) and a 64 x 64 annulus
 * r in [0.05, 1.05], dt 1e-5, tau 1e-3, Q 1, omega1 = omega2 = 0, FP32. */
int dbm_params_default(dbm_params *p);

/* Host-only validation of *p (no GPU needed).  Checks sizes, radii, dt, tau,
 * rate constants and the Courant condition of Sec. II.C,
 *   max over velocities, rows and radii of |C_r| + |C_theta| <= 1,
 *   C_r = v_kir dt / dr, C_theta = v_kith dt / (r dtheta);
 * writes that maximum to *cfl when cfl is not NULL.
 * Returns DBM_OK, DBM_EINVAL or DBM_ECFL. */
int dbm_check(const dbm_params *p, double *cfl);

/* Host-only: bytes of caller device memory dbm_create needs for *p (two f
 * buffers, two lambda buffers, geometry tables, status and reduction words),
 * or 0 if *p is invalid. */
size_t dbm_state_bytes(const dbm_params *p);

/* Host-only: the work split of one simulation's step.  The grid is cut into
 * strips of `width` radial sites (the kernel's W: dbm_launch_info's threads
 * minus the producer warp's 32) by runs of *rows_per_item theta rows; the
 * ceil(nr / width) x ceil(ntheta / rows) items are dealt round-robin to
 * `slots` persistent CTAs (SMs x resident CTAs per SM), and each loads its
 * rows plus two halo rows.  rows_requested > 0 fixes the rows (at most
 * ntheta); 0 picks the rows that minimise the busiest CTA's loaded rows,
 * ceil(items / slots) x (rows + 2), with the fewest items on ties.  This is
 * the split dbm_create and dbm_set_variant use.  Writes *rows_per_item and
 * *items (either may be NULL).  Errors: DBM_EINVAL (a size below 1 or a
 * negative rows_requested). */
int dbm_plan_items(int32_t nr, int32_t ntheta, int32_t width, int32_t slots, int32_t rows_requested,
                   int32_t *rows_per_item, int64_t *items);

/* Runtime call; no passage of the paper corresponds to it (the paper
 * describes the update, not its bookkeeping).
 * Bind a simulation to caller device memory dev_buf (dev_bytes >=
 * dbm_state_bytes(p), 256-byte aligned, on the current device).  Uploads the
 * geometry tables and clears the buffer on the legacy default stream and
 * waits for that stream only (work in flight on non-blocking streams goes on;
 * none of it may touch dev_buf).  The caller keeps ownership of dev_buf and
 * must keep it alive until dbm_destroy.
 * Errors: DBM_EINVAL, DBM_ECFL, DBM_ENOMEM (buffer too small), DBM_ECUDA. */
int dbm_create(const dbm_params *p, void *dev_buf, size_t dev_bytes, dbm_t **out);

/* Runtime call; no passage of the paper corresponds to it.
 * Release the handle (not dev_buf).  First waits until the GPU has finished
 * the last work enqueued on the handle's buffers: the handle's own calls
 * (steps, init, moments, non-equilibrium moments) and the batched steps in
 * which it was active, so dev_buf may be reused once this returns.  Work the
 * caller captured into its own CUDA graphs is the caller's to finish.
 * Errors: DBM_EINVAL (NULL), DBM_ECUDA (that work failed; the handle is
 * released all the same). */
int dbm_destroy(dbm_t *h);

/* Set the state at t = 0 from host fields rho, u_r, u_theta, T, lambda
 * ([ntheta][nr] doubles each, caller-owned, read during the call): f = f^eq
 * (Eq. feq, Sec. II.B) of the fields at every site, lambda copied (reading:
 * the paper gives macroscopic initial data only).  f^eq is evaluated in the
 * state's precision with the arithmetic of the step's own equilibrium.  The
 * fields are copied to the device and checked there by the init kernel;
 * the call synchronises `stream` once at the end, so the host arrays may be
 * reused on return.  Resets the step counter.
 * Errors: DBM_EINVAL (NULL array, or some rho <= 0, T <= 0 or non-finite
 * value: the state is then undefined until the next init), DBM_ECUDA. */
int dbm_init_state(dbm_t *h, const double *rho, const double *ur, const double *uth,
                   const double *T, const double *lam, void *stream);

/* As dbm_init_state with device-resident fields: d_fields points to
 * 5 * ntheta * nr doubles laid out [field][ntheta][nr] in the order rho, u_r,
 * u_theta, T, lambda (read by the GPU in stream order).  Asynchronous: an
 * invalid value is reported as DBM_EINVAL by the next dbm_status or
 * dbm_moments. */
int dbm_init_state_device(dbm_t *h, const double *d_fields, void *stream);

/* Enqueue nsteps time steps (Eq. LB_evolution_equation + Eq. Eqlambda) on
 * `stream`; asynchronous.  nsteps = 0 is a no-op.  Uses a CUDA graph of the
 * step kernel for long runs.  Errors: DBM_EINVAL (nsteps < 0), DBM_ECUDA. */
int dbm_step(dbm_t *h, int64_t nsteps, void *stream);

/* Macroscopic fields of the current state, copied to host arrays (any may be
 * NULL): rho = sum f, u = sum f v / rho in polar components, T = sum f
 * (v - u)^2 / (2 rho) (Sec. II.B), lambda.  Each site's moments are
 * evaluated in the state's precision: FP64 states in FP64; FP32 states in
 * FP32 ring by ring, the very values the step computes, widened to double.
 * totals (may be NULL) receives the area-weighted sums {mass, momentum_x,
 * momentum_y, energy}, energy = rho T + rho u^2 / 2, weight r dr dtheta,
 * accumulated over sites in FP64.  Synchronises `stream`.
 * Errors: DBM_ENONFINITE (some moment is NaN/inf; outputs still written),
 * DBM_ETIMEOUT (a step kernel's bounded wait expired), DBM_EINVAL (the last
 * dbm_init_state_device found an invalid field value), DBM_ECUDA. */
int dbm_moments(dbm_t *h, double *rho, double *ur, double *uth, double *T, double *lam,
                double totals[4], void *stream);

/* As dbm_moments into device memory d_out (5 * ntheta * nr doubles,
 * [field][ntheta][nr], order rho, u_r, u_theta, T, lambda); asynchronous, no
 * totals, no status check. */
int dbm_moments_device(dbm_t *h, double *d_out, void *stream);

/* Non-equilibrium manifestations of Sec. II.E (Eqs. M_absolute,
 * D_absolute): Delta*_m = M*_m(f) - M*_m(f^eq) with the central moments
 * M*_2 = sum f v* v*, M*_3 = sum f v* v* v*, M*_{3,1} = sum (1/2) f |v*|^2 v*,
 * M*_{4,2} = sum (1/2) f |v*|^2 v* v*, v* = v - u, polar components,
 * evaluated in FP64 from f.  out: host array of DBM_NONEQ * ntheta * nr
 * doubles, [component][ntheta][nr], components rr, r-theta, theta-theta of
 * Delta*_2; rrr, rr-theta, r-theta-theta, theta-theta-theta of Delta*_3;
 * r, theta of Delta*_{3,1}; rr, r-theta, theta-theta of Delta*_{4,2}.
 * Synchronises `stream`. */
#define DBM_NONEQ 12
int dbm_noneq(dbm_t *h, double *out, void *stream);

/* As dbm_noneq into device memory d_out (same layout); asynchronous. */
int dbm_noneq_device(dbm_t *h, double *d_out, void *stream);

/* Steps taken since the last init or import. */
int64_t dbm_steps_done(const dbm_t *h);

/* Runtime call; no passage of the paper corresponds to it.
 * Host-only: device addresses of the current state inside the handle's
 * buffer, for callers that read it in place (for example
 * dbm_totals_noalloc).  *d_f: f[33][ntheta][ld] and *d_lam: lam[ntheta][ld]
 * in the handle's precision, ld = nr rounded up to a multiple of 32 (*ld);
 * lam holds the stored reaction variable as in dbm_export_state.  The state
 * alternates between two buffers: the addresses are those the next step
 * reads, valid for work enqueued (in stream order) before the next
 * dbm_step, dbm_batch_step, init or import of the handle.  Any output may be
 * NULL.  Errors: DBM_EINVAL (NULL handle). */
int dbm_state_device(const dbm_t *h, const void **d_f, const void **d_lam, int64_t *ld);

/* Synchronise `stream` and report the sticky device status word: DBM_OK,
 * DBM_ETIMEOUT (a bounded wait in a step kernel expired), DBM_EDEVICE (a
 * device-side self-check failed and the step skipped the offending copy or
 * store; dbm_last_error says which), DBM_EINVAL (the last init found an
 * invalid field value) or DBM_ECUDA. */
int dbm_status(dbm_t *h, void *stream);

/* Checkpoint: copy the raw state to host memory.  f receives 33 * ntheta * nr
 * values and lam ntheta * nr values in the handle's precision (float for
 * DBM_FP32, double for DBM_FP64), layout f[v][ntheta][nr]; *steps receives the
 * step counter.  lam holds the stored reaction variable: lambda for DBM_FP64,
 * the unburnt fraction 1 - lambda for DBM_FP32 (floats near 1 are too coarse
 * for the last stages of burning).  Synchronises `stream`. */
int dbm_export_state(dbm_t *h, void *f, void *lam, int64_t *steps, void *stream);

/* Restore a state written by dbm_export_state (same layout and precision);
 * resuming is bitwise identical to an uninterrupted run.  Synchronises. */
int dbm_import_state(dbm_t *h, const void *f, const void *lam, int64_t steps, void *stream);

/* Launch shape of the handle (any pointer may be NULL): persistent CTAs in
 * the grid, threads per CTA, dynamic shared memory per CTA, theta rows per
 * work item, work items per step and the step-kernel variant. */
int dbm_launch_info(const dbm_t *h, int *grid, int *threads, int *smem_bytes,
                    int *rows_per_item, int *items, int *variant);

/* Self-test of the FP32 step's reciprocal (hardware approximation refined by
 * one Newton-Raphson step): writes it and the correctly rounded 1/x for n
 * device floats d_x into d_approx and d_ieee (device arrays); asynchronous. */
int dbm_selftest_rcp(const float *d_x, float *d_approx, float *d_ieee, int n, void *stream);

/* Self-test of the bounded wait that every device-side wait of the step
 * kernels uses (an mbarrier wait that gives up after a cycle limit, sets a
 * status bit and returns instead of hanging).  One CTA waits on an mbarrier
 * for at most limit_cycles (1 .. 2^31; the step kernels use 2^31, about a
 * second): with arrive = 0 nothing arrives, the wait runs out and the kernel
 * ORs 1 (the step kernels' "wait timed out" bit, reported by dbm_status as
 * DBM_ETIMEOUT) into the device int *d_status; with arrive = 1 another warp
 * arrives and *d_status is left unchanged.  Asynchronous on `stream`.
 * Errors: DBM_EINVAL, DBM_ECUDA. */
int dbm_selftest_wait(int *d_status, int arrive, int64_t limit_cycles, void *stream);

/* Number of step-kernel variants for a precision (0 if invalid).  Variants
 * differ only in how the work is staged (pipeline, ring depth, registers);
 * every variant computes the same update bit for bit. */
int dbm_num_variants(int precision);

/* Switch the handle to step-kernel variant 1..dbm_num_variants(). */
int dbm_set_variant(dbm_t *h, int variant);

/* Autotuner: time every variant on the handle's own state for `steps`
 * launches each (after 2 untimed ones) with CUDA events on `stream`, switch
 * the handle to the fastest and remember it for the handle's size class
 * (precision x ceil(log2 nr) x ceil(log2 ntheta)), which dbm_create then uses
 * for params with variant 0 for the rest of the process.  The timing steps
 * advance the simulation (num_variants x (steps + 2) steps).  *best receives
 * the chosen variant, ms_per_step[v-1] (may be NULL) each variant's time. */
int dbm_autotune(dbm_t *h, int steps, void *stream, int *best, float *ms_per_step);

/* ---- allocation-free conservation totals -------------------------------- */
/*
 * The paper has no counterpart to this entry point.  It computes the same
 * totals as dbm_moments for callers that cannot hand the library any device
 * scratch memory: a component holding only raw device pointers to a state that
 * another component owns (a checkpoint writer or a monitoring thread), or code
 * under a fixed device-memory budget whose allocator refuses new allocations
 * once a run has started.  It allocates nothing and calls no cudaMalloc,
 * cudaFree or allocating library routine: its reduction scratch (4 FP64 sums
 * per theta row) is a static device array of DBM_NOALLOC_MAX_ROWS rows
 * (512 KB) that every GPU loading the library holds until the process exits.
 *
 *   d_f       device array f[33][ntheta][ld] in p->precision (float or double):
 *             a live state in place (dbm_state_device gives its address and
 *             ld) or the unpadded layout dbm_export_state writes (ld = nr);
 *             read in stream order.  Each site's sums are taken as dbm_moments
 *             takes them for that precision, accumulated in FP64.
 *   ld        elements between consecutive theta rows, >= nr; 0 means nr.
 *   d_totals  device array of 4 doubles receiving {mass, momentum_x,
 *             momentum_y, energy}, area-weighted as in dbm_moments.
 *   stream    cudaStream_t as void* (NULL: legacy default stream); the call
 *             only enqueues two kernels and returns.
 *
 * The first call on a device (and again after that device's context was
 * replaced, e.g. by cudaDeviceReset) looks up the device address of the
 * static array with that device current; make that first call before any
 * stream capture.  All calls share the one array and it keeps the last
 * call's contents; each call rewrites every row it reads, so nothing needs
 * clearing, but calls whose work overlaps on the GPU (for example on two
 * concurrent streams) race on it.
 * Errors: DBM_EINVAL (NULL pointer, ld < nr, invalid grid or precision),
 * DBM_ENOMEM (ntheta > DBM_NOALLOC_MAX_ROWS: the state does not fit the
 * static scratch), DBM_ECUDA (symbol lookup or launch failed; the failure
 * is recorded for dbm_last_error). */
#define DBM_NOALLOC_MAX_ROWS 16384
int dbm_totals_noalloc(const dbm_params *p, const void *d_f, int64_t ld, double *d_totals, void *stream);

/* ---- batches: many uneven simulations, one persistent launch per step ---- */
/*
 * A batch advances the simulations attached to its slots together: each time
 * step is ONE launch of the persistent step kernel over a device table of
 * work items (W radial sites x rows_per_item theta rows) drawn from every
 * attached simulation, interleaved so that every CTA gets a share of each.
 * A device-side step counter T decides which slots are active in a step
 * (slot s advances while start_s <= T < end_s), so a captured CUDA graph of
 * 32 steps stays valid while slots come and go.  The update of each
 * simulation is exactly the single-instance update (same kernel body).
 * All simulations of a batch share one precision.  While attached, a
 * simulation must not be stepped on its own.
 *
 * Batches and the server below are runtime machinery (scheduling many
 * simulations on one GPU); no passage of the paper corresponds to them.
 */
typedef struct dbm_batch_s dbm_batch_t;

/* Host-only: device bytes for a batch of max_slots slots and at most
 * max_items work items (0 if an argument is invalid). */
size_t dbm_batch_bytes(int max_slots, int64_t max_items, int precision);

/* Host-only: the work items of a batched step (what dbm_batch_step launches
 * after a commit).  Slot s holds an nr[s] x ntheta[s] simulation (nr[s] = 0:
 * empty), cut into strips of `width` radial sites (the kernel's W) by runs of
 * rows_per_item[s] theta rows.  The items of all slots are interleaved; when
 * they outnumber the `grid` persistent CTAs, they are balanced over the CTAs
 * longest-processing-time-first with the cost estimate
 * (rows + 2) (0.3 + 0.7 active lanes / width), and laid out so that CTA c runs
 * items c, c + grid, c + 2 grid, ..., padded with empty items (slot -1); the
 * interleaved order is kept if the padded table would exceed max_items.
 * items (may be NULL): room for max_items quadruples (slot, first radial site,
 * first theta row, end row).  *n_items receives the count.
 * Errors: DBM_EINVAL, DBM_ENOMEM (more than max_items items). */
int dbm_batch_plan(int32_t nslots, const int32_t *nr, const int32_t *ntheta, const int32_t *rows_per_item,
                   int32_t width, int32_t grid, int64_t max_items, int32_t *items, int64_t *n_items);

/* Create a batch on caller device memory (256-byte aligned, >=
 * dbm_batch_bytes).  rows_per_item: theta rows per work item (0 = 16; -1 =
 * scaled to each simulation: 16 up to 512 theta rows, 32 up to 1024, else 64).
 * Allocates a pinned host staging buffer for the tables and takes max_slots
 * entries of the device's batch constant table (per-slot constants read by
 * the batched kernel from constant memory; DBM_BATCH_CONST_FP32 /
 * DBM_BATCH_CONST_FP64 entries per device and precision, shared by all live
 * batches of the process, given back by dbm_batch_destroy).  Synchronous.
 * Errors: DBM_EINVAL, DBM_ENOMEM (buffer too small, or fewer than max_slots
 * free table entries), DBM_ECUDA. */
#define DBM_BATCH_CONST_FP32 256
#define DBM_BATCH_CONST_FP64 128
int dbm_batch_create(int max_slots, int64_t max_items, int precision, int rows_per_item,
                     void *dev_buf, size_t dev_bytes, dbm_batch_t **out);

/* Runtime call; no passage of the paper corresponds to it.  Free the batch
 * (not the attached simulations or dev_buf) after waiting for the batched
 * steps already enqueued, which read its tables in dev_buf. */
int dbm_batch_destroy(dbm_batch_t *b);

/* Attach simulation h to a free slot to advance nsteps steps from the batch's
 * current step on (it keeps its own state buffers).  Takes effect at the next
 * dbm_batch_step.  Errors: DBM_EINVAL (bad slot, precision mismatch, h
 * already attached), DBM_EBUSY (slot taken). */
int dbm_batch_attach(dbm_batch_t *b, int slot, dbm_t *h, int64_t nsteps);

/* Free a slot; the simulation keeps the steps it took (its step counter and
 * buffer index are up to date after every dbm_batch_step).
 * Errors: DBM_EINVAL, DBM_ENOTFOUND (slot empty). */
int dbm_batch_detach(dbm_batch_t *b, int slot);

/* Steps the slot's simulation still has to take (-1 if the slot is empty). */
int64_t dbm_batch_remaining(const dbm_batch_t *b, int slot);

/* The batch's step counter T (host view). */
int64_t dbm_batch_time(const dbm_batch_t *b);

/* Upload the slot and item tables (stream-ordered; done automatically by
 * dbm_batch_step after attach/detach) and pick the batch kernel: the
 * precision's default (tensor-map row loads for FP32) when every attached
 * simulation has usable tensor maps, else the bulk-copy variant.  A change of
 * kernel waits for `stream` to drain and drops the captured step graph.
 * Errors: DBM_ENOMEM (more items than max_items), DBM_ECUDA. */
int dbm_batch_commit(dbm_batch_t *b, void *stream);

/* Advance the step counter nsteps steps on `stream` (asynchronous); every
 * attached simulation advances while it has steps left. */
int dbm_batch_step(dbm_batch_t *b, int64_t nsteps, void *stream);

/* Autotuner of a batch: times the precision's default kernel and the
 * bulk-copy kernel, each with 16, 32, 64 and size-scaled (-1) theta rows per
 * work item, for twice `steps` batched steps each (after 32 untimed steps;
 * the better of the two timings counts) with CUDA events on `stream`, and
 * keeps the fastest.  The trials advance every attached simulation
 * (8 x (32 + 2 steps) steps at most); attach them with enough steps left.  *variant and *rows_per_item receive the choice;
 * ms_per_step[8] (may be NULL) the time per step of each candidate in the
 * order (default, 16), (default, 32), (default, 64), (default, -1), then the
 * same for the bulk-copy kernel; 0 for a candidate not run.
 * Errors: DBM_EINVAL, DBM_ECUDA. */
int dbm_batch_autotune(dbm_batch_t *b, int steps, void *stream, int *variant, int *rows_per_item,
                       float *ms_per_step);

/* Launch shape: persistent grid, current number of work items, rows per item,
 * kernel variant (as of the last commit).  Null outputs are skipped. */
int dbm_batch_launch_info(const dbm_batch_t *b, int *grid, int *items, int *rows_per_item,
                          int *variant);

/* ---- serving: continuous batching behind submit / poll ------------------ */
/*
 * A server owns a batch and a scheduler thread.  dbm_submit queues a request
 * (parameters, host initial fields, number of steps); the scheduler admits
 * queued requests into free batch slots as soon as its device pool has room
 * (first fit in arrival order; a request passed over max_bypass times blocks
 * later ones until it starts), advances all resident simulations quantum by
 * quantum in shared launches, and retires finished ones: their moments go to
 * host memory and dbm_poll hands them out.  A quantum is `quantum` steps or
 * fewer: it ends when the first resident simulation finishes, so the work
 * items are rebalanced over the GPU for the simulations still running.  Two
 * quanta are kept in flight, so admission, table updates and retirement on
 * the host overlap the GPU.  Per-request upload and download run on a second
 * stream and overlap the batched steps.  Each result equals the result of
 * running the request alone (same kernel, same bits).
 */
typedef struct dbm_server_s dbm_server_t;

typedef struct dbm_server_config {
    int32_t max_slots;      /* simulations resident at once (batch slots)          */
    int32_t max_queue;      /* queued requests beyond which dbm_submit is EBUSY    */
    int32_t quantum;        /* steps per scheduling round (32 | quantum: graphs)   */
    int32_t precision;      /* DBM_FP32 or DBM_FP64, shared by all requests        */
    int64_t max_items;      /* capacity of the batch's work-item table             */
    int32_t rows_per_item;  /* theta rows per work item (0 = 16, -1 = size-scaled) */
    int32_t max_bypass;     /* how often a queued request may be passed over       */
} dbm_server_config;

typedef struct dbm_fields {  /* host arrays [ntheta][nr], read during dbm_submit */
    const double *rho, *ur, *uth, *T, *lam;
} dbm_fields;

typedef struct dbm_result {
    int32_t status;          /* DBM_OK, DBM_ECANCELLED, DBM_ENONFINITE, ...        */
    int32_t nr, ntheta;
    int32_t pad;
    int64_t steps;           /* steps taken                                       */
    double *rho, *ur, *uth, *T, *lam; /* library-owned host arrays [ntheta][nr]   */
                                      /* (NULL unless status is OK or ENONFINITE) */
    double totals[4];        /* as dbm_moments                                    */
    double t_submit, t_start, t_end;  /* seconds on the server's clock            */
} dbm_result;

typedef struct dbm_server_stats {
    double submitted, completed, failed, cancelled;
    double queued, running;
    double updates;            /* site x velocity updates of completed requests  */
    double executed;           /* site x velocity updates enqueued in all quanta  */
    double pool_free_largest;  /* bytes                                           */
    double batch_time;         /* steps of the batch clock                        */
    int32_t status;            /* first error of the batched steps, or DBM_OK     */
    int32_t pad;
} dbm_server_stats;

/* Host-only: device bytes the server itself needs inside its pool (the batch
 * tables); the rest of the pool holds the resident simulations. */
size_t dbm_server_min_bytes(const dbm_server_config *cfg);

/* Start a server on caller device memory (256-byte aligned), on the current
 * device.  The caller keeps ownership of dev_pool until dbm_server_destroy.
 * Its batch takes max_slots entries of the batch constant table (see
 * dbm_batch_create).  Errors: DBM_EINVAL, DBM_ENOMEM, DBM_ECUDA. */
int dbm_server_create(const dbm_server_config *cfg, void *dev_pool, size_t pool_bytes,
                      dbm_server_t **out);

/* Runtime call; no passage of the paper corresponds to it.
 * Queue a simulation: params (precision must match the server's), initial
 * fields (copied before return), nsteps.  *ticket identifies it.
 * Errors: DBM_EINVAL, DBM_ECFL, DBM_ENOMEM (larger than the whole pool),
 * DBM_EBUSY (queue full), or the error that ended the server's work.
 *
 * A batched step that fails (DBM_ECUDA, DBM_EDEVICE, ...) ends the server's
 * work: nothing more is launched, and every queued or resident request whose
 * steps are not all done finishes with that status and no arrays (the stats'
 * status holds it).  Requests that finished before it keep their results.
 * For tests of this path, DBM_SERVER_FAIL_QUANTUM=n in the environment at
 * dbm_server_create makes quantum n (from 0) fail with DBM_ECUDA on the host,
 * without a launch. */
int dbm_submit(dbm_server_t *s, const dbm_params *p, const dbm_fields *init, int64_t nsteps,
               uint64_t *ticket);

/* Runtime call; no passage of the paper corresponds to it.
 * Wait up to timeout_us (0: do not wait, < 0: forever) for a request.  On
 * DBM_OK *out holds its result (status inside) and the ticket is consumed;
 * free the arrays with dbm_result_free.  DBM_ENOTREADY (timeout_us = 0 and
 * still queued or running), DBM_ETIMEOUT, DBM_ENOTFOUND. */
int dbm_poll(dbm_server_t *s, uint64_t ticket, dbm_result *out, int64_t timeout_us);

/* Free the host arrays of a polled result. */
int dbm_result_free(dbm_result *res);

/* Cancel a queued or running request (its result status becomes
 * DBM_ECANCELLED; a running one leaves the batch at the next quantum). */
int dbm_cancel(dbm_server_t *s, uint64_t ticket);

/* Counters of the server. */
int dbm_server_stats_get(dbm_server_t *s, dbm_server_stats *out);

/* Cancel what is left, stop the scheduler, free everything but dev_pool. */
int dbm_server_destroy(dbm_server_t *s);

#ifdef __cplusplus
}
#endif
#endif /* DBM_H */
