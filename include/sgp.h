/*
 * sgp.h -- C ABI of the GB300 propagator for the rotating spin-orbit-coupled
 * spin-2 Gross-Pitaevskii system, integrated with the compact splitting
 * Fourier spectral method of arXiv 2603.25282.
 *
 * Model (Sec. 1, Eq. (CGPEs)):
 *   i d/dt Psi = (H0 I + c1 F.f - gamma S) Psi + c2 A00 A conj(Psi),
 *   H0 = -Lap/2 + V + c0 rho - Omega L_z,  V = (gx^2 x^2 + gy^2 y^2 [+ gz^2 z^2])/2.
 * Method (Sec. 3): in the rotating frame of Eq. (mapping) the linear flow
 * (Laplace + SOC + Omega f_z, Eq. (linearEQ2)) is exact per Fourier mode
 * (Eq. (sl1)); the nonlinear flow is exact per grid point (Eq. (solution2))
 * with the trap taken at R(t)x; they are composed as TS2 (Algorithm 1) or TS4
 * (Sec. 3.3).
 *
 * Conventions shared by every entry point:
 *   - Field layout: complex interleaved (re, im), shape
 *     [batch][5][nz][ny][nx] with x fastest; component order l = 2,1,0,-1,-2
 *     (Sec. 1, the vector Psi).  2D grids have nz = 1.
 *   - Element type: complex64 (two floats) for SGP_F32 contexts, complex128
 *     (two doubles) for SGP_F64 contexts.  SGP_F32 contexts still keep the
 *     time t, the rotation angle Omega t, the linear-flow phase angles and all
 *     observable sums in FP64.
 *   - Grid: x_j = -L + j h, h = 2L/N, N even (Sec. 3.1); supported N per
 *     axis: 2^a 3^b with 16 <= N <= 1024 (b <= 1).
 *   - Frame: the context stores the rotating-frame field
 *     phi_l(x,t) = exp(-i l Omega t) psi_l(R(t) x, t) of Eq. (mapping); at
 *     t = 0 it equals the lab-frame field.
 *   - Ownership: every pointer argument stays owned by the caller; the
 *     context owns its device buffers and frees them in sgp_destroy.
 *   - Streams: all device work of a context is issued on the CUDA stream
 *     given at creation (a cudaStream_t passed as void*).  With NULL the
 *     context creates and owns a private non-blocking stream; device-pointer
 *     copies in or out are then ordered only on that stream (call
 *     sgp_synchronize before touching a device destination from another
 *     stream, and have a device source ready before the call).  Calls
 *     documented as asynchronous return before the GPU work completes.
 *   - Errors: every call returns an sgp_status; on failure the context keeps
 *     a message readable with sgp_last_error.  No call throws or aborts.
 *     A context is not thread-safe: one host thread at a time.
 */
#ifndef SGP_H
#define SGP_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sgp_ctx sgp_ctx;

typedef enum {
  SGP_OK = 0,
  SGP_EINVAL = 1,        /* bad argument (size, pointer, parameter, dt)   */
  SGP_ENOMEM = 2,        /* device or host allocation failed              */
  SGP_ECUDA = 3,         /* a CUDA runtime call failed (see last_error)   */
  SGP_ETIMEOUT = 4,      /* a bounded device-side wait gave up (ensembles, tile loads) */
  SGP_ENONFINITE = 5,    /* a NaN/Inf was detected in the observables     */
  SGP_ESTATE = 6,        /* call out of order (e.g. step before set_state)*/
  SGP_EUNSUPPORTED = 7,  /* valid request the library does not implement */
  SGP_EDRIFT = 8         /* the health check saw the mass drift too far   */
} sgp_status;

typedef enum { SGP_F32 = 32, SGP_F64 = 64 } sgp_prec;

/* Compositions of Sec. 3.3.  TS2: N(tau/2) L(tau) N(tau/2) (Algorithm 1).
 * TS4: N(a1 tau) L(b1 tau) N(a2 tau) L(b2 tau) N(a2 tau) L(b1 tau) N(a1 tau)
 * with the fourth-order coefficients of Sec. 3.3, the nonlinear flow taking
 * the a_j and the linear flow the b_j.  The same compositions with the two
 * flows' roles exchanged (the other reading of the coefficient list, equally
 * valid, with a different error constant): TS2_LNL: L(tau/2) N(tau) L(tau/2);
 * TS4_LOUTER: L(a1 tau) N(b1 tau) L(a2 tau) N(b2 tau) L(a2 tau) N(b1 tau)
 * L(a1 tau).  Time advances in the L substeps. */
typedef enum { SGP_TS2 = 0, SGP_TS4 = 1, SGP_TS2_LNL = 2, SGP_TS4_LOUTER = 3 } sgp_scheme;

/* Caller-supplied device allocator (optional).  alloc returns a device
 * pointer of at least `bytes` bytes on `device` (usable on the context
 * stream `stream`), or NULL on failure; free releases such a pointer. */
typedef void* (*sgp_alloc_fn)(size_t bytes, int device, void* stream, void* user);
typedef void (*sgp_free_fn)(void* ptr, int device, void* stream, void* user);

/* Flags of sgp_autotune. */
enum { SGP_TUNE_FORCE = 1 };

/* Substep kinds for sgp_substep. */
typedef enum { SGP_SUB_NONLINEAR = 0, SGP_SUB_LINEAR = 1 } sgp_substep_kind;

/* Parameters of Eq. (CGPEs) and the harmonic trap (harmonic). */
typedef struct {
  double omega;   /* angular velocity Omega                       */
  double gamma;   /* spin-orbit coupling strength gamma           */
  double c0, c1, c2;  /* mean-field, spin-exchange, singlet-pairing */
  double gx, gy, gz;  /* trap frequencies gamma_x, gamma_y, gamma_z */
} sgp_params;

/* Observables of Sec. 2 for one batch member, lab-frame quantities computed
 * from the rotating-frame field (mass, <L_z>, |grad|^2, the rho/F/A00 terms
 * and the SOC term are frame invariant; the trap and widths use R(t)x).
 * Integrals are h^d-weighted grid sums; derivatives are spectral. */
typedef struct {
  double t;             /* current time                                   */
  double mass;          /* N(t) = sum_l ||psi_l||^2                        */
  double energy;        /* E(t), Sec. 2 "Mass and energy"                  */
  double magnetization; /* M(t) = sum_l l ||psi_l||^2                      */
  double lz;            /* <L_z>(t)                                        */
  double comp_mass[5];  /* ||psi_l||^2, l = 2..-2                          */
  double width2[3];     /* delta_x, delta_y, delta_z of Eq. (ConWid)       */
  double e_kin;         /* sum (1/2)|grad psi|^2                           */
  double e_pot;         /* sum V rho                                       */
  double e_rot;         /* -Omega <L_z>                                    */
  double e_int;         /* c0/2 rho^2 + c1/2 (|F+|^2+Fz^2) + c2/2 |A00|^2  */
  double e_soc;         /* -gamma Psi^H S Psi                              */
} sgp_obs;

/* Library version as MAJOR*10000 + MINOR*100 + PATCH.  Cannot fail. */
int sgp_version(void);

/* Human-readable name of a status code (static storage; "unknown"
 * for a value outside the enum).  Cannot fail. */
const char* sgp_status_string(sgp_status s);

/* Create a context for `batch` independent fields on a dim-D grid
 * (Sec. 3.1 grids).  n[0..dim-1] and L[0..dim-1] are given in (x, y, z)
 * order; L is the half-width of [-L, L].  prec is SGP_F32 or SGP_F64.
 * device is the CUDA ordinal; stream a cudaStream_t (or NULL).
 * Allocates the field, the FFT twiddle tables and the observable scratch on
 * `device`.  Errors: SGP_EINVAL for dim not in {2,3}, unsupported N, L <= 0,
 * batch outside [1, 65535] or a NULL out; SGP_ENOMEM/SGP_ECUDA on allocation
 * failure (no context is returned then).  Parameters default to all zero
 * with unit trap frequencies; the field to zero at t = 0. */
sgp_status sgp_create_grid(int dim, const int* n, const double* L, int batch,
                           int prec, int device, void* stream, sgp_ctx** out);

/* Set the physical parameters (Sec. 1) of every batch member to *p.
 * Synchronous on the host (waits for the context stream); takes effect for
 * work issued afterwards.  Errors: SGP_EINVAL for NULL or non-finite values. */
sgp_status sgp_set_params(sgp_ctx* ctx, const sgp_params* p);

/* Per-member parameters: p[m] for member m, count == batch.  Members may
 * differ in every parameter; when they differ in Omega or gamma the
 * linear-flow tables are built per member.  Same synchronisation and errors
 * as sgp_set_params, plus SGP_EINVAL for count != batch. */
sgp_status sgp_set_params_batch(sgp_ctx* ctx, const sgp_params* p, int count);

/* Device memory of the contexts (and ensemble groups) created after this
 * call comes from `alloc` and goes back through `free_fn`: the field, the
 * twiddle and mode tables, the observables scratch, the adjoint checkpoints
 * and the autotuner's scratch.  Each context keeps the pair it was created
 * with until sgp_destroy; frees synchronise the context stream first.
 * Returned blocks must be 16-byte aligned (the kernels move 16-byte
 * pieces); a misaligned block is handed back to free_fn at once and counts
 * as a failed allocation.
 * alloc = free_fn = NULL restores cudaMalloc/cudaFree.  Process-wide, not
 * thread-safe against concurrent sgp_create_grid.  An allocation failure
 * makes the calling entry point return SGP_ENOMEM or SGP_ECUDA.  Errors:
 * SGP_EINVAL if exactly one of the two functions is NULL. */
sgp_status sgp_set_allocator(sgp_alloc_fn alloc, sgp_free_fn free_fn, void* user);

/* Copy a field into the context and set the time to t0.  `src` holds
 * batch*5*nz*ny*nx complex elements of the context precision in the layout
 * above; src_on_device != 0 means a device pointer on the context device.
 * At t0 the rotating frame coincides with the lab frame only if t0 = 0;
 * otherwise `src` is taken as the rotating-frame field at t0.  The copy is
 * ordered on the context stream; a host `src` may be reused on return.
 * Errors: SGP_EINVAL for NULL or non-finite t0. */
sgp_status sgp_set_state(sgp_ctx* ctx, const void* src, int src_on_device,
                         double t0);

/* Copy the current (rotating-frame) field out, same layout as set_state
 * (the caller owns dst, batch*5*nz*ny*nx elements).  With dst_on_device ==
 * 0 the call synchronises the context stream before returning; with a
 * device pointer it is asynchronous.  Errors: SGP_EINVAL for NULL; SGP_ECUDA
 * for a failed copy. */
sgp_status sgp_get_state(sgp_ctx* ctx, void* dst, int dst_on_device);

/* Lab-frame field at the current time t (Sec. 3.1): psi_l(x, t) =
 * exp(i l Omega t) phi_l(R(t)^T x, t), the inverse of the mapping
 * (mapping), evaluated on the grid as in Eq. (RSDA2).  The rotation by
 * Omega t (each member its own Omega) is done as exact quarter turns, which
 * need a square x-y grid (equal N and L) and are only used when
 * |Omega t| mod pi/2 leaves a remainder beyond pi/4, and three shears
 * exp(a y d_x) exp(b x d_y) exp(a y d_x), a = -tan(r/2), b = sin(r), for the
 * remainder r (each a line FFT, a phase per mode with its angle in FP64,
 * the inverse FFT).  In 3D the rotation is about z.  Accurate to the
 * spectral accuracy of the grid for fields that decay inside the domain
 * (the shears are periodic translations).  dst: the state layout of
 * sgp_get_state, on the device if dst_on_device, else host memory.  The
 * context's state is not changed.  Synchronises.  Errors: SGP_EINVAL for
 * NULL dst, dim 1, or a non-square grid when quarter turns are needed. */
sgp_status sgp_get_state_lab(sgp_ctx* ctx, void* dst, int dst_on_device);

/* Current time t (host copy, FP64) into *t.  Errors: SGP_EINVAL for NULL. */
sgp_status sgp_get_time(const sgp_ctx* ctx, double* t);

/* Advance every batch member by nsteps steps of size dt with the given
 * composition (Sec. 3.3; TS2 is Algorithm 1, sgp_scheme lists all four).
 * Substeps of the same kind where consecutive steps meet are merged: the
 * nonlinear ones at the same time into one exact nonlinear flow (the flow
 * property of Eq. (solution2)), the linear ones (time-independent in the
 * rotating frame) into one linear flow, so a call costs nsteps linear and
 * nsteps+1 nonlinear substeps for TS2 (the reverse for TS2_LNL, which also
 * opens and closes the run with an x-transform pass).  Runs of 128 steps
 * or more are issued as replays of a captured CUDA graph of 64 steps (one
 * extra nonlinear pass per 64 steps, where the chunks meet); the time is
 * kept on the device in FP64 and advanced inside the graph.  The field is
 * in physical space on return.  Asynchronous on the context stream.
 * Errors: SGP_EINVAL for nsteps < 0, dt <= 0 or non-finite dt; SGP_ESTATE
 * before sgp_set_state; SGP_ECUDA if a launch fails. */
sgp_status sgp_step(sgp_ctx* ctx, long long nsteps, double dt, int scheme);

/* The substeps that nsteps steps of `scheme` issue (Sec. 3.3), host only
 * (no device work): the per-step sequence of nonlinear ('N') and linear
 * ('L') flows with the flows of the same kind that meet at a step boundary
 * merged into one (N(a) N(b) = N(a + b) at equal time; L is
 * time-independent in the rotating frame).  Entry k: kinds[k], its step
 * deltas[k] and toffs[k], relative to the start of the run, the time at
 * which a nonlinear flow acts or at which a linear one starts (time
 * advances in the linear flows).  Writes the
 * first min(cap, count) entries (arrays of cap elements, owned by the
 * caller; may be NULL when cap = 0) and the total number of entries into
 * *count.  sgp_step issues exactly this list (in chunks of 64 steps for
 * graph replay, each chunk a list of its own).  Errors: SGP_EINVAL for an
 * unknown scheme, nsteps < 0, dt <= 0 or non-finite, NULL count, or NULL
 * arrays with cap > 0. */
sgp_status sgp_substep_plan(int scheme, long long nsteps, double dt, long long cap, char* kinds,
                            double* deltas, double* toffs, long long* count);

/* Host-to-host propagation with the copies overlapped: the same result, bit
 * for bit, as sgp_set_state(ctx, host_in, 0, t0); sgp_step(ctx, nsteps,
 * dt, scheme); sgp_get_state(ctx, host_out, 0), but the batch is split into
 * `chunks` groups of consecutive members and the copies of the other groups
 * (to the device on one copy stream, back on another) run while a group is
 * propagated on the context stream (members are independent, Sec. 3).
 * host_in, host_out: [batch][5][nz][ny][nx] complex in the context's
 * precision, owned by the caller, may be the same buffer; page-locked
 * memory is needed for the overlap (pageable memory gives the same result
 * without it).  Returns when host_out holds the state at t0 + nsteps*dt.
 * Each group runs its steps with direct launches (no graph replay); the
 * health check does not run in this call.  Errors: SGP_EINVAL for NULL
 * buffers, chunks outside [1, batch], nsteps < 0, dt <= 0 or non-finite,
 * non-finite t0, an unknown scheme; SGP_ECUDA for a failed copy or launch
 * (the host buffers are no longer in use when the call returns). */
sgp_status sgp_step_host(sgp_ctx* ctx, const void* host_in, double t0, void* host_out,
                         long long nsteps, double dt, int scheme, int chunks);

/* Health check of sgp_step (off by default).  With every > 0, sgp_step
 * runs in chunks of at most `every` steps and after each chunk sums every
 * member's mass h^d sum |phi|^2 in FP64 on the device (Sec. 2: the scheme
 * conserves it exactly) and compares it with the mass at the last
 * sgp_set_state (taken at the first checked step after it).  It returns
 * SGP_ENONFINITE if a mass is NaN or Inf and SGP_EDRIFT if |m/m0 - 1| >
 * drift_tol for some member, with the member, its mass and the step count
 * in sgp_last_error; the steps up to that check have been taken and the
 * time advanced accordingly.  Each check synchronises the context stream.
 * every = 0 turns the check off.  Errors: SGP_EINVAL for every < 0 or a
 * negative or non-finite drift_tol. */
sgp_status sgp_set_health_check(sgp_ctx* ctx, long long every, double drift_tol);

/* Enable (default) or disable graph replay in sgp_step (results are the
 * same either way).  Errors: SGP_EINVAL for a NULL ctx. */
sgp_status sgp_set_graphs(sgp_ctx* ctx, int enable);

/* ---------------------------------------------------------------------
 * Kernel variants (FFT tile and radix schedules) and the autotuner.
 * Every pass kernel exists in up to six variants per line length N, and
 * 3D grids have a plane-level variant of the x-pass:
 *   0  default: x-pass CTAs of about 256 threads (rows side by side), line
 *      pass up to 512 threads with TILE >= 4 (FP32) / 2 (FP64) columns;
 *   1  CTAs of about half the threads (line pass TILE down to 1);
 *   2  CTAs of about a quarter of the threads;
 *   3  FP32 only: for N a power of two the radix-4 plan (4 elements per
 *      thread instead of 8), for N = 3*2^k 12 elements per thread (radix
 *      6 then 4s) in CTAs of 128 threads;
 *   4  FP32 only: the line pass of variant 1 with its tile brought into
 *      shared memory by tensor copies (TMA) instead of per-thread loads
 *      (bit for bit variant 1); for the x-pass the same as variant 1;
 *   5  FP32, x axis of 3D grids with NX = NY = 64 or 128 only: the
 *      x-passes of sgp_step and sgp_substep become xy-plane passes, one
 *      thread-block cluster of NX/16 CTAs per z plane that also does the
 *      y transforms (the plane moves between the CTAs through distributed
 *      shared memory), so a step runs no y-line passes: two passes per
 *      linear/nonlinear pair instead of four.  Other x-passes (gradients,
 *      observables) are those of variant 1;
 *   6  x-pass: CTAs of variant 2's rows with the nonlinear flow shared by
 *      256 threads (for small grids, whose CTAs are few, each thread takes
 *      fewer points through the flow); line pass: the same as variant 2.
 * A plan is one variant per axis (x-pass, y lines, z lines).  Variants
 * compute the same transforms with different rounding (variant 3 has a
 * different radix plan), so results agree to rounding, not bit for bit;
 * variant 4 agrees with variant 1 bit for bit, and variant 5 with variant
 * 1 when the y axis runs variant 0, 1, 2 or 4; x-pass variant 6 agrees
 * with variant 2 to rounding.
 * ------------------------------------------------------------------- */
/* 1 if variant v exists for line length n at precision prec, else 0
 * (also for arguments out of range, and for variant 5, which depends on
 * the whole grid: sgp_set_plan takes it as stated above).  Cannot fail. */
int sgp_variant_exists(int prec, int n, int variant);
/* Set the plan: variants[a] for axis a < dim.  Synchronises the context
 * stream; drops captured graphs.  SGP_EINVAL for a variant that does not
 * exist (nothing is changed then). */
sgp_status sgp_set_plan(sgp_ctx* ctx, const int* variants);
/* Current plan into variants[0..2] (0 for absent axes; caller-owned array
 * of 3).  Errors: SGP_EINVAL for NULL. */
sgp_status sgp_get_plan(const sgp_ctx* ctx, int* variants);
/* Autotuner: axis by axis (the other axes at their current variant), run
 * `reps` Strang steps (1..1000) of dt = 1e-3 with each variant of that
 * axis on a scratch copy of the field, after one warm-up step, timed with
 * CUDA events on the context stream; keep the fastest (a higher-numbered
 * variant must be at least 1.5% faster to replace a lower one).  The state
 * and the time are not changed.  Results are cached per process by
 * (device, precision, grid, batch); a cached plan is reused unless flags
 * has SGP_TUNE_FORCE or ms_out is given.  ms_out (may be NULL): 3 x 7
 * doubles, ms per step of [axis][variant], -1 where the variant or axis
 * does not exist, for variant 4 of the x-pass (which is variant 1) and for
 * variant 6 of the line passes (which is variant 2).
 * Synchronises.  Allocates one field-sized scratch buffer
 * for the duration of the call.  Errors: SGP_EINVAL for a NULL ctx or reps
 * outside [1, 1000]; SGP_ENOMEM / SGP_ECUDA for the scratch or a launch. */
sgp_status sgp_autotune(sgp_ctx* ctx, int reps, int flags, double* ms_out);

/* Apply one substep of size delta (delta may be negative, Sec. 3.3 TS4):
 * SGP_SUB_NONLINEAR applies the exact flow (solution2) at the current time;
 * SGP_SUB_LINEAR applies the exact flow (sl1) and advances the time by delta.
 * Asynchronous.  Errors: SGP_EINVAL for a NULL ctx, an unknown kind or a
 * non-finite delta; SGP_ESTATE before sgp_set_state; SGP_ECUDA. */
sgp_status sgp_substep(sgp_ctx* ctx, int kind, double delta);

/* Observables of Sec. 2 for every batch member into out[0..batch-1].
 * Synchronises the context stream.  Returns SGP_ENONFINITE (with out
 * filled) if any sum is NaN or Inf. */
sgp_status sgp_observables(sgp_ctx* ctx, sgp_obs* out);

/* ---------------------------------------------------------------------
 * Adjoint (gradients of a terminal-time objective J(Phi(T))).
 * ------------------------------------------------------------------- */
/* Like sgp_step, and also stores the state at the start of every chunk of
 * `interval` steps (interval = 0: ceil(sqrt(nsteps))) in device memory
 * owned by the context, for sgp_backward.  The record stays valid until the
 * next sgp_set_state, sgp_set_params(_batch), sgp_step, sgp_substep or
 * sgp_record.  Memory: ceil(nsteps/interval) states for the checkpoints and,
 * for one recomputed segment in sgp_backward, interval*(substeps per step)
 * + 1 states (3 for TS2, 7 for TS4) plus interval*(linear substeps per
 * step) states for the linear substeps' outputs in transform space; when it
 * can be had, a second such buffer (the next segment is then recomputed on
 * a second stream during the sweep through the current one).  Errors: SGP_EINVAL for nsteps <= 0,
 * interval < 0 or dt/scheme as in sgp_step; SGP_ESTATE before
 * sgp_set_state; SGP_ENOMEM/SGP_ECUDA on allocation or launch failure. */
sgp_status sgp_record(sgp_ctx* ctx, long long nsteps, double dt, int scheme,
                      long long interval);

/* Vector-Jacobian product of the recorded run (Sec. 3.3 compositions taken
 * substep by substep in reverse; the flows of Eqs. (sl1) and (solution2)
 * are exact, time-reversible and symplectic).  g_T: dJ/dRe Phi(T) +
 * i dJ/dIm Phi(T) in the state layout (batch, 5, [nz,] ny, nx) and precision
 * of the context, on the device if g_T_on_device, else on the host.  Writes
 * the same quantity for the state at the start of the record into g_0
 * (device if g_0_on_device; may alias g_T) and, if dparams is not NULL, the
 * partial derivatives dJ/d(Omega, gamma, c0, c1, c2) through the dynamics
 * into dparams[5*m + 0..4] for member m (host memory; a dependence of J on
 * Omega through the frame R(T) is the caller's).  Each segment is recomputed
 * from its checkpoint (overlapping the sweep through the segment after it
 * when the second segment buffer fits; same result).  Synchronises the
 * context stream.  The record stays
 * valid (several objectives can be differentiated).  Errors: SGP_EINVAL for
 * NULL buffers; SGP_ESTATE without a valid record; SGP_ECUDA. */
sgp_status sgp_backward(sgp_ctx* ctx, const void* g_T, int g_T_on_device, void* g_0,
                        int g_0_on_device, double* dparams);

/* ---------------------------------------------------------------------
 * Ensembles: independent runs on different grids advanced together.
 * Members are grouped by grid; each group is one batched context.  All
 * members share the time and the composition; each has its own
 * parameters.
 *
 * 2D ensembles whose line lengths are all in {64, 96, 128, 192, 256, 384,
 * 512} run in ONE persistent kernel launch per 64 steps (captured in a CUDA
 * graph and replayed; a shorter rest is launched directly).  Its CTAs take
 * work items, each one CTA tile of one pass (the x-pass with the nonlinear
 * flow of Eq. (solution2), or the y-line pass with the linear flow of Eq.
 * (sl1), Sec. 3) of one member, from a device queue ordered pass by pass;
 * a per-member counter of finished tiles makes a member's pass wait for
 * its previous passes.  Every such wait is bounded (sgp_ensemble_set_wait_
 * limit); when one gives up the kernel stops and the step call returns
 * SGP_ETIMEOUT.  The passes use the default kernel geometry (the autotuner's
 * choices do not apply) and give the same results as the per-group launches
 * with plan {0, 1}.  Other ensembles (3D, other line lengths, or with the
 * persistent kernel switched off) issue every group's passes as parallel
 * branches of one captured graph per 64 steps.
 * ------------------------------------------------------------------- */
typedef struct sgp_ens sgp_ens;

/* count members; n[m*dim + a] and L[m*dim + a] are member m's grid.
 * stream as in sgp_create_grid.  Errors as sgp_create_grid per member. */
sgp_status sgp_ensemble_create(int dim, int count, const int* n, const double* L,
                               int prec, int device, void* stream, sgp_ens** out);
/* Number of grid groups (0 for NULL). */
int sgp_ensemble_groups(const sgp_ens* ens);
/* p[0..count-1], one parameter set per member (synchronous).  Errors as
 * sgp_set_params_batch, for the member group that fails. */
sgp_status sgp_ensemble_set_params(sgp_ens* ens, const sgp_params* p);
/* Copy member m's field (5*nz*ny*nx elements of its grid) in or out; layout
 * and on_device as sgp_set_state/sgp_get_state (host copies synchronise).
 * All members share t0.  Errors: SGP_EINVAL for NULL, a member out of
 * range, a non-finite t0 or, once a state is set, a t0 other than the
 * ensemble's time; SGP_ECUDA for a failed copy. */
sgp_status sgp_ensemble_set_member_state(sgp_ens* ens, int member, const void* src,
                                         int src_on_device, double t0);
sgp_status sgp_ensemble_get_member_state(sgp_ens* ens, int member, void* dst,
                                         int dst_on_device);
/* Advance every member by nsteps steps.  Asynchronous, except with the
 * persistent kernel, where the call waits for the work to finish so that
 * it can report a wait that gave up.  Errors as sgp_step: SGP_EINVAL for
 * nsteps < 0, dt <= 0 or non-finite, an unknown scheme; SGP_ESTATE before
 * any member state; SGP_ECUDA; SGP_ETIMEOUT when a bounded device-side wait
 * of the persistent kernel gave up (the members' states are then undefined
 * and must be set again before the next step). */
sgp_status sgp_ensemble_step(sgp_ens* ens, long long nsteps, double dt, int scheme);
/* Use (enable = 1, the default when the ensemble qualifies) or not the
 * persistent work-queue kernel for sgp_ensemble_step and
 * sgp_ensemble_step_host.  Errors: SGP_EINVAL for NULL; SGP_EUNSUPPORTED to
 * enable it for an ensemble that does not qualify (3D, or a line length it
 * is not compiled for). */
sgp_status sgp_ensemble_set_persistent(sgp_ens* ens, int enable);
/* 1 if the steps run in the persistent kernel, else 0 (also for NULL). */
int sgp_ensemble_persistent(const sgp_ens* ens);
/* Limit of every device-side wait of the persistent kernel, in seconds of
 * the GPU's nominal SM clock (default 1 s; at most 3600).  Errors:
 * SGP_EINVAL for NULL or a limit outside (0, 3600]; SGP_ECUDA. */
sgp_status sgp_ensemble_set_wait_limit(sgp_ens* ens, double seconds);
/* Fault injection for tests of the bounded waits (no counterpart in the
 * paper): in the next step call, the first work item of `member` does not
 * signal its completion, so the member's second pass waits until the wait
 * limit and the call returns SGP_ETIMEOUT.  Nothing traps or hangs; the
 * ensemble stays usable once its states are set again.  Errors: SGP_EINVAL
 * for NULL or a member out of range; SGP_EUNSUPPORTED when the persistent
 * kernel is not in use. */
sgp_status sgp_ensemble_inject_stall(sgp_ens* ens, int member);
/* Host round trip of the whole ensemble in one call: every member's state
 * from host_in[m] at time t0, nsteps steps, every member's state to
 * host_out[m] (arrays of count pointers; member m's buffer holds its
 * 5*nz*ny*nx elements; host_in[m] may equal host_out[m]).  The same result
 * as count sgp_ensemble_set_member_state calls, sgp_ensemble_step and count
 * sgp_ensemble_get_member_state calls, with the copies issued
 * asynchronously in stream order and a single synchronisation at the end.
 * When every buffer is page-locked and mapped into the device's address
 * space (cudaHostAlloc, or cudaHostRegister with mapping) and 16-byte
 * aligned, all copies of one direction are a single kernel launch that
 * reads or writes the host buffers through that mapping (two launches per
 * call); otherwise one copy per member and direction.  Returns when
 * every host_out[m] holds its result.  Errors: SGP_EINVAL for NULL arrays
 * or buffers, non-finite t0, nsteps < 0, dt <= 0, an unknown scheme;
 * SGP_ECUDA for a failed copy or launch. */
sgp_status sgp_ensemble_step_host(sgp_ens* ens, const void* const* host_in, double t0,
                                  void* const* host_out, long long nsteps, double dt, int scheme);
/* Observables of every member into out[0..count-1] (synchronises).
 * Errors: SGP_EINVAL for NULL; SGP_ESTATE before any member state;
 * SGP_ENONFINITE as sgp_observables (all members are still written). */
sgp_status sgp_ensemble_observables(sgp_ens* ens, sgp_obs* out);
/* sgp_autotune for every grid group of the ensemble (flags as there);
 * drops the ensemble's captured graphs.  Errors as sgp_autotune. */
sgp_status sgp_ensemble_autotune(sgp_ens* ens, int reps, int flags);
/* Wait for the ensemble's work.  Errors: SGP_EINVAL for NULL; SGP_ECUDA. */
sgp_status sgp_ensemble_synchronize(sgp_ens* ens);
/* Kernels launched by the ensemble so far (0 for NULL). */
long long sgp_ensemble_launch_count(const sgp_ens* ens);
/* Message of the last failing call on ens, or of a failed creation for
 * NULL; valid until the next call. */
const char* sgp_ensemble_last_error(const sgp_ens* ens);
/* Free the ensemble and its groups (synchronises first).  NULL is a no-op. */
sgp_status sgp_ensemble_destroy(sgp_ens* ens);

/* Allocation-free observables (no counterpart in the paper; a service of
 * this library).  Computes the same quantities as sgp_observables for a
 * field the caller already holds on the device, without a context and
 * without allocating anything: no cudaMalloc, cudaFree or other allocating
 * call is made.  It is meant for callers that cannot allocate device memory
 * at this point: code whose device memory is entirely reserved by another
 * allocator's pool, code on a latency-critical path where cudaMalloc's
 * implicit device synchronisation is not acceptable, and code that only
 * holds a device pointer to a field produced elsewhere.
 *
 * All scratch (per-block partial sums, FFT twiddles, final sums, member
 * parameters) lives in
 * file-scope device arrays of fixed size that every GPU which loads the
 * library keeps until the process exits.  Limits: each n[a] as in
 * sgp_create_grid (<= 1024), batch <= 64, and at most 2^19 per-block partial
 * sums (batch * ny * nz / rows-per-block * 13, e.g. batch 64 at 512^2 in
 * FP32); larger requests return SGP_EINVAL with a message.
 *
 * Arguments: the grid and precision as in sgp_create_grid; p the
 * parameters, one set applied to every member of the batch; t the time;
 * field_dev a device pointer (on `device`) to batch*5*nz*ny*nx elements in
 * the layout of sgp_set_state, read only; stream a cudaStream_t (or NULL);
 * out[0..batch-1] host results.
 *
 * The first call on a device is a set-up: with that device current it looks
 * up the device addresses of the scratch arrays (cudaGetSymbolAddress) and
 * loads every kernel this entry point can launch, for all line lengths and
 * both precisions.  CUDA loads a library's device code and file-scope
 * arrays lazily, at first use, and that loading takes device memory; so
 * make the first call while memory can still be allocated, as a warm-up.
 * Every later call on that device allocates no device memory at all.
 * No call may be made on a stream that is being captured: every call
 * synchronises `stream` and copies the sums to host memory.  Every call
 * uses the same scratch and overwrites what the previous call left there,
 * so calls that may overlap on the GPU (other streams, other host threads)
 * race and must be serialised by the caller.  Errors (SGP_EINVAL for bad
 * arguments or sizes beyond the limits, SGP_ECUDA, SGP_ENONFINITE for a
 * non-finite observable) leave their message in sgp_last_error(NULL). */
sgp_status sgp_observables_static(int dim, const int* n, const double* L, int batch,
                                  int prec, const sgp_params* p, double t,
                                  const void* field_dev, int device, void* stream,
                                  sgp_obs* out);

/* Wait for all work issued on the context stream.  Errors: SGP_EINVAL for
 * NULL; SGP_ECUDA with the first asynchronous failure; SGP_ETIMEOUT when a
 * bounded wait of line-pass variant 4 for its tile's tensor copies gave up
 * since the last call (the state is then undefined until it is set again;
 * the word is cleared). */
sgp_status sgp_synchronize(sgp_ctx* ctx);

/* Number of kernels this context has launched so far (for accounting; graph
 * replays count their kernels).  0 for NULL. */
long long sgp_launch_count(const sgp_ctx* ctx);

/* Per-kernel timing with CUDA events recorded on the context stream around
 * every launch while enabled (adds one event pair per launch).  Kinds:
 * 0 x-pass, 1 line pass along y, 2 line pass along z, 3 tables,
 * 4 observables, 5 other.  sgp_get_profile synchronises, writes the number
 * of launches and the summed device milliseconds of each kind into
 * launches[0..5] and ms[0..5] (caller-owned arrays of 6), and clears the
 * record.  Enabling clears too.  Graph replay is off while profiling.
 * Errors: SGP_EINVAL for NULL; SGP_ECUDA. */
sgp_status sgp_set_profiling(sgp_ctx* ctx, int enable);
sgp_status sgp_get_profile(sgp_ctx* ctx, long long* launches, double* ms);

/* Free the context and its device memory (synchronises first, through the
 * allocator it was created with).  NULL is a no-op.  Always SGP_OK. */
sgp_status sgp_destroy(sgp_ctx* ctx);

/* Message of the last failing call on ctx ("" if none).  For a NULL ctx:
 * the message of the last failing call made without a context
 * (sgp_create_grid, sgp_set_allocator, sgp_ensemble_create,
 * sgp_observables_static; all but sgp_set_allocator clear it when they
 * start),
 * in static storage.  Valid until the next call on ctx (or, for NULL, the
 * next call without a context). */
const char* sgp_last_error(const sgp_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* SGP_H */
