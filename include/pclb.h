/*
 * pclb.h -- C ABI of the GB300 polar-coordinate lattice Boltzmann library.
 *
 * The library advances the discrete distribution f of the polar-coordinate
 * finite-difference lattice Boltzmann model (Lin, Xu, Zhang, Li & Succi,
 * "Polar coordinate lattice Boltzmann modeling of compressible flows") on an
 * annulus R1 <= r <= R2, 0 < theta <= 2 pi N_f / N_i, one GPU, one stream.
 *
 * One time step is the combined scheme of Eq. (38): at every node and for
 * every discrete velocity, the analytic BGK relaxation of Eq. (19) towards
 * the equilibrium of Eq. (10) (weights Eqs. 11a-12, Table I), minus the
 * Modified Warming-Beam increments of Eq. (28) (switch function Eq. 37) in r
 * and in theta, all evaluated from the distribution at time t.  Boundary
 * nodes follow Sec. II C: two radial ghost layers per wall in equilibrium
 * with extrapolated (Eq. 39) or prescribed macroscopic values, and periodic
 * azimuthal ghosts with the direction label rotated by N_f (Eq. 40).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  * Velocity index q: q = 0 is the rest velocity; q = 1 + (k-1) N_i + (i-1)
 *    for shell k = 1..4 and direction i = 1..N_i, v_ki = v_k (cos phi_i,
 *    sin phi_i), phi_i = 2 pi (i-1)/N_i (Eq. 2).  Q = 1 + 4 N_i.  Labels are
 *    fixed in Cartesian space.
 *  * Nodes: r = R1 + i_r dr, i_r = 0..n_r-1, dr = (R2-R1)/(n_r-1) (both walls
 *    are nodes); theta = (i_t + 1) dtheta, i_t = 0..n_theta-1,
 *    dtheta = 2 pi n_f / (n_dirs n_theta).
 *  * Field arrays are [n_theta][n_r], r fastest, contiguous.  Distribution
 *    arrays are [Q][n_theta][n_r], contiguous.  The element type is float for
 *    PCLB_FP32 and double for PCLB_FP64.  Velocities are polar (u_r,
 *    u_theta) at the node's theta.  T is the temperature, equal to the
 *    internal energy E for the paper's gamma = 2.
 *  * Pointers marked "device" must be CUDA device memory (or managed memory)
 *    of the context's device; "host" pointers are ordinary host memory.
 *    Caller pointers are borrowed for the duration of the call (device
 *    pointers until the work queued on the context's stream has run).
 *  * All device work is queued on the context's CUDA stream and is
 *    asynchronous unless stated otherwise.  Calls on one context must not be
 *    made from two host threads at once.
 *  * Every call returns a pclb_status; PCLB_OK is 0.  On failure nothing has
 *    been queued unless stated, and pclb_last_error() describes the cause.
 *    No C++ exception crosses this interface.
 *
 * Precision: PCLB_FP32 stores f in float and computes the step in float.
 * The parts whose rounding would otherwise dominate are carried in
 * float-float (a pair of floats, ~44 significant bits): the velocity moments
 * are accumulated across shells with two-sum / two-product corrections, the
 * temperature recovery T = (e - |j|^2 / (2 rho)) / rho and the weights F_k(T)
 * of Eq. (11) are evaluated in float-float, and so is x = v.u / T with
 * float-float velocity constants.  The adjoint step (PCLB_FP32) takes each
 * node's state from the same float-float moments, rounded to float, and
 * evaluates the cotangents in float (the ghost states at the walls in
 * double).  PCLB_FP64 computes everything in double.
 */
#ifndef PCLB_H
#define PCLB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PCLB_VERSION_MAJOR 0
#define PCLB_VERSION_MINOR 1

typedef enum {
  PCLB_OK = 0,
  PCLB_EINVAL = 1,       /* invalid argument: NULL pointer, size, parameter out of range */
  PCLB_ENOMEM = 2,       /* the workspace given is smaller than pclb_workspace_size() */
  PCLB_ECUDA = 3,        /* a CUDA runtime call or kernel launch failed */
  PCLB_ENONPHYS = 4,     /* a node or ghost node had rho <= 0, T <= 0 or a non-finite value */
  PCLB_ETIMEOUT = 5,     /* a bounded wait for the stream (or a device-side wait) ran out */
  PCLB_ECFL = 6,         /* max over velocities and nodes of |C_r| + |C_theta| exceeds 1 */
  PCLB_ESTATE = 7,       /* call out of order, e.g. pclb_step before any state was set */
  PCLB_EUNSUPPORTED = 8  /* configuration the library does not implement (e.g. n_dirs not 8, 16, 24) */
} pclb_status;

typedef enum { PCLB_FP32 = 0, PCLB_FP64 = 1 } pclb_precision;

typedef enum {
  PCLB_BC_EXTRAP = 0,    /* rho, u, T of both ghost layers by linear extrapolation, Eq. (39) */
  PCLB_BC_WALL = 1,      /* rho, T extrapolated; u_r, u_theta prescribed at the ghost nodes */
  PCLB_BC_DIRICHLET = 2  /* rho, u_r, u_theta, T prescribed at the ghost nodes */
} pclb_bc_kind;
/* Convection schemes (Sec. II B 3; the paper compares them in its Fig. 5).
 * Each advances psi_t + a psi_xi = 0 by psi_j -= M_j with C = a dt / dxi. */
typedef enum {
  PCLB_SCHEME_MWB = 0,     /* Modified Warming-Beam with the switch S(eta), Eq. (28): the default */
  PCLB_SCHEME_WB = 1,      /* Warming-Beam, Eq. (25) */
  PCLB_SCHEME_LW = 2,      /* Lax-Wendroff: centred differences in the Taylor expansion of Eq. (22) */
  PCLB_SCHEME_UPWIND2 = 3  /* forward-Euler step with the second-order upwind derivative of Eq. (23) */
} pclb_scheme;

/* Relaxation (Sec. II B 2). */
typedef enum {
  PCLB_RELAX_EXACT = 0,  /* f^eq + (f - f^eq) exp(-dt/tau), Eq. (19): the default */
  PCLB_RELAX_EULER = 1   /* f - dt/tau (f - f^eq), Eq. (18); requires dt <= 2 tau */
} pclb_relaxation;

/* Flag added to a kind: the ghost nodes carry, besides f^eq of their
 * macroscopic state, the departure f - f^eq of the wall node (the
 * non-equilibrium microscopic boundary of Sec. II C 1, in the form of the
 * extrapolation scheme it cites: the non-equilibrium part of the nearest
 * fluid node).  The adjoint entry points differentiate it too (the ghosts'
 * cotangent reaches the wall node's f directly and through its own
 * equilibrium). */
#define PCLB_BC_NEQ 8

/* Device status bits accumulated by the kernels (pclb_status_flags). */
#define PCLB_FLAG_NONPHYS 1u   /* rho <= 0 or T <= 0 at a node or ghost node */
#define PCLB_FLAG_NONFINITE 2u /* a non-finite moment or distribution value */
#define PCLB_FLAG_TIMEOUT 4u   /* a kernel gave up waiting for its own asynchronous copies */

/* Annulus and its grid (Sec. II C). */
typedef struct {
  int32_t n_r;      /* radial nodes, >= 3 */
  int32_t n_theta;  /* azimuthal nodes, >= 2 */
  double r_in;      /* R1 > 0 */
  double r_out;     /* R2 > R1 */
  int32_t n_f;      /* 1 <= n_f <= n_dirs; n_f == n_dirs is the full circle */
} pclb_grid;

/* Discrete velocity model (Sec. II A): N_k = 4 shells of n_dirs directions
 * plus the rest velocity, Q = 1 + 4 n_dirs labels.  n_dirs = 8 (the octagon)
 * runs the tuned kernels and every entry point.  n_dirs = 16 and 24 (Table I,
 * rows 2-3; B from that table) run the forward path only (in FP32 a tiled
 * step kernel that streams the opposite-velocity plane pairs, in FP64 and for
 * the field operations generic kernels): pclb_set_state, pclb_set_f,
 * pclb_get_f, pclb_step (every scheme and relaxation), pclb_moments,
 * pclb_diagnostics, pclb_noneq, pclb_run_host and the state save / load
 * calls; the reverse-mode entry points and pclb_diagnostics_noalloc return
 * PCLB_EUNSUPPORTED for them. */
typedef struct {
  int32_t n_dirs;    /* N_i: 8, 16 or 24 */
  double speeds[5];  /* v_0 .. v_4; the paper uses 0, 1, 2.92, 2.99, 4.49 */
  double B[5];       /* B[n] = B_n of Table I (octagon: 8, -1/4, 1, -6, 48) */
} pclb_dvm;

/* Radial boundary conditions (Sec. II C 1).  values[s] (host, copied by
 * pclb_create) holds double [2][4][n_theta]: ghost layer (0 = next to the
 * wall, 1 = outer), field (rho, u_r, u_theta, T), theta node.  It may be
 * NULL for PCLB_BC_EXTRAP.  Side 0 is the inner wall, side 1 the outer. */
typedef struct {
  int32_t kind[2];
  const double* values[2];
} pclb_bc;

typedef struct pclb_ctx pclb_ctx;

/* Library version as major * 100 + minor. */
int32_t pclb_version(void);

/* Text of the last error on ctx, or of the last failed pclb_create /
 * pclb_workspace_size on this host thread when ctx is NULL.  Never NULL;
 * valid until the next call on the same context or thread. */
const char* pclb_last_error(const pclb_ctx* ctx);

/* Bytes of device workspace pclb_create needs for this problem: two
 * ping-pong copies of f with two azimuthal ghost rows on each side and rows
 * padded to 32 elements, small tables, the status word and reduction
 * scratch, three more state-sized buffers for the adjoint (a state copy and
 * two adjoint variables) and host-I/O staging.  Host-only; queues nothing. */
pclb_status pclb_workspace_size(const pclb_grid* grid, const pclb_dvm* dvm, pclb_precision prec,
                                size_t* bytes);

/* Create a context.  tau > 0 is the relaxation time and dt > 0 the time step
 * of Eq. (38).  workspace (device, 256-byte aligned, at least
 * pclb_workspace_size() bytes) is owned by the caller and must outlive the
 * context; the library allocates no device memory of its own.  stream is a
 * cudaStream_t (NULL = the legacy default stream).  Validates every argument
 * and the Courant numbers before queuing anything; then uploads the tables
 * on the stream.  The state is undefined until pclb_set_state or
 * pclb_set_f. */
pclb_status pclb_create(const pclb_grid* grid, const pclb_dvm* dvm, double tau, double dt,
                        pclb_precision prec, const pclb_bc* bc, void* workspace,
                        size_t workspace_bytes, void* stream, pclb_ctx** out);

/* Release the host-side context (the workspace stays the caller's).
 * Synchronizes the context's stream first (bounded wait). */
pclb_status pclb_destroy(pclb_ctx* ctx);

/* Queue later work of ctx on another stream (cudaStream_t). */
pclb_status pclb_set_stream(pclb_ctx* ctx, void* stream);

/* f = f^eq(rho, u, T) at every node (the initial equilibrium of Sec. III).
 * rho, u_r, u_theta, T: device, [n_theta][n_r], context precision.
 * Non-physical inputs set PCLB_FLAG_NONPHYS in the status word. */
pclb_status pclb_set_state(pclb_ctx* ctx, const void* rho, const void* u_r, const void* u_theta,
                           const void* T);

/* Copy a distribution in / out: device, [Q][n_theta][n_r], context
 * precision.  Bitwise; used for checkpoints. */
pclb_status pclb_set_f(pclb_ctx* ctx, const void* f);
pclb_status pclb_get_f(pclb_ctx* ctx, void* f);

/* Advance n >= 0 time steps of Eq. (38).  One fused kernel launch per step
 * (ghost nodes are computed inside it).  Asynchronous; errors found on the
 * device are reported by pclb_status_flags. */
pclb_status pclb_step(pclb_ctx* ctx, int32_t n);

/* The same n steps as pclb_step, launched as one CUDA graph: the first call
 * for a given (n, current state buffer) captures the n launches on a private
 * stream and instantiates the graph (cached per context, up to four, dropped
 * by pclb_set_scheme and pclb_destroy); later calls replay it on the
 * context's stream.  Results are bitwise those of pclb_step.  For grids
 * small enough that launch overhead matters (no paper section: an execution
 * detail). */
pclb_status pclb_step_graph(pclb_ctx* ctx, int32_t n);

/* Macroscopic fields of the current state (Eqs. 3-5): device,
 * [n_theta][n_r], context precision; any pointer may be NULL. */
pclb_status pclb_moments(pclb_ctx* ctx, void* rho, void* u_r, void* u_theta, void* T);

/* Select the convection scheme and the relaxation of subsequent steps (the
 * variants the paper compares; a new context uses PCLB_SCHEME_MWB and
 * PCLB_RELAX_EXACT).  Errors: PCLB_EINVAL (unknown value), PCLB_ECFL
 * (PCLB_RELAX_EULER with dt > 2 tau, where it is unstable).  The adjoint
 * entry points support PCLB_SCHEME_MWB only (PCLB_EUNSUPPORTED otherwise);
 * both relaxations are supported. */
pclb_status pclb_set_scheme(pclb_ctx* ctx, int32_t scheme, int32_t relaxation);

/* How long a step or adjoint kernel (pclb_step, pclb_step_graph,
 * pclb_step_states, pclb_run_host, pclb_adjoint_state, pclb_adjoint_step)
 * waits for the TMA copies of its own stencil window before it gives the
 * tile up and sets PCLB_FLAG_TIMEOUT; the default is
 * 2000000000 ns (2 s), the maximum 60 s.  A tile given up stores no more;
 * its copies still get the default limit to land before its block exits, so
 * the context stays usable, but the state (or cotangent) after such a step is undefined
 * (reload it) and pclb_status_flags returns PCLB_ETIMEOUT.  A limit of 0
 * gives every tile up without waiting, which exercises that path.  No paper
 * counterpart: an execution detail.  Drops cached step graphs.  Errors:
 * PCLB_EINVAL (limit above the maximum). */
pclb_status pclb_set_wait_limit(pclb_ctx* ctx, uint64_t limit_ns);

/* Non-equilibrium manifestations of the current state (Sec. IV).  At every
 * node, with c = v (plain) or c = v - u (central, u the node's velocity) in
 * polar components at the node, and w = f (moments) or w = f - f^eq
 * (departures, f^eq the equilibrium of Eq. 10 at the node's own moments):
 *   M_2 = sum w c c, M_3 = sum w c c c, M_{3,1} = sum w (c.c/2) c,
 *   M_{4,2} = sum w (c.c/2) c c.
 * groups: bitwise OR of PCLB_NEQ_* (1..15).  out: device, context precision,
 * [n_groups x 12][n_theta][n_r], the selected groups in bit order, each as
 * 12 fields: M_2 rr, r theta, theta theta; M_3 rrr, rr theta, r theta theta,
 * theta theta theta; M_{3,1} r, theta; M_{4,2} rr, r theta, theta theta.
 * Errors: PCLB_EINVAL (groups out of range, out NULL), PCLB_ESTATE (no
 * state). */
#define PCLB_NEQ_M 1      /* M_m(f) */
#define PCLB_NEQ_DELTA 2  /* Delta_m = M_m(f - f^eq) */
#define PCLB_NEQ_MSTAR 4  /* M*_m(f), central */
#define PCLB_NEQ_DSTAR 8  /* Delta*_m = M*_m(f - f^eq) */
pclb_status pclb_noneq(pclb_ctx* ctx, int32_t groups, void* out);

/* Global integrals of the current state with the area element r dr dtheta,
 * summed in double: out[0] mass, out[1] x-momentum, out[2] y-momentum,
 * out[3] total energy (rho (E + u^2/2)), out[4] min rho, out[5] min T,
 * out[6] number of nodes, out[7] reserved (0).  out: host, 8 doubles.
 * Synchronizes the stream (bounded wait). */
pclb_status pclb_diagnostics(pclb_ctx* ctx, double* out);

/* Read (and if clear != 0, reset) the device status word that the kernels
 * set (PCLB_FLAG_*).  flags: host.  Synchronizes the stream (bounded wait).
 * Returns PCLB_ENONPHYS when any flag other than the timeout flag is set,
 * PCLB_ETIMEOUT when the timeout flag is set, else PCLB_OK. */
pclb_status pclb_status_flags(pclb_ctx* ctx, uint32_t* flags, int32_t clear);

/* Wait for all work queued on the context's stream, polling for at most
 * timeout_ms milliseconds (PCLB_ETIMEOUT when it runs out). */
pclb_status pclb_sync(pclb_ctx* ctx, int32_t timeout_ms);

/* End-to-end call with host buffers: bring rho, u_r, u_theta, T (host,
 * [n_theta][n_r], context precision) to the device, set f = f^eq, advance n
 * steps, compute the moments and bring them back to the host arrays
 * out_rho .. out_T (any may be NULL).  The fields pass through the workspace
 * tail (pclb_workspace_size reserves it).  When every buffer is page-locked
 * (cudaHostAlloc / cudaHostRegister, e.g. torch's pin_memory) and n_dirs = 8,
 * the grid is processed in azimuthal slabs of whole tile rows: each slab's
 * copies run on the copy engines (streams of the context's own) while the
 * set-state, step and moment kernels of other slabs run, the first and the
 * last step slab by slab and the steps in between on the whole grid; the
 * results are bit for bit those of the plain sequence.  Otherwise the copies
 * and kernels run one after another on the context's stream.  Either way an
 * output array may be an input array (input rows are read before the same
 * output rows are written).  The call returns after the results are on the
 * host (bounded wait). */
pclb_status pclb_run_host(pclb_ctx* ctx, const void* rho, const void* u_r, const void* u_theta,
                          const void* T, int32_t n, void* out_rho, void* out_u_r,
                          void* out_u_theta, void* out_T);

/* ---------------------------------------------------------------------------
 * Reverse mode.  The adjoint of one step (the vector-Jacobian product of the
 * map f^n -> f^{n+1} of Eq. 38, including the radial ghost nodes of Eq. 39
 * and the azimuthal periodicity of Eq. 40) is derived from the same
 * equations; |x| in the switch function of Eq. (37) is differentiated on its
 * active branch (d|x|/dx = sign x, sign 0 = 0).  The context holds one
 * adjoint variable lam (the cotangent of the current distribution) in its
 * workspace, in the same stored layout as f.
 * ------------------------------------------------------------------------- */

/* Bytes of one stored state (distribution in the library's internal layout:
 * azimuthal ghost rows and padded rows).  Host-only. */
pclb_status pclb_state_bytes(pclb_ctx* ctx, size_t* bytes);

/* Copy the current state to / from a caller buffer of pclb_state_bytes bytes
 * (device, 16-byte aligned).  Bitwise; used for checkpoints and for the
 * states the adjoint needs. */
pclb_status pclb_save_state(pclb_ctx* ctx, void* state);
pclb_status pclb_load_state(pclb_ctx* ctx, const void* state);

/* One step of Eq. (38) from the state in f_from to f_to, both buffers of
 * pclb_state_bytes bytes in the layout pclb_save_state writes (device,
 * 16-byte aligned, distinct); the context's own state is left alone.  Lets a
 * backward pass recompute a segment's states straight into the buffers the
 * adjoint steps read.  Asynchronous, one kernel launch (two for n_dirs 16,
 * 24). */
pclb_status pclb_step_states(pclb_ctx* ctx, const void* f_from, void* f_to);

/* Set / read the adjoint variable: device, [Q][n_theta][n_r], context
 * precision. */
pclb_status pclb_lambda_set(pclb_ctx* ctx, const void* lam);
pclb_status pclb_lambda_get(pclb_ctx* ctx, void* lam);

/* One adjoint step: lam <- J(f)^T lam, where f is the state the forward step
 * started from: f_state (device, a buffer filled by pclb_save_state) or, if
 * NULL, the context's current state.  Asynchronous, three kernel launches:
 * the wall feedback and the tiles next to the walls on a side stream of the
 * context, forked from and joined back to the context's stream with events,
 * and the interior tiles on the context's stream; to the caller it is one
 * stream-ordered operation. */
pclb_status pclb_adjoint_state(pclb_ctx* ctx, const void* f_state);

/* Convenience form in the packed layout: lam_n = J(f_n)^T lam_np1, all three
 * device, [Q][n_theta][n_r].  Replaces the context's adjoint variable with
 * lam_n; leaves the forward state alone. */
pclb_status pclb_adjoint_step(pclb_ctx* ctx, const void* f_n, const void* lam_np1, void* lam_n);

/* lam <- (d fields / d f)^T g at the current state, where fields = (rho,
 * u_r, u_theta, T) as pclb_moments returns them (Eqs. 3-5).  g_*: device,
 * [n_theta][n_r], context precision; NULL means a zero cotangent. */
pclb_status pclb_moments_vjp(pclb_ctx* ctx, const void* g_rho, const void* g_ur, const void* g_ut,
                             const void* g_T);

/* Gradients of <lam, f^eq(rho, u_r, u_theta, T)> with respect to the fields
 * (the adjoint of pclb_set_state, Eq. 10): fields as for pclb_set_state,
 * outputs g_* device [n_theta][n_r] (any may be NULL). */
pclb_status pclb_set_state_vjp(pclb_ctx* ctx, const void* rho, const void* u_r, const void* u_theta,
                               const void* T, void* g_rho, void* g_ur, void* g_ut, void* g_T);

/* Global integrals of a distribution, as pclb_diagnostics computes them, but
 * without a context and without allocating any device memory.  The paper has
 * no counterpart: this entry point exists for callers that cannot call
 * cudaMalloc -- code running inside an allocator's own callbacks (which
 * would re-enter the allocator), plug-ins that own no memory pool, hosts that
 * have handed all device memory to another framework.  They pass only the
 * input and the output; the reduction's scratch is a fixed file-scope device
 * array.
 *
 * grid, dvm, prec: as for pclb_create (host, read during the call).
 * f: device, [Q][n_theta][n_r] in prec's element type, not modified.
 * out: host, 8 doubles laid out as in pclb_diagnostics.
 * stream: cudaStream_t the kernels are queued on; the call waits for it
 * (bounded wait, PCLB_ETIMEOUT) before copying the 8 results to out.
 * On a stream that is being captured it returns PCLB_EUNSUPPORTED and
 * queues nothing.
 *
 * Limit: n_theta <= 16384 (one 8-double partial per azimuthal row); larger
 * grids are rejected with PCLB_EINVAL and a message.  The scratch array,
 * (16384 + 1) x 8 doubles = 1 MiB, is held by every device that loads the
 * library until the process exits.  The first call on a device looks up the
 * array's device address with that device current.  Every call overwrites
 * every slot it reads, so nothing needs clearing, and the array keeps the
 * last call's contents.  All calls share the one array: calls that overlap
 * on the GPU (other streams, other host threads) race on it and must be
 * serialized by the caller.  After PCLB_ETIMEOUT the call's kernels may
 * still be queued and will write the array later: synchronize the stream
 * before the next call.  Allocates nothing: no cudaMalloc, cudaFree or
 * allocating library routine. */
pclb_status pclb_diagnostics_noalloc(const pclb_grid* grid, const pclb_dvm* dvm, pclb_precision prec,
                                     const void* f, double* out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PCLB_H */
