/*
 * lbm.h -- C ABI of libhemelb_gb300.so: the sparse lattice-Boltzmann
 * (LBGK) collide-and-stream hot path of HemeLB (arXiv 1906.11925) on one
 * GB300 GPU (sm_103a).
 *
 * The paper's statement of the problem (Section 2): the vessel is a lattice
 * of sparse fluid sites; each site holds a single-particle distribution over
 * a finite set of lattice vectors (D3Q19, Fig. 1); a time step is a collision
 * followed by propagation to the neighbouring site along each vector.
 * Section 2 and Section 3.2 name the boundary families (walls and
 * inlets/outlets, "iolets"); Section 4 states simple bounce-back walls.
 * This library implements:
 *   - LBGK collision, f*_i = f_i - (f_i - feq_i)/tau, with the compressible
 *     second-order equilibrium feq_i = w_i rho (1 + 3 c.u + 9/2 (c.u)^2
 *     - 3/2 u.u), on D3Q15 or D3Q19;
 *   - halfway bounce-back at wall links;
 *   - density (pressure) iolets: the population entering from iolet k is
 *     feq(rho_k(t), u(x, t)), rho_k(t) = mean_k + amp_k sin(2 pi t/period_k
 *     + phase_k) evaluated at the start of step t (period 0 = constant);
 *   - wall shear stress from the non-equilibrium stress.
 *
 * Direction order (both lattices): 0 is the rest vector; after it opposite
 * vectors are adjacent, opp(i) = i + 1 for odd i and i - 1 for even i > 0.
 *   D3Q15: 1..6 = +x -x +y -y +z -z; 7..14 = (1,1,1) (-1,-1,-1) (1,1,-1)
 *          (-1,-1,1) (1,-1,1) (-1,1,-1) (-1,1,1) (1,-1,-1).
 *   D3Q19: 1..6 as D3Q15; 7..18 = (1,1,0) (-1,-1,0) (1,-1,0) (-1,1,0)
 *          (1,0,1) (-1,0,-1) (1,0,-1) (-1,0,1) (0,1,1) (0,-1,-1) (0,1,-1)
 *          (0,-1,1).
 *
 * Conventions for every call:
 *   - "caller order" is the order of the site list given to lbm_create; the
 *     library reorders sites internally along a Morton (Z-order) curve and
 *     converts back on every output.
 *   - Canonical link tables are direction-major: nbr[i * n + x] is the
 *     caller index of the site x + c_i, or -1 when that voxel is not fluid;
 *     link[i * n + x] is 0 (fluid), 1 (wall) or 2 + k (iolet k).  For i = 0,
 *     nbr = x and link = 0.
 *   - Pointers named *_d are device pointers owned by the caller; the call
 *     enqueues work on the context's stream and returns without waiting.
 *     Every other pointer is host memory; calls that write host memory
 *     synchronise the context's stream before returning.
 *   - No call throws, aborts or traps.  Arguments are validated before any
 *     allocation.  On error the context stays usable unless the status is
 *     LBM_ERR_CUDA.  lbm_last_error() gives a message.
 *   - A context is not thread-safe; distinct contexts are independent.
 */
#ifndef HEMELB_GB300_LBM_H
#define HEMELB_GB300_LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LBM_OK = 0,
    LBM_ERR_ARG = 1,      /* bad argument (NULL, range, unsupported q/storage) */
    LBM_ERR_TABLE = 2,    /* link table inconsistent (range, symmetry, flags)   */
    LBM_ERR_NOMEM = 3,    /* not enough free device memory (checked up front)   */
    LBM_ERR_CUDA = 4,     /* a CUDA call failed; the context must be destroyed  */
    LBM_ERR_UNSTABLE = 5, /* non-finite state detected                          */
    LBM_ERR_STATE = 6     /* call not valid in the context's current state      */
} lbm_status;

enum { LBM_STORE_FP32 = 0, LBM_STORE_FP16 = 1, LBM_STORE_I16 = 2 };
enum { LBM_STREAM_PULL = 0, LBM_STREAM_AA = 1 };
enum { LBM_IOLET_DENSITY = 0, LBM_IOLET_VELOCITY = 1 };
enum { LBM_MAX_IOLETS = 64 };
enum { LBM_ORDER_MORTON_RUNS = 0, LBM_ORDER_MORTON = 1, LBM_ORDER_ROWS = 2, LBM_ORDER_SLABS = 3 };

typedef struct lbm_ctx lbm_ctx; /* opaque */

/* Parameters of a simulation (copied by lbm_create).
 *   q          15 or 19.
 *   storage    LBM_STORE_FP32: populations stored as float deviations
 *              d_i = f_i - w_i rho0; LBM_STORE_FP16: stored as IEEE half
 *              h_i = RN((f_i - w_i rho0) * 2^fp16_scale_log2); LBM_STORE_I16:
 *              stored as int16 fixed point k_i = RN((f_i - w_i rho0) *
 *              2^fp16_scale_log2) with |k_i| <= 32766 (the same two bytes as
 *              fp16 with a uniform step 2^-S instead of 11 significant bits:
 *              finer for the large deviations that dominate a flowing site,
 *              but the caller must choose S so that every deviation stays
 *              below 32766 * 2^-S; a value beyond that saturates, and the
 *              saturated slot reads as NaN everywhere outside the step
 *              kernels, so lbm_mass reports LBM_ERR_UNSTABLE).  Arithmetic is
 *              float32 in every form.
 *   tau        relaxation time, tau > 0.5 (kinematic viscosity (tau - 1/2)/3).
 *   rho0       reference density of the deviation storage and of the initial
 *              rest state, > 0.
 *   fp16_scale_log2  S in [0, 24] for LBM_STORE_FP16, in [0, 30] for
 *              LBM_STORE_I16; ignored for LBM_STORE_FP32.
 *   n_iolets   K in [0, LBM_MAX_IOLETS]; the four arrays hold K doubles each
 *              (host memory, may be NULL when K = 0).
 *   iolet_kind K int32 or NULL (all density iolets): LBM_IOLET_DENSITY, or
 *              LBM_IOLET_VELOCITY: a link into the iolet bounces back from a
 *              boundary moving with u_b = velocity_weight[x] U_k(t) n_k (Ladd's
 *              moving-wall rule, f_opp(i) = f*_i - 6 w_i rho c_i.u_b); the paper
 *              drives its inlet this way (Sections 2 and 3.2, Table I).  For a
 *              velocity iolet the schedule (rho_mean, amp, period, phase) gives
 *              the speed U_k(t), and the driven densities of lbm_step_driven
 *              are speeds too.
 *   iolet_normal  K x 3 doubles (unit inward normals of the velocity iolets);
 *              may be NULL when there is none.
 *   velocity_weight  n doubles, caller order, or NULL (all 1): the per-site
 *              profile of the velocity iolets (the paper's velocity weights
 *              file, Section 3.2).
 *   streaming  LBM_STREAM_PULL: two population buffers, every step gathers
 *              through the neighbour table.  LBM_STREAM_AA: one buffer updated
 *              in place by the AA pattern (even steps touch only a site's own
 *              slots, odd steps gather and scatter through the table): half
 *              the population memory and half the table traffic; identical
 *              results (the same collision arithmetic).
 *   wall_q     q x n doubles, caller order, or NULL (every wall half-way):
 *              for a wall link (link[i][x] == 1) the fraction of the link
 *              from x along c_i that lies in the fluid, in (0, 1], rounded to
 *              a multiple of 2^-24; ignored elsewhere.  A wall link with
 *              q != 1/2 uses the Bouzidi-Firdaouss-Lallemand interpolation
 *              (the paper's BFL wall boundary, Section 3.2), with x_b = x - c_i:
 *              q < 1/2 and x_b fluid: f_opp(i)(x, t+1) = 2q f*_i(x) + (1 - 2q) f*_i(x_b);
 *              q >= 1/2: f_opp(i)(x, t+1) = f*_i(x) / (2q) + (1 - 1/(2q)) f*_opp(i)(x);
 *              q < 1/2 without a fluid x_b: the half-way rule.  Both
 *              streaming forms (bitwise the same results); differentiated
 *              by lbm_objective_grad like the half-way walls.
 *   site_order the order the device keeps the sites in (every result is the
 *              same, outputs are in caller order; the sites with iolet or
 *              interpolated-wall links come last in all of them):
 *              LBM_ORDER_MORTON_RUNS (0, default): runs of 32 sites along x
 *              (from x multiples of 32) kept contiguous, the runs ordered
 *              along the Morton curve of (x / 32, y, z): a warp's 32 sites
 *              then have neighbours in a few contiguous runs, which makes the
 *              scattered stores of the AA odd step nearly coalesced (the
 *              sites after the bulk, a shell on the walls and iolets, stay in
 *              plain Morton order);
 *              LBM_ORDER_MORTON (1): the Morton (Z-order) curve of (x, y, z);
 *              LBM_ORDER_ROWS (2): (z, y, x) row order;
 *              LBM_ORDER_SLABS (3): row order, and with LBM_STREAM_AA the
 *              bulk sites are cut into chunks of whole z planes (about 1 MB
 *              of populations each) and lbm_step runs each even step and the
 *              odd step after it as one persistent launch over them: the odd
 *              step of a chunk runs once the even steps of the chunk and its
 *              two neighbours are done, 14 chunks behind the even steps, and
 *              reads the even step's output back from L2 instead of HBM (the
 *              same results to the bit; about 40% fewer HBM bytes per step,
 *              but not faster than the unfused form in float32 and slower
 *              with 16-bit storage, whose unfused even step runs at higher
 *              occupancy).  Where a site's neighbour lies more than one
 *              chunk away (a periodic z axis) the pairs run unfused. */
typedef struct {
    int32_t q;
    int32_t storage;
    double tau;
    double rho0;
    int32_t fp16_scale_log2;
    int32_t n_iolets;
    const double *rho_mean;
    const double *amp;
    const double *period;
    const double *phase;
    int32_t streaming;
    const int32_t *iolet_kind;
    const double *iolet_normal;
    const double *velocity_weight;
    const double *wall_q;
    int32_t site_order;
} lbm_params;

/* Neighbour-link table of a sparse site list (Section 2: every fluid site
 * propagates to its neighbour along each lattice vector), built on the host.
 *   xyz       int32 [n][3] fluid voxel coordinates, all distinct, each in
 *             [-2^19, 2^19).
 *   io_xyz    int32 [n_io][3] non-fluid voxels that belong to iolet io_id[m]
 *             (0 <= io_id < LBM_MAX_IOLETS); a link into such a voxel is an
 *             iolet link, a link into any other non-fluid voxel is a wall.
 *   periodic  int32 [3] or NULL: axis a wraps modulo periodic[a] when > 0.
 *   nbr, link outputs, [q][n] each, caller-allocated (canonical tables).
 * Errors: LBM_ERR_ARG for a bad q, NULL pointer with n > 0, duplicate
 * coordinates, a coordinate or iolet id out of range.  No GPU is used. */
lbm_status lbm_links_build(int32_t q, int64_t n, const int32_t *xyz, int64_t n_io,
                           const int32_t *io_xyz, const int32_t *io_id,
                           const int32_t *periodic, int32_t *nbr, uint8_t *link);

/* Create a simulation on the current CUDA device from the canonical tables.
 * Validates params and tables (range, symmetry nbr[opp i][nbr[i][x]] == x,
 * fluid iff nbr >= 0, iolet ids < n_iolets), computes the Morton order of
 * xyz (int32 [n][3]), uploads the internal tables and initialises the fluid
 * at rest, f_i = w_i rho0, time t = 0.  All inputs are copied; the caller
 * keeps ownership.  cuda_stream is a cudaStream_t (NULL = legacy default
 * stream) on which every later call enqueues its work.  n = 0 is allowed
 * (every step is then a no-op).  On success *out receives the context. */
lbm_status lbm_create(lbm_ctx **out, const lbm_params *params, int64_t n,
                      const int32_t *xyz, const int32_t *nbr, const uint8_t *link,
                      void *cuda_stream);

/* Destroy a context and free its device memory (NULL is a no-op). */
void lbm_destroy(lbm_ctx *ctx);

/* Message of the last failed call on ctx, or of the last failed call
 * without a context on this thread when ctx is NULL.  Never NULL. */
const char *lbm_last_error(const lbm_ctx *ctx);

/* Change the stream used by later calls.  Work that later calls queue on
 * the new stream starts after the work already queued on the old one (an
 * event recorded on the old stream, waited for by the new one). */
lbm_status lbm_set_stream(lbm_ctx *ctx, void *cuda_stream);

/* Advance nsteps >= 0 time steps (Section 2: collision then propagation),
 * asynchronous on the context's stream.  Step t uses the iolet densities
 * rho_k(t).  Each step is one fused collide-and-stream launch over the bulk
 * sites and one over the sites with iolet links; whole chunks of 32 steps
 * run as one replay of a CUDA graph of those launches (captured on first
 * use, bitwise the same results), except while the caller is capturing the
 * context's stream itself.  The host may wait here for the copy of an
 * earlier chunk's iolet values when it runs more than 8 chunks ahead. */
lbm_status lbm_step(lbm_ctx *ctx, int64_t nsteps);

/* Advance nsteps steps with iolet densities supplied by the caller instead
 * of the sinusoidal schedule (the paper drives its inlet from a file,
 * Table I): rho_io_host is host memory, double [nsteps][n_iolets], row s
 * used by step s.  If mass_host is not NULL it receives the total mass
 * (see lbm_mass) after every step, double [nsteps].  Synchronous. */
lbm_status lbm_step_driven(lbm_ctx *ctx, int64_t nsteps, const double *rho_io_host,
                           double *mass_host);

/* Current time step counter t (number of steps taken since t = 0 or the
 * last lbm_set_time). */
lbm_status lbm_get_time(const lbm_ctx *ctx, int64_t *t);
lbm_status lbm_set_time(lbm_ctx *ctx, int64_t t);

/* Density, velocity and wall shear stress of the current state f(t), float32,
 * in caller order: rho_d [n], u_d [n][3], wss_d [n] (device pointers; any may
 * be NULL to skip it).  Wall shear stress: sigma = -(1 - 1/(2 tau))
 * sum_i (f_i - feq_i) c_i c_i, traction s = sigma n with the unit wall normal
 * n = -normalize(sum of c_i over the site's wall links), wss = |s - (n.s) n|;
 * 0 at sites without wall links or whose wall vectors sum to zero.
 * Asynchronous. */
lbm_status lbm_macros(lbm_ctx *ctx, float *rho_d, float *u_d, float *wss_d);

/* Total mass sum_x sum_i f_i(x, t), accumulated in float64 in a fixed order
 * (deterministic for a given context).  Synchronous.  Returns
 * LBM_ERR_UNSTABLE (and stores the value) when the sum is not finite.  Also
 * reads the error flag of the step kernels: when a step kernel gave up
 * waiting for its table copies (or, in the checked build, met a table entry
 * out of range) it returns LBM_ERR_CUDA, the stored state is undefined, and
 * lbm_step, lbm_step_driven and lbm_objective_grad return LBM_ERR_STATE
 * until lbm_set_state or lbm_set_populations replaces the state. */
lbm_status lbm_mass(lbm_ctx *ctx, double *out);

/* Weighted sum over the sites of the current state f(t), accumulated in
 * float64 in a fixed order (deterministic): sum_x weight[x] q(x), with q the
 * wall shear stress of lbm_macros (kind LBM_OBJ_WSS) or the density
 * (LBM_OBJ_DENSITY).  weight_d: device float64 [n], caller order, or NULL
 * for all ones (e.g. the mean WSS over a site subset is a 0/1 weight divided
 * by its count).  Synchronous. */
lbm_status lbm_weighted_sum(lbm_ctx *ctx, int32_t kind, const double *weight_d, double *out);

/* Failure detection, checked on its own: the table-staged steps wait for
 * their bulk copies on mbarriers with a bounded number of polls (about 4M),
 * and the blocks of a fused AA step pair (LBM_ORDER_SLABS) wait for the even
 * steps of neighbouring chunks on counters, again with a bounded number of
 * polls (about 2M, a second or so); a step kernel that gives up sets an
 * error flag and returns, and lbm_mass reports LBM_ERR_CUDA.  A copy it gave
 * up on may still land afterwards, and a fused pair that gave up has updated
 * only part of the sites, so the output of that launch is undefined (see
 * lbm_mass).  This call runs both bounded waits, with `limit` polls each
 * (1 .. 2^24), on a barrier that no copy completes and on a counter that
 * nothing raises, and stores 1 in *gave_up when both waits gave up (they
 * always should).  The context and the device stay usable.  Synchronous on
 * cuda_stream.  The paper has no counterpart. */
lbm_status lbm_check_wait_timeout(uint32_t limit, void *cuda_stream, int32_t *gave_up);

/* Failure detection: an instability check on the stored state.  With
 * every > 0, lbm_step checks the state after every `every` of its steps and
 * after its last one: a stored value that is not finite, or a site whose own
 * stored slots give a density <= 0 or a speed |j| / rho above u_max (lattice
 * units; the collision keeps rho and j, so these are the moments of the
 * site's last post-collision state, approximately so at iolet and
 * interpolated-wall sites), is reported as LBM_ERR_UNSTABLE with the step
 * range of the first failing check; lbm_step then waits for its stream
 * before returning.  every = 0 (the default) turns the check off and leaves
 * lbm_step asynchronous.  every < 0 or u_max not finite and > 0: LBM_ERR_ARG.
 * The paper has no counterpart (its GUI can only interrupt a run). */
lbm_status lbm_set_stability_check(lbm_ctx *ctx, int64_t every, double u_max);

/* Guard words (an out-of-range write check in place of a memory sanitizer):
 * the padding slots [n, npad) of every plane of the context's population
 * buffers and one extra row of 128 slots after the last plane hold a fixed
 * NaN bit pattern that no kernel writes.  Stores 1 in *intact when every
 * guard word still holds it, else 0.  The raw state blob of lbm_get_state
 * includes the plane padding, so lbm_set_state of a blob whose padding was
 * changed shows here.  Synchronous. */
lbm_status lbm_check_guards(lbm_ctx *ctx, int32_t *intact);

/* Populations f(t) as float64 [q][n], caller order (host memory).  Sync. */
lbm_status lbm_get_populations(lbm_ctx *ctx, double *f_host);

/* Same result as lbm_get_populations, for callers that cannot let the
 * library call cudaMalloc or cudaFree (device memory owned by their own pool
 * allocator, or a fixed memory budget; cudaFree would also synchronise the
 * whole device).  The paper has no counterpart: this is a memory-management
 * variant of the call above.  The float64 staging buffer is a static device
 * array of 2^20 values (8 MiB, held by every GPU that loads the library until
 * the process exits); q * n above 2^20 is rejected with LBM_ERR_ARG.  No
 * cudaMalloc, cudaFree or other allocating routine is called.  The first call
 * on a device looks up the array's device address (cudaGetSymbolAddress,
 * with the context's device made current for the lookup) and keeps it for
 * the life of the process, so the device must not be reset
 * (cudaDeviceReset) while the library is loaded.  The call copies to host
 * memory and waits for the context's stream, so it must never be made while
 * that stream is being captured into a CUDA graph: it then returns
 * LBM_ERR_STATE without doing anything.  All calls share the one array: calls whose
 * work overlaps on the GPU (several contexts on different streams, or several
 * threads) race on it and must be serialised by the caller.  Every call
 * overwrites the first q * n values before reading them, so nothing needs
 * clearing between calls.  Synchronous. */
lbm_status lbm_get_populations_noalloc(lbm_ctx *ctx, double *f_host);

/* Replace the state by f (float64 [q][n], caller order, host memory),
 * rounded to the storage format.  Does not change t.  A value that is not
 * finite, or whose deviation f_i - w_i rho0 does not fit the storage format
 * (|deviation| * 2^S > 65504 for fp16), gives LBM_ERR_UNSTABLE and leaves
 * the state unchanged.  Synchronous. */
lbm_status lbm_set_populations(lbm_ctx *ctx, const double *f_host);

/* Raw stored state (checkpoint/resume): lbm_state_bytes gives the size of
 * the blob, the stored population buffer plus an 8-byte trailer holding the
 * AA layout phase; get/set copy it to/from host memory byte-for-byte, so
 * that a resumed run is bit-identical.  A blob is only valid for a context
 * with the same q, n, storage and streaming.  Synchronous. */
lbm_status lbm_state_bytes(const lbm_ctx *ctx, size_t *bytes);
lbm_status lbm_get_state(lbm_ctx *ctx, void *host, size_t bytes);
lbm_status lbm_set_state(lbm_ctx *ctx, const void *host, size_t bytes);

/* The link table the kernels use, converted back to canonical caller-order
 * form (nbr, link: [q][n] host memory), for verification.  Synchronous. */
lbm_status lbm_get_links(lbm_ctx *ctx, int32_t *nbr, uint8_t *link);

/* ------------------------------------------------------------------ adjoint
 * Gradients of a time-windowed objective by the discrete adjoint of the step
 * (reverse mode), with binomial checkpointing of raw state snapshots.  Not in
 * the paper, whose method is the forward solver only (Section 2); this is
 * the differentiation of that solver.  Velocity (Ladd) iolets are
 * differentiated too (their mean, amp and phase are those of the speed
 * schedule U_k(t)), and so are interpolated (BFL) walls. */
enum { LBM_OBJ_WSS = 0, LBM_OBJ_DENSITY = 1 };

/* J = scale * sum over the states f(t) with t_begin <= t < t_end (t counted
 * like lbm_get_time) of sum_x weight[x] q(x, t); q is the wall shear stress
 * of lbm_macros (LBM_OBJ_WSS) or the density (LBM_OBJ_DENSITY).  weight is
 * host memory, float64 [n], caller order. */
typedef struct {
    int32_t kind;
    const double *weight;
    int64_t t_begin;
    int64_t t_end;
    double scale;
} lbm_objective;

/* Run nsteps steps from the current state f(t0) (t0 = the context's time),
 * accumulate J over the window, and compute by the discrete adjoint
 *   dJ_dtau, dJ_dmean[k], dJ_damp[k], dJ_dphase[k] (k < n_iolets; derivatives
 *   with respect to the parameters of rho_k(t) = mean + amp sin(2 pi t /
 *   period + phase); amp and phase give 0 for a constant iolet), and
 *   dJ_df0 = dJ/df(t0), float64 [q][n] caller order.
 * Every output pointer except J may be NULL.  Forward arithmetic is that of
 * lbm_step (fp32 or fp16 storage), the adjoint state is float32, and every
 * time accumulation (J and all derivatives) is float64; results are bitwise
 * reproducible and do not depend on n_snap.  An LBM_STREAM_AA context runs
 * the sweep in the AA form (states in the AA layouts, the adjoint steps in
 * place on one buffer, the adjoint of every other step without the table);
 * its results are those of the pull form to the bit.  n_snap >= 1 device
 * snapshots of the stored state are used (one holds f(t0)); the schedule is Griewank's
 * binomial checkpointing, lbm_revolve_steps forward steps in total.  Device
 * memory: (n_snap + 1) state buffers + 2 float32 adjoint buffers + small,
 * allocated on the first call and kept in the context for later calls
 * (lbm_release_workspace); LBM_ERR_NOMEM before allocating if the part not
 * yet held does not fit.  On return the
 * context holds f(t0 + nsteps) and its time is t0 + nsteps, as after
 * lbm_step(nsteps).  Synchronous. */
lbm_status lbm_objective_grad(lbm_ctx *ctx, const lbm_objective *obj, int64_t nsteps,
                              int32_t n_snap, double *J, double *dJ_dtau, double *dJ_dmean,
                              double *dJ_damp, double *dJ_dphase, double *dJ_df0);

/* Forward steps lbm_objective_grad takes for nsteps steps and n_snap
 * snapshots: r nsteps - C(n_snap + r, n_snap + 1) + 1 with r the smallest
 * integer such that C(n_snap + r, n_snap) >= nsteps (the final state is
 * formed once more).  Host only. */
lbm_status lbm_revolve_steps(int64_t nsteps, int32_t n_snap, int64_t *forward_steps);

/* Forward and adjoint steps of the last lbm_objective_grad call, and the
 * device time of its forward-and-adjoint sweep (CUDA events on the context's
 * stream, allocation and read-back excluded).  Any output may be NULL. */
lbm_status lbm_adjoint_counts(const lbm_ctx *ctx, int64_t *forward_steps, int64_t *adjoint_steps,
                              double *sweep_ms);

/* lbm_objective_grad keeps its device workspace (snapshots, adjoint buffers)
 * in the context for later calls; this frees it (lbm_destroy does too). */
lbm_status lbm_release_workspace(lbm_ctx *ctx);

/* Change tau (> 0.5) or the iolet schedules (same n_iolets) of a context,
 * e.g. between objective evaluations; the state is unchanged. */
lbm_status lbm_set_tau(lbm_ctx *ctx, double tau);
lbm_status lbm_set_iolets(lbm_ctx *ctx, int32_t n_iolets, const double *rho_mean,
                          const double *amp, const double *period, const double *phase);

/* Sizes: number of sites, padded plane length, and device bytes held. */
lbm_status lbm_info(const lbm_ctx *ctx, int64_t *n, int64_t *npad, size_t *device_bytes);

/* Number of slab chunks over which the context's AA step pairs run fused
 * (LBM_ORDER_SLABS with LBM_STREAM_AA), or 0 when its steps run one by one
 * (any other order or streaming, fewer than two chunks, or a neighbour more
 * than one chunk away).  Host only. */
lbm_status lbm_slab_chunks(const lbm_ctx *ctx, int32_t *count);

/* ------------------------------------------------------------------------
 * Volume rendering (Section 3.3.2).  The paper's visualisation renders the
 * flow on the GPU by ray marching (direct volume rendering), with the volume
 * in a 3D texture, the viewing parameters and the transfer-function look-up
 * table in constant memory, and zoom, rotation and the scale and offset of
 * the transfer function as the steerable parameters.  Here the image goes to
 * a caller-owned device buffer (there is no display path).  Definitions:
 *   volume   float v[nz][ny][nx]; voxel (i, j, k) is centred at (i, j, k) and
 *            the box is [-1/2, n - 1/2] on each axis; a sample is the
 *            trilinear interpolation between voxel centres, its coordinates
 *            clamped to [0, n - 1].
 *   camera   pinhole at eye looking at center; forward f = normalize(center -
 *            eye), right r = normalize(f x up), up' = r x f.  Pixel (px, py)
 *            (py = 0 is the top row) looks along f + s_x r + s_y up', with
 *            s_x = ((px + 1/2) / W * 2 - 1) tan(fov_y / 2) W / H and
 *            s_y = (1 - (py + 1/2) / H * 2) tan(fov_y / 2).
 *   march    the ray's piece inside the box (from the eye when the eye is
 *            inside) is cut into segments of length dt, the last one
 *            shorter, with one sample at each segment's midpoint.
 *   transfer s = clamp((v - tf_offset) tf_scale, 0, 1); (r, g, b, alpha) is
 *            the LUT linearly interpolated at s * 255 (alpha = opacity per
 *            unit length); a segment of length l has opacity min(1, alpha l).
 *   compose  front to back, C += (1 - A) a (r, g, b), A += (1 - A) a; the
 *            ray stops before a sample once A >= a_stop.
 * The pixel is (C_r, C_g, C_b, A), float32.  Arithmetic is float32. */
typedef struct lbm_volume lbm_volume;

enum { LBM_QTY_DENSITY = 0, LBM_QTY_SPEED = 1, LBM_QTY_WSS = 2 };
enum { LBM_FILTER_TEXTURE = 0, LBM_FILTER_EXACT = 1 };

/* One view.  filter: LBM_FILTER_TEXTURE samples with the texture unit's
 * trilinear filter (one fetch; its weights are quantised to 1/256), and
 * LBM_FILTER_EXACT with eight texel fetches and float32 weights.
 * skip_empty = 1 lets rays jump over 8^3 bricks whose samples are all
 * exactly 0 whenever the LUT gives value 0 zero opacity; the image is then
 * bitwise the one of the full march (0 marches every segment).  Limits:
 * 1 <= width, height <= 16384; 0 < fov_y < 3.1; dt >= 1e-3 with at most 2^24
 * segments along the box diagonal; 0 < a_stop <= 1 (1: no early stop);
 * every value finite; up not parallel to center - eye.  counters_d, when
 * not NULL (device, 2 x uint64, 8-byte aligned), receives += the number of
 * samples composited and of brick jumps (a slightly slower kernel). */
typedef struct {
    int32_t width, height;
    double eye[3], center[3], up[3];
    double fov_y;
    double dt;
    double tf_scale, tf_offset;
    double a_stop;
    int32_t filter;
    int32_t skip_empty;
    unsigned long long *counters_d;
    float lut[256][4];
} lbm_view;

/* A volume of nx x ny x nz float voxels (1..16384 each) held as a 3D CUDA
 * array with a trilinear and a point-sampling texture and a surface, plus
 * its 8^3 brick occupancy.  Created holding zeros.  Synchronous.  Errors of
 * the volume calls are read with lbm_last_error(NULL). */
lbm_status lbm_volume_create(int32_t nx, int32_t ny, int32_t nz, lbm_volume **out);
void lbm_volume_destroy(lbm_volume *vol);

/* Copy v_d (device, float [nz][ny][nx], dense) into the volume and rebuild
 * the brick occupancy from its non-zero voxels; lbm_volume_download copies
 * the volume out to v_d.  Asynchronous on cuda_stream. */
lbm_status lbm_volume_upload(lbm_volume *vol, const float *v_d, void *cuda_stream);
lbm_status lbm_volume_download(const lbm_volume *vol, float *v_d, void *cuda_stream);

/* Bounding box of the context's sites: lo[3] (smallest coordinates) and
 * dims[3] (extent, 0 for no sites). */
lbm_status lbm_lattice_box(const lbm_ctx *ctx, int32_t *lo, int32_t *dims);

/* Write a quantity of the current state f(t) into the volume: the site at
 * coordinates xyz goes to voxel xyz - origin[3] (sites outside the volume
 * are left out); voxels without a site hold 0.  quantity: LBM_QTY_DENSITY
 * (rho), LBM_QTY_SPEED (|u|) or LBM_QTY_WSS (as lbm_macros).  Refilling from
 * the same context and origin rewrites only the sites' voxels.  Asynchronous
 * on the context's stream. */
lbm_status lbm_volume_from_lattice(lbm_volume *vol, lbm_ctx *ctx, int32_t quantity,
                                   const int32_t *origin);

/* Ray-march the volume into rgba_d (device, float [height][width][4],
 * 16-byte aligned).  Asynchronous on cuda_stream; the caller orders it
 * after the fill or upload when those run on another stream. */
lbm_status lbm_render(const lbm_volume *vol, const lbm_view *view, float *rgba_d, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* HEMELB_GB300_LBM_H */
