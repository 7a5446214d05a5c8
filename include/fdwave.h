/*
 * fdwave.h -- C ABI of libfdwave, a GB300 (sm_103a) finite-difference solver
 * for the damped, variable-velocity acoustic wave equation
 *
 *     m u_tt + eta u_t - lap(u) = q                     (arXiv 1609.03361, Sec. 5, Eq. 3)
 *
 * with explicit second-order time stepping, central space orders 2..16, an
 * absorbing damping layer, multilinear source injection / receiver sampling
 * (Sec. 5.2, Listing 8), the adjoint propagator (Sec. 5.1, Listing 7) and the
 * FWI gradient with wavefield checkpointing (Sec. 5.4, "gradient test").
 *
 * Conventions shared by every call
 * --------------------------------
 *  Grid.    `shape` is the PHYSICAL grid (points per axis).  The library adds
 *           `nbl` damping-layer points on every side; the COMPUTATIONAL shape is
 *           shape[a] + 2*nbl.  Axis order is (x, y, z) in 3D and (x, z) in 2D,
 *           the last axis (depth) being contiguous in memory.  Fields exchanged
 *           with the library are dense row-major float32 arrays in either the
 *           physical or the computational shape, as each call states.
 *  Units.   Spacing in metres, time in milliseconds, velocity in km/s (m/ms),
 *           squared slowness m = 1/v^2 in ms^2/m^2.
 *  Points.  Coordinates are double [npts][ndim] in metres relative to the
 *           physical origin; every coordinate must lie in [0, (N_a-1) h_a].
 *  Time.    u^{-1} = u^0 = 0.  Step n = 0..nt-2 makes u^{n+1} and adds the
 *           source sample q^n into it, scaled by dt^2 / (m + eta dt/2).
 *           Receivers record rec^n = P_r u^n for n = 0..nt-1.  Time series are
 *           float32 [nt][npts] (row n holds sample n of every point).
 *  Memory.  Array arguments may be HOST or DEVICE pointers (the library asks
 *           the CUDA runtime which); host arrays are staged through
 *           library-owned device buffers.  The caller owns every array it
 *           passes; the library keeps no pointer past the call except where
 *           stated.  Device arrays must live on the context's device.
 *  Streams. `stream` is a cudaStream_t (NULL = the legacy default stream).
 *           Work is queued in stream order and the calls do not synchronise,
 *           except that a host output array in pageable memory is complete
 *           when the call returns.  Calls on one context must be ordered
 *           (one stream, or synchronised by the caller).  Errors raised by
 *           queued GPU work (a bounded wait that timed out) are reported by
 *           fdw_sync and by the next call on the context.
 *  Errors.  Every call returns fdw_status; FDW_OK = 0.  fdw_last_error gives
 *           a message for the last failure on a context.
 */
#ifndef FDWAVE_H
#define FDWAVE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fdw_ctx fdw_ctx;      /* one shot: grid, model, wavefields, points, checkpoints */
typedef struct fdw_batch fdw_batch;  /* several contexts stepped together in one launch per step */

typedef enum {
  FDW_OK = 0,
  FDW_ERR_ARG = 1,            /* null / inconsistent argument */
  FDW_ERR_SHAPE = 2,          /* ndim not 2 or 3, a dimension < 2, or too large */
  FDW_ERR_ORDER = 3,          /* space order odd, < 2 or > 16 */
  FDW_ERR_CFL = 4,            /* dt above the stability limit for vmax */
  FDW_ERR_OUT_OF_DOMAIN = 5,  /* a point outside the physical domain */
  FDW_ERR_OOM = 6,            /* device allocation failed */
  FDW_ERR_CUDA = 7,           /* CUDA runtime error, or no usable GPU */
  FDW_ERR_TIMEOUT = 8,        /* a device-side bounded wait gave up */
  FDW_ERR_STATE = 9           /* call out of order (e.g. model not set) */
} fdw_status;

/* Storage types for the model and the checkpoint snapshots. */
enum { FDW_F32 = 0, FDW_F16 = 1, FDW_BF16 = 2 };
/* Layout of a field exchanged with the library. */
enum { FDW_LAYOUT_PHYSICAL = 0, FDW_LAYOUT_COMPUTATIONAL = 1 };

/* ---------------------------------------------------------------- host helpers */

/* Library version as 10000*major + 100*minor + patch. */
int fdw_version(void);

/* Text of a status code (static string). */
const char* fdw_status_string(fdw_status st);

/* Central second-derivative weights c_0..c_r (r = p/2, c must hold r+1
 * doubles) of order p, unscaled (multiply by 1/h^2).  Sec. 3.1: the order of
 * the `dx2` expansion is a parameter; for p = 2 the paper prints [1, -2, 1].
 * FDW_ERR_ORDER for an invalid p, FDW_ERR_ARG for c == NULL.  Host only. */
fdw_status fdw_fd_weights(int space_order, double* c);

/* Stability limit of the explicit scheme (von Neumann, undamped):
 * dt_max = 2 / (vmax sqrt(sum_a S / h_a^2)) with S the largest |symbol| of the
 * 1-D stencil.  Returns a negative value for invalid arguments.  Host only. */
double fdw_dt_max(int ndim, const double* spacing, int space_order, double vmax);

/* ---------------------------------------------------------------- context */

/* Create a context on CUDA device `device` for one problem:
 *   ndim          2 or 3
 *   shape         physical points per axis [ndim], each >= 2
 *   spacing       grid spacing per axis [ndim], metres, > 0
 *   space_order   even, 2..16
 *   nbl           damping-layer points per side, >= 0
 *   dt, nt        time step (ms) and number of time samples (>= 1)
 *   vmax          largest velocity of any model that will be set (km/s); it
 *                 sets the damping strength (Sec. 5, Eq. 3: eta is the
 *                 spatially varying damping of the absorbing layer) and the
 *                 stability check: dt > fdw_dt_max(...) gives FDW_ERR_CFL.
 * Allocates the two wavefield buffers and the model buffer.  *out receives the
 * context, or NULL on failure.  The damping is the built-in quadratic profile
 * eta = sum_a 3 ln(1000) / (2 nbl h_a vmax) (d_a / nbl)^2 (d_a: cells into the
 * layer along axis a) until fdw_set_damping replaces it. */
fdw_status fdw_create(fdw_ctx** out, int ndim, const int64_t* shape, const double* spacing,
                      int space_order, int nbl, double dt, int nt, double vmax, int device);

/* Free a context and everything it owns (NULL is ignored).  Synchronises the
 * device first. */
void fdw_destroy(fdw_ctx* ctx);

/* Message of the last failure on this context ("" when none). */
const char* fdw_last_error(const fdw_ctx* ctx);

/* Set the squared slowness m (float32, host or device).  layout
 * FDW_LAYOUT_PHYSICAL: m has the physical shape and is extended into the layer
 * by repeating the edge values; FDW_LAYOUT_COMPUTATIONAL: m has the
 * computational shape.  m_dtype selects the STORAGE type on the device
 * (FDW_F32, FDW_F16 or FDW_BF16); arithmetic stays float32.  m must be > 0. */
fdw_status fdw_set_model(fdw_ctx* ctx, const float* m, int layout, int m_dtype, void* stream);

/* Replace the built-in damping by a user field eta (float32, computational
 * shape, >= 0, host or device), or restore the built-in profile with
 * eta == NULL.  A field costs one more read per point and step. */
fdw_status fdw_set_damping(fdw_ctx* ctx, const float* eta, void* stream);

/* Source and receiver positions (Sec. 5.2: sparse points with their own
 * coordinates).  xyz is double [n][ndim] (host), n >= 0.  The multilinear
 * weights and the per-tile lists are built on the host and kept by the
 * context.  FDW_ERR_OUT_OF_DOMAIN if a point lies outside the physical grid. */
fdw_status fdw_set_sources(fdw_ctx* ctx, int nsrc, const double* xyz);
fdw_status fdw_set_receivers(fdw_ctx* ctx, int nrec, const double* xyz);

/* --------------------------------------------------------------- propagation */

/* Forward modelling (Sec. 5.1, Listing 6, with the injection and sampling of
 * Sec. 5.2): q [nt][nsrc] in, receiver traces rec [nt][nrec] out. */
fdw_status fdw_forward(fdw_ctx* ctx, const float* q, float* rec, void* stream);

/* Forward modelling that also keeps checkpoints for fdw_gradient: the pair
 * (u^{jk}, u^{jk-1}) every k = ckpt_every steps, stored as snap_dtype
 * (FDW_F32, FDW_F16 or FDW_BF16; 16-bit snapshots carry one float32 scale per
 * snapshot), plus a copy of q.  The checkpoints live on the device until the
 * next checkpointed forward or fdw_destroy.  Gradient accuracy against the
 * exact FP64 discrete gradient (64^3 grid, order 8, 400 steps, k = 10):
 * FP32 checkpoints about 1e-6, FP16 snapshots about 1.4e-4 (within 1e-3);
 * BF16 snapshots about 1.3e-3, which does NOT meet a 1e-3 bound: their 8-bit
 * significand rounds every stored value by up to 2^-9 relative, and a scale
 * cannot help because bfloat16 already has float32's exponent range. */
fdw_status fdw_forward_ckpt(fdw_ctx* ctx, const float* q, float* rec, int ckpt_every,
                            int snap_dtype, void* stream);

/* Adjoint modelling (Sec. 5.1, Listing 7): the receivers inject d [nt][nrec]
 * backward in time and the sources sample qadj [nt][nsrc] (out), so that
 * <F q, d> = <q, F^T d> (Sec. 5.3, Eq. 4).  qadj^n = P_s lambda^{n+1}. */
fdw_status fdw_adjoint(fdw_ctx* ctx, const float* d, float* qadj, void* stream);

/* FWI gradient (Sec. 5.4) with respect to m of sum_n <r^n, P_r u^n>, where
 * r = resid - resid_sub ([nt][nrec] each; resid_sub may be NULL) and u is the
 * wavefield of the last fdw_forward_ckpt.  For the misfit
 * J = 1/2 sum |rec - d_obs|^2 pass resid = rec, resid_sub = d_obs.
 * grad (out, float32) has the computational shape (grad_layout
 * FDW_LAYOUT_COMPUTATIONAL), or the physical shape with the layer cells summed
 * onto the edge cells they repeat (FDW_LAYOUT_PHYSICAL, the gradient with
 * respect to a physical model set with FDW_LAYOUT_PHYSICAL).
 * FDW_ERR_STATE without a preceding checkpointed forward. */
fdw_status fdw_gradient(fdw_ctx* ctx, const float* resid, const float* resid_sub, float* grad,
                        int grad_layout, void* stream);

/* Copy the newest wavefield u^{nt-1} of the last forward call (or lambda^1 of
 * the last adjoint when which == 1) to out (float32, computational shape). */
fdw_status fdw_get_wavefield(fdw_ctx* ctx, int which, float* out, void* stream);

/* Wait for the context's queued work and report device-side errors. */
fdw_status fdw_sync(fdw_ctx* ctx);

/* ------------------------------------------------------------------ tuning */

/* Brute-force search over tile shapes, x-chunk lengths and pipeline depths
 * (Sec. 3.3.3: block sizes found by a brute-force search), timing `steps`
 * forward steps each on the current model (injecting zeros and sampling into
 * scratch rows, as a real step does), then timing the four fastest again,
 * interleaved and longer, and keeping the best.  The choice is kept by the
 * context and, when the environment variable FDW_AUTOTUNE_CACHE names a file,
 * cached there per (GPU, order, shape, model type).  Synchronises. */
fdw_status fdw_autotune(fdw_ctx* ctx, int steps);

/* Checkpoint memory budget of fdw_forward_ckpt / fdw_gradient: at most
 * `max_pairs` checkpoint pairs (u^{n}, u^{n-1}) are stored (each the size of
 * two fields in the snapshot type).  0 (the default) stores one pair per
 * ckpt_every steps, (nt-1)/ckpt_every pairs, and the gradient recomputes each
 * segment of ckpt_every steps once.  A smaller positive budget makes both
 * calls follow a binomial checkpoint schedule over those segments (Griewank,
 * "revolve"; the paper has no counterpart: it extends the checkpointed
 * gradient of Sec. 5.4): the forward call stores the pairs that the schedule
 * takes on its first sweep, and the gradient re-advances from stored pairs,
 * storing and freeing pairs as it reverses, with the fewest forward steps any
 * schedule with that many pairs can use (fdw_checkpoint_schedule gives the
 * schedule).  With FP32 snapshots the gradient is bit for bit the one of the
 * unlimited budget.  Takes effect at the next fdw_forward_ckpt (a gradient
 * before it gives FDW_ERR_STATE).  Under a budget the gradient reuses the
 * slots as it goes, so it consumes the checkpoints: each fdw_gradient needs
 * its own fdw_forward_ckpt (FDW_ERR_STATE otherwise).  FDW_ERR_ARG if
 * max_pairs < 0.  Host only. */
fdw_status fdw_set_checkpoint_budget(fdw_ctx* ctx, int max_pairs);

/* The binomial schedule used for nseg segments with nslots pairs, as (op, arg)
 * pairs of ints: op 1 = advance the current state to the start of segment
 * arg, 2 = store the current state in slot arg, 3 = make slot arg (-1: the
 * zero state at time 0) the current state, 4 = recompute segment arg from the
 * current state (its start) and run its adjoint steps.  The state at the
 * start of segment 0 is current at the beginning.  Writes at most cap pairs
 * into actions[2*cap] and returns the number of actions (larger than cap when
 * actions was too short: nothing is written then), -1 for nseg < 1,
 * nslots < 0, cap < 0 or actions NULL with cap > 0.  Host only. */
int fdw_checkpoint_schedule(int nseg, int nslots, int* actions, int cap);

/* Force a tile configuration: tile index (0..9, -1 = default: 9 on 3D grids,
 * 3 on 2D grids; 3 is meant for 2D grids, 6 keeps per-plane tiles in a
 * second ring, 7 and 8 are 4 and 6 with the x-direction queue in tensor
 * memory, 9 is 7 with each pipeline
 * stage holding exactly one plane's reads: the halo plane x, its tiles and
 * the centre tile of plane x + r), x-chunk length (0 = default) and pipeline
 * depth of the forward and adjoint steps (>= r + 2 with r = space_order / 2,
 * >= 2 for tile 9, 0 = default; the gradient step picks its own).  Every tile computes each point with the same arithmetic,
 * so the results do not depend on the tiling, bit for bit.  FDW_ERR_ARG
 * outside these ranges. */
fdw_status fdw_set_tiling(fdw_ctx* ctx, int tile, int xchunk, int stages);

/* Run plain forward modelling (fdw_forward, and fdw_batch_forward when every
 * context of the batch asks for it) and the plain adjoint (fdw_adjoint) as one
 * persistent launch over all time steps (on = 1, the default) or as one
 * launch per step (on = 0).  With on = 1 the checkpointed forward
 * (fdw_forward_ckpt without a checkpoint budget) runs one persistent launch
 * per segment of ckpt_every steps, each followed by the storing of its
 * snapshot pair, and the gradient recomputes each segment in one launch; the
 * gradient's adjoint steps, and every step under a checkpoint budget, keep
 * one launch per step.  The schemes of Sec. 5 (Eq. 3) and Sec. 5.1 are
 * unchanged, and so are the results, bit for bit: the launch takes work units
 * step by step, and a unit of step n + 1 starts as soon as every unit that
 * updated the planes it reads (its own x chunk and the neighbouring ones, all
 * column tiles) has finished step n, instead of after the whole step; the
 * paper has no counterpart (it is a scheduling change of the same time loop).
 * Slab contexts (which never run whole time loops) step one launch at a time.
 * The autotuner times the mode the context is in.  FDW_ERR_STATE for on = 1
 * on a slab context. */
fdw_status fdw_set_persistent(fdw_ctx* ctx, int on);

/* Tile configuration in use: out[0] = tile index, out[1] = x-chunk length,
 * out[2] = pipeline stages, out[3] = CTAs per launch, out[4] = work units. */
fdw_status fdw_get_tiling(fdw_ctx* ctx, int* out5);

/* Temporal blocking of plain forward modelling (fdw_forward, and
 * fdw_batch_forward when every context of the batch asks for it): with
 * steps_per_pass = 2 each launch advances the scheme of Sec. 5 (Eq. 3) by two
 * time steps, u^{n+1} and u^{n+2} from u^{n-1} and u^n, reading the two old
 * fields and the model once and writing the two new ones (the first step is
 * recomputed on a halo of r rows / planes around each tile and kept in shared
 * memory).  Sources and receivers are handled as in the one-step loop and the
 * traces agree with it to rounding.  The paper has no counterpart: it is a
 * memory-traffic optimisation of the same scheme.  Only 3D grids, space orders
 * 2 and 4 and the built-in damping profiles: FDW_ERR_ARG for a 2D grid,
 * FDW_ERR_ORDER above order 4, FDW_ERR_STATE on a slab context; a damping
 * field set with fdw_set_damping makes fdw_forward run one step per launch.
 * The context then holds four wavefield buffers instead of two (allocated
 * here; FDW_ERR_OOM if that fails).  Checkpointed forward runs, the adjoint
 * and the gradient always step one step per launch.  variant: 0 (output tiles
 * of 16 rows at order 2, 12 at order 4, two CTAs per SM) or 1 (32 / 28 rows,
 * one CTA per SM), -1 = default 0; xchunk: x planes per work unit (0 =
 * default); stages: pipeline depth (>= 2r + 1, 0 = default).  steps_per_pass =
 * 1 restores one step per launch. */
fdw_status fdw_set_time_blocking(fdw_ctx* ctx, int steps_per_pass, int variant, int xchunk,
                                 int stages);

/* out[0] = steps per pass; with 2: out[1] = variant, out[2] = x-chunk length,
 * out[3] = pipeline stages, out[4] = work units (needs the model set). */
fdw_status fdw_get_time_blocking(fdw_ctx* ctx, int* out5);

/* -------------------------------------------------------------- batched shots */

/* Group contexts that share order, spacing, dt, nt and model storage type so
 * that every time step of all of them runs as one launch over one table of
 * work units (grids may differ in size).  The contexts must outlive the
 * batch.  The batch keeps its own tiling (fdw_batch_autotune). */
fdw_status fdw_batch_create(fdw_batch** out, int nshots, fdw_ctx* const* ctxs);
void fdw_batch_destroy(fdw_batch* b);
const char* fdw_batch_last_error(const fdw_batch* b);

/* Forward modelling of every shot: q[s] and rec[s] as in fdw_forward. */
fdw_status fdw_batch_forward(fdw_batch* b, const float* const* q, float* const* rec,
                             void* stream);

/* Checkpointed forward and gradient of every shot, as fdw_forward_ckpt and
 * fdw_gradient per shot (resid_sub may be NULL, or hold NULL entries). */
fdw_status fdw_batch_forward_ckpt(fdw_batch* b, const float* const* q, float* const* rec,
                                  int ckpt_every, int snap_dtype, void* stream);
fdw_status fdw_batch_gradient(fdw_batch* b, const float* const* resid,
                              const float* const* resid_sub, float* const* grad,
                              int grad_layout, void* stream);

fdw_status fdw_batch_autotune(fdw_batch* b, int steps);
fdw_status fdw_batch_get_tiling(fdw_batch* b, int* out5);

/* ------------------------------------------------ single-shot domain split */

/* One x slab of a grid too large for one GPU (Sec. 6 names MPI parallelism
 * only between whole inversion operators; splitting one grid across devices
 * is an extension the paper does not have): the context holds the
 * computational x planes [x_begin, x_end) of the grid that fdw_create would
 * build from the same arguments, plus r = space_order/2 ghost planes on either
 * side, and updates only its own planes.  x_end - x_begin >= r.  The model
 * (fdw_set_model, either layout) and damping field (fdw_set_damping) are given
 * for the whole grid, and source and receiver coordinates for the whole
 * domain: the slab injects the source corners in its planes and records the
 * receivers whose base plane (the lower x corner) it owns, leaving zeros in the
 * other receivers' columns, so that summing the slabs' traces gives the traces
 * of the whole grid.  Whole time loops (fdw_forward, fdw_forward_ckpt,
 * fdw_adjoint, fdw_gradient, batches) give FDW_ERR_STATE / FDW_ERR_ARG on a
 * slab: it advances with fdw_step, and after each step the caller copies
 * each neighbour's send planes into this slab's ghost planes
 * (fdw_halo_planes).  FDW_ERR_SHAPE for a range outside the grid. */
fdw_status fdw_create_slab(fdw_ctx** out, int ndim, const int64_t* shape, const double* spacing,
                           int space_order, int nbl, double dt, int nt, double vmax, int device,
                           int64_t x_begin, int64_t x_end);

/* One forward time step n (0 <= n <= nt-2) of any context: u^{n+1} from u^n
 * and u^{n-1} (Sec. 5, Eq. 3 and Listing 6), injection of q^n, and the
 * receiver samples rec^n of u^n; n = nt-1 records rec^{nt-1} only (for a slab,
 * after the last ghost exchange).  n = 0 first clears the wavefields.  Calls
 * n = 0 .. nt-1 in order compute what fdw_forward computes.  q [nt][nsrc] and
 * rec [nt][nrec] are device arrays (FDW_ERR_ARG otherwise); stream-ordered. */
fdw_status fdw_step(fdw_ctx* ctx, int n, const float* q, float* rec, void* stream);

/* Device addresses, in the field u^{n+1} that fdw_step(n) produced, of a
 * slab's first r and last r own planes (send_lo, send_hi) and of its lower and
 * upper ghost planes (recv_lo, recv_hi), each a contiguous block of *count
 * floats (r planes of ny x nzp; nzp = nz rounded up to a multiple of 32 in 3D,
 * the same layout in every slab of a grid).  Before step n+1 the caller copies
 * the lower neighbour's send_hi into recv_lo and the upper neighbour's send_lo
 * into recv_hi (the outermost slabs keep zero ghosts: the zero halo of the
 * scheme).  FDW_ERR_ARG for a context that is not a slab.  Host only. */
fdw_status fdw_halo_planes(fdw_ctx* ctx, int n, float** send_lo, float** send_hi,
                           float** recv_lo, float** recv_hi, int64_t* count);

/* The exchange after step n between two neighbouring slabs of one grid held
 * by this process (lower: the one with the smaller x planes), possibly on
 * different devices: lower's send_hi to upper's recv_lo and upper's send_lo to
 * lower's recv_hi, enqueued on `stream`.  FDW_ERR_ARG for slabs that are not
 * neighbours of one grid. */
fdw_status fdw_exchange_ghosts(fdw_ctx* lower, fdw_ctx* upper, int n, void* stream);

/* Copies between a slab's ghost-plane blocks after step n and caller buffers
 * of *count floats each (fdw_halo_planes), host or device, for exchanges
 * through a communication library: dir 0 copies the send planes out (send_lo
 * to lo, send_hi to hi), dir 1 copies lo into recv_lo and hi into recv_hi.  A
 * NULL buffer skips its side.  Stream-ordered. */
fdw_status fdw_halo_copy(fdw_ctx* ctx, int n, int dir, float* lo, float* hi, void* stream);

/* ---------------------------------------------------------- allocation-free */

/* Forward modelling that allocates nothing.  The paper has no counterpart:
 * this is a service for callers that cannot call cudaMalloc, such as code
 * that must stay inside a device-memory budget owned by another allocator or
 * a loop that may not touch the allocator once it runs.  It computes what
 * fdw_create + fdw_set_model (physical layout, FDW_F32) + fdw_set_sources +
 * fdw_set_receivers + fdw_forward compute, with the built-in damping, for a
 * small problem, keeping all of its scratch (wavefields, model, tables) in one
 * 16 MiB static device array that every GPU loading the library holds until
 * the process exits.
 *   m     device, float32, physical shape (squared slowness, > 0)
 *   q     device, float32 [nt][nsrc];  rec  device, float32 [nt][nrec] (out)
 *   src_xyz, rec_xyz  host, double [n][ndim], metres
 *   other arguments as in fdw_create.
 * Limits: at most 4096 computational points per axis, at most 2^20 points per
 * field with rows padded to a multiple of 32, at most 4096 sources and 4096
 * receivers, at most 8192 work units; FDW_ERR_SHAPE beyond them.  The first
 * call on a device looks up the array's device address, so make it before any
 * stream capture.  Every call rewrites the array and clears the wavefields;
 * calls that overlap on the GPU (other streams or host threads) race on it.
 * Sizes, order, stability and point locations are checked on the host before
 * any CUDA call; m, q and rec must then be device (or managed) memory, else
 * FDW_ERR_ARG (a host buffer never reaches a kernel).  The call waits for its
 * stream and returns FDW_ERR_TIMEOUT if a device-side bounded wait gave up
 * (FDW_ERR_CUDA for any other device-side fault or a failed CUDA call).  Its
 * traces are bit for bit those of fdw_forward on a context with the tiling
 * fdw_set_tiling(ctx, 0 (3D) or 3 (2D), 64, space_order/2 + 3). */
fdw_status fdw_forward_static(int ndim, const int64_t* shape, const double* spacing,
                              int space_order, int nbl, double dt, int nt, double vmax,
                              const float* m, int nsrc, const double* src_xyz, const float* q,
                              int nrec, const double* rec_xyz, float* rec, void* stream);

/* ---------------------------------------------------------- 2D diffusion */

/* The diffusion example of Sec. 4: u_t = alpha (u_xx + u_yy) (Eq. 1), forward
 * Euler in time and second-order 3-point differences per axis, on an
 * [nx][ny] grid whose boundary rows and columns keep their initial values
 * (only interior points are updated).  One step is
 *   u'(i,j) = wc u(i,j) + wx (u(i-1,j) + u(i+1,j)) + wy (u(i,j-1) + u(i,j+1))
 * with wx = dt alpha/dx^2, wy = dt alpha/dy^2, wc = 1 - 2wx - 2wy, in float32.
 *   u       device float32 [nx][ny], y contiguous: the initial field on entry,
 *           the field after `steps` steps once the stream reaches that point
 *   tmp     device float32 [nx][ny] scratch, not overlapping u (its contents
 *           on entry are ignored and undefined afterwards)
 *   nx, ny  >= 3 (FDW_ERR_ARG), <= 2^31 (FDW_ERR_SHAPE)
 *   dx, dy, alpha, dt  > 0 (FDW_ERR_ARG); dt above the Eq. 2 limit
 *           dx^2 dy^2 / (2 alpha (dx^2 + dy^2)) gives FDW_ERR_CFL
 *   steps   >= 0
 *   steps_per_pass  time steps fused into one pass over memory: 1, 2, 4 or 8
 *           (0 selects 4).  Results do not depend on it: every point sees the
 *           same float32 operations in the same order.
 *   stream  CUDA stream (NULL: the legacy default stream)
 * The caller owns u and tmp.  Stream-ordered: the call returns once the work
 * is enqueued; host or non-device pointers give FDW_ERR_ARG, a failed launch
 * FDW_ERR_CUDA.  Allocates nothing. */
fdw_status fdw_diffusion2d(float* u, float* tmp, int64_t nx, int64_t ny, double dx, double dy,
                           double alpha, double dt, int steps, int steps_per_pass, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* FDWAVE_H */
