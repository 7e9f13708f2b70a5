/*
 * mrgb.h -- C ABI of the GB300 multiresolution stencil library.
 *
 * The library advances scalar advection on a periodic forest of octrees of
 * collocated nb^3 blocks with interpolating-wavelet grid adaptation, after
 * T. Gillis and W. M. van Rees, "MURPHY - A scalable multiresolution
 * framework for scientific computing on 3D block-structured collocated
 * grids" (arXiv 2112.07537).  All compute runs in CUDA kernels on the device
 * the grid was created on; nothing here falls back to the CPU.
 *
 * Conventions shared by every call
 *  - Return value: MR_OK (0) or a negative MR_ERR_* code.  No call throws or
 *    aborts.  MR_ERR_CUDA means a CUDA runtime call failed; the message of
 *    the last failure is available from mr_last_error().
 *  - Asynchrony: calls enqueue work on the grid's stream and return, except
 *    where a call's comment says it synchronises (those that return host
 *    values: mr_grid_leaves, mr_adapt, mr_query, mr_field_copy_out to host).
 *  - Ownership: the caller owns host buffers and the device workspace passed
 *    to mr_grid_create (for example a torch uint8 tensor); the grid carves all
 *    its device arrays (block pool, octree tables, scratch) out of that
 *    workspace and never calls cudaMalloc.  The workspace must outlive the grid.
 *  - Leaves: a leaf is (level L, anchor a[3]) with 0 <= a[d] < ntree[d]*2^L,
 *    in units of level-L blocks.  The grid keeps its leaves sorted by Morton
 *    key (anchor scaled to lmax, bits interleaved x lowest); the block pool
 *    slot of a leaf is its rank in that order.
 *  - Field layout: leaf-major in slot order, nb^3 values per leaf, x fastest
 *    (v[slot*nb^3 + i + nb*(j + nb*k)]); point i of a level-L leaf with
 *    anchor a sits at x = (a*nb + i) * tree_len / (nb * 2^L) (vertex-aligned,
 *    Sec. 2.2: coarse point k coincides with fine point 2k); periodic in every
 *    direction.  Element type: float for MR_F32, double for MR_F64.
 *  - Padded layout (ghost fill output): per leaf (nb+2G)^3 values over
 *    [-G, nb+G)^3, x fastest.
 */
#ifndef MRGB_H
#define MRGB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MR_OK 0
#define MR_ERR_INVALID (-1)     /* bad argument or descriptor */
#define MR_ERR_NOMEM (-2)       /* workspace or leaf capacity too small */
#define MR_ERR_CUDA (-3)        /* a CUDA runtime call failed */
#define MR_ERR_TIMEOUT (-4)     /* a bounded device/host loop hit its cap */
#define MR_ERR_UNSUPPORTED (-5) /* valid request outside what is built */
#define MR_ERR_BALANCE (-6)     /* leaves are not 2:1 balanced, or a ghost
                                   shell reaches beyond the +-1 level ring */

#define MR_F32 0
#define MR_F64 1

/* right-hand side schemes (supplementary "Finite differences scheme") */
#define MR_CONS3 0  /* Table SM3 with the ideal weights 1/3, 2/3 */
#define MR_CONS5 1  /* Table SM4 with the ideal weights 1/10, 3/5, 3/10 */
#define MR_WENOZ5 2 /* Table SM4 with WENO-Z weights (Borges et al. 2008) */

/* analytic initial fields for mr_field_set */
#define MR_INIT_GAUSSIAN 0    /* params: cx cy cz sigma amp; nearest image  */
#define MR_INIT_TANH_SPHERE 1 /* params: cx cy cz radius width             */
#define MR_INIT_TAYLOR_GREEN 2 /* params: component(0,1,2) scale phase    */
#define MR_INIT_GAUSSIAN_SUM 3 /* params: n, then n x (cx cy cz sigma amp), n <= 51 */
/* params: cx cy cz sigma beta amp; amp exp(-(r^2/sigma^2)/(1 - r^2/beta^2))
 * for r < beta, else 0 (nearest image; the initial field of Sec. 5.3)      */
#define MR_INIT_COMPACT_GAUSSIAN 4
/* params: component(0,1,2) scale; the incompressible deformation field of
 * Sec. 5.3 in its published divergence-free form
 * (2 sin^2(pi x) sin(2 pi y) sin(2 pi z), -sin(2 pi x) sin^2(pi y) sin(2 pi z),
 *  -sin(2 pi x) sin(2 pi y) sin^2(pi z)) times scale                     */
#define MR_INIT_DEFORMATION 5
/* params as MR_INIT_GAUSSIAN_SUM; the sum is added to the field's current
 * values (sums of more than 51 Gaussians in several calls)                */
#define MR_INIT_GAUSSIAN_SUM_ADD 6

/* adaptation flags */
#define MR_ADAPT_REFINE 1
#define MR_ADAPT_COARSEN 2
/* FP32 grids: adapt the fields other than the criterion field with FP64
 * arithmetic (their ghost fill, refinement, coarsening and update step, as
 * the criterion field's).  Without it they run in FP32 (padded blocks,
 * wavelet sums and the update's details in FP32): their values then differ
 * from exact arithmetic by a few FP32 roundings of the field maximum, while
 * the criterion field and every refine/coarsen decision stay as with the
 * flag.  No effect on FP64 grids.                                         */
#define MR_ADAPT_OTHERS_FP64 4

typedef struct {
  int ntree[3];     /* trees per direction (the forest tiles the domain)   */
  double tree_len;  /* edge of one tree                                    */
  int nb;           /* points per block edge: even, 8..32                  */
  int lmin, lmax;   /* level bounds used by the adaptation policy          */
  int wav_N;        /* interpolation order N: 2, 4 or 6                    */
  int wav_Nt;       /* lifting order N~: 0 or 2                            */
  int precision;    /* MR_F32 or MR_F64                                    */
  int nfields;      /* user fields held in the block pool (>= 1)           */
  int capacity;     /* maximum number of leaves                            */
  void *stream;     /* cudaStream_t the grid enqueues on (NULL: legacy)    */
  int flags;        /* MR_GRID_FIXED_TREE: no adaptation buffers (smaller
                       workspace); mr_adapt*, mr_criterion and
                       mr_ghost_fill64 then return MR_ERR_UNSUPPORTED      */
} mr_grid_desc;

#define MR_GRID_FIXED_TREE 1
#define MR_GRID_VELOCITY 2 /* reserve the ghost-filled velocity cache used by
                              mr_step_vel / mr_rhs_advect_vel              */
/* Every tree of the forest is its own periodic domain: a batch of
 * independent grids (one per tree, each with its own leaves, fields and
 * adaptation) advanced together -- every call is one launch per phase over
 * the leaves of all of them.  2:1 balance, ghosts, neighbours and the
 * adaptation policy never cross a tree boundary; each tree wraps onto
 * itself.  mr_field_set evaluates its analytic fields in every tree's own
 * coordinates [0, tree_len)^3.  The paper has no counterpart (its instances
 * are separate runs); each tree computes exactly what a one-tree grid with
 * the same leaves and values computes. */
#define MR_GRID_INDEPENDENT_TREES 4
/* Physical boundaries (Sec. 2.4): the domain ends at x_d = 0 and
 * x_d = ntree[d] * tree_len along each axis d flagged here instead of
 * wrapping around.  Ghost values beyond a boundary come from a polynomial of
 * degree < N (the wavelet's order) through grid values next to it, applied
 * as the paper orders it: to the coarse values before refinement, to each
 * block before substitution and coarsening, and once more when every ghost
 * is known.  The layout is vertex-aligned, so the lower boundary is grid
 * point 0 and the upper boundary lies one spacing beyond the last point.
 * Condition (default: extrapolation through the N nearest points):
 * MR_GRID_BC_DIRICHLET0 -- zero value: through 0 at the boundary and the
 * N-1 nearest points off it; MR_GRID_BC_ZERO -- plain zeros.  Such grids run
 * a general point-wise ghost path (one thread per padded point, the tensor
 * sums of Alg. SM1/SM2 evaluated directly) and the per-block stage kernel;
 * the criterion's extended region stops at the boundary, neighbours and the
 * update step never reach beyond it, and every adaptation iteration
 * ghost-fills every field in full with FP64 padded blocks.
 * mr_ghost_fill_static returns MR_ERR_UNSUPPORTED on them, and
 * mr_grid_create / mr_workspace_size refuse MR_GRID_INDEPENDENT_TREES
 * combined with a bounded axis (MR_ERR_UNSUPPORTED). */
#define MR_GRID_BOUNDED_X 8
#define MR_GRID_BOUNDED_Y 16
#define MR_GRID_BOUNDED_Z 32
#define MR_GRID_BC_DIRICHLET0 64
#define MR_GRID_BC_ZERO 128

typedef struct {
  int nleaf;
  int count_per_level[32];
  int min_level, max_level;
} mr_stats;

typedef struct mr_grid mr_grid;

/* Last error message recorded by any call in this process (static string). */
const char *mr_last_error(void);

/* Device workspace (bytes) a grid with this descriptor needs.  Covers the
 * block pool (nfields user fields, two RK temporaries, and the second pool
 * adaptation writes into), the padded ghost buffers for the widest shell the
 * adaptation uses (Table 2.2), and the octree tables (the owner map holds
 * prod_d ntree[d]*2^lmax int32 entries). */
int mr_workspace_size(const mr_grid_desc *desc, size_t *bytes);

/* Create a grid on the current CUDA device.  workspace: device pointer,
 * 256-byte aligned, at least mr_workspace_size bytes, owned by the caller.
 * lev/anc: host arrays of nleaf leaves (any order) forming a 2:1-balanced
 * complete forest (face, edge and corner neighbours differ by <= 1 level).
 * Synchronises.  Errors: MR_ERR_INVALID (bad descriptor, overlapping or
 * missing leaves), MR_ERR_NOMEM (capacity/workspace), MR_ERR_BALANCE.      */
int mr_grid_create(const mr_grid_desc *desc, void *workspace, size_t workspace_bytes,
                   const int32_t *lev, const int32_t *anc, int nleaf, mr_grid **out);
int mr_grid_destroy(mr_grid *grid);

/* Current leaves in slot (Morton) order and their Morton keys (keys may be
 * NULL).  Synchronises.  cap: capacity of the host arrays.                 */
int mr_grid_leaves(mr_grid *grid, int32_t *lev, int32_t *anc, uint64_t *keys, int cap,
                   int *nleaf);

/* Copy a whole field in (from host or device memory) or out, in the field
 * layout above with the current leaf count.  Copies to host synchronise.   */
int mr_field_copy_in(mr_grid *grid, int fid, const void *src, int src_on_device);
int mr_field_copy_out(mr_grid *grid, int fid, void *dst, int dst_on_device);

/* Evaluate an analytic field on the device at every point (MR_INIT_*). */
int mr_field_set(mr_grid *grid, int fid, int kind, const double *params, int nparams);

/*
 * Ghost reconstruction (Alg. SM1 then Alg. SM2, Sec. 2.2.2 and 2.2.4) of
 * field fid with a shell of G points:
 *   1. every leaf takes same-level points as copies, points inside a coarser
 *      leaf from the zero-detail refinement (J^s, K^s) of the coarse-level
 *      values, points inside a finer leaf as the coincident value;
 *   2. leaves next to a coarser leaf substitute their band (Table 2.2 coarse
 *      region extension, mirrored) degree by degree (eqs 2.23, 2.27-2.29);
 *      the substituted values overwrite the field;
 *   3. points inside a finer leaf F become the tensor H^a coarsening of F's
 *      data from steps 1-2.
 * padded: device buffer of nleaf*(nb+2G)^3 elements receiving the padded
 * blocks, or NULL (only the substitution of the field happens then).
 * G: 1..MR_MAX_SHELL(=12) and G <= nb/2 (MR_ERR_BALANCE otherwise).        */
int mr_ghost_fill(mr_grid *grid, int fid, int G, void *padded);

/* As mr_ghost_fill, but the padded blocks are computed and returned in FP64
 * (from the stored field values, FP32 fields upcast): the path the
 * adaptation uses, so that refinement and coarsening decisions do not depend
 * on FP32 rounding.  padded: nleaf*(nb+2G)^3 doubles or NULL.             */
int mr_ghost_fill64(mr_grid *grid, int fid, int G, double *padded);

/* Ghost fill that allocates nothing, for callers that cannot obtain device
 * memory when they call it (no cudaMalloc, no pool or framework allocator:
 * for example code running inside another runtime's fixed memory budget).
 * The paper has no counterpart: this is a packaging variant of
 * mr_ghost_fill, with the same arguments, semantics and results (the same
 * kernels in the same precision: where mr_ghost_fill computes the padded
 * blocks of an FP32 grid in FP64 -- internal shells wider than the stencil
 * shell -- so does this call, and it returns MR_ERR_UNSUPPORTED wherever
 * mr_ghost_fill does).
 * Its scratch -- the padded blocks and the fine-to-coarse side buffer --
 * lives in one 64 MiB array of static device memory that every GPU loading
 * the library keeps until the process exits; grids whose
 * 2 * nleaf * (nb + 2*Gi)^3 padded elements (Gi >= G: the internal shell;
 * 8 bytes each on the FP64 path, else the field's element size) exceed it
 * are rejected with MR_ERR_NOMEM.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current;
 * make that first call before any stream capture (a first call made while
 * the grid's stream is capturing is refused with MR_ERR_INVALID).  All calls
 * share the array: calls that overlap on the GPU (different streams, or
 * grids used concurrently) race on it; serialise them.  Nothing in the array
 * needs to start at zero (every value read is written first in the same
 * call).                                                                  */
int mr_ghost_fill_static(mr_grid *grid, int fid, int G, void *padded);

/* Wait for the grid's stream and report device-side errors recorded by the
 * kernels since the last check (MR_ERR_BALANCE: a ghost point was owned by
 * a leaf more than one level away, or a shell exceeded the stored padding). */
int mr_sync(mr_grid *grid);

/* rhs = -sum_d (F_{i+1/2} - F_{i-1/2}) / h for d(phi)/dt + div(u phi) = 0,
 * with u = u_const (host, 3 doubles).  Includes the ghost fill of phi (and
 * its substitution).  scheme: MR_CONS3 / MR_CONS5 / MR_WENOZ5.             */
int mr_rhs_advect(mr_grid *grid, int phi_fid, const double *u_const, int out_fid, int scheme);

/* RK3-TVD stage (supplementary "Time integration scheme"):
 *   stage 0: out = y + dt*rhs
 *   stage 1: out = 3/4 u + 1/4 (y + dt*rhs)
 *   stage 2: out = 1/3 u + 2/3 (y + dt*rhs)
 * elementwise over the current leaves; out may alias u or y.               */
int mr_rk_stage(mr_grid *grid, int stage, double dt, int u_fid, int y_fid, int rhs_fid,
                int out_fid);

/* As mr_rhs_advect with a velocity field u = (field vel_fid[0], vel_fid[1],
 * vel_fid[2]) instead of a constant: interface velocity (u_i + u_{i+1})/2
 * selects the upwind side.  The grid needs MR_GRID_VELOCITY.  The velocity
 * components are substituted and ghost-filled once per tree (the velocity
 * does not change in time, and substitution is idempotent, so these equal
 * the ghosts of a fill at every stage): the cache is
 * rebuilt after every adaptation that changes the leaves; a caller that
 * writes new velocity values must call mr_velocity_invalidate.            */
int mr_rhs_advect_vel(mr_grid *grid, int phi_fid, const int *vel_fid, int out_fid, int scheme);

/* One RK3 step of phi (in place) advected by the velocity fields vel_fid[3]
 * (see mr_rhs_advect_vel).                                                 */
int mr_step_vel(mr_grid *grid, int phi_fid, double dt, const int *vel_fid, int scheme);

/* As mr_step_vel with a time-dependent velocity s(t) u(x): stage_scale[3]
 * (host) are s at the three RK3 stage times t, t + dt, t + dt/2 (Sec. 5.3
 * multiplies the deformation field by cos(pi t / 3)).  The scale multiplies
 * the velocity before the interface velocity picks the upwind side, so a
 * negative scale reverses the flow.  MR_ERR_INVALID for a non-finite scale. */
int mr_step_vel_scaled(mr_grid *grid, int phi_fid, double dt, const int *vel_fid, int scheme,
                       const double *stage_scale);

/* Stable time step (Sec. 5.1 takes dt = CFL h_f / U; in 3D the reading used
 * here is dt = CFL * h_min / max_x sum_d |u_d|, which equals it for an
 * axis-aligned velocity): h_min is the spacing of the finest leaf present,
 * and the velocity is either the constant u_const (host, 3 doubles) or the
 * fields vel_fid[3] (exactly one of the two non-NULL), whose maximum of
 * |u_0| + |u_1| + |u_2| over every point is reduced on the device in FP64
 * (max is exact, so the result is independent of the order).  *dt (host)
 * receives +inf for a zero velocity.  Synchronises.  Errors:
 * MR_ERR_INVALID for a non-positive or non-finite CFL, both or neither of
 * u_const / vel_fid, or a bad field id.                                  */
int mr_dt(mr_grid *grid, double cfl, const double *u_const, const int *vel_fid, double *dt);

/* CUDA-graph mode of the RK steps (mr_step, mr_step_vel, mr_step_vel_scaled):
 * with enable = 1 a step's kernels (the three stages) are captured once into
 * a CUDA graph on the grid's stream and the graph is replayed by every later
 * step with the same key -- step kind, field ids, dt, velocity or stage
 * scales, scheme, diffusion term, leaves (any adaptation changes the key)
 * and pools; a different key captures the step again.  Results are bit-for-
 * bit those of the stream-ordered step.  The velocity cache is rebuilt
 * outside the capture.  While a step is being captured the launch registry
 * records no events (mr_profile times steps run without graphs); replays
 * count their kernels in mr_launch_count.  enable = 0 releases the graph
 * (synchronises).  mr_graph_replays returns the replays since creation.    */
int mr_use_graphs(mr_grid *grid, int enable);
int mr_graph_replays(mr_grid *grid, long long *n);

/* Launch-shape autotuner.  With enable = 1, the first launch of each tunable
 * kernel configuration (kernel, wavelet, nb, precision, shell, mode) on this
 * grid times every candidate CTA size on the grid's own data -- the ghost
 * gather, pre-pass and merge, the criterion, the interpolation, and the fused
 * stage kernel (one grid line per thread or two), each only on launches that
 * overwrite their outputs from unchanged inputs, so repeating them changes
 * nothing -- and keeps the fastest in a table shared by every grid of the
 * process (later launches of that configuration use it whether or not their
 * grid tunes).  Results do not depend on the CTA size: every output point is
 * computed with the same arithmetic whatever the size.  On FP32 grids left
 * at mr_set_stage_kernel(grid, 0) the tuner also picks the faster of the two
 * stage kernels (see there: equal up to the last bit).  No tuning happens
 * while a step is being captured into a CUDA graph.  The paper has no
 * counterpart (its code runs one block after the other per MPI rank).
 * mr_autotune_table writes one line per tuned configuration (chosen size
 * and the time of every candidate) into buf (NUL-terminated; MR_ERR_NOMEM
 * if truncated); *nentries receives the number of entries.
 * mr_autotune_clear empties the table.                                   */
int mr_autotune(mr_grid *grid, int enable);
int mr_autotune_table(char *buf, size_t len, int *nentries);
int mr_autotune_clear(void);

/* Which kernel runs the FP32 stage (ghost faces + rhs + RK3 stage, the
 * supplement's "Finite differences" and "Time integration" schemes) of
 * mr_step, mr_step_vel, mr_step_vel_scaled, mr_rhs_advect and
 * mr_rhs_advect_vel: 1 = k_fused (the ghost-extended block in shared memory,
 * one thread per grid line), 2 = k_march (the block traversed plane by plane,
 * one thread per grid column, two CTAs per SM), 0 = chosen by the autotuner
 * on grids with mr_autotune enabled (the faster of the two for that
 * configuration), else k_fused (the default).  k_march
 * needs 12 <= nb <= 24; other block sizes always use k_fused.  Both evaluate
 * every value with the same operations in the same order; they may differ in
 * the last bit where the compiler fuses a multiply and an add differently
 * (measured within 1e-6 of the field maximum).  FP64 grids are unaffected.
 * MR_ERR_INVALID for which outside 0..2.                                  */
int mr_set_stage_kernel(mr_grid *grid, int which);

/* Bounds of the adaptation loops: mr_adapt runs at most max_iter iterations
 * (default 64) and each iteration at most max_sweeps policy sweeps (default
 * 256); beyond either the call returns MR_ERR_TIMEOUT with the leaves of the
 * last completed iteration in place.  MR_ERR_INVALID for values < 1.      */
int mr_set_adapt_limits(mr_grid *grid, int max_iter, int max_sweeps);

/* Drop the cached ghost-filled velocity (after changing velocity values). */
int mr_velocity_invalidate(mr_grid *grid);

/* One RK3 step of phi (in place): three times ghost fill + fused rhs/stage,
 * using the grid's two internal temporaries.  Constant velocity u_const.   */
int mr_step(mr_grid *grid, int phi_fid, double dt, const double *u_const, int scheme);

/* Per-leaf max |detail| over the block and its coarse-region extension
 * (Sec. 2.2.5, eqs 2.24-2.26), from the field as stored after a ghost fill
 * with the adaptation shell in FP64: evaluated in FP64 on FP64 grids and in
 * float pairs (two FP32 numbers, about 48 significant bits, on the FP32
 * pipe) on FP32 grids; either agrees with exact arithmetic to about 1e-14 of
 * the field maximum.  maxdet: device array of nleaf doubles.               */
int mr_criterion(mr_grid *grid, int fid, double *maxdet);

/* Grid adaptation (Alg. SM3) of every field, driven by field crit_fid, run
 * until no leaf changes (at most 64 iterations, else MR_ERR_TIMEOUT).
 * flags: MR_ADAPT_REFINE | MR_ADAPT_COARSEN, optionally | MR_ADAPT_OTHERS_FP64
 * (the criterion field always adapts in FP64 arithmetic; the other fields of
 * an FP32 grid in FP32 unless that flag is given).  Synchronises once per
 * iteration; *n_changed (may be NULL) receives the total number of leaves
 * that refined or coarsened.                                               */
int mr_adapt(mr_grid *grid, int crit_fid, double eps_refine, double eps_coarsen, int flags,
             int *n_changed);

/* One iteration of mr_adapt; *n_changed receives the leaves changed. */
int mr_adapt_iter(mr_grid *grid, int crit_fid, double eps_refine, double eps_coarsen,
                  int flags, int *n_changed);

/* Block norms (max |detail| per leaf, Sec. 2.2.5) that the last adaptation
 * iteration took its decisions with, in the slot order of the tree that
 * iteration started from (*n leaves; after an mr_adapt that converged, the
 * current tree).  dst: nleaf doubles (host or device), or NULL to query *n.
 * Synchronises.                                                           */
int mr_last_block_norms(mr_grid *grid, double *dst, int cap, int *n);

/* Sum over leaves of h^3 * sum(phi) in FP64 (eq 2.18 with p = 0), written
 * to *mass (host).  Synchronises.                                          */
int mr_mass(mr_grid *grid, int fid, double *mass);

/* Leaf counts.  Synchronises. */
int mr_query(mr_grid *grid, mr_stats *stats);

/* Diffusion term of the stencil step: every following mr_rhs_advect,
 * mr_rhs_advect_vel, mr_step and mr_step_vel adds nu times the central
 * Laplacian of the same ghost-filled field to the advection right-hand side,
 *   d phi / dt = -div(u phi) + nu * Laplacian(phi),
 * order 2: DIFF-2, sum_d (f[i-1] - 2 f[i] + f[i+1]) / h^2;
 * order 4: DIFF-4, sum_d (-f[i-2] + 16 f[i-1] - 30 f[i] + 16 f[i+1] - f[i+2]) / (12 h^2)
 * (Sec. 4.3 names second- and fourth-order central Laplacians; h is the
 * leaf's grid spacing).  order 0 or nu = 0 removes the term (the default).
 * The time step stays the caller's: explicit diffusion also needs
 * dt <= c h_min^2 / nu.  Errors: MR_ERR_INVALID for a negative or non-finite
 * nu or another order.  No device work. */
int mr_set_diffusion(mr_grid *grid, double nu, int order);

/* Launch registry (the per-operation timers of the library).
 * mr_profile(grid, 1) clears the records and brackets every following kernel
 * launch with CUDA events on the grid's stream (up to 4096 launches);
 * mr_profile(grid, 0) stops recording.  mr_profile_read synchronises and
 * returns, for kernel id kid (0 .. MR_NUM_KERNELS-1), the summed device time
 * of its recorded launches, their number and the kernel's name (static
 * string).  mr_launch_count returns every kernel launch since creation.    */
#define MR_NUM_KERNELS 18
int mr_profile(mr_grid *grid, int enable);
int mr_profile_read(mr_grid *grid, int kid, double *total_ms, int *nlaunch, const char **name);
int mr_launch_count(mr_grid *grid, long long *n);
/* Algorithmic bytes of the recorded launches of kernel kid (the roofline
 * numerator), accumulated on the device while profiling is on.  Defined for
 * the ghost pre-pass (kid 0) and the ghost gather (kid 1): every point of the
 * requested shell G of each leaf the launch reconstructs is written once and
 * its source value read once, ((nb + 2G)^3 - nb^3) * (source + padded
 * element size) per leaf -- the internal shell the kernels also fill (wider
 * where substitution or the fine-to-coarse coarsening reads further) counts
 * as time, not bytes; leaves a launch skips (need mask, stencil pre-pass of
 * a leaf without coarser neighbours) count zero.  0 for other kernels.
 * Synchronises; *bytes (host) receives the sum since the last mr_profile(1). */
int mr_profile_bytes(mr_grid *grid, int kid, double *bytes);

/* Compute throughput of the current device, measured by short probe
 * kernels (8 CTAs of 256 threads per SM, 8 independent dependency chains per
 * thread; about half a second): out[0] FP32 fused multiply-add TFLOP/s,
 * out[1] FP64 FMA TFLOP/s, out[2] FP32 fast divisions (__fdividef) in G/s,
 * out[3] FP32 IEEE divisions G/s, out[4] FP64 divisions G/s.  These are the
 * compute-roofline denominators of the stencil and wavelet kernels beside
 * the copy bandwidth (the paper has no counterpart: it reports CPU-cluster
 * timings only).  Runs on the legacy stream and synchronises it; allocates
 * nothing.  out: host array of MR_NUM_PEAKS doubles.                     */
#define MR_NUM_PEAKS 5
int mr_device_peaks(double *out);

/* Device pointer of field fid (slot-major layout above). */
int mr_field_ptr(mr_grid *grid, int fid, void **ptr);

#ifdef __cplusplus
}
#endif
#endif /* MRGB_H */
