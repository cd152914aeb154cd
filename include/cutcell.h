/*
 * cutcell.h -- C ABI of the GB300 cut-cell step library (libcutcell.so).
 *
 * The library advances the fully compressible, quasi-flux-form equations of
 * Yamazaki, Satomura & Nikiforakis, "3D cut-cell modelling for
 * high-resolution atmospheric simulations" (arXiv 1509.02572), Sec 2.1
 * (Eqs. momentum_u .. continuity), on Cartesian grids cut by bilinear terrain
 * (Sec 2.3), with the finite-volume discretisation and three-step velocity of
 * Sec 2.4 and leapfrog + Robert-Asselin time stepping (Sec 2.2).
 *
 * Conventions shared by every entry point
 *   - A model holds one or more independent domains ("ensemble"); each domain
 *     is one uniform block, periodic in x and y (cyclic lateral boundaries,
 *     Sec 3), with a free-slip (or no-slip) terrain surface and a rigid lid.
 *   - The library owns all device memory it allocates; the caller owns every
 *     host buffer it passes.  Host buffers are FP64 for every precision mode.
 *   - Every call returns a cc_status; CC_OK is 0.  On error the message of
 *     cc_last_error() describes the failure.  A model is bound to the CUDA
 *     stream given at creation; calls on one model are not thread-safe.
 *   - Cell (i,j,k), 0 <= i < nx, 0 <= j < ny, 0 <= k < nz, has its centre at
 *     ((i+1/2)dx, (j+1/2)dy, (k+1/2)dz).  Corner (I,J,K) sits at
 *     (I dx, J dy, K dz) and carries the co-located velocity components of the
 *     semi-staggered arrangement (Sec 2.3, Fig. 7).
 *   - Host cell arrays: nz*ny*nx doubles, x fastest.  Host corner arrays:
 *     (nz+5)*ny*nx doubles for levels K = -2 .. nz+2, x fastest (the levels
 *     below the floor and above the lid carry boundary values).
 */
#ifndef CUTCELL_H
#define CUTCELL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  CC_OK = 0,
  CC_EINVAL = 1,    /* invalid argument (null pointer, bad size, bad index) */
  CC_ECUDA = 2,     /* a CUDA runtime call failed                           */
  CC_EGEOM = 3,     /* merge or boundary stencil cannot be formed           */
  CC_ENUMERIC = 4,  /* NaN or Inf in the state (cc_diagnostics), or the step watchdog raised */
  CC_ENOMEM = 5,    /* device allocation failed                             */
  CC_ESTATE = 6,    /* call out of order (e.g. step before geometry)        */
  CC_ETIMEOUT = 7   /* a bounded wait inside a kernel ran out (step watchdog) */
} cc_status;

enum { CC_FP64 = 0, CC_FP32 = 1 };
/* prognostic fields; CC_UB = boundary-point velocity (3 per column corner) */
enum { CC_RHOP = 0, CC_PP = 1, CC_MX = 2, CC_MY = 3, CC_MZ = 4, CC_UB = 5 };

/* One domain.  Reading of the paper's constants: g, R, cp, p0 physical
 * constants (p0 = 1e5 Pa, Sec 2.1); base state of constant Brunt-Vaisala
 * frequency N with surface potential temperature theta0 at pressure p_surf;
 * ra_nu Robert-Asselin coefficient (Sec 2.2); c4 strength of the fourth-order
 * artificial diffusion (Sec 2.1), applied as -(c4/(16 dt)) sum delta^4 on
 * momentum and (rho theta)'; sponge: Rayleigh damping of momentum toward
 * (rho_bar U, 0, 0) above (1 - sponge_frac) of the domain height with peak
 * rate tau_max (Sec 3, Klemp-Lilly layer); bc_slip 1 = free slip (Sec 3),
 * 0 = no slip (Sec 2.4). */
typedef struct {
  int nx, ny, nz;
  double dx, dy, dz;
  double dt;
  double U, N, theta0, p_surf, p0, g, R, cp;
  double ra_nu, c4, sponge_frac, tau_max;
  int bc_slip;
} cc_config;

/* Conservation and sanity diagnostics of one domain, level "current". */
typedef struct {
  double mass;        /* sum over merged cells of V_G rho'_G (kg)           */
  double mass_comp;   /* compensation term of the Neumaier sum              */
  double max_u;       /* max |u| over corners above the terrain (m/s)       */
  double max_w;       /* max |w| over corners above the terrain (m/s)       */
  long long nonfinite;/* number of non-finite prognostic values             */
  long long steps;    /* steps taken since cc_init_state                    */
  double heat;        /* sum over merged cells of V_G (rho theta)'_G (kg K);
                         the scheme does not conserve it (diagnostic)       */
  double heat_comp;   /* compensation term of its Neumaier sum              */
} cc_diag;

typedef struct cc_model cc_model;

/* Create a model of n independent domains (cfgs[0..n-1]) computing in
 * precision CC_FP64 or CC_FP32 (FP32 perturbations about an FP64-evaluated
 * hydrostatic base state; geometry always FP64).  stream: a cudaStream_t or
 * NULL for the default stream.  Allocates all device memory.  The domains
 * share the physical constants R, cp and p0 (CC_EINVAL otherwise; the other
 * parameters are free per domain).  *out receives the model; on failure *out
 * is NULL and the status says why. */
cc_status cc_create(const cc_config *cfgs, int n, int precision, void *stream, cc_model **out);

/* Release every device and host resource of the model.  Null is accepted. */
cc_status cc_destroy(cc_model *m);

/* Last error message of the model (static storage owned by the model), or of
 * the last failed cc_create when m is NULL. */
const char *cc_last_error(const cc_model *m);

/* Terrain of domain d: corner heights h(I dx, J dy) for I < nx, J < ny
 * (periodic), ny*nx doubles x fastest, every value >= 0 and below the lid.
 * Copied to the device; Sec 2.3, Eq. bilin and its coefficients. */
cc_status cc_set_terrain(cc_model *m, int d, const double *corner_h);

/* Analytic terrain shapes of cc_set_terrain_analytic. */
enum { CC_HILL_BELL = 0, CC_HILL_ELLIPSOID = 1, CC_HILL_COSINE = 2 };

/* Terrain of domain d from an analytic hill evaluated on the GPU at the
 * corners (I dx, J dy), I < nx, J < ny.  params = {h0, a, xc, yc}: height,
 * half-width (bell) or radius (ellipsoid, cosine), and the centre in metres
 * from corner (0, 0); r is the horizontal distance from the centre.
 *   CC_HILL_BELL       h0 / (1 + r^2/a^2)^(3/2)          (Sec 3.1.1)
 *   CC_HILL_ELLIPSOID  h0 sqrt(max(0, 1 - r^2/a^2))      (Sec 3.1.2; the
 *                      hemisphere when h0 = a)
 *   CC_HILL_COSINE     h0 (1 + cos(pi r / a)) / 2 for r < a, else 0 (appendix)
 * The heights then pass the checks of cc_set_terrain; when one fails the
 * domain is left without terrain (CC_EINVAL).  CC_EINVAL also for an
 * unknown kind, h0 < 0, a <= 0 or non-finite parameters. */
cc_status cc_set_terrain_analytic(cc_model *m, int d, int kind, const double *params);

/* Corner heights of domain d as last set, ny*nx doubles x fastest, into a
 * host array.  CC_ESTATE before the domain has terrain. */
cc_status cc_get_terrain(const cc_model *m, int d, double *corner_h);

/* Build the cut-cell geometry of every domain on the GPU in FP64 (Sec 2.3 and
 * 2.4): column gradients (Eqs. xgrad, ygrad), volumes and apertures by exact
 * integration of the bilinear surface, cell classes, merge targets of the
 * Fig. 6 pseudocode, merge groups, velocity-point classes, boundary-point
 * normals and nearest-plane stencils, merged-face interpolation weights,
 * and the compacted group lists.  CC_EGEOM when a merge chain ends below the
 * terrain or loops, or a stencil cannot be formed. */
cc_status cc_build_geometry(cc_model *m);

/* Copy domain d's geometry to host buffers (any pointer may be NULL):
 *   vf, ax, ay: nz*ny*nx (volume fraction; apertures of the faces x = I dx and
 *   y = J dy of cell (I,J,k)); az: (nz+1)*ny*nx (face z = K dz of column
 *   (i,j)); cls: nz*ny*nx (0 below terrain, 1 full, 2 cut, 3 absorbed);
 *   root: nz*ny*nx (cell id (k*ny+j)*nx+i of the group's host, -1 below
 *   terrain); vcls: (nz+5)*ny*nx corner classes for K = -2..nz+2 (0 at or
 *   below terrain, 1 predicted, 2 merged face, 3 lid). */
cc_status cc_get_geometry(const cc_model *m, int d, double *vf, double *ax, double *ay, double *az,
                          int8_t *cls, int32_t *root, int8_t *vcls);

/* Boundary-point and merged-face stencils of domain d (any pointer may be
 * NULL): per column corner (ny*nx): bK level of the nearest plane, bI, bJ its
 * low corner, ba, bb the weights alpha and beta, bn the unit normal (3 each);
 * per corner ((nz+5)*ny*nx): mK the level of the predicted point above a
 * merged-face point, mg its weight gamma. */
cc_status cc_get_stencils(const cc_model *m, int d, int32_t *bK, int32_t *bI, int32_t *bJ, double *ba,
                          double *bb, double *bn, int32_t *mK, double *mg);

/* Compacted merge-group list of domain d, ascending by host cell id.
 * *ngroups and *nmembers receive the sizes; if host and start/members are
 * non-NULL they receive: host[g], start[g] (ngroups+1 entries), members
 * (ascending cell ids of each group, host included).  Call once with NULLs to
 * get the sizes. */
cc_status cc_get_groups(const cc_model *m, int d, int *ngroups, int *nmembers, int32_t *host,
                        int32_t *start, int32_t *members);

/* Initial state of every domain: zero perturbations, uniform wind U on the
 * predicted velocity points, diagnosed boundary / merged-face / lid values. */
cc_status cc_init_state(cc_model *m);

/* Replace one field of domain d at level 0 (filtered previous) or 1 (current)
 * with a host array in the layout above (cells, corners or 3*ny*nx for
 * CC_UB).  The next step uses the uploaded values.  Copies through pinned
 * staging; synchronous with respect to the model's stream. */
cc_status cc_upload_state(cc_model *m, int d, int field, int level, const double *host);

/* Copy one field of domain d at level 0 or 1 to a host array (same layout). */
cc_status cc_download_state(const cc_model *m, int d, int field, int level, double *host);

/* Derived output fields of cc_download_derived. */
enum { CC_U = 0, CC_V = 1, CC_W = 2, CC_THETA_P = 3 };

/* A derived field of domain d at level 0 or 1 into a host array.
 *   CC_U, CC_V, CC_W (level 1 only: the boundary-point velocity is
 *     diagnosed for the current level alone): the velocity at the corners
 *     K = 0 .. nz,
 *     (nz+1)*ny*nx doubles x fastest, as every flux formula uses it (Sec 2.4):
 *     at corners at or below the terrain the boundary-point velocity of the
 *     column, elsewhere momentum over the corner density (the mean total
 *     density of the 8 cells around the corner), in the model's arithmetic;
 *   CC_THETA_P: the potential-temperature perturbation theta - theta_bar of
 *     every cell, nz*ny*nx doubles, with theta = rho theta / rho and rho theta
 *     from the pressure by the equation of state (Sec 2.1), evaluated in FP64
 *     from the stored perturbations; absorbed cells carry their group's
 *     state, cells below the terrain give 0.
 * Computed on the GPU; synchronous with respect to the model's stream.
 * CC_EINVAL for a bad domain, field or level, CC_ESTATE before a state. */
cc_status cc_download_derived(const cc_model *m, int d, int which, int level, double *host);

/* Global error norms of the appendix accuracy test ("Estimation of global
 * accuracy"): the corner velocity component `which` (CC_U, CC_V, CC_W) of the
 * current level of domain da of model a against domain db of model b, a
 * finer solution of the same problem taken as exact, at the corners the two
 * grids share, over the N shared corners of a with K dz > zmin (the grid
 * points above the hill top; zmin = -inf takes every corner level 0 .. nz):
 *   out[0] = L1 = (1/N) sum |psi_a - psi_b|,
 *   out[1] = L2 = ((1/N) sum (psi_a - psi_b)^2)^(1/2),   out[2] = N.
 * The spacings must be in one ratio dx_a / dx_b = p / q >= 1 (integers in
 * lowest terms, q <= 16) in x, y and z over the same extents (CC_EINVAL
 * otherwise); corner I of a is corner I p / q of b when q divides I, and only
 * those corners count (every corner for an integer ratio).  The models may
 * differ in precision.  Both on the current device; waits for b's stream, computes on
 * a's and synchronises it.  Errors are reported on a. */
cc_status cc_error_norms(const cc_model *a, int da, const cc_model *b, int db, int which, double zmin, double *out);

/* The same transfers queued on the model's stream without waiting (no
 * counterpart in the paper; for callers that move whole states every step):
 * the host buffer must stay valid and unchanged (upload) or unread
 * (download) until the stream has passed the transfer (cc_synchronize).
 * With pinned host buffers the copies run asynchronously; transfers, steps
 * and other calls on the model stay in stream order. */
cc_status cc_upload_state_async(cc_model *m, int d, int field, int level, const double *host);
cc_status cc_download_state_async(const cc_model *m, int d, int field, int level, double *host);

/* The same four transfers with FP32 host buffers (same layouts), for FP32
 * models only, whose prognostic fields are FP32: the values are copied
 * unchanged, with half the host-device bytes of the FP64 calls.  An FP64
 * model returns CC_EINVAL.  The _async forms follow the rules above. */
cc_status cc_upload_state_f32(cc_model *m, int d, int field, int level, const float *host);
cc_status cc_download_state_f32(const cc_model *m, int d, int field, int level, float *host);
cc_status cc_upload_state_f32_async(cc_model *m, int d, int field, int level, const float *host);
cc_status cc_download_state_f32_async(const cc_model *m, int d, int field, int level, float *host);

/* The two-time-level state of every domain in one host buffer (no
 * counterpart in the paper; for callers that move whole states every step):
 * for each domain d = 0 .. ndom-1 in turn, the fields CC_RHOP, CC_PP, CC_MX,
 * CC_MY, CC_MZ in that order, each at level 0 then level 1, every array in
 * the host layout of cc_upload_state, back to back.  cc_state_elems sets *n
 * to the buffer's element count.  cc_upload_all_async and
 * cc_upload_all_f32_async (FP32 models only, FP32 host values copied
 * unchanged) queue the upload on the model's stream as the _async transfers
 * do, with one host-to-device copy per domain instead of one per array, into
 * a device staging buffer of the whole state made on first use (CC_ENOMEM
 * when it cannot be made); the host buffer must stay valid and unchanged
 * until cc_synchronize.  CC_EINVAL for a null argument or an FP64 model with
 * FP32 values, CC_ESTATE before a state. */
cc_status cc_state_elems(const cc_model *m, long long *n);
cc_status cc_upload_all_async(cc_model *m, const double *host);
cc_status cc_upload_all_f32_async(cc_model *m, const float *host);

/* Checkpoint and resume (no counterpart in the paper; long runs are split
 * over several jobs).  cc_save writes the whole state of every domain -- all
 * four time levels of the five fields and of the boundary-point velocity in
 * the device layout and the model's precision, with the time-level roles and
 * step counts -- to the file `path` (synchronises the stream).  cc_load reads
 * it into a model created with the same configurations and precision whose
 * geometry is built; the model then continues bit for bit as the saved one
 * would.  CC_EINVAL when the file is not a checkpoint, is truncated, cannot be
 * opened, or does not match the model's precision, domain count or sizes;
 * a file found truncated after the header checks leaves the model without a
 * state (CC_ESTATE on cc_step until cc_init_state or a good cc_load). */
cc_status cc_save(const cc_model *m, const char *path);
cc_status cc_load(cc_model *m, const char *path);

/* Advance every domain by n steps (leapfrog; the first step after
 * cc_init_state is forward Euler).  Asynchronous on the model's stream.
 *
 * Step watchdog (no counterpart in the paper): every step's full-cell stencil
 * raises a flag when it writes a non-finite value or when a corner's
 * advective Courant number sum_d |u_d| dt / d_d exceeds 1 (the stability
 * limit of centred leapfrog advection), and a third when one of its bounded
 * waits for the TMA copies of a plane ran out (after two seconds; the block
 * then stops, waits a bounded time for its copies in flight and returns, so
 * the step is void but the context stays usable).  Each call queues a copy of
 * the flags to the host after its steps; a later cc_step whose copy has
 * arrived (checked without waiting) and cc_synchronize return CC_ENUMERIC
 * (first two) or CC_ETIMEOUT (third), with the reason in cc_last_error,
 * instead of stepping on.  cc_init_state and cc_load clear the flags. */
cc_status cc_step(cc_model *m, int n);

/* Failure detection test (no counterpart in the paper): with on != 0, every
 * TMA plane barrier of the FP32 stencil's refined-box kernel expects 16 bytes
 * more than its copies bring, so each of its bounded waits runs out and the
 * step watchdog reports CC_ETIMEOUT; nothing faults and the context stays
 * usable.  Periodic domains (cyclic gather, no barriers) are not affected.
 * Off by default; drops the captured graphs. */
cc_status cc_inject_wait_timeout(cc_model *m, int on);

/* CUDA graphs (no counterpart in the paper): with graphs on (the default),
 * cc_step captures the launches of one step (one cycle of level 0 of a
 * refined model) once per arrangement of time levels and schedules, on a
 * private stream, and replays the graph on the model's stream; the results
 * are the same bits as launching the kernels one by one.  Forward-Euler
 * starts and steps taken with profiling on always launch directly. */
cc_status cc_graphs_enable(cc_model *m, int on);

/* Diagnostics of domain d at the current level; synchronises the stream.
 * Returns CC_ENUMERIC when non-finite values are present. */
cc_status cc_diagnostics(cc_model *m, int d, cc_diag *out);

/* Wait for all work queued on the model's stream; CC_ENUMERIC or
 * CC_ETIMEOUT if the step watchdog (see cc_step) was raised by a step since
 * the last cc_init_state or cc_load. */
cc_status cc_synchronize(cc_model *m);

/* Number of kernels the last cc_step launched (for launch accounting). */
long long cc_last_launch_count(const cc_model *m);

/* Schedule of the full-cell stencil (no counterpart in the paper): tile
 * height in y (FP32: 16 or 8, FP64: 8 or 4; tiles are 32 cells wide) and the
 * number of work items one launch aims for (304 or 912; the z-columns are cut
 * into chunks to reach it).  The schedule changes only how the work is
 * distributed over thread blocks, never the result (bit for bit).
 * cc_autotune times every schedule (FP32: with each warp-role form, below)
 * reps times on the model's current state
 * and keeps the fastest, for the whole ensemble or for each level of a
 * refined model; the state is left unchanged (the stencil writes only the
 * levels the next step overwrites).  Needs cc_init_state; synchronises.
 * cc_get_schedule / cc_set_schedule read or set the schedule of domain d
 * (of an ensemble: the one shared by all domains); CC_EINVAL for a pair not
 * in the list. */
cc_status cc_autotune(cc_model *m, int reps);
cc_status cc_get_schedule(const cc_model *m, int d, int *tile_y, int *items_per_launch);
cc_status cc_set_schedule(cc_model *m, int d, int tile_y, int items_per_launch);

/* Warp roles of the FP32 full-cell stencil (no counterpart in the paper; the
 * paper's OpenMP code updates all variables of a cell in one thread).
 * roles = 1: every thread updates rho', p' and the three momenta of its two
 * cells.  roles = 2: each thread block holds two warpgroups over the same
 * tile, one updating rho' and p' (Sec 2.4, the scalar fluxes and their
 * divergence), the other the momenta (Eqs. momentum_u_d .. momentum_w_d);
 * the two read the same staged planes, and each thread keeps the live values
 * of one update only, so that twice as many warps fit per SM.  The result is
 * the same either way.  cc_autotune times both with every schedule and keeps
 * the fastest pair.  cc_get_warp_roles / cc_set_warp_roles read or set the
 * roles of domain d's launch (of an ensemble: the one shared by all domains;
 * of a refined model: every block of d's level).  CC_EINVAL for roles other
 * than 1 or 2, or 2 on an FP64 model (its stencil has one form). */
cc_status cc_get_warp_roles(const cc_model *m, int d, int *roles);
cc_status cc_set_warp_roles(cc_model *m, int d, int roles);

/* Kernel timing for measurement (no counterpart in the paper).  When enabled,
 * cc_step brackets each stage with CUDA events on the model's stream;
 * cc_profile_read synchronises and returns the summed device time (ms) and the
 * number of timed launches of one stage since the last cc_profile_reset. */
enum { CC_K_FULL = 0, CC_K_GROUPS = 1, CC_K_DIAGNOSE = 2, CC_K_REFINE = 3 };
cc_status cc_profile_enable(cc_model *m, int on);
cc_status cc_profile_read(cc_model *m, int kernel, double *total_ms, long long *launches);
cc_status cc_profile_reset(cc_model *m);

/* ------------------------------------------------------------------------
 * Block-structured refinement with subcycling (Sec 2.2).
 *
 * A refined model holds nlev levels as domains 0 .. nlev-1 of one model.
 * Level 0 is `base` (periodic, rigid lid).  Level l >= 1 is the box
 * boxes[l-1] = {nx, ny, nz, ox, oy}: nx x ny x nz cells of spacing 2^-l of
 * the base spacing, resting on the floor, whose cell i covers cell
 * (i + ox) / 2 of level l-1 (likewise j with oy; cell k covers k / 2).  Its
 * time step is 2^-l dt: every step of level l-1 takes two steps of level l
 * first (subcycling), then the coarse step, then the exchange:
 *   - coarse -> fine: every ghost cell of level l outside the cells it
 *     integrates (-2 .. n+1 laterally, k < nz+2) takes the value of the
 *     coarse cell covering it; every ghost corner outside the corners it
 *     integrates (-1 .. n+1, K < nz+2) the coarse momentum interpolated
 *     linearly along each axis;
 *   - fine -> coarse: coarse cells of the covered box within 4 cells of its
 *     boundary take the mean of their 8 fine cells; coarse corners strictly
 *     inside it (within 4) the coincident fine corner;
 *   - flux register: a coarse face on the boundary of the covered box
 *     carries, for the mass and rho-theta updates of the coarse cell outside
 *     the box, the mean over the two fine substeps of the sum of its 2 x 2
 *     fine face fluxes, so the fluxes leaving one level enter the other.
 * With the Robert-Asselin filter off, the two-time-level perturbation mass
 * over the active cells of all levels (cc_refine_mass) is then conserved to
 * round-off.
 * Constraints (CC_EINVAL otherwise): 2 <= nlev <= 8; nx, ny, nz, ox, oy even;
 * the covered box (ox/2 .. (ox+nx)/2, oy/2 .. (oy+ny)/2, 0 .. nz/2) at least
 * 8 cells inside the coarser level's edges and below its top.  Terrain: a
 * box level takes corner heights for I < nx, J < ny (cc_set_terrain) that
 * are zero within 8 corners of its edges; at cc_build_geometry every coarser
 * level must be flat (zero heights) within 4 cells of each covered box
 * (CC_EGEOM otherwise).  Host arrays of a box level cover its cells and
 * corners 0 .. n-1 (the layouts above with its nx, ny, nz).
 * cc_init_state, cc_step (n steps of level 0, each a full cycle),
 * cc_upload_state / cc_download_state / cc_diagnostics (domain = level) work
 * on refined models as on ensembles. */
typedef struct {
  int nx, ny, nz, ox, oy;
} cc_box;

/* Create a refined model of nlev levels: level 0 from *base, levels 1 ..
 * nlev-1 from boxes[0 .. nlev-2] (spacings and time step halved per level,
 * every other constant from *base; the sponge of every level is measured
 * against the top of level 0).  Precision, stream and ownership as in
 * cc_create. */
cc_status cc_create_refined(const cc_config *base, int nlev, const cc_box *boxes, int precision,
                            void *stream, cc_model **out);

/* Sibling blocks (Sec 2.2: a level is made of blocks, each with its own ghost
 * shell, filled by copies from the blocks next to it on the same level and by
 * injection from the coarser level elsewhere).  As cc_create_refined, with
 * the box of the finest level cut at the nxcut x positions xcut[] and the
 * nycut y positions ycut[] (its cells; even, strictly increasing, every block
 * at least 18 cells wide) into (nxcut + 1)(nycut + 1) blocks of uneven sizes,
 * each spanning the level's height.  The blocks are domains nlev - 1 ..
 * nlev - 2 + (nxcut + 1)(nycut + 1), by y block, then x block; each has its own
 * padded arrays, cc_set_terrain heights (its corners, zero within 8 corners
 * of its edges, so the terrain stays clear of the cuts) and host layouts of
 * its nx, ny.  After every step of the level each block's ghost shell
 * (4 deep) where it lies in a sibling takes the sibling's cells, corners and
 * boundary-point velocities (the two time levels the next step reads); the
 * coarse-fine injection, restriction and flux register run per block over the
 * faces and cells of the level's outer boundary only.  All blocks of the
 * level advance in the same launches (one work list over the blocks).  The
 * arithmetic of every cell is that of the undivided box, so the results equal
 * its results bit for bit.  nxcut = nycut = 0 is cc_create_refined. */
cc_status cc_create_refined_blocks(const cc_config *base, int nlev, const cc_box *boxes, int nxcut,
                                   const int *xcut, int nycut, const int *ycut, int precision, void *stream,
                                   cc_model **out);

/* Level of domain d (0 for every domain of a model made by cc_create) and the
 * origin of its block in the level's box (fine cells; 0, 0 for an undivided
 * level).  Null outputs are skipped. */
cc_status cc_domain_block(const cc_model *m, int d, int *level, int *ox, int *oy);

/* Two-time-level perturbation mass of a refined model (Sec 2.2, reading of
 * the conservation check): sum over the levels of V rho' over the merged cells
 * of each level outside the box covered by the next finer level, at the
 * current level, plus the same sum at the previous level when both != 0.
 * out[0] receives the sum (kg).  Synchronises the stream. */
cc_status cc_refine_mass(cc_model *m, int both, double *out);

/* Number of domains (ensemble members, or levels and blocks of a refined
 * model). */
int cc_domain_count(const cc_model *m);

/* A cube of the block-structured layout: its refinement level and its index
 * in cube units of that level (cube (ci, cj, ck) of level l covers cells
 * ci*c .. (ci+1)*c - 1 of that level in x, and so on). */
typedef struct {
  int level, ci, cj, ck;
} cc_cube;

/* Block-structured cube layout (Sec 2.2, grid generation of the cube-based
 * Cartesian mesh); host code, no GPU needed.  The level-0 domain of
 * nx0 x ny0 x nz0 cells at spacing H is divided into cubes of cube^3 cells;
 * cubes near the terrain are split into eight, level after level, up to
 * level nlev-1 (spacing H / 2^l, every cube holding cube^3 cells); the sizes
 * are then adjusted so that cubes touching across a face, an edge or a corner
 * differ by at most one level (2:1); cubes completely inside the terrain are
 * dropped.  Refinement test (the paper only says that cubes close to the
 * terrain surface are split; this test gives its cube counts 64, 148, 232 for
 * its hemisphere grids): a cube below the finest level is split when its
 * bottom lies below the highest terrain point and its footprint lies within
 * one cube width, horizontally, of a finest-level corner where the terrain
 * is raised above its lowest value.  Lateral boundaries are periodic.
 *   h_finest: corner heights of the finest level, (ny0 2^(nlev-1)) x
 *             (nx0 2^(nlev-1)) doubles, x fastest (host array);
 *   out:      capacity cubes, sorted by (level, ck, cj, ci), or NULL to get
 *             the count only; *count receives the number of cubes.
 * CC_EINVAL for extents that are not multiples of cube, nlev outside 1 .. 12,
 * non-finite heights, or a capacity below the count (the count is still
 * set). */
cc_status cc_cbcm_cubes(int nx0, int ny0, int nz0, int cube, double H, int nlev, const double *h_finest,
                        cc_cube *out, int capacity, int *count);

/* Fused multiply-add peak of the current GPU (no counterpart in the paper;
 * the denominator of the roofline of the plain FP64 form, which is bound by
 * the FP64 pipe rather than by memory): independent chains x <- x a + b in
 * registers on 8 blocks of 256 threads per SM, iters steps per chain, one
 * warm-up launch and one launch timed with CUDA events on `stream`.
 * *flops_per_s receives 2 x the fused multiply-adds per second.  precision:
 * CC_FP64 or CC_FP32.  CC_EINVAL for a bad argument, CC_ECUDA for a CUDA
 * error (also when an earlier call left one pending, which is not cleared).
 * Synchronises `stream`; changes no clock or other GPU setting. */
cc_status cc_fma_peak(int precision, int iters, void *stream, double *flops_per_s);

/* Allocation-free mass sum (the paper has no counterpart; it is an entry
 * point for callers that cannot call cudaMalloc -- code running inside
 * another framework's memory pool, or a host application that reserves all
 * device memory up front and must not allocate afterwards).
 * Computes, on `stream`, the Neumaier-compensated sum that cc_diagnostics
 * reports as the mass: out[0] = sum_i volume[i] * rho_prime[i] and
 * out[1] = its compensation term, from device buffers the caller owns:
 *   rho_prime: n device values (double for CC_FP64, float for CC_FP32);
 *   volume:    n device doubles (cell volumes in m^3);
 *   out:       2 device doubles, overwritten.
 * The scratch is a fixed array inside the library holding
 * CC_NOALLOC_MAX_PARTS partial sums (16 KiB per GPU that loads the library,
 * kept until the process exits); the call uses nparts of them and rejects
 * nparts outside 1..CC_NOALLOC_MAX_PARTS with CC_EINVAL.  Nothing is
 * allocated and nothing is freed.  The first call on a device looks up the
 * array's device address with that device current, so make that first call
 * before any stream capture.  Every call shares the array: calls that overlap
 * on the GPU (for example on two streams) race, so serialise them.
 * Errors (CC_EINVAL, CC_ECUDA) are described by cc_noalloc_last_error(). */
#define CC_NOALLOC_MAX_PARTS 1024 /* the message of cc_noalloc_last_error() quotes this limit */
cc_status cc_mass_sum_noalloc(const void *rho_prime, int precision, const double *volume, long long n,
                              int nparts, double *out, void *stream);
const char *cc_noalloc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* CUTCELL_H */
