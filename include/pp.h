/*
 * pp.h — C ABI of the GB300 pressure-recovery and surface-force library.
 *
 * Method (Verma, Abbati, Novati, Koumoutsakos, "Computing the force distribution
 * on the surface of complex, deforming geometries using vortex methods and
 * Brinkman penalization"):
 *   1. source of the pressure-Poisson equation from the velocity, Eq. PoissonFinal
 *      (Sec. 2.2):  lap P = -rho (grad u^T : grad u) + rho lambda div(chi (u_s - u));
 *   2. P = sum_x' G(x, x') f(x') h^2, G = log|x - x'| / (2 pi)   (Eqs. green2D,
 *      greenSum, Appendix A.1), by a quadtree fast multipole method at the grid
 *      cells and by a tree-code at off-grid surface points (Appendix A.2);
 *   3. surface tractions -P n and 2 mu D . n, and their closed-surface integrals
 *      (Eqs. Fpress, FpressNet, CdP, Fvisc, FviscNet, CdNu, Sec. 2.3).
 *
 * Conventions shared by every call
 *  - Grid: n x n cells, n = 8 * 2^k (8 <= n <= 16384), cell-centred, uniform
 *    spacing h, cell (i, j) centred at (x0 + (i + 1/2) h, y0 + (j + 1/2) h).
 *    Grid fields are row-major: element (i, j) at index j * n + i.
 *  - Precision: a PP_FP64 plan takes and returns grid fields as double; a
 *    PP_MIXED plan takes and returns them as float (FP32 expansions and near
 *    field, FP64 monopole/constant terms and FP64 force integration).  Surface
 *    arrays (points, normals, dS, per-point output, forces) are always double.
 *  - Memory: every array argument is a DEVICE pointer owned by the caller,
 *    except `forces` of pp_surface_traction, which may be host or device memory.
 *    The plan owns its device workspace (source weights, expansions, tables).
 *  - Ordering: calls are stream-ordered on the plan's stream (pp_options.stream,
 *    NULL = the legacy default stream).  pp_pressure_solve and
 *    pp_surface_traction need a prior pp_rhs on the same plan.
 *  - Errors: every call returns a pp_status; nothing is thrown across the ABI.
 *    PP_ERR_ARG / PP_ERR_STATE leave the plan unchanged.  After PP_ERR_CUDA the
 *    plan is marked dead and only pp_plan_destroy is accepted.
 */
#ifndef PP_H
#define PP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PP_OK = 0,
    PP_ERR_ARG = 1,      /* invalid argument (size, pointer, option) */
    PP_ERR_STATE = 2,    /* call order violated, or plan dead after a CUDA error */
    PP_ERR_OOM = 3,      /* device allocation failed */
    PP_ERR_CUDA = 4,     /* a CUDA runtime call or kernel launch failed */
    PP_ERR_TIMEOUT = 5,  /* a bounded device wait gave up */
    PP_ERR_BUDGET = 6    /* request does not fit the memory budget */
} pp_status;

enum { PP_FP64 = 0, PP_MIXED = 1 };
enum { PP_NEAREST = 0, PP_BILINEAR = 1 };

typedef struct pp_plan_s* pp_plan;

/* n x n cell-centred grid with lower-left corner (x0, y0). */
typedef struct {
    int n;
    double x0, y0;
} pp_grid;

typedef struct {
    double rho;        /* fluid density (default 1) */
    int precision;     /* PP_FP64 (default) or PP_MIXED */
    double lift;       /* offset along n where grad u is sampled (Sec. 2.3.2): <0 -> 2h (rigid
                          body, the paper's choice), 0 -> on the surface (deforming body) */
    int interp;        /* PP_NEAREST (default, the paper's nearest-neighbour rule) or PP_BILINEAR */
    double uinf_x;     /* direction of U_inf for drag/lift (default (1, 0)), Eq. CdP */
    double uinf_y;
    void* stream;      /* cudaStream_t for all launches (default NULL) */
    int tile;          /* mixed-precision near field: 8 or 16 target cells per thread on the FP32 cores,
                          or 128 for 128-leaf tiles on the tensor cores (default 16) */
    double theta_surface; /* acceptance parameter of the tree-code at the surface points
                          (0.25..0.95), independent of the grid's theta; 0 (default) ->
                          min(theta, 0.6).  A few thousand points make a strict value cheap,
                          and the forces integrate the surface pressure. */
    int m2l_tensor;    /* mixed plans of order 12 with theta >= 0.5: 1 -> the multipole-to-local
                          translations of a solve into a 16-byte aligned output run on the
                          tensor cores (tcgen05, one dense split-FP16 operator per list entry,
                          sources from a shared-memory halo, 4 x 128 target boxes per tile),
                          0 (default) -> on the FP32 cores; the results agree to FP32
                          rounding.  Other orders and theta take the FP32 cores either way
                          (pp_plan_info reports which). */
} pp_options;

/* Fill *opt with the defaults listed above. */
void pp_options_default(pp_options* opt);

/*
 * Create a plan for an n x n grid of spacing h, multipole order p = `order`
 * (Eq. pressTruncated truncation, 2 <= p <= 40) and acceptance parameter theta
 * (0.25 <= theta <= 0.95): two equal boxes at centre distance d are well
 * separated when their half-diagonals r satisfy 2 r < theta d, and a box is
 * accepted for a point target when r < theta d (Sec. A.2, "sufficiently large
 * distances").  Allocates the plan's device workspace on the current device.
 * opt may be NULL (defaults).  On success *out receives the plan.
 * Errors: PP_ERR_ARG (bad n, h, order, theta, options), PP_ERR_OOM, PP_ERR_CUDA.
 */
int pp_plan_create(pp_plan* out, pp_grid grid, double h, int order, double theta,
                   const pp_options* opt);

/*
 * Device memory a plan would hold (host only, allocates nothing): the bytes pp_plan_create
 * allocates for an n x n grid at this order, theta and options (precision and near-field
 * tile decide the arrays), plus the surface scratch grown for pp_surface_traction calls of
 * up to npts points (0: the scratch a new plan starts with).  The zero-padded FFT solve's
 * buffers are not included.  pp_plan_info's workspace_bytes reports the same figure for a
 * live plan.  Used by the solve server's admission against its memory budget.
 * Errors: PP_ERR_ARG (NULL bytes, or an argument pp_plan_create would reject).
 */
int pp_plan_bytes(int n, int order, double theta, const pp_options* opt, int npts, int64_t* bytes);

/* Release the plan and its device memory (synchronises its stream). NULL is a no-op. */
int pp_plan_destroy(pp_plan plan);

/* Change the stream later calls are ordered on. */
int pp_plan_set_stream(pp_plan plan, void* stream);

/*
 * Source of the pressure-Poisson equation, Eq. PoissonFinal (Sec. 2.2), and the
 * leaf multipole expansions, Eq. alphaK:
 *   f = -rho (u_x^2 + 2 u_y v_x + v_y^2) + rho lambda [d_x(chi (us_x - u)) + d_y(chi (us_y - v))],
 * second-order central differences (one-sided second order on the edge rows and
 * columns), q = f h^2 kept on the device for the solve.
 * u, v, chi, us_x, us_y: n*n row-major device arrays of the plan's precision.
 * f_out: optional (NULL allowed) n*n row-major device array receiving f.
 * Errors: PP_ERR_ARG (NULL field pointer), PP_ERR_STATE, PP_ERR_CUDA.
 */
int pp_rhs(pp_plan plan, const void* u, const void* v, const void* chi, const void* us_x,
           const void* us_y, double lambda, void* f_out);

/*
 * Pressure at every grid cell, Eq. greenSum, by the fast multipole method:
 * upward pass (Eqs. alphaK, expandedBeta), multipole-to-local and local-to-local
 * translations of the log series (Eq. logExpansion), local evaluation plus the
 * direct near-field sum over the theta-near leaves.  The self term uses
 * |x - x'| clamped below at h exp(pi/4 - 3/2 - log(2)/2) (the mean of log r over a cell).
 * p_out: optional n*n row-major device array of the plan's precision (NULL: run
 * the passes, keep nothing but the expansions).  Any element alignment; in mixed plans
 * a 16-byte aligned p_out takes the vector-store kernels (tensor-core near field, the
 * two-launch downward pass), others the scalar-store ones, with equal results up to
 * FP32 rounding order.
 * Errors: PP_ERR_STATE (no prior pp_rhs), PP_ERR_CUDA.
 */
int pp_pressure_solve(pp_plan plan, void* p_out);

/*
 * Pressure at every grid cell by the Fourier-based fast Poisson solver of Hockney, which
 * Appendix A.1 names as an alternative to the tree-code: the zero-padded (2n x 2n) FFT
 * convolution of the weights q = f h^2 with the kernel (1/2pi) log max(h |dx|, rho_h).  It is
 * the same discrete sum as pp_pressure_solve (Eq. greenSum, same self-term clamp) without
 * truncation error, so it serves as an independent whole-grid check of the multipole solve
 * and as a speed comparison on uniform grids.  Computed in the plan's precision (FP32 for
 * PP_MIXED, FP64 for PP_FP64).
 * p_out: n*n row-major device array of the plan's precision.
 * The first call on a plan forms the transformed kernel in FP64: it allocates the plan's FFT
 * buffers (n (n + 4) complex values, (n + 1) 2n reals and under n complex twiddles, in the
 * plan's precision), uses 2 x (2n)^2 x 16 bytes of
 * temporary device memory and synchronises the plan's stream; it may not be captured into a
 * graph.  Later calls allocate nothing (three kernel launches on the plan's stream).
 * Errors: PP_ERR_ARG (NULL p_out, n > 4096), PP_ERR_STATE (no prior pp_rhs, or a first call
 *         inside a stream capture), PP_ERR_OOM (first call), PP_ERR_CUDA.
 */
int pp_pressure_solve_fft(pp_plan plan, void* p_out);

/*
 * Surface pressure by the tree-code (Eq. pressTruncated per accepted box, Eq.
 * greenSum on leaves that are not accepted) at `npts` off-grid points, and the
 * surface tractions of Sec. 2.3:
 *   t_P = -P n (Eq. Fpress, P at the surface point itself),
 *   t_nu = 2 rho nu D . n, D = (grad u + grad u^T)/2 (Eq. Fvisc), grad u by central
 *   differences at the cell holding the lifted point x + lift n (nearest-neighbour rule)
 *   or bilinearly interpolated from the four surrounding cells (PP_BILINEAR),
 *   F = sum (t_P + t_nu) dS (Eqs. FpressNet, FviscNet), drag = F . U_hat (Eq. CdP),
 *   lift = F . (-U_hat_y, U_hat_x).
 * u, v: the plan-precision velocity (normally those given to pp_rhs).
 * points, normals: npts x 2 device doubles (x, y), normals outward from the body.
 * dS: npts device doubles, or NULL for trapezoid weights on the closed polygon
 *     (points in order around the body).
 * per_point: optional npts x 5 device doubles (P, tPx, tPy, tnux, tnuy).
 * forces: optional 6 doubles (FPx, FPy, Fnux, Fnuy, drag, lift), host or device
 *     memory; host memory is written before the call returns (stream synchronised).
 * Errors: PP_ERR_ARG (npts < 1 or > 2^24, NULL points/normals/u/v), PP_ERR_STATE,
 *         PP_ERR_OOM, PP_ERR_CUDA.
 */
int pp_surface_traction(pp_plan plan, const void* u, const void* v, int npts,
                        const double* points, const double* normals, const double* dS,
                        double nu, double* per_point, double* forces);

/*
 * Penalisation force, Eq. dragPenal (Sec. 3.1): the volume integral of the Brinkman term,
 *   F = sum over cells of lambda chi (u - u_s) h^2
 * (the paper's static-body form lambda chi u when u_s = 0), with drag = F . U_hat and
 * lift = F . (-U_hat_y, U_hat_x) for the plan's free-stream direction.  The paper uses it
 * as a cross-check of the surface-force drag; it needs only the fields, no prior call.
 * u, v, chi, us_x, us_y: n*n row-major device arrays of the plan's precision.
 * forces: 4 doubles (Fx, Fy, drag, lift), host or device memory; host memory is written
 *     before the call returns (stream synchronised).
 * The reduction order is fixed, so repeated calls give identical results.
 * Errors: PP_ERR_ARG (NULL pointer, non-finite lambda), PP_ERR_STATE (dead plan), PP_ERR_CUDA.
 */
int pp_penal_force(pp_plan plan, const void* u, const void* v, const void* chi, const void* us_x,
                   const void* us_y, double lambda, double* forces);

/*
 * Mass and centre-of-mass velocity of the body marked by chi, for the acceleration of a
 * deforming body (Sec. 3.3): Eq. aSF divides the surface force F_P + F_nu by the body's mass
 * M, Eq. aPenal differences the centre-of-mass velocity u_CM over time steps.  With the
 * body's density taken as the fluid's (rho of the plan) and its volume as sum chi h^2:
 *   out[0] = M = rho h^2 sum chi,  out[1..2] = u_CM = sum chi (u, v) / sum chi.
 * u, v, chi: n*n row-major device arrays of the plan's precision.  out: 3 doubles, host or
 * device memory; host memory is written before the call returns (stream synchronised).  Sums
 * in a fixed order (compensated FP32 per thread in mixed plans, FP64 block trees): repeated
 * calls give identical results.  A chi that sums to zero gives NaN velocities.
 * Errors: PP_ERR_ARG (NULL pointer), PP_ERR_STATE (dead plan), PP_ERR_CUDA.
 */
int pp_body_moments(pp_plan plan, const void* u, const void* v, const void* chi, double* out);

/* Static description of a plan (host memory). */
typedef struct {
    int n, order, levels, precision;
    double h, theta;
    int n_near;            /* leaves in the near field of a leaf (theta-near offsets) */
    int n_m2l[4];          /* multipole-to-local offsets per child position */
    int64_t near_pairs;    /* near-field source/target cell pairs of one full-grid solve */
    int64_t m2l_pairs;     /* box-to-box translations of one full-grid solve */
    int64_t workspace_bytes;
    int64_t launches;      /* kernel launches issued by this plan so far */
    int64_t m2l_pairs_leaf; /* translations at the leaf level (part of m2l_pairs) */
    double theta_surface;  /* acceptance parameter the surface tree-code uses */
    int near_kernel;       /* near-field kernel a solve runs: 128 = tensor cores (tcgen05,
                              128-leaf tiles), 16 / 8 = FP32 cores with 16 / 8 targets per
                              thread, 0 = the generic leaf kernel (FP64 plans) */
    int downward;          /* downward pass of a solve into a 16-byte aligned output: 2 = two
                              launches (every level's multipole-to-local translations in one,
                              then the local-to-local shifts and the evaluation per subtree of
                              the level L - 3 boxes), 3 = the same with the translations on the
                              tensor cores (option m2l_tensor), 1 = one launch per level,
                              0 = generic per-level kernels */
} pp_plan_info_t;

int pp_plan_info(pp_plan plan, pp_plan_info_t* info);

/*
 * Device status flags of the tensor-core kernels, which bound every wait on the tensor cores
 * and copies and, when one gives up, set a flag and finish without their result instead of
 * hanging: flags[0] the surface tree-code's list overflow, flags[1] the tensor-core near field,
 * flags[2] the tensor-core translations, flags[3] reserved; 0 = no failure, else the code of
 * the wait that gave up.  Synchronises the plan's stream, copies the four ints to host memory
 * `flags` and clears them on the device.
 * Errors: PP_ERR_ARG (NULL), PP_ERR_CUDA; PP_ERR_TIMEOUT when a tensor-core flag is set.
 */
int pp_plan_device_status(pp_plan plan, int* flags);

/*
 * Stage timing (tracing aid).  When enabled, each call records CUDA events on the
 * stream it runs on; pp_plan_stage_times waits for the last recorded event and
 * writes the latest duration of each stage in milliseconds:
 *   0 source + leaf multipoles (pp_rhs), 1 upward pass, 2 downward pass
 *   (multipole-to-local + local-to-local; all levels, or all but the leaf level
 *   when the leaf level runs fused as stage 4), 3 leaf evaluation (near field, plus
 *   the local expansion when not fused; in mixed precision it runs on a side
 *   stream concurrently with stages 1-2), 4 leaf-level multipole-to-local fused
 *   with the local expansion at every cell, 5 surface (tree-code, tractions, sums).
 * A stage that has not run since timing was enabled reports -1.
 * Returns the number of stages (6) or a negative pp_status.
 */
int pp_plan_enable_timing(pp_plan plan, int on);
int pp_plan_stage_times(pp_plan plan, double* ms, int cap);

/*
 * Copy expansion coefficients of one tree level to device memory `dst`
 * (testing aid).  kind 0 = multipoles, kind 1 = locals.  Layout: 4^level boxes
 * in row-major box order, each (order + 1) complex numbers as (re, im) doubles,
 * scaled by the box side s: multipole entry k = alpha_k / s^k (entry 0 = S),
 * local entry l = b_l s^l (entry 0 = b_0), for the potential 2 pi P.
 */
int pp_get_expansion(pp_plan plan, int kind, int level, double* dst);

/*
 * Host-only helpers (no device needed): the same-level offsets (dx, dy) that are
 * not well separated at acceptance parameter theta (the near field of a leaf),
 * and the multipole-to-local offsets of a box at child position `child`
 * (0..3 = (x & 1) + 2 (y & 1)).  Writes up to `cap` pairs into out[2 * i],
 * out[2 * i + 1] and returns the count, or -PP_ERR_ARG.
 */
int pp_near_offsets(double theta, int* out, int cap);
int pp_m2l_offsets(double theta, int child, int* out, int cap);
/*
 * The interaction list a box at child position `child` actually uses: triplets
 * (dx, dy, kind) in out[3 i .. 3 i + 2].  kind 0: the same-level box at offset (dx, dy);
 * kind 1: the parent-level box at offset (dx, dy) from the box's parent, standing for its
 * four children when all four are well separated and the parent itself is accepted
 * (r_box + r_parent < theta d; the tie counts as not accepted).  pp_m2l_offsets lists the
 * same-level boxes the entries cover.  Returns the count or -PP_ERR_ARG.
 */
int pp_m2l_entries(double theta, int child, int* out, int cap);

/*
 * Adaptive quadtree for multiresolution grids (host only, no device needed).  The paper's
 * grids are block-structured and adaptive (Sec. 3 cites wavelet-adapted multiresolution
 * grids; Appendix A.2 groups the sources hierarchically).  The caller gives nleaf leaf
 * blocks (level[i] in 0..20, column ix[i] and row iy[i] in 0..2^level - 1, side 2^-level of
 * the unit domain); they must tile the domain exactly.  The tree holds every leaf and all
 * of its ancestors, the four children of a box stored together (child c = (x & 1) + 2 (y & 1)).
 * Interaction lists come from a dual-tree walk with the grid solve's acceptance test
 * (r_A + r_B < theta d, r the half-diagonal, ties not separated): multipole-to-local pairs
 * (target box, source box; the levels may differ) and near-field pairs (target leaf, source
 * leaf), each list sorted by target then source.  Every (target leaf, source leaf) pair is
 * covered exactly once: by one near-field pair or by one multipole-to-local pair of their
 * ancestors.
 * pp_atree_sizes: sizes[0..3] = boxes, multipole-to-local pairs, near-field pairs, deepest level.
 * pp_atree_boxes: per box (any output may be NULL) its level, ix, iy, parent (-1 at the root),
 *     first child (-1 for a leaf; the four children follow it) and leaf index (the position of
 *     the leaf in the caller's arrays, -1 for an internal box).
 * pp_atree_lists: m2l[2 i], m2l[2 i + 1] and p2p[2 i], p2p[2 i + 1] (either may be NULL).
 * Errors: PP_ERR_ARG (nleaf < 1, NULL arrays, theta outside [0.25, 0.95], a level or index out
 *         of range, duplicate or overlapping leaves, leaves that leave a gap), PP_ERR_OOM.
 */
typedef struct pp_atree_s* pp_atree;
int pp_atree_create(int nleaf, const int* level, const int* ix, const int* iy, double theta, pp_atree* out);
/*
 * The same tree and the same sorted lists built on the GPU from DEVICE arrays level, ix, iy
 * (nleaf ints each, caller-owned): Morton keys of the leaf blocks at level 20, a radix sort of
 * them, a one-pass check that the sorted blocks tile the domain (each Z-order range starts
 * where the previous one ends), the boxes level by level from scans of the flags "this leaf
 * opens a box of level k", and the lists from a breadth-first dual-tree walk with the same
 * acceptance test, radix-sorted by (target, source).  Work is ordered on `stream` (NULL: the
 * legacy default stream); the call allocates device temporaries, synchronises the stream and
 * returns a tree whose queries and solves behave exactly as for pp_atree_create.
 * Errors: as pp_atree_create (PP_ERR_ARG for a layout that does not tile the domain), and
 *         PP_ERR_CUDA, PP_ERR_OOM.
 */
int pp_atree_create_device(int nleaf, const int* level, const int* ix, const int* iy, double theta, void* stream,
                           pp_atree* out);
int pp_atree_sizes(pp_atree tree, int64_t* sizes);
int pp_atree_boxes(pp_atree tree, int* level, int* ix, int* iy, int* parent, int* first_child, int* leaf);
int pp_atree_lists(pp_atree tree, int* m2l, int* p2p);
int pp_atree_destroy(pp_atree tree);

/*
 * Pressure at every cell of the adaptive grid, FP64: Eq. greenSum over cells of several sizes
 * (each source cell clamped at its own rho_h = h exp(pi/4 - 3/2 - ln2/2), h = its side) by the
 * fast multipole method on the tree's lists: leaf multipoles, shifts up the tree,
 * multipole-to-local over the pair list (boxes of any two levels), local shifts down the tree,
 * local evaluation plus the near field over the near-field pairs (Appendix A.2's series and
 * their standard local shifts, in units of each box's side).
 * q: nleaf*64 device doubles, the weights f h^2 of the cells, leaf-major in the order the
 *    leaves were given to pp_atree_create, cell (cx, cy) of a block at cy*8 + cx (8 x 8 cells
 *    per block, cell side = block side / 8).
 * p_out: nleaf*64 device doubles, same layout.  order: 2..30.  stream: a CUDA stream or NULL.
 * Near field: between leaves of one level from a table of log|D| over integer cell offsets
 * (built once in FP64), between leaves of different levels directly.
 * The first solve on a tree uploads the tree, the lists and the table and allocates the
 * expansions (synchronising the stream); so does a solve at a higher order than before.  They
 * stay with the tree until pp_atree_destroy, so later solves allocate nothing and only launch
 * kernels on the stream.  Solves on one tree share its arrays: order them on one stream.
 * Errors: PP_ERR_ARG (NULL tree, q or p_out, order out of range), PP_ERR_OOM, PP_ERR_CUDA.
 */
int pp_atree_solve(pp_atree tree, int order, const double* q, double* p_out, void* stream);

/*
 * The same solve in mixed precision: q and p_out are nleaf*64 device floats (same layout);
 * expansions in FP32 (in units of each box's side), the box monopoles S and the constant
 * terms of the locals in FP64, the leaf multipoles and the shifts from tables built on the
 * host in FP64, each translation's geometry (tau, rho in target-side units, log|tau| +
 * log s in FP64) computed on the host once per tree, the near field in FP32 with compensated
 * sums (each same-level source leaf's log h part, S log h, in FP64).  Agrees with
 * pp_atree_solve to FP32 rounding of the expansions and the near field.  Its first call on a
 * tree also uploads those tables (synchronising the stream).  It leaves the tree's FP64
 * multipoles stale: pp_atree_surface_pressure then needs a pp_atree_solve first.
 * Errors: as pp_atree_solve.
 */
int pp_atree_solve_mixed(pp_atree tree, int order, const float* q, float* p_out, void* stream);

/*
 * Pressure at npts off-grid points (the body's surface points, Sec. 2.3.1) on an adaptive grid,
 * FP64, by the tree-code over the adaptive tree (Appendix A.2: a group is accepted for a
 * target at a sufficient distance): depth-first from the root, a box whose half-diagonal r
 * is below theta d (d the distance of the point from its centre) contributes its multipole
 * (Eq. pressTruncated about the box centre), a leaf that is not accepted is summed directly
 * over its 64 cells, each clamped at its own rho_h (Eq. greenSum), any other box opens its
 * children.  Uses the multipoles of the last pp_atree_solve on this tree (its order), so q
 * must be the weights that solve was given.
 * points: npts x 2 device doubles; P_out: npts device doubles; theta: 0.25..0.95.
 * Synchronises the stream (the stack-overflow flag is read back).
 * Errors: PP_ERR_ARG (NULL pointer, npts < 1 or > 2^24, theta out of range), PP_ERR_STATE (no
 *         prior solve on the tree, or a walk deeper than its stack), PP_ERR_CUDA.
 */
int pp_atree_surface_pressure(pp_atree tree, const double* q, int npts, const double* points, double theta,
                              double* P_out, void* stream);

/*
 * Tractions and drag/lift from a given surface pressure, allocating nothing.
 * The paper has no counterpart: this is a deployment variant of the traction and
 * force-integration step of pp_surface_traction for callers that cannot allocate
 * device memory (a flow solver that reserved the whole device up front, or a
 * loop that must not pay the implicit synchronisation of cudaMalloc).  It needs
 * no plan: the caller passes the grid, the velocity (u, v: n*n row-major device
 * arrays, double for PP_FP64 or float for PP_MIXED), npts device points and
 * outward normals (npts x 2 doubles), optional dS (NULL: trapezoid weights on the
 * closed polygon), the pressure at the points P_points (npts device doubles, e.g.
 * column 0 of pp_surface_traction's per_point), rho, nu, lift (<0: 2h), interp,
 * and the U_inf direction.  Outputs as in pp_surface_traction: per_point (npts x 5
 * device doubles, nullable) and forces (6 doubles, host or device, nullable; host
 * memory is written before return after a stream synchronisation).
 * Scratch: the per-block partial sums live in one fixed device array of
 * PP_NOALLOC_SCRATCH_BYTES (4 doubles per 64-point block of the largest request plus
 * 8 doubles: 4 * 16384 + 8 doubles, about 512 KB) that every device loading the
 * library keeps until the process exits.  Every call looks up that array's device
 * address in the current context (cudaGetSymbolAddress, which allocates nothing);
 * the first call on a device may also load the library's device code, so make the
 * first call on a device before any stream capture.  All calls share the array, so
 * calls that overlap on the GPU (different streams or host threads) race: order
 * them on one stream.  Nothing in it needs clearing: every partial sum that is read
 * was written by the same call.
 * Errors: PP_ERR_ARG (npts < 1 or > PP_NOALLOC_MAX_POINTS, bad grid/options, NULL
 * inputs), PP_ERR_CUDA.
 */
#define PP_NOALLOC_MAX_POINTS (1 << 20)
#define PP_NOALLOC_SCRATCH_BYTES ((4 * (PP_NOALLOC_MAX_POINTS / 64) + 8) * 8)
int pp_surface_forces_noalloc(int precision, pp_grid grid, double h, const void* u, const void* v,
                              int npts, const double* points, const double* normals, const double* dS,
                              const double* P_points, double rho, double nu, double lift, int interp,
                              double uinf_x, double uinf_y, double* per_point, double* forces,
                              void* stream);

/*
 * One whole step as a CUDA graph: pp_rhs + pp_pressure_solve (+ pp_surface_traction
 * when npts > 0) with fixed arguments, captured once and replayed with
 * pp_step_graph_launch on any stream.  Replays recompute everything from the
 * current contents of the argument buffers, so a caller refills u, v, chi, us_x,
 * us_y (and points, normals) in place between launches.  forces must be device
 * memory (or NULL).  The plan's own stream is not used by replays; after creation
 * the plan's call-order state is that of a completed step.  Destroy the graph
 * before its plan.
 * Errors: PP_ERR_ARG (as in the three calls; host forces), PP_ERR_STATE, PP_ERR_CUDA.
 */
typedef struct pp_graph_s* pp_graph;
int pp_step_graph_create(pp_plan plan, const void* u, const void* v, const void* chi, const void* us_x,
                         const void* us_y, double lambda, void* p_out, int npts, const double* points,
                         const double* normals, const double* dS, double nu, double* per_point,
                         double* forces, pp_graph* out);
int pp_step_graph_launch(pp_graph graph, void* stream);
int pp_step_graph_destroy(pp_graph graph);

/*
 * A batch of independent snapshots (possibly of different grid sizes) solved by ONE
 * graph launch: each step graph becomes an independent branch of one CUDA graph, so
 * the small snapshots' work overlaps on the device.  The step graphs (and their plans
 * and buffers) must outlive the batch; the batch copies their graphs at creation.  Each
 * graph must come from a different plan: the branches run at once and a plan's workspace
 * holds one solve.
 * Errors: PP_ERR_ARG (count < 1, NULL graph, two graphs of one plan), PP_ERR_STATE (a plan
 *         is dead), PP_ERR_CUDA.
 */
typedef struct pp_batch_s* pp_batch;
int pp_batch_create(int count, const pp_graph* graphs, pp_batch* out);
int pp_batch_launch(pp_batch batch, void* stream);
int pp_batch_destroy(pp_batch batch);

/*
 * Continuous-batching solve server (no counterpart in the paper: the deployment loop
 * around the method).  Requests for snapshots of any grid size are admitted in
 * arrival order whenever one of `slots` streams is free and the plans they need fit
 * in `budget_bytes` of device memory; admitted requests run concurrently.  Plans stay
 * resident and are reused by later requests of the same grid and options; idle plans
 * are evicted least-recently-used to make room.  A dispatcher thread issues all CUDA
 * work on the device that was current at pp_server_create; completion is detected
 * by polling events, and every host wait takes a timeout.
 */
enum { PP_SERVER_QUEUED = 0, PP_SERVER_RUNNING = 1, PP_SERVER_DONE = 2, PP_SERVER_FAILED = 3,
       PP_SERVER_CANCELLED = 4 };

typedef struct {
    int64_t budget_bytes; /* device memory the server's plans may hold (default 8 GiB) */
    int slots;            /* requests in flight at once, one stream each (1..64, default 8) */
    int precision;        /* PP_MIXED (default) or PP_FP64 */
    int order;            /* expansion order of every plan (default 12) */
    double theta;         /* acceptance parameter (default 0.6) */
    int tile;             /* near-field tile: 8, 16 or 128 (tensor cores), as in pp_options (default 16) */
    double theta_surface; /* surface tree-code acceptance, as in pp_options (default 0: min(theta, 0.6)) */
} pp_server_config;

/* One solve request.  All arrays are caller-owned device memory that must stay valid
 * until the request is finished; outputs may be NULL. */
typedef struct {
    pp_grid grid;
    double h;
    const void *u, *v, *chi, *us_x, *us_y; /* plan-precision n*n fields */
    double lambda, nu, rho, lift;          /* lift < 0: 2h */
    int interp;
    double uinf_x, uinf_y;
    int npts;                              /* 0: no surface part */
    const double *points, *normals, *dS;
    void* p_out;                           /* n*n pressure, plan precision */
    double* per_point;                     /* npts x 5 */
    double* forces;                        /* 6 doubles, device memory */
} pp_request;

typedef struct {
    int64_t queued, running, completed, failed;
    int64_t plans_resident, plans_created, plans_evicted, bytes_held;
} pp_server_stats_t;

void pp_server_config_default(pp_server_config* cfg);
typedef struct pp_server_s* pp_server;
int pp_server_create(const pp_server_config* cfg, pp_server* out);
/* Queue a request; *id identifies it.  PP_ERR_ARG: invalid request; PP_ERR_BUDGET: its plan
 * alone exceeds the budget. */
int pp_server_submit(pp_server server, const pp_request* req, int64_t* id);
/* Cancel a request that has not started (PP_ERR_STATE once it is on the device). */
int pp_server_cancel(pp_server server, int64_t id);
/* Status (PP_SERVER_*), the request's pp_status if it failed, and host times in seconds
 * since server creation: submitted, started, finished (times may be NULL). */
int pp_server_query(pp_server server, int64_t id, int* status, int* error, double times[3]);
/* Wait up to timeout_s seconds: PP_OK when done, PP_ERR_TIMEOUT if still unfinished,
 * PP_ERR_STATE if cancelled, else the request's error. */
int pp_server_wait(pp_server server, int64_t id, double timeout_s);
int pp_server_stats(pp_server server, pp_server_stats_t* stats);
/* Cancel queued requests, let in-flight ones finish, release everything. */
int pp_server_destroy(pp_server server);

/*
 * Streaming solves from HOST memory (no counterpart in the paper: the transfer loop
 * around the method).  Each submitted snapshot is copied host->device, solved by a
 * step graph (pp_rhs + pp_pressure_solve + pp_surface_traction) and its pressure and
 * forces copied device->host.  Two device slots alternate, with the uploads, the solve
 * and the downloads on three streams, so snapshot k+1's upload and snapshot k-1's
 * download overlap snapshot k's solve.  lambda, nu, npts and dS are fixed at creation;
 * the points and normals are uploaded with every snapshot (the body moves).
 *  - Host buffers: u, v, chi, us_x, us_y (n*n, plan precision), points and normals
 *    (npts x 2 doubles), p_out (n*n, plan precision, may be NULL) and forces (6
 *    doubles, may be NULL).  They should be page-locked (cudaHostAlloc or
 *    cudaHostRegister) for the copies to overlap; pageable memory is accepted but
 *    its copies serialise with the host.  A snapshot's buffers must stay valid and
 *    unmodified until pp_pipeline_wait returns.
 *  - dS: optional npts device doubles (NULL: trapezoid weights), as in
 *    pp_surface_traction.
 *  - The pipeline owns two sets of device buffers and step graphs on `plan`; the plan
 *    must not be used otherwise while the pipeline exists, and outlives it.
 * Errors: PP_ERR_ARG (NULL buffers, npts < 0, plan without a grid), PP_ERR_STATE (plan
 * dead), PP_ERR_OOM, PP_ERR_CUDA.
 */
typedef struct pp_pipeline_s* pp_pipeline;
int pp_pipeline_create(pp_plan plan, double lambda, int npts, const double* dS, double nu, pp_pipeline* out);
int pp_pipeline_submit(pp_pipeline pipe, const void* u, const void* v, const void* chi, const void* us_x,
                       const void* us_y, const double* points, const double* normals, void* p_out,
                       double* forces);
/* Wait until every submitted snapshot's results are in host memory. */
int pp_pipeline_wait(pp_pipeline pipe);
int pp_pipeline_destroy(pp_pipeline pipe);

/*
 * Measured throughput of the ALU pipes the rooflines of this library's kernels divide by (no
 * counterpart in the paper: measurement support).  Three kernels fill every SM with warps
 * running independent dependency chains of one instruction: FP32 fused multiply-add, the
 * special-function unit's base-2 logarithm (lg2.approx), FP64 fused multiply-add.  Each is
 * timed with CUDA events on `stream` (NULL: the legacy default stream), after one warm-up
 * round, best of `reps` (1..1000) launches of about 1-3 ms.  Allocates nothing.
 * out (host, 7 doubles): FP32 TFLOP/s (2 flops per FMA), lg2 results in 1e9 per second,
 * FP64 TFLOP/s, the three best kernel times in ms, and the SM count.  The rates hold at the
 * SM clock the device ran during the call; sample it alongside to scale them.
 * Errors: PP_ERR_ARG (NULL out, reps out of range), PP_ERR_CUDA.
 */
int pp_measure_alu_peaks(double* out, int reps, void* stream);

/* Static text for a status code. */
const char* pp_error_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* PP_H */
