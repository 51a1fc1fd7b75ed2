/*
 * kifmm.h - C-ABI of the GB300 kernel-independent FMM for the Zheleznyak
 * integral photoionization model (Lin, Zhuang, Cai, Zeng, Bao, arXiv:2006.03515).
 *
 * What it computes (Sec. 3, Eq. (summation) with the discrete kernel G):
 *
 *   S_i = C * ( sum_{j != i} K(|x_i - x_j|) I_j h_j^3  +  sigma(h_i) I_i ),
 *   K(R) = (exp(-aR) - exp(-bR)) / (4 pi R^3 ln(b/a))        (Eqs. (integral), (gfun))
 *
 * for cell centres x_i of cubic cells of edge h_i, a = chi_min p_O2,
 * b = chi_max p_O2, and C = xi (omega/alpha) p_q / (p + p_q) (Eq. (Ifun)).
 * The far part of the sum is approximated by the kernel-independent FMM of
 * Sec. 3 (equivalent/check surfaces, S2M, M2M, M2L, L2L, outline steps 1-4)
 * on an adaptive octree; the near part is summed directly (Eq. (nearfar)).
 *
 * Conventions for every entry point:
 *  - Pointers named *_dev are DEVICE pointers (cudaMalloc'd or torch CUDA
 *    tensors) on the current device; *_host are host pointers. All arrays are
 *    dense and C-contiguous. Points are N x 3 FP64 in cm, row-major (x, y, z).
 *  - The caller keeps ownership of every array it passes. A plan copies what
 *    it needs into device buffers it owns; they are freed by kifmm_destroy.
 *  - Errors are reported by the return status only; no entry point aborts,
 *    throws, or traps on the device. kifmm_last_error() gives a message for the
 *    last failing call of the calling thread.
 *  - A plan is not re-entrant: one kifmm_eval at a time per plan. All work of a
 *    plan is issued on the stream given in its options (0 = legacy default).
 *  - kifmm_eval does not allocate memory; every buffer it uses is created by
 *    kifmm_plan.
 */
#ifndef KIFMM_H
#define KIFMM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct kifmm_plan_s* kifmm_plan_t;

typedef enum {
    KIFMM_OK = 0,
    KIFMM_ERR_ARG = -1,             /* invalid argument (size, NULL, range)         */
    KIFMM_ERR_OOM = -2,             /* device allocation failed                     */
    KIFMM_ERR_CUDA = -3,            /* a CUDA call or kernel launch failed          */
    KIFMM_ERR_TIMEOUT = -4,         /* a bounded device wait ran out                */
    KIFMM_ERR_DUPLICATE_POINT = -5, /* two points with identical coordinates        */
    KIFMM_ERR_NONFINITE = -6,       /* NaN/Inf in points or cell sizes              */
    KIFMM_ERR_NUMERIC = -7          /* an operator could not be built (SVD failed)  */
} kifmm_status;

typedef enum { KIFMM_FP64 = 0, KIFMM_MIXED = 1 } kifmm_precision;
typedef enum { KIFMM_SELF_CELL_EXACT = 0, KIFMM_SELF_PAPER_GL2 = 1 } kifmm_self_mode;
typedef enum { KIFMM_REPR_SURFACE = 0, KIFMM_REPR_CHEB = 1 } kifmm_repr;
typedef enum { KIFMM_F32 = 0, KIFMM_F64 = 1 } kifmm_dtype;

typedef struct {
    /* KIFMM_FP64: every step in FP64.
     * KIFMM_MIXED: near-field sums, check-surface and target evaluations in FP32
     * (box-local coordinates, compensated sums); M2L, L2L and the M2M translations as
     * 3-term FP16 splits (hi*hi + hi*lo + lo*hi, power-of-two scaled) on the tensor cores
     * with FP32 accumulation (SIMT FP32 for small levels); the upward pseudo-inverse
     * applications c = Sigma^+ U^T chk to FP64 accuracy (exact integer slices on the
     * tensor cores, or the FP64 pipe); on a uniform lattice of full leaves the near field
     * as 27 per-offset kernel matrices on the tensor cores (same FP16 x 3 form). */
    int precision;
    /* Value of the i == j term of the discrete kernel G (Sec. 3):
     * KIFMM_SELF_CELL_EXACT: the exact integral of K over the cell (default);
     * KIFMM_SELF_PAPER_GL2: the paper's 2-point Gauss-Legendre value h^3 K(h/2). */
    int self_mode;
    /* Relative cut-off of the truncated-SVD pseudo-inverse (Sec. 3, after the
     * outline): singular values below pinv_eps * sigma_max are dropped.
     * Default 1e-5. Must lie in (0, 1). */
    double pinv_eps;
    /* Root cube. has_root = 0: origin = min_i(x_i - h_i/2) per axis and
     * side = the largest extent of max_i(x_i + h_i/2) - origin. has_root = 1:
     * root = {origin_x, origin_y, origin_z, side}; every cell must lie inside. */
    int has_root;
    double root[4];
    /* cudaStream_t on which the plan runs all of its work (NULL = default stream). */
    void* stream;
    /* Far-field representation. KIFMM_REPR_SURFACE (default): the paper's equivalent and
     * check surfaces with m0 = surface_order (Sec. 3). KIFMM_REPR_CHEB: values at the
     * p^3 tensor Chebyshev nodes of each box, p = surface_order (2..10), with polynomial
     * interpolation in place of the pseudo-inverses (a volumetric representation, not in
     * the paper, that reaches the direct sum to ~1e-7 at p = 8). */
    int repr;
    /* Radii of the surfaces of the surface representation, in box half-widths (Sec. 3,
     * Fig. fmulloc): radii[0] for the upward equivalent and downward check surfaces,
     * radii[1] for the upward check and downward equivalent surfaces. Default {1.05, 2.95},
     * the reading that reproduces the FMM accuracy the paper reports at its own test sizes
     * (Sec. 4: E_V 0.10-0.40 % against the paper's 0.15-0.69 %); {0, 0} also selects the
     * default. The schematic figure draws {1.2, 2.6} (E_V 1.2-2.2 % on the same cases, at a
     * higher kept rank). Need 1 < radii[0] < radii[1] < 3 (the equivalent surface encloses
     * the box and the check surface stays inside its near range). Ignored by the Chebyshev
     * representation. */
    double radii[2];
    /* Rectangular cells (the paper's Sec. 4.2 grid): when all three are > 0, every cell is
     * the box cell_dims[0] x cell_dims[1] x cell_dims[2] (cm, along x, y, z), cell_h_dev must
     * be NULL and uniform_h is ignored. The weights are the cell volume hx hy hz, the self
     * term the box's own value (exact integral of K over the box, or the paper's
     * 3 g(rho) / (pi sum h^2) per unit volume with rho = sqrt(sum h^2 / 12)), and the root
     * rule takes each axis' own half extent. {0, 0, 0} (default): cubic cells. */
    double cell_dims[3];
    /* Kernel of the sum (kernel independence: the same FMM for any of them), with
     * p_O2 = a / chi_min (a, b as in kifmm_plan): KIFMM_KERNEL_ZHELEZNYAK (default), the
     * paper's K; KIFMM_KERNEL_HELMHOLTZ3, the three-exponential approximation of Sec. 2.2
     * (Eq. (gexp), Table Helcoeff), sum_j C_j p_O2^2 exp(-lambda_j p_O2 R) / (4 pi R), the
     * free-space solution of the modified Helmholtz equations (Hel); KIFMM_KERNEL_THREEGROUP,
     * the three-group model of Sec. 2.3 (Eq. (rtetoint), Table threegroupcoeff),
     * sum_j A_j p_O2 exp(-lambda_j p_O2 R) / (4 pi R^2). The self term follows the kernel
     * (exact cell integral, or hx hy hz K(sqrt(sum h^2 / 12)) for the paper's rule). The
     * comparison kernels run in the FP64 form (KIFMM_ERR_ARG with KIFMM_MIXED). */
    int kernel;
    /* Nonzero: when the points are every cell centre of a box of n_x x n_y x n_z cubic cells
     * (uniform_h, no cell_h or cell_dims, no root given) and leaf_size = nc^3 (nc >= 2), the
     * plan appends zero-weight cells (I = 0) that extend the box to multiples of 2 nc cells
     * per axis, and takes the root at the box's corner with side nc h 2^L. Every leaf is then
     * a full nc^3 block of one level, so that the lattice paths (near field on the tensor
     * cores, tabulated S2M / L2P) serve grids of any size. The padding adds nothing to the
     * discrete sum (its weights are 0) and S is returned for the caller's points only; the
     * FMM's approximation follows the padded tree. Other point sets are planned unpadded
     * (kifmm_info.n_padding = 0). The surrogate's photo_solve refuses padded plans. */
    int pad_lattice;
} kifmm_opts;

typedef enum { KIFMM_KERNEL_ZHELEZNYAK = 0, KIFMM_KERNEL_HELMHOLTZ3 = 1, KIFMM_KERNEL_THREEGROUP = 2 } kifmm_kernel;

/* Fills *opts with the defaults above (FP64, cell-exact self term, eps 1e-5,
 * automatic root, default stream, surface representation, radii {1.05, 2.95}, cubic
 * cells). */
void kifmm_default_opts(kifmm_opts* opts);

/*
 * Builds a plan for N cell-centred points (outline step 1 and the operators of
 * Eqs. (s2m)-(l2l)): root cube, 63-bit Morton keys (21 bits per axis, one FP64
 * subtraction and one FP64 multiplication per coordinate), stable radix sort,
 * levelled octree split while a box holds more than leaf_size points (at most
 * 20 levels; empty children are not created), U/V/W/X interaction lists,
 * per-level surfaces with surface_order (m0) points per side, truncated-SVD
 * pseudo-inverses and the M2M/M2L/L2L matrices, and the self-cell values.
 *
 *   points_dev   device, N x 3 FP64, cell centres (cm). Must be finite and distinct.
 *   n            number of points, 1 <= n < 2^31.
 *   cell_h_dev   device, N FP64 cell edges (cm), or NULL to use uniform_h for all.
 *   uniform_h    cell edge when cell_h_dev is NULL (> 0); ignored with opts->cell_dims.
 *   leaf_size    m >= 1: a box with more than m points is split.
 *   surface_order m0 in [3, 12]: lattice points per side of each surface.
 *   a, b         chi_min p_O2 and chi_max p_O2 in 1/cm, 0 < a < b.
 *   opts         options, or NULL for kifmm_default_opts().
 * On success *out receives the plan. Statuses: KIFMM_ERR_ARG,
 * KIFMM_ERR_NONFINITE, KIFMM_ERR_DUPLICATE_POINT, KIFMM_ERR_OOM,
 * KIFMM_ERR_CUDA, KIFMM_ERR_NUMERIC. The call synchronises its stream.
 */
int kifmm_plan(kifmm_plan_t* out, const double* points_dev, int64_t n,
               const double* cell_h_dev, double uniform_h, int leaf_size,
               int surface_order, double a, double b, const kifmm_opts* opts);

/*
 * One evaluation of S (outline steps 2-4): S_dev[i] = C * (far field through
 * the FMM + near field by direct summation + sigma(h_i) I_i), in input order.
 *   I_dev  device, N values of I (cm^-3 s^-1, caller order), dtype F32 or F64.
 *   S_dev  device, N outputs (same dtype), fully overwritten (never accumulated).
 *   C      scale factor (1.0 gives the raw sum).
 * Asynchronous on the plan's stream; allocates nothing; no host synchronisation.
 * Mixed plans with the lattice near field run its sums on a second stream owned by the
 * plan, forked from and joined back into the plan's stream by events within the call, so
 * the whole evaluation stays ordered on the plan's stream (and inside a capture of it).
 * Statuses: KIFMM_ERR_ARG (NULL, bad dtype), KIFMM_ERR_CUDA (launch failure). A bounded
 * device wait that gives up is reported by kifmm_check (below), not by this call.
 */
int kifmm_eval(kifmm_plan_t plan, const void* I_dev, void* S_dev, int dtype, double C);

/*
 * The same evaluation from host buffers: copies I_host to the device, runs
 * kifmm_eval, copies S back to S_host and synchronises the plan's stream.
 * Host buffers may be pageable or pinned (pinned is faster). Returns KIFMM_ERR_TIMEOUT when a
 * bounded device wait of the evaluation gave up (as kifmm_check).
 */
int kifmm_eval_host(kifmm_plan_t plan, const void* I_host, void* S_host, int dtype, double C);

/*
 * Evaluates `count` fields (each a plan with its own I and S, possibly of different
 * sizes and pressures; the batched workload of many streamer fields) as one unit of
 * work ordered on plan[0]'s stream.
 *   lanes    1: the fields run back to back on plan[0]'s stream. lanes > 1 (at most
 *            KIFMM_MAX_LANES): plan[0]'s stream forks into that many concurrent
 *            streams owned by plan[0]; every distinct plan is placed on one lane
 *            (largest fields first, each onto the lane with the fewest points so far;
 *            entries repeating a plan share its lane and run in order, because they
 *            share its workspace), and all lanes join back before the call's work
 *            completes on plan[0]'s stream. Fields are independent, so the device
 *            schedules one field's kernels beside another's (a small field's levels
 *            and a large field's near field fill the SMs together). Results are those
 *            of one kifmm_eval per field.
 *   capture  != 0: the whole batch, fork and join included, is recorded once into a
 *            CUDA graph held by plan[0] and replayed on later calls with the same
 *            arguments (plans, buffers, count, dtype, lanes and the values of C); any
 *            other call records a new graph. Plans are told apart by an id that is never
 *            reused, so a plan created at a destroyed plan's address is a new plan.
 * Completion is ordered on plan[0]'s stream only: synchronise it (not the other
 * plans' streams) before reading S or destroying a plan. Statuses: KIFMM_ERR_ARG
 * (NULL plan or buffer, count < 1, lanes out of range, capture on the legacy default
 * stream), KIFMM_ERR_CUDA.
 */
#define KIFMM_MAX_LANES 8
int kifmm_eval_batch(kifmm_plan_t* plans, const void* const* I_dev, void* const* S_dev,
                     int count, int dtype, const double* C, int capture, int lanes);

/*
 * Autotuner: picks the leaf size m for a point set by measurement. For each of the
 * ncand candidate leaf sizes it builds a plan (same points, cell sizes, m0, a, b, opts),
 * runs one untimed and `reps` timed evaluations of a unit source on the plan's stream
 * (CUDA events) and keeps the fastest. The leaf size trades near-field pairs (P2P,
 * ~27 m per point) against the number of boxes (M2L, M2M, L2L per box), so its best value
 * depends on N, the pressure and the precision. Writes the best candidate to *best_leaf
 * and, if ms_out is not NULL, the mean time of each candidate (ms) to ms_out[0..ncand).
 * Allocates and frees its own temporary device buffers. Statuses as kifmm_plan.
 */
int kifmm_autotune(const double* points_dev, int64_t n, const double* cell_h_dev, double uniform_h,
                   const int* leaf_candidates, int ncand, int surface_order, double a, double b,
                   const kifmm_opts* opts, int reps, int* best_leaf, float* ms_out);

/*
 * Status of the device work issued so far for the plan: synchronises the plan's stream and
 * reads the plan's device error word. A bounded wait inside a tensor-core kernel that gave
 * up (instead of hanging) leaves a code there; the evaluation it belonged to is then not
 * valid. Returns KIFMM_ERR_TIMEOUT in that case and clears the word (each event is reported
 * once), KIFMM_OK otherwise, KIFMM_ERR_CUDA if the stream reports an error. kifmm_eval_host
 * makes this check itself; callers of the asynchronous kifmm_eval and kifmm_eval_batch
 * call it for each plan when they synchronise.
 */
int kifmm_check(kifmm_plan_t plan);

/*
 * Constants of the Zheleznyak model (Sec. 2.1, Eqs. (gfun), (Ifun)) for a gas pressure p
 * and an oxygen partial pressure p_O2 (Torr): a = chi_min p_O2 and b = chi_max p_O2 with
 * chi_min = 0.035 and chi_max = 2 /(cm Torr), and the scale C = xi (omega/alpha) p_q / (p + p_q)
 * for the quenching pressure p_q (Torr) and the factor xi (omega/alpha) of Eq. (Ifun)
 * (0.06 and 30 Torr in the paper's tests). Any output pointer may be NULL.
 * KIFMM_ERR_ARG unless p > 0, p_O2 > 0, p_q > 0 and xi_omega_alpha > 0 are finite.
 */
int kifmm_model_constants(double p_torr, double p_o2_torr, double p_q_torr, double xi_omega_alpha, double* a,
                          double* b, double* C);

/*
 * Accuracy-targeted autotuner: the fastest (leaf size, surface order, surface radii) whose
 * estimated error meets a target. For every candidate of leaf[0..nleaf) x order[0..norder) x
 * radii pairs radii[2j], radii[2j+1] (j < nradii; nradii = 0: opts' radii), it builds a plan
 * with opts (precision, root, cells, stream ...), evaluates the representative source I_dev
 * (device, N FP64, caller order; C = 1), estimates the relative L2 error against the FP64
 * direct sum of the discrete integral (Sec. 3, Eq. (summation)) at k_samples (1..4096)
 * targets drawn in proportion to the first candidate's field (probability 0.5 |S_i| / sum |S|
 * + 0.5 / N, importance weights), and times reps evaluations (CUDA events on the plan's
 * stream). A candidate is accepted when its estimate is at most target / 2 (the factor
 * covers the estimate's sampling error); *best receives the fastest accepted candidate, or
 * the most accurate one with ok = 0 when none is accepted. entries (may be NULL) receives
 * every candidate, leaf-major then order then radii. Allocates and frees its own work space.
 * Statuses as kifmm_plan, and KIFMM_ERR_ARG for empty candidate lists or target <= 0.
 */
typedef struct {
    int leaf;           /* leaf size m */
    int order;          /* surface order m0 (Chebyshev order p) */
    double radii[2];    /* surface radii */
    float ms;           /* mean evaluation time */
    double err;         /* estimated relative L2 error against the discrete sum */
    int ok;             /* err <= target / 2 */
} kifmm_tune_entry;
int kifmm_tune(const double* points_dev, int64_t n, const double* cell_h_dev, double uniform_h, const double* I_dev,
               double a, double b, const kifmm_opts* opts, const int* leaf, int nleaf, const int* order, int norder,
               const double* radii, int nradii, double target, int k_samples, int reps, kifmm_tune_entry* entries,
               kifmm_tune_entry* best);

/* Frees every device buffer of the plan (synchronising its stream). NULL is a no-op. */
void kifmm_destroy(kifmm_plan_t plan);

/* Message of the last failing call on this thread ("" if none). Owned by the library. */
const char* kifmm_last_error(void);

/* ---- introspection (tests of the tree and lists; host copies) ---- */

typedef struct {
    int64_t n_points;           /* points of the tree: the caller's, then n_padding padding cells */
    int64_t n_boxes;
    int32_t n_levels;
    int32_t surface_points;     /* S = m0^3 - (m0-2)^3 (Chebyshev representation: p^3) */
    int64_t n_leaves;
    int64_t list_len[4];        /* total entries of U, V, W, X */
    double origin[3];
    double side;
    double pinv_rank_min;       /* smallest kept rank over the levels' pseudo-inverses */
    int64_t eval_launches;      /* kernels launched by one kifmm_eval of this plan */
    int64_t p2p_pairs;          /* near-field pair evaluations of one kifmm_eval */
    int64_t m2l_tensor;         /* 1 if M2L runs on the tensor cores (mixed form) */
    int64_t device_error;       /* nonzero if a bounded device wait ran out (synchronises) */
    double m2l_flops;           /* algorithmic M2L flop of one kifmm_eval: 2 r_l^2 per V pair */
    double upward_flops;        /* upward pseudo-inverse work (FP64-equivalent): 2 r_l S per leaf and parent */
    double upward_mma_flops;    /* FP16 tensor-core flop executed for it by the exact slice products (0 on the FP64 pipe) */
    int64_t near_tensor;        /* 1 if the near field runs on the tensor cores: mixed form, points on a uniform
                                 * lattice with full leaves of one level (per-offset kernel matrices) */
    int64_t lattice_far;        /* 1 if, on such a lattice (surface form, no W / X lists), S2M and the local
                                 * part of L2P apply one tabulated check-surface matrix to every leaf */
    int64_t m2m_tensor_levels;  /* levels whose M2M translations run on the tensor cores (mixed form) */
    int64_t l2l_tensor_levels;  /* levels whose L2L translations run on the tensor cores (mixed form) */
    int64_t upward_tensor_levels; /* levels whose upward pseudo-inverse runs as exact slices on the tensor cores */
    int64_t n_padding;          /* zero-weight padding cells (kifmm_opts.pad_lattice); perm values >= the caller's
                                 * n (n_points - n_padding) are padding cells */
} kifmm_info;

/* Plan sizes and counters. Reads the device error word, so it synchronises the plan's stream. */
int kifmm_get_info(kifmm_plan_t plan, kifmm_info* info);

/* Copies the tree to caller-allocated host arrays (any pointer may be NULL):
 * perm[n_points] (input index of each sorted point), keys[n_points] (Morton keys
 * in sorted order), level/parent/pstart/pend/leaf[n_boxes], anchor[3*n_boxes]
 * (integer coordinates at the box's level), child[8*n_boxes] (-1 for empty). */
int kifmm_get_tree(kifmm_plan_t plan, int64_t* perm, uint64_t* keys, int32_t* level,
                   int32_t* parent, int64_t* pstart, int64_t* pend, int32_t* leaf,
                   int32_t* anchor, int32_t* child);

/* Copies interaction list `which` (0 = U, 1 = V, 2 = W, 3 = X) in CSR form:
 * offsets[n_boxes + 1], items[list_len[which]] (box ids, ascending per box). */
int kifmm_get_list(kifmm_plan_t plan, int which, int64_t* offsets, int32_t* items);

/* Copies per-point self-cell values sigma(h_i) in sorted order (n_points FP64). */
int kifmm_get_sigma(kifmm_plan_t plan, double* sigma);

/* Copies the upward coefficients c (the truncated-SVD coordinates of each box's upward
 * equivalent density, c = Sigma^+ U^T q^u, Sec. 3) of the last evaluation:
 * n_boxes x *stride FP64 host array (*stride receives the row stride, >= the rank). With
 * c == NULL only *stride is written, so that the caller can size the array. */
int kifmm_get_upward(kifmm_plan_t plan, double* c, int* stride);

/* Per-phase device times (ms) of the last kifmm_eval when KIFMM_TIMING=1 in
 * the environment at plan time: [scatter, P2M, M2M, M2L, S2L+L2L+DC2DE,
 * L2P+M2P, P2P] and, where the tensor-core lattice near field ran its sums on
 * the plan's own second stream beside the far field, an eighth entry: the
 * span of those sums (P2P then holds the join and the output combination).
 * Returns the number of phases written (<= cap). */
int kifmm_get_phase_times(kifmm_plan_t plan, float* ms, int cap);

/* ---- learned surrogate: 3D spectral neural operator ---- */

/*
 * A spectral neural operator on an n^3 grid that maps u = I / max I to S / (C max I) (the
 * amplitude-normalised form of the linear map I -> S); the paper has no learned part (it
 * stands in for the solve inside a time loop, with the FMM as judge and fallback). Layers: lift 1 -> width; `layers` times z = SpecConv(v) + W v + b,
 * v = GELU(z) (no GELU after the last); projection width -> proj_width (GELU) -> 1.
 * SpecConv keeps the frequencies {0..m-1} U {n-m..n-1} on the first two axes and {0..m-1}
 * on the last (the real field's conjugate half), mixes channels per frequency with a complex
 * width x width matrix (BF16 weights, FP32 accumulation) and transforms back.
 * Limits: n >= 4, 1 <= modes <= n/2, width <= 64, proj_width <= 128.
 * Fields are device FP32 arrays [batch][n^3], point index i*n^2 + j*n + k (k = last axis).
 * Parameters form one flat FP32 vector (order: lift W, b; per layer R real, R imag
 * ([(2m)(2m)m][width][width]), W [width][width], b; then Q1 [proj][width], q1, Q2, q2).
 * The model owns its device memory (allocated by sno_create, all activations for
 * max_batch fields) and runs its work on `stream`; calls on one model must not overlap.
 * Errors: KIFMM_ERR_ARG for bad sizes or pointers, KIFMM_ERR_OOM, KIFMM_ERR_CUDA.
 */
typedef struct sno_model_s* sno_model_t;
int sno_create(sno_model_t* out, int n, int width, int modes, int layers, int proj_width, int max_batch,
               void* stream);
void sno_destroy(sno_model_t model);
int64_t sno_num_params(sno_model_t model);
/* host copies of the flat parameter / gradient vectors (sno_num_params floats) */
int sno_set_params(sno_model_t model, const float* theta_host);
int sno_get_params(sno_model_t model, float* theta_host);
int sno_get_grads(sno_model_t model, float* grad_host);
/* parameters to / from a file ("SNO1" header with the model's sizes, then the FP32 vector);
   loading checks the sizes against the model's and resets the optimiser state */
int sno_save(sno_model_t model, const char* path);
int sno_load(sno_model_t model, const char* path);
/* training checkpoint to / from a file ("SNO2" header with the model's sizes, the Adam step
   count, then the FP32 parameters and Adam's two moment vectors): training resumed from a
   checkpoint takes the same steps as training that never stopped. Loading checks the sizes
   against the model's. Statuses: KIFMM_ERR_ARG (NULL, unreadable or mismatched file),
   KIFMM_ERR_CUDA. */
int sno_save_checkpoint(sno_model_t model, const char* path);
int sno_load_checkpoint(sno_model_t model, const char* path);
/* 1: spectral weights used in BF16 (default); 0: in FP32 (gradient checks) */
int sno_set_bf16(sno_model_t model, int on);
/* y = network(u) for `batch` fields (batch <= max_batch) */
int sno_forward(sno_model_t model, const float* u_dev, float* y_dev, int batch);
/* mean squared error of network(u) against t, and its gradient (kept in the model) */
int sno_loss_grad(sno_model_t model, const float* u_dev, const float* t_dev, int batch, double* loss_host);
/* one Adam step with the gradient of the last sno_loss_grad */
int sno_adam_step(sno_model_t model, float lr, float beta1, float beta2, float eps);

/*
 * Period of the network's truncated transforms: N with n <= N <= 4n and 2 modes <= N
 * (default n). The n^3 grid is then the corner of a zero-padded N^3 grid: the exponentials
 * are e^{-2 pi i k x / N}, the kept frequencies {0..m-1} U {N-m..N-1} (last axis {0..m-1}),
 * and the spectral convolution is no longer periodic on the grid itself (the
 * photoionization sum is a linear, not a periodic, convolution).
 */
int sno_set_period(sno_model_t model, int period);

/*
 * Exact near part added to the model's output: with u the model's input,
 *   y += sigma u(x) + sum_{0 < |d| <= r_out} K(h |d|) w(|d|) h^3 u(x + d),
 * K the photoionization kernel of Eq. (gfun) (a, b as in kifmm_plan), h the grid's cell edge,
 * sigma the self-cell value of self_mode, |d| in cells, w = 1 up to r_in and
 * cos^2(pi/2 (|d| - r_in)/(r_out - r_in)) up to r_out, u = 0 outside the grid. With
 * u = I / max I and targets S / (C max I) (photo_solve's amplitude-normalised form) this is
 * the short-range part of Eq. (summation) (Sec. 3) computed exactly, and the network learns
 * the smooth remainder. 0 <= r_in < r_out <= 8. a = b = 0 switches the near part off.
 * It is a fixed addend: sno_loss_grad's gradients are those of the network alone.
 */
int sno_set_near_field(sno_model_t model, double a, double b, double h, int self_mode, double r_in, double r_out);

/*
 * Initialises the network at the far part of the sum (needs sno_set_near_field): channel 0
 * carries, through layer 0's spectral weights, the Fourier multiplier on the N-periodic grid
 * of the far kernel K(h |d|) (1 - w(|d|)) h^3 (computed in FP64 on the device), and passes
 * unchanged through the later layers (bias `shift`, e.g. 8, keeps GELU linear); the weights
 * into and out of channel 0 and projection row 0 are set accordingly, every other parameter
 * keeps its value (so a small random start elsewhere lets training use the other channels).
 * The network's output is then the far convolution truncated to the kept modes. Resets the
 * optimiser state.
 */
int sno_init_far_field(sno_model_t model, double shift);

/*
 * Surrogate-first solve on the plan's points, which must be the model's n^3 grid in the
 * model's index order (FP64 I and S on the device, caller order). The map I -> S is linear
 * (Sec. 3, Eq. (summation)), so the network works in the amplitude-normalised form: with
 * s = max |I| (computed on the device), u = I / s and S = C s y, y = network(u) (plus the near
 * part when set; it must then have been set for the plan's a, b, cell edge and self term).
 * The result is judged against the direct sum of the discrete integral (the plan's kernel,
 * self terms and C) at k_samples (1..4096) targets drawn from `seed`; when the judged
 * relative L2 error exceeds tol, kifmm_eval's result replaces it. *used_fallback is set to 1
 * in that case and *judged_err to the judged error. Runs on the plan's stream and returns
 * after the judge (host synchronisation).
 */
int photo_solve(kifmm_plan_t plan, sno_model_t model, const double* I_dev, double* S_dev, double C, double tol,
                int k_samples, uint64_t seed, int* used_fallback, double* judged_err);

/*
 * photo_solve for `count` fields at once (1 <= count <= the model's max_batch): field b
 * has its own plan plans[b] (the model's grid; no padding), source I_dev[b], result
 * S_dev[b] and scale C[b] (NULL: 1). One forward pass of the network over the batch on
 * plans[0]'s stream, then the judge of each field (targets from seed + b), then one
 * kifmm_eval_batch of the fields judged above tol. used_fallback[b] and judged_err[b]
 * (either array may be NULL) as in photo_solve. Returns when every S_dev[b] is complete.
 */
int photo_solve_batch(kifmm_plan_t* plans, int count, sno_model_t model, const double* const* I_dev,
                      double* const* S_dev, const double* C, double tol, int k_samples, uint64_t seed,
                      int* used_fallback, double* judged_err);

/* ---- streamer time loop (Sec. 5, Eq. (eM)) ---- */

/*
 * The discharge model that the photoionization sum feeds (Sec. 5, Eq. (eM)):
 *   dn_e/dt - div(mu_e E n_e) - div(D_e grad n_e) = S_i + S_ph,
 *   dn_p/dt + div(mu_p E n_p) = S_i + S_ph,   -Laplace(phi) = (e / eps0)(n_p - n_e),  E = -grad(phi),
 *   S_i = mu_e n_e alpha(|E|) |E|, alpha = 5.7 p exp(-260 p / |E|) cm^-1,
 *   S_ph = kifmm_eval of S_i with scale C (Eqs. (integral), (Ifun)),
 * on nx x ny x nz cubic cells of edge h (cm) of the box [0, nx h] x [0, ny h] x [0, nz h],
 * fields [z][y][x] (x fastest, cell (i, j, k) centred at ((i + 1/2) h, (j + 1/2) h, (k + 1/2) h)).
 * phi = 0 on the face z = 0 and phi0 on the face z = nz h, homogeneous Neumann conditions for
 * phi on the side faces and for the densities on every face. Drift fluxes from MUSCL face
 * values with the Koren limiter, diffusion by central differences, Heun's second-order
 * explicit scheme (S_ph twice per step), the Poisson equation by multigrid V-cycles to a
 * relative residual of mg_tol (FP64 residual and potential, FP32 error equations). FP64
 * densities and fields; every array argument is a device pointer of nx ny nz doubles owned
 * by the caller.
 */
typedef struct streamer_s* streamer_t;
typedef struct {
    double p;          /* gas pressure, Torr */
    double phi0;       /* potential of the top electrode, V (Sec. 5: 52 kV) */
    double mu_e, mu_p; /* mobilities, cm^2 / (V s) (Sec. 5: 2.9e5 / p and 2.6e3 / p) */
    double D_e;        /* electron diffusion coefficient, cm^2 / s (Sec. 5: 1800) */
    double C;          /* scale of S_ph: xi (omega / alpha) p_q / (p + p_q) (Eq. (Ifun)) */
    double mg_tol;     /* relative residual of the Poisson solve (Sec. 5: 1e-8) */
    int mg_max_cycles; /* V-cycles before KIFMM_ERR_TIMEOUT */
    /* Local, thresholded photoionization (the saving the paper suggests at the end of Sec. 5.1):
     * region = {x0, x1, y0, y1, z0, z1} cell ranges [x0, x1) ... of the sub-box where S_ph is
     * evaluated, from the sources inside it (the plan is then over the sub-box's cell centres,
     * x fastest); all zero: the whole grid. Sources with S_i < threshold max S_i are left out
     * (threshold 0: none). S_ph is 0 outside the region. */
    int region[6];
    double threshold;
} streamer_params;

/* The paper's parameters of Sec. 5 at pressure p (phi0 52 kV, xi omega / alpha = 0.06,
 * p_q = 30 Torr, mg_tol 1e-8, 100 cycles). */
void streamer_default_params(streamer_params* prm, double p_torr);

/* plan: a kifmm plan over the nx ny nz cell centres in the fields' order (or over the region's
 * cells in that order when a region is set; the FMM of S_ph, built once and reused at every
 * evaluation), or NULL for a run without photoionization.
 * stream: the cudaStream_t of every launch. The densities start at 0.
 * KIFMM_ERR_ARG on invalid sizes or parameters, or a plan of another point count. */
int streamer_create(streamer_t* out, int nx, int ny, int nz, double h, const streamer_params* prm,
                    kifmm_plan_t plan, void* stream);
/* Copies the densities n_e, n_p in. */
int streamer_set(streamer_t s, const double* ne_dev, const double* np_dev);
/* Copies out n_e, n_p, and phi and S_ph of the last right-hand-side evaluation (any NULL). */
int streamer_get(streamer_t s, double* ne_dev, double* np_dev, double* phi_dev, double* sph_dev);
/* The right-hand side L(n_e, n_p) of the current densities: (dn_e/dt, dn_p/dt). */
int streamer_rhs(streamer_t s, double* dne_dev, double* dnp_dev);
/* nsteps steps of Heun's method with step dt (s). KIFMM_ERR_TIMEOUT when a Poisson solve does
 * not reach mg_tol within mg_max_cycles. */
int streamer_step(streamer_t s, double dt, int nsteps);
/* The potential for the charge term rho_dev (the right-hand side of -Laplace(phi) = rho, V /
 * cm^2) with the boundary conditions above, into phi_dev; synchronises; *rel_residual and
 * *cycles (either may be NULL) report the solve. */
int streamer_poisson(streamer_t s, const double* rho_dev, double* phi_dev, double* rel_residual, int* cycles);
/* Multigrid levels and the last solve's cycles and relative residual. */
int streamer_info(streamer_t s, int* mg_levels, int* last_cycles, double* last_residual);
void streamer_destroy(streamer_t s);

/* ---- evaluation without device allocation ---- */

/* Largest point count kifmm_direct_noalloc accepts (its fixed work space: 8 bytes per point). */
#define KIFMM_NOALLOC_MAX_POINTS 65536

/*
 * The same sum as kifmm_eval for cells of one edge h, evaluated directly (every pair,
 * FP64) and without allocating device memory:
 *   S_dev[i] = C * ( sum_{j != i} K(|x_i - x_j|) I_j h^3  +  sigma(h) I_i ).
 * The paper has no counterpart of this entry point. It serves callers that cannot
 * allocate device memory when they need S: a stream that is being captured into a CUDA
 * graph, a real-time loop that forbids allocation after start-up, or a process whose
 * device memory belongs to another allocator. Its only work space is a fixed array in
 * device memory (KIFMM_NOALLOC_MAX_POINTS + 32 doubles, about 512 KB) that every GPU
 * loading this library holds until the process exits.
 *
 *   points_dev  device, n x 3 FP64 cell centres (distinct); n <= KIFMM_NOALLOC_MAX_POINTS
 *   h           cell edge (> 0); a, b as in kifmm_plan; C scale; self_mode as kifmm_opts
 *   I_dev, S_dev  device, n FP64 each (S fully overwritten)
 *   stream      cudaStream_t (NULL = default stream); the call is asynchronous on it.
 * The first call on a device looks up the work space's device address (with that
 * device current); make that first call before any stream capture. Every call shares
 * the work space and writes it before reading it, so nothing carries over from one call
 * to the next, but calls that overlap on the GPU (other streams, other threads) race on
 * it and must be serialised by the caller. Returns KIFMM_ERR_ARG for n beyond the limit
 * or invalid arguments, KIFMM_ERR_CUDA if a launch fails. Calls no cudaMalloc/cudaFree.
 */
int kifmm_direct_noalloc(const double* points_dev, int64_t n, double h, const double* I_dev, double* S_dev,
                         double a, double b, double C, int self_mode, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* KIFMM_H */
