/*
 * sem.h - C ABI of a GB300 (sm_103a) spectral-element screened-Poisson solver.
 *
 * Problem (Sec. 2, Eq. pde / Eq. pdeweak of Remacle, Gandham & Warburton,
 * "GPU accelerated spectral finite elements on all-hex meshes"):
 *     -div(grad u) + lambda u = s  on an unstructured all-hex mesh,
 *     u = 0 on the Dirichlet part of the boundary,
 * discretised with order-n GLL spectral elements and solved with matrix-free
 * preconditioned conjugate gradients (Algorithm 1) and the two-scale additive
 * Schwarz preconditioner P = P^c + P^f (Sec. 4).
 *
 * Conventions shared by every call
 *  - Every function returns an int status: 0 = SEM_OK, < 0 an error (see the
 *    SEM_ERR_* codes; sem_last_error() gives a message), > 0 a solver outcome.
 *  - "_dev" pointers are CUDA device pointers, "_host" pointers host pointers.
 *    The caller owns every buffer it passes; the library never frees them and
 *    keeps no reference after the call returns.
 *  - Global vectors have sem_num_dofs() float64 entries in the library's own
 *    DOF numbering; sem_dof_coords() gives the position of each DOF.
 *  - All device work is enqueued on the handle's CUDA stream (given at create,
 *    changeable with sem_set_stream). Calls that return host-visible results
 *    (sem_solve, sem_num_dofs) synchronise that stream; the other calls are
 *    asynchronous with respect to the host.
 *  - A handle is not thread safe; different handles are independent.
 */
#ifndef SEM_H
#define SEM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sem_s sem_t;

/* status codes */
#define SEM_OK             0
#define SEM_ERR_ARG       (-1)  /* bad argument (NULL pointer, order out of 2..8, sizes) */
#define SEM_ERR_JACOBIAN  (-2)  /* |J| <= 0 at some GLL node (inverted or mirrored hex) */
#define SEM_ERR_MESH      (-3)  /* non-conforming / non-manifold mesh (a face on > 2 hexes) */
#define SEM_ERR_CUDA      (-4)  /* a CUDA runtime call failed */
#define SEM_ERR_OOM       (-5)  /* device or host allocation failed */
#define SEM_ERR_NAN       (-6)  /* NaN/Inf or a non-positive p^T A p met in the solver */
#define SEM_ERR_SINGULAR  (-7)  /* coarse matrix not SPD (e.g. pure Neumann with lambda = 0) */
#define SEM_MAXIT          1    /* sem_solve: maxit reached before the tolerance */

/* sem_create flags */
#define SEM_GEOM_STORED     0x0  /* store G1..G6 and m per GLL node (Sec. 3.1, 7 factors) */
#define SEM_GEOM_RECOMPUTE  0x1  /* recompute them from the 8 vertices in the operator (Sec. 3.1) */
#define SEM_NEUMANN         0x10 /* no Dirichlet nodes (default: Dirichlet on every boundary face) */
#define SEM_MIXED           0x100 /* also keep the stored factors in FP32 and BF16, for
                                       SEM_PREC_FP32 and SEM_PREC_BF16 */
#define SEM_PATCH_FULL      0x1000 /* P^f patches with the edge and corner layers too: all (n+3)^3
                                      box nodes of Sec. 4.2 (default: face layers only) */

/* arithmetic of the operator and the preconditioner (sem_set_precision) */
#define SEM_PREC_FP64  0   /* FP64 vectors, dot products, alpha/beta and residual updates; the element
                              kernels (operator with stored or recomputed factors, patch solves) compute in
                              double-FP32: pairs of FP32 numbers with error-free sums and products on
                              the FP32 pipe, every step within a few 2^-48 of its operands' magnitudes
                              (binary64: 2^-53), which matches binary64 results to about 1e-14 of
                              their magnitude (default). On GB300 the FP64 pipe is 1/64 of the FP32
                              pipe, and these kernels were bound by it. Vector entries below 2^-80 in
                              magnitude enter with FP32 precision, below 2^-126 as zero */
#define SEM_PREC_FP32  1   /* Ax and P in FP32; vectors, dots, alpha/beta, residual updates in
                              FP64; the residual is recomputed with the FP64 operator whenever it
                              fell by 1e3 and before convergence is accepted */
#define SEM_PREC_P32   2   /* P alone in FP32 (patch solves from the FP64 residual, FP32
                              prolongation sums; the coarse AMG stays FP64); Ax, vectors, dots and
                              recurrences in FP64, so no residual replacement is needed */
#define SEM_PREC_BF16  3   /* sem_apply_A with the stored factors rounded to BF16 (half the bytes
                              of the FP32 copy) and FP32 arithmetic:
                              |y - A x| <= (2^-8 + gamma_K u32) |A|(|x|) per result, K = 4(n+1) + 16;
                              sem_apply_P* as in SEM_PREC_FP32. Needs stored geometry and SEM_MIXED.
                              The solves refuse it (SEM_ERR_ARG): on the smooth components that PCG
                              leaves last, A x is far below |A|(|x|), and the mixed solve stalls */

#define SEM_PREC_FP64_NATIVE 4  /* everything in binary64 on the FP64 pipe (the reference
                                    arithmetic for SEM_PREC_FP64) */

/* coarse solver P_0 of the two-scale preconditioner (sem_set_coarse_solver) */
#define SEM_COARSE_VCYCLE  0  /* smoothed aggregation, three V(1,1) damped-Jacobi cycles: a fixed SPD
                                 operator, plain PCG (default) */
#define SEM_COARSE_KCYCLE  1  /* the paper's (Sec. 4.1): unsmoothed aggregation, one recursive K-cycle
                                 with damped Jacobi; nonlinear, so sem_solve switches to flexible PCG */

/* how sem_solve and sem_solve_many drive the iterations (sem_set_loop) */
#define SEM_LOOP_HOST    0  /* one graph replay per iteration, the host reads the state in between */
#define SEM_LOOP_DEVICE  1  /* the whole solve is one graph (a device-evaluated while loop); with
                               sem_solve_many all solves are one graph launch (default) */
#define SEM_LOOP_EAGER   2  /* the host loop, each iteration's kernels launched one by one without
                               a graph (for profilers that list single launches) */

/* preconditioner choice for sem_solve (sem_set_precond) */
#define SEM_PRECOND_TWO_SCALE 0  /* P = P^c + P^f (Sec. 4) */
#define SEM_PRECOND_FINE      1  /* P = P^f only (Table 1, fine-scale rows) */
#define SEM_PRECOND_NONE      2  /* P = I */

/*
 * sem_create - build a problem on a hex mesh (Sec. 2.1-2.4 set-up, Sec. 4 tables).
 *   vert_xyz_host  3*n_vert doubles, x y z interleaved.
 *   hex2vert_host  8*n_hex vertex ids in 0..n_vert-1, VTK/gmsh hex corner order
 *                  (corner c has reference signs (-,-,-),(+,-,-),(+,+,-),(-,+,-),
 *                  then the same four with zeta = +1).
 *   order          polynomial order n, 2 <= n <= 8 ((n+1)^3 GLL nodes per hex). At n = 1 the
 *                  one-node patch extension reaches the neighbour's far vertex, the pencil
 *                  has no Dirichlet node and the patch problem is singular, so n = 1 is refused.
 *   lambda         screening coefficient c >= 0 (kappa = 1).
 *   flags          SEM_GEOM_* | SEM_NEUMANN.
 *   cuda_stream    cudaStream_t to enqueue work on (NULL = legacy default stream);
 *                  borrowed, must outlive its use by the handle.
 *   out            receives the handle; free it with sem_destroy.
 * The library copies the mesh; it allocates its own device work space here and
 * frees it in sem_destroy. Errors: SEM_ERR_ARG, SEM_ERR_JACOBIAN, SEM_ERR_MESH,
 * SEM_ERR_CUDA, SEM_ERR_OOM, SEM_ERR_SINGULAR.
 */
int sem_create(const double* vert_xyz_host, int64_t n_vert,
               const int64_t* hex2vert_host, int64_t n_hex,
               int order, double lambda, int flags, void* cuda_stream, sem_t** out);

/* sem_destroy - free a handle and all its device memory (NULL is ignored). */
void sem_destroy(sem_t* h);

/* sem_set_stream - enqueue the handle's later work on another stream. */
int sem_set_stream(sem_t* h, void* cuda_stream);

/* sem_num_dofs - number of global GLL nodes N (Sec. 2.2). */
int sem_num_dofs(const sem_t* h, int64_t* n_dof_host);

/* sem_num_elements - number of hexes N_E. */
int sem_num_elements(const sem_t* h, int64_t* n_hex_host);

/* sem_dof_coords - xyz_dev[3*N]: physical position of every DOF (x y z interleaved). */
int sem_dof_coords(const sem_t* h, double* xyz_dev);

/* sem_mass - m_dev[N]: assembled lumped GLL mass m_N = sum of m_{ijk;e} (Sec. 2.4, Sec. 4.1). */
int sem_mass(const sem_t* h, double* m_dev);

/* sem_get_mask / sem_set_mask - mask_dev[N] bytes, 1 = Dirichlet node, 0 = free.
 * The default mask is every node on a boundary face (or none with SEM_NEUMANN).
 * sem_set_mask rebuilds the coarse space (free vertices) and its AMG hierarchy. */
int sem_get_mask(const sem_t* h, uint8_t* mask_dev);
int sem_set_mask(sem_t* h, const uint8_t* mask_dev);

/* sem_boundary_mask - the Dirichlet mask (Eq. pde, u = 0 on the boundary part of the
 * problem statement): the same as sem_get_mask, under the name of the problem statement's
 * boundary call. The mask is handle state (set at create, changed by sem_set_mask) rather
 * than an argument of every apply and solve, because the coarse space, the AMG hierarchy
 * and the patch pencils of Sec. 4 are built from it once per change. */
int sem_boundary_mask(const sem_t* h, uint8_t* mask_dev);

/* sem_apply_mass - b_dev[N] = m_N s_N on free DOFs and 0 on Dirichlet DOFs: the load
 * vector of the weak form (Eq. pdeweak) by GLL quadrature, with the lumped mass m_N of
 * sem_mass (Sec. 2.4). s_dev[N]: the source s sampled at the DOF positions of
 * sem_dof_coords. Both are caller-owned device buffers of N doubles; they may be the
 * same buffer. Asynchronous on the handle's stream. Errors: SEM_ERR_ARG, SEM_ERR_CUDA. */
int sem_apply_mass(const sem_t* h, const double* s_dev, double* b_dev);

/* sem_coarse_levels - sizes of the coarse solver's hierarchy (Sec. 4.1): sizes_host[0] is
 * the number of free vertices (the Q1 coarse space), then one entry per aggregation level
 * below it, the last being the level solved by the dense inverse. Up to max_levels entries
 * are written (sizes_host may be NULL when max_levels is 0); *n_levels_host receives the
 * full count, 0 when there is no coarse space (no free vertex, or its set-up failed).
 * Host-only; no device work. Errors: SEM_ERR_ARG. */
int sem_coarse_levels(const sem_t* h, int max_levels, int64_t* sizes_host, int* n_levels_host);

/* sem_apply_A - y = A_D x (Eq. R / Algorithm 2 then gather, Eq. gather):
 * rows and columns of Dirichlet nodes are replaced by the identity, so
 * y_i = x_i on masked nodes. x_dev and y_dev: N doubles, must not alias. */
int sem_apply_A(sem_t* h, const double* x_dev, double* y_dev);

/* sem_apply_A_f32 - y = A x with FP32 vectors in and out (device pointers, G floats each,
 * caller-owned, x != y): the FP32 element arithmetic of SEM_PREC_FP32 (BF16 factors under
 * SEM_PREC_BF16) with no FP64 vector at all, so no conversions. Masked DOFs return x. For
 * x exactly representable in FP32 the result agrees with what sem_apply_A returns in FP32
 * precision to within 4 FP32 ulps of max|y| (the two instantiations may contract differently). Needs FP32 factors: SEM_MIXED at create, or recomputed geometry
 * (SEM_ERR_ARG otherwise). Asynchronous on the handle's stream. */
int sem_apply_A_f32(sem_t* h, const float* x_dev, float* y_dev);

/* sem_status - synchronise the handle's stream and report whether a kernel gave up a
 * bounded wait on one of its barriers since the last check (the bulk copies of the FP32
 * operator, the MMAs of the tensor-core patch solve): SEM_ERR_CUDA then, with the flag
 * cleared and that launch's results unspecified; SEM_OK otherwise. Every solve makes the
 * same check when it finishes; the asynchronous applies leave it to this call. */
int sem_status(sem_t* h);

/* sem_apply_P / sem_apply_Pf / sem_apply_Pc - z = P r with P = P^c + P^f (Sec. 4),
 * the fine overlapping-patch part P^f alone (Sec. 4.2, Eq. z) or the coarse part
 * P^c alone (Sec. 4.1, Eq. coarse). r is read as 0 on masked nodes and z is 0
 * there. r_dev and z_dev: N doubles, must not alias. */
int sem_apply_P(sem_t* h, const double* r_dev, double* z_dev);
int sem_apply_Pf(sem_t* h, const double* r_dev, double* z_dev);
int sem_apply_Pc(sem_t* h, const double* r_dev, double* z_dev);

/* sem_set_precision - SEM_PREC_FP64, SEM_PREC_FP32, SEM_PREC_P32 or SEM_PREC_BF16 for
 * sem_apply_A, sem_apply_P* and sem_solve. FP32 with stored geometry, and BF16, need
 * SEM_MIXED at create (SEM_ERR_ARG otherwise; BF16 also refuses recomputed geometry).
 * In FP32, sem_apply_A / sem_apply_P* return FP64 vectors computed with FP32 element
 * arithmetic and FP64 sums over the local copies; sem_solve still reaches rtol on the true
 * FP64 residual (the returned history holds the recomputed residual at replacements). */
int sem_set_precision(sem_t* h, int precision);

/* sem_set_patch_solver - arithmetic of the patch solves of P^f (Sec. 4.2, Eq. z) under
 * SEM_PREC_FP32, SEM_PREC_P32 and SEM_PREC_BF16:
 *   SEM_PATCH_SOLVE_FP32     FP32 on the FP32 pipe (default);
 *   SEM_PATCH_SOLVE_BF16_TC  the six contractions with S and S^T as BF16 matrix products on the
 *                            tensor cores (tcgen05, FP32 accumulation in tensor memory; box
 *                            values, S and every stage's input rounded to BF16): each patch
 *                            result within about 7 * 2^-9 of |S||S^T|(|r|). The rounding between
 *                            stages makes P^f slightly nonlinear, so sem_solve then uses the
 *                            flexible (Polak-Ribiere) beta. Handles with natural-boundary sides
 *                            (free element faces) keep the FP32 kernel, which needs no per-element
 *                            pencils in a shared tile. SEM_PREC_FP64 is unaffected.
 * Errors: SEM_ERR_ARG, SEM_ERR_OOM. A bounded wait of the tensor-core kernel that runs out is
 * reported by the next sem_solve as SEM_ERR_CUDA. */
#define SEM_PATCH_SOLVE_FP32     0
#define SEM_PATCH_SOLVE_BF16_TC  1
int sem_set_patch_solver(sem_t* h, int kind);

/* sem_set_precond - choose SEM_PRECOND_* for sem_solve (default two-scale). */
int sem_set_precond(sem_t* h, int which);

/* sem_set_loop - SEM_LOOP_DEVICE (default), SEM_LOOP_HOST or SEM_LOOP_EAGER. All run the same
 * kernels in the same order, so results are bit-identical. With the device loop a solve is captured once
 * per configuration (precision, preconditioner, coarse solver, tiles, network, rtol, maxit)
 * as a graph whose while node runs one iteration per round until the device state says
 * done (never more than maxit + 2 rounds); with profiling on (sem_profile) the host loop
 * is used. Errors: SEM_ERR_ARG. */
int sem_set_loop(sem_t* h, int mode);

/* sem_set_overlap - in the FP32 path the coarse branch (a chain of small AMG kernels) runs
 * beside the patch solves of P^f; those CTAs are then capped to fill all but reserve_sms SMs
 * (their kernel loops over the elements), so the coarse kernels find free slots instead of
 * queueing behind them. 0 = no cap. Default 48 of the GPU's 152 SMs (measured best for the
 * 32^3, n = 7 mixed solve among 24..56). Results do not depend on it. Errors: SEM_ERR_ARG. */
int sem_set_overlap(sem_t* h, int reserve_sms);

/* sem_set_weights - overlap-weighted P^f (not in the paper, which sums the patch corrections,
 * Sec. 4.2): weighted != 0 scales the residual entering the patch solves and their summed
 * result by w_N = c_N^-1/2, c_N the number of patches that contain DOF N, i.e. W P^f W, still
 * symmetric positive definite; 0 restores the paper's unweighted sum (the default). Fewer
 * iterations on the same work per iteration. Errors: SEM_ERR_ARG. */
int sem_set_weights(sem_t* h, int weighted);

/* sem_set_coarse_solver - choose P_0 (SEM_COARSE_*); rebuilds the AMG hierarchy on the host
 * (Sec. 4.1). With SEM_COARSE_KCYCLE each coarse level above the dense one takes two
 * flexible-CG steps preconditioned by the K-cycle below it, combined as the A-orthogonal
 * projection onto their span; sem_solve then uses beta_k = z_k.(r_k - r_k-1) / (z_k-1.r_k-1).
 * Errors: SEM_ERR_ARG, SEM_ERR_CUDA, SEM_ERR_OOM. */
int sem_set_coarse_solver(sem_t* h, int kind);

/*
 * sem_solve - PCG (Algorithm 1) for A_D x = b from x_0 = 0.
 *   b_dev          N doubles, read as 0 on masked nodes.
 *   x_dev          N doubles, output solution (0 on masked nodes).
 *   rtol, maxit    stop when ||r_k||_2 <= rtol ||b||_2 (recursive residual), or after
 *                  maxit operator applications.
 *   iters_host     receives the number of iterations (operator applications).
 *   res_hist_host  NULL or maxit+1 doubles: ||r_k|| / ||b|| for k = 0..iters.
 *   true_rel_res_host  NULL or receives ||b - A_D x|| / ||b|| computed afresh.
 * Returns SEM_OK on convergence, SEM_MAXIT, or an error (SEM_ERR_NAN, ...).
 * Synchronises the handle's stream.
 */
int sem_solve(sem_t* h, const double* b_dev, double* x_dev, double rtol, int maxit,
              int* iters_host, double* res_hist_host, double* true_rel_res_host);

/*
 * sem_solve_block - k independent PCG solves (Algorithm 1) of A_D x_j = b_j on one handle,
 * advanced together: every kernel of an iteration (operator, patch solves, coarse restriction
 * and V-cycles, P-sum, vector updates) is one launch over all k right-hand sides (its grid's
 * second dimension), so the tables and stored factors of the mesh serve the k solves within
 * each launch and small problems fill the GPU k times better. Each right-hand side keeps its
 * own alpha, beta and stop test; one that has converged stops changing while the others go
 * on. The whole block is one graph launch. Results are bit-identical to k sem_solve calls.
 *   k              1..SEM_MAX_BLOCK.
 *   b_dev, x_dev   k * N doubles each (right-hand side j at offset j * N), must not alias.
 *   iters_host, status_host, true_rel_res_host   NULL or k entries: iteration count,
 *                  sem_solve status (SEM_OK, SEM_MAXIT or an error) and ||b_j - A x_j|| / ||b_j||.
 * Needs SEM_PREC_FP64 or SEM_PREC_FP64_NATIVE, the V-cycle coarse solver and no attached
 * network (SEM_ERR_ARG otherwise). The first call with a larger k than before grows the
 * handle's solver work space to k slices (and rebuilds the coarse work vectors). Returns
 * SEM_OK when all converged, else the most severe status. Synchronises the handle's stream.
 */
#define SEM_MAX_BLOCK 8
int sem_solve_block(sem_t* h, int k, const double* b_dev, double* x_dev, double rtol, int maxit,
                    int* iters_host, int* status_host, double* true_rel_res_host);

/*
 * sem_solve_many - the PCG solves of `count` independent handles advanced together (the
 * batched form of Algorithm 1). With the device loop (SEM_LOOP_DEVICE, the default, on every
 * handle) all the solves are the parallel branches of one graph, launched once, each branch a
 * device-evaluated while loop; otherwise every round reads back the state of all active
 * solves, then replays each one's iteration graph on its own stream. Give every handle its
 * own CUDA stream (sem_create / sem_set_stream); a handle may appear once. b_dev[i] /
 * x_dev[i]: load and solution of handles[i], as in sem_solve (rtol, maxit shared).
 * iters_host[i] and status_host[i] (either may be NULL) receive each solve's iteration count
 * and sem_solve status. Returns SEM_OK, or the first error (or SEM_MAXIT) met. Synchronises
 * all the handles' streams.
 */
int sem_solve_many(int count, sem_t* const* handles, const double* const* b_dev,
                   double* const* x_dev, double rtol, int maxit, int* iters_host, int* status_host);

/*
 * sem_solve_many_block - sem_solve_block on `count` handles at once: every handle's block of
 * k right-hand sides (b_dev[i], x_dev[i]: k * N_i doubles, column j at offset j * N_i) is one
 * branch of one graph, launched once, so problems of different sizes and orders share the GPU
 * and each problem's kernels cover its k loads (one persistent, graph-captured launch for a
 * batch of problems with several loads each). Requirements as for sem_solve_block on every
 * handle; a handle may appear once. iters_host and status_host: NULL or count * k entries
 * (handle i's column j at i * k + j). Results are bit-identical to sem_solve_block on each
 * handle. Returns SEM_OK, or the most severe status. Synchronises the first handle's stream
 * (the graph's) and every handle's own.
 */
int sem_solve_many_block(int count, sem_t* const* handles, int k, const double* const* b_dev,
                         double* const* x_dev, double rtol, int maxit, int* iters_host, int* status_host);

/*
 * sem_set_tiles / sem_autotune - tile shapes of the element kernels: the number of
 * elements one CTA of the operator (epb_ax) and of the patch solve (epb_sw) processes,
 * 1, 2, 4 or 8 (at low order an element has only (n+1)^2 and (n+3)^2 threads). A shape not
 * compiled for the handle's order (shared-memory or thread limits) is refused with
 * SEM_ERR_ARG. sem_set_tiles sets the shapes of the FP64 and the FP32 kernels alike.
 * sem_autotune times every compiled shape on the handle's own mesh and keeps the fastest,
 * for the kernels of the precision in use only: the operator in FP32 under
 * SEM_PREC_FP32, the patch solve in FP32 under SEM_PREC_FP32 and SEM_PREC_P32, the FP64
 * kernels otherwise (so tuning once per precision tunes both sets). It overwrites the
 * handle's work vectors, so call it between solves. Results are bit-identical for every
 * shape.
 */
int sem_set_tiles(sem_t* h, int epb_ax, int epb_sw);
int sem_autotune(sem_t* h, int* epb_ax_host, int* epb_sw_host);

/*
 * sem_selfcheck_convert - checks the library's binary64 -> binary32 conversion (integer
 * operations on the IEEE-754 bit layouts, used by the PCG vector kernels that write FP32
 * copies of FP64 vectors) against the GPU's conversion instruction: each of the n 64-bit
 * patterns in bits_dev (device memory, caller-owned) as a binary64, rounded to binary32
 * (nearest, ties to even). Any bit difference counts (a NaN matches any NaN);
 * *mismatches_host (host) receives the count, 0 when they agree. Runs on the default
 * stream and synchronises. Errors: SEM_ERR_ARG, SEM_ERR_OOM, SEM_ERR_CUDA.
 */
int sem_selfcheck_convert(const uint64_t* bits_dev, int64_t n, int64_t* mismatches_host);

/*
 * sem_measure_fma_peak - arithmetic peak of one pipe, measured with the library's own
 * multiply-add loop: every thread of 8 CTAs of 256 threads per SM runs 8 independent
 * chains of `iters` fused multiply-adds in FP64 (precision = SEM_PREC_FP64) or FP32
 * (SEM_PREC_FP32) on the current device's default stream. *tflops_host receives
 * 2 x (multiply-adds) / (shortest of three timed launches, after one warm-up launch) in
 * TFLOP/s, *ms_host that launch's time. It is the denominator of the element kernels'
 * arithmetic roofline (Sec. 5 reports the kernels' GFLOP/s against the device peak). It
 * allocates and frees a small output buffer and synchronises. Errors: SEM_ERR_ARG,
 * SEM_ERR_OOM, SEM_ERR_CUDA.
 */
int sem_measure_fma_peak(int precision, int64_t iters, double* tflops_host, double* ms_host);

/*
 * sem_profile / sem_profile_read - per-kernel timing of the library's own launches.
 * While enabled, a CUDA event pair is recorded on the handle's stream around each
 * kernel launch (or launch group: "coarse_amg" is the whole AMG V-cycle sequence),
 * and the elapsed times are summed per kernel name when the stream is synchronised.
 * sem_profile(h, 1) resets the counters and enables; sem_profile(h, 0) disables.
 * sem_profile_read fills up to max_kernels entries: names_host (64 bytes each, NUL
 * terminated), launches_host (kernels launched under that name) and total_ms_host
 * (any may be NULL) and sets
 * *n_kernels_host to the number of distinct kernels seen. Synchronises the stream.
 * (Not in the paper: the tracing the paper's GFLOP/s and GB/s tables rest on.)
 */
int sem_profile(sem_t* h, int enable);
int sem_profile_read(sem_t* h, int max_kernels, char* names_host, int64_t* launches_host,
                     double* total_ms_host, int* n_kernels_host);

/*
 * sem_apply_A_noalloc - y = A_D x without any device allocation.
 * For callers that cannot call cudaMalloc: code running while a stream is being
 * captured into a CUDA graph (allocation is not allowed there), components whose
 * device memory is owned and handed out by a host framework, or loops where an
 * allocator call is not permitted. The caller passes every input and output; the
 * only scratch (one FP64 value per local GLL node, written by the element kernel and
 * summed by the gather kernel) is a file-scope static device array of
 * SEM_NOALLOC_MAX_LOCAL_NODES doubles (16 MiB), held by every GPU that loads the
 * library until the process exits. It calls no cudaMalloc, cudaFree or allocating
 * library routine. The paper has no counterpart; it computes y = A_D x with the
 * geometric factors recomputed from the vertices.
 *   order          2..8.  n_hex, n_dof: sizes; n_hex*(order+1)^3 must not exceed
 *                  SEM_NOALLOC_MAX_LOCAL_NODES, else SEM_ERR_ARG.
 *   lambda         screening coefficient >= 0.
 *   elem_xyz_dev   [n_hex][8][3] vertex coordinates of each hex, VTK corner order.
 *   l2g_dev        int32 [n_hex*(order+1)^3]: global DOF of local node i + p(j + p k).
 *   g2l_off_dev    int32 [n_dof+1], g2l_idx_dev int32 [n_hex*(order+1)^3]: for each DOF
 *                  the local nodes (element*(order+1)^3 + local) that share it.
 *   mask_dev       uint8 [n_dof], 1 = Dirichlet (y = x there), 0 = free.
 *   x_dev, y_dev   n_dof doubles each, must not alias.
 *   cuda_stream    stream to enqueue on (NULL = legacy default stream).
 * The first call on each device, with that device current, resolves the static
 * arrays' device addresses and copies the GLL tables there (a synchronous copy);
 * make that first call before any stream capture. Every call on a device shares
 * the one scratch array, which keeps the last call's contents (nothing in it needs
 * to start at zero: every entry is written before it is read), so calls that
 * overlap on the GPU (other streams, other threads) race and must be serialised by
 * the caller. Errors: SEM_ERR_ARG, SEM_ERR_CUDA (message in sem_last_error).
 */
#define SEM_NOALLOC_MAX_LOCAL_NODES 2097152
int sem_apply_A_noalloc(int order, int64_t n_hex, int64_t n_dof, double lambda,
                        const double* elem_xyz_dev, const int32_t* l2g_dev,
                        const int32_t* g2l_off_dev, const int32_t* g2l_idx_dev,
                        const uint8_t* mask_dev, const double* x_dev, double* y_dev,
                        void* cuda_stream);

/*
 * sem_heat_step - one backward-Euler step of the heat equation (Sec. 5, heat experiment).
 * The model problem c u - div(kappa grad u) = s with c = 1/dt and s = u_prev/dt + Q/(rho c_p),
 * divided by kappa, is this handle's operator with lambda = 1/(kappa dt) (give that lambda
 * to sem_create):  A u = M (lambda u_prev + g),  g = Q / (rho c_p kappa).
 *   u_prev_dev  previous field (sem_num_dofs doubles; 0 on masked DOFs).
 *   g_dev       scaled source g at the DOFs (its masked entries are ignored).
 *   u_dev       new field (may alias u_prev_dev, not g_dev).
 * The step solves A d = M (lambda u_prev + g) - A u_prev (residual with the FP64 operator)
 * by sem_solve's method (handle precision, preconditioner, network) from d = 0, i.e. with
 * u_prev as the initial guess, stopping when the residual is <= rtol ||M (lambda u_prev + g)||,
 * then u = u_prev + d. iters_host and true_rel_res_host (relative to the full right-hand
 * side) may be NULL. Returns like sem_solve. Synchronises the handle's stream.
 */
int sem_heat_step(sem_t* h, const double* u_prev_dev, const double* g_dev, double* u_dev,
                  double rtol, int maxit, int* iters_host, double* true_rel_res_host);

/*
 * Learned correction (not in the paper; an extension of the preconditioner of Sec. 4).
 * A network N maps the residual left by the two-scale preconditioner to a correction:
 * z = P r + N(r - A P r), inside flexible PCG: beta_k = z_k.(r_k - r_k-1) / (z_k-1.r_k-1)
 * (Polak-Ribiere form of Algorithm 1's beta), alpha as in Algorithm 1. For an input
 * vector v (v = r - A P r in the solver), per element e on its (order+1)^3 GLL grid:
 *   hbar = mean of the element's three box sizes (the h of the Sec. 4.2 patch solve),
 *   s_l = (v_N / m_N) hbar^2 at the node's DOF N (m_N = sem_mass), sigma_e = rms of s_l,
 *   input channels (s / sigma_e, hx/hbar, hy/hbar, hz/hbar, lambda hbar^2 / (1 + lambda hbar^2)),
 *   three 3x3x3 zero-padded correlations 5 -> 8 -> 8 -> 1 (ReLU after the first two),
 *   local correction y_l sigma_e; N(r) at a DOF = mean over its local copies; 0 on masked DOFs.
 * Weights are BF16 copies of FP32 master weights; activations and sums are FP32.
 * The flat parameter vector (sem_net_num_params() = 3041 floats) is
 * [W1, b1, W2, b2, W3, b3], W[co][ci][a][c][d] the weight of tap (a, c, d) along (i, j, k)
 * of the local node index i + p(j + p k). Inside a solve, with z0 = P r and c = N(r - A z0),
 * an iteration's direction uses z0 + c only if (z0 + c).r >= accept_theta z0.r (else z0:
 * every step stays a descent step), and the correction is switched off for the rest of the
 * solve at the first iteration k >= W with ||r_k|| >= stall_ratio ||r_k-W||, W = stall_window
 * (both set by sem_set_learned).
 *
 * sem_net_create     new network on the current device; He-normal first two layers from
 *                    the seed, last layer zero (an untrained network adds nothing).
 * sem_net_destroy    frees it; detach it from every handle (sem_set_learned(h, NULL)) first.
 * sem_net_get_params / sem_net_set_params  copy the FP32 master parameters (n must equal
 *                    sem_net_num_params()); set also resets the optimiser state.
 * sem_net_apply      out_dev = N(v_dev) for the handle's mesh (sem_num_dofs doubles each).
 * sem_net_pair       one training pair from a PCG iterate x_k of A x = b with solution x_star:
 *                    r = b - A x_k, z0 = P r (the handle's preconditioner and precision),
 *                    s_dev = r - A z0 (the network input), delta_dev = x_star - x_k - z0
 *                    (the wanted correction), all 0 on masked DOFs; r_dev and z0_dev receive
 *                    r and z0 unless NULL. Uses the solver's scratch vectors: do not overlap
 *                    it with sem_solve on the same handle.
 * sem_net_gradient   training loss of one sample (input v_dev, target t = target_dev, e.g.
 *                    the pair's s and delta) and its gradient (grad_host:
 *                    sem_net_num_params() floats, or NULL). loss_kind:
 *                    SEM_NET_LOSS_L2      mean over local nodes of (y_l - t_N / sigma_e)^2,
 *                                         y = N's local output;
 *                    SEM_NET_LOSS_ENERGY  1 + (c^T A c - 2 c^T v) / (t^T v) for c = N(v): with
 *                                         v = A t this is ||t - c||_A^2 / ||t||_A^2, the error
 *                                         norm CG minimises (one more operator application,
 *                                         in the handle's precision);
 *                    SEM_NET_LOSS_ANGLE   1 - z^T r / sqrt((z^T A z)(e^T r)) for z = z0_dev + c
 *                                         and e = t + z0_dev, with the pair's r_dev and z0_dev
 *                                         (A e = r): 1 - cos of the A-angle between z and e
 *                                         (an exact line search along z leaves 1 - cos^2 of
 *                                         ||e||_A^2), invariant to positive scaling of z.
 *                    r_dev and z0_dev may be NULL for the first two losses.
 * sem_net_train_step the same, then one Adam step (beta1 0.9, beta2 0.999, eps 1e-8) with
 *                    learning rate lr on the master weights.
 * sem_set_learned    attaches net (or detaches with NULL) to the handle's sem_solve, with the
 *                    stall rule's window (0..8; 0 = never switch off) and ratio (> 0) and the
 *                    acceptance threshold accept_theta (8, 0.5 and 0.25 recommended: the
 *                    residual norm of two-scale PCG can rise over its first few iterations;
 *                    -inf accepts every correction); the handle allocates its forward work
 *                    space (22 floats per local node).
 * sem_learned_iterations  iterations of the handle's last sem_solve whose direction used the
 *                    correction.
 * These calls synchronise the handle's stream (gradient, train, set_learned) or enqueue on
 * it (apply). Errors: SEM_ERR_ARG, SEM_ERR_OOM, SEM_ERR_CUDA.
 */
typedef struct sem_net_s sem_net_t;
int sem_net_create(uint64_t seed, sem_net_t** out);
void sem_net_destroy(sem_net_t* net);
int sem_net_num_params(void);
int sem_net_get_params(const sem_net_t* net, float* params_host, int n);
int sem_net_set_params(sem_net_t* net, const float* params_host, int n);
int sem_net_apply(sem_net_t* net, sem_t* h, const double* v_dev, double* out_dev);
int sem_net_pair(sem_t* h, const double* b_dev, const double* x_star_dev, const double* x_k_dev,
                 double* s_dev, double* delta_dev, double* r_dev, double* z0_dev);
#define SEM_NET_LOSS_L2      0
#define SEM_NET_LOSS_ENERGY  1
#define SEM_NET_LOSS_ANGLE   2
int sem_net_gradient(sem_net_t* net, sem_t* h, const double* v_dev, const double* target_dev,
                     const double* r_dev, const double* z0_dev, int loss_kind,
                     float* grad_host, double* loss_host);
int sem_net_train_step(sem_net_t* net, sem_t* h, const double* v_dev, const double* target_dev,
                       const double* r_dev, const double* z0_dev, int loss_kind, float lr,
                       double* loss_host);
int sem_set_learned(sem_t* h, sem_net_t* net, int stall_window, double stall_ratio,
                    double accept_theta);
int sem_learned_iterations(const sem_t* h, int* used_host);

/* sem_last_error - message for the last error raised on this thread ("" if none). */
const char* sem_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SEM_H */
