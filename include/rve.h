/*
 * librve -- batched RVE computational homogenisation on one NVIDIA GB300.
 *
 * C ABI of the hot path of Ullah, Kaczmarczyk, Grammatikos, Evernden, Pearce,
 * "Multi-scale computational homogenisation to predict the long-term
 * durability of composite structures" (arXiv 1610.03484):
 *
 *   macro Gauss point (T, c, t) --degradation law (Sec. 4)--> constituent
 *   tensors --RVE cell problems (Sec. 2)--> homogenised stiffness C (6x6),
 *   thermal conductivity K (3x3) and moisture diffusivity D (3x3).
 *
 * Conventions shared by every call
 *  - Return value: RVE_OK (0) or a negative RVE_ERR_* code.  rve_strerror()
 *    names a code; rve_last_error() returns a thread-local detail string for
 *    the last failing call on the calling thread.
 *  - Handles (rve_ctx, rve_mesh) are opaque and library-owned.  All device
 *    memory behind them is allocated by the library with cudaMalloc on the
 *    context's device and freed by rve_mesh_free / rve_destroy.
 *  - Host arrays passed in are read during the call only (copied); host
 *    arrays passed out are written before the call returns.  Functions whose
 *    name ends in _dev take device pointers instead and run on the context's
 *    stream; they return after enqueueing all work and the caller synchronises.
 *  - Units are SI on input and output (Pa, W/(m K), m^2/s, deg C, hours).
 *  - Voigt order is the paper's (Sec. 2, definition of the macro strain):
 *    strain (e11, e22, e33, 2e12, 2e23, 2e31), stress (s11, s22, s33, s12,
 *    s23, s31).  C is returned row-major, C[6*i + j] = dsigma_i / deps_j.
 *  - Not thread-safe per context: calls on one rve_ctx must be serialised.
 */
#ifndef RVE_H
#define RVE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ error codes */
#define RVE_OK                    0
#define RVE_ERR_INVALID_ARGUMENT (-1)  /* null pointer, size or enum out of range */
#define RVE_ERR_BAD_MESH         (-2)  /* degenerate tet, bad index, unmatched periodic faces */
#define RVE_ERR_NOT_SPD          (-3)  /* constituent tensor not positive definite */
#define RVE_ERR_NOT_CONVERGED    (-4)  /* PCG hit max_iter before rtol (results still written) */
#define RVE_ERR_NUMERIC          (-5)  /* NaN / Inf met in a reduction */
#define RVE_ERR_CUDA             (-6)  /* a CUDA runtime call failed (detail in rve_last_error) */
#define RVE_ERR_NO_DEVICE        (-7)  /* no CUDA device or wrong architecture */
#define RVE_ERR_OUT_OF_MEMORY    (-8)  /* device allocation failed */
#define RVE_ERR_STATE            (-9)  /* call order violated (e.g. homogenise before set_materials) */
#define RVE_ERR_TIMEOUT         (-10)  /* a bounded device wait gave up */
#define RVE_ERR_BOUNDS          (-11)  /* checking build only: an element's DOF index or column was
                                          out of range; the element was skipped (rve_debug_bounds) */

/* ------------------------------------------------------------- enumerations */
/* RVE boundary conditions of Sec. 2 (unified constraint approach,
 * Eqs. eq_RVE_disc_Eqs / eq_mat_C_and_D). */
#define RVE_BC_DIRICHLET 0   /* linear boundary displacement: fluctuation = 0 on the boundary */
#define RVE_BC_PERIODIC  1   /* periodic fluctuation, anti-periodic traction */
#define RVE_BC_NEUMANN   2   /* uniform traction t = sigma_bar n */

#define RVE_PREC_FP64    0   /* FP64 operator, vectors and reductions */
#define RVE_PREC_MIXED   1   /* FP32 operator and vectors, FP64 scalars, FP64 residual refinement */

#define RVE_MODE_PCG     0   /* macro_update_gauss_points: plain batched PCG for every point */

#define RVE_KERNEL_AUTO      0   /* operator kernel of the mixed inner solve (rve_options) */
#define RVE_KERNEL_CUDA_CORE 1
#define RVE_KERNEL_TENSOR    2

/* ------------------------------------------------------------------ types */
typedef struct rve_ctx_s*  rve_ctx;
typedef struct rve_mesh_s* rve_mesh;

typedef struct rve_options {
    int     device;          /* CUDA device ordinal (default 0) */
    int     precision;       /* RVE_PREC_FP64 or RVE_PREC_MIXED (default FP64) */
    double  rtol;            /* relative residual target of the cell solves (default 1e-10) */
    int     max_iter;        /* PCG iteration cap per solve (default 20000) */
    double  inner_rtol;      /* MIXED: relative tolerance of each FP32 inner solve (default 1e-6) */
    int     max_refine;      /* MIXED: maximum FP64 refinement sweeps (default 4) */
    int     check_every;     /* unused: the PCG loop tests convergence on the device every iteration */
    int     batch;           /* RVEs solved together in macro_update_gauss_points, 0 = auto */
    void*   stream;          /* cudaStream_t to run on; NULL = library-created stream */
    int     profile;         /* 1: time every operator launch with CUDA events (rve_stats.op_*) */
    int     warm_start;      /* macro_update_gauss_points: >0 solves each mesh's points in order of
                                their degradation factor and starts every batch from the previous
                                batch of the same call: 1 the nearest solution, 2 the line and 3
                                the parabola in the factor through 2 or 3 of them, 4 (default)
                                the energy-optimal (Galerkin) combination of up to three of them
                                for the mechanics without constraint rows (one operator pass over
                                the sources and a few inner products per batch; otherwise the
                                parabola, and the transport fields take the nearest);
                                0 starts every batch from zero */
    int     transport_once;  /* macro_update_gauss_points: 1 solves the thermal and moisture cell
                                problems once per mesh and call and gives all the mesh's points
                                those K and D (transport is not degraded, Sec. 5, so they are the
                                same problems); 0 (default) solves all twelve load cases for
                                every point */
    int     operator_kernel; /* MIXED inner solve, mechanics at p = 2 and 3: RVE_KERNEL_AUTO
                                (default) takes the kernel rve_autotune_schedule chose for the
                                mesh, else the matrix-free CUDA-core kernel; RVE_KERNEL_CUDA_CORE
                                that kernel; RVE_KERNEL_TENSOR the tensor-core kernel (element
                                matrices stored once per mesh and materials, 3 x TF32 products
                                with FP32 accumulation).  Other cases always use the matrix-free
                                kernel. */
    int     deterministic;   /* 1: bit-reproducible cell solves.  The scatter kernels (operator,
                                true residual, right-hand side) run once per element colour (no
                                two elements of a colour share a DOF; greedy colouring of the DOF
                                map at rve_set_bc), so every entry receives its element
                                contributions in one fixed order; forces the CUDA-core operator.
                                Slower (one launch per colour).  0 (default): one launch, the
                                atomic additions in arrival order (results agree to rounding).
                                The Jacobi diagonal is always formed colour by colour. */
} rve_options;

/* Isotropic matrix phase (Sec. 1, Sec. 7). */
typedef struct rve_matrix_props {
    double E;    /* Young's modulus [Pa] */
    double nu;   /* Poisson ratio */
    double k;    /* thermal conductivity [W/(m K)] */
    double d;    /* moisture diffusivity [m^2/s] */
} rve_matrix_props;

/* Transversely isotropic yarn, axis 1 along the local fibre direction (Sec. 6). */
typedef struct rve_yarn_props {
    double E1, E2, G12, nu12, nu23;   /* [Pa], [Pa], [Pa], -, - */
    double k1, k2;                    /* conductivity along / across the fibre */
    double d1, d2;                    /* diffusivity along / across the fibre */
} rve_yarn_props;

/* Degradation law of Sec. 4 (Eqs. alphaT, Model_final1):
 *   1 - omega = exp(-c * beta * ln(1 - T/Tg) * t), T and Tg in kelvin,
 *   c = clamp(c_wt / c_sat_wt, 0, 1), t in days = t_h / 24.
 * It scales the matrix Young's modulus (Sec. 5: only the matrix degrades);
 * apply_to_yarn != 0 scales the yarn moduli by the same factor. */
typedef struct rve_degradation {
    double beta;        /* [1/day], paper: -0.001682 */
    double Tg_C;        /* glass transition [deg C], paper: 126 */
    double c_sat_wt;    /* moisture content that maps to c = 1 [wt%] */
    int    apply_to_yarn;
} rve_degradation;

typedef struct rve_mesh_stats {
    int64_t n_vertices, n_edges, n_faces, n_tets;   /* after periodic folding if periodic */
    int64_t n_scalar_dofs;                          /* V + (p-1)E + (p-1)(p-2)/2 F */
    int64_t n_constrained;                          /* Dirichlet-masked scalar DOFs */
    int32_t p, bc;
    double  volume;
} rve_mesh_stats;

typedef struct rve_stats {
    int32_t iterations_mech;      /* PCG iterations, mechanical solve (max over RHS and batch) */
    int32_t iterations_scalar;    /* PCG iterations, thermal + moisture solve */
    int32_t refine_sweeps;        /* MIXED: FP64 residual refinement sweeps */
    int32_t converged;            /* 1 if every RHS reached rtol */
    double  rel_residual_mech;    /* final relative residual (max over RHS) */
    double  rel_residual_scalar;
    double  hill_mandel_mech;     /* |C_energy - C_sigma| / |C| (Eq. Hill_prin check) */
    double  hill_mandel_scalar;
    double  seconds;              /* wall time of the call */
    int64_t kernel_launches;      /* device kernels launched by the call */
    double  op_ms;                /* summed device time of operator launches (profile mode) */
    int64_t op_launches;          /* operator launches counted in op_ms */
    double  op_bytes;             /* algorithmic bytes of those launches: x read + y written
                                     (2 n_rows ncols sizeof(real)) + element data once */
    double  op_flops;             /* algorithmic flops of those launches (FMA = 2) */
    /* profile mode, the PCG vector kernels of the same iterations: */
    double  update_ms, update_bytes;     /* x, r read+written, p, q read (6 n_rows ncols s) */
    double  pupdate_ms, pupdate_bytes;   /* r, p read, p, q written (4 n_rows ncols s) */
    double  finalize_ms;                 /* alpha and beta/multiplier kernels */
    /* profile mode, outside the PCG iterations: */
    double  residual_ms;                 /* true residual r = b - K x: FP64 operator (FP64 mode) or
                                            double-float operator (mixed mode) */
    int64_t residual_launches;           /* true-residual applications counted in residual_ms */
    double  op_active_frac;              /* active columns / columns, averaged over operator launches */
    /* the operator launches above by class k = 2 (p - 1) + (scalar field ? 1 : 0) */
    double  op_class_ms[6];
    int64_t op_class_launches[6];
    double  op_class_bytes[6];
    double  op_class_flops[6];
    double  op_class_active_frac[6];
    /* every call: host time spent capturing and instantiating the PCG graphs, and their number */
    double  graph_host_ms;
    int64_t graphs;
} rve_stats;

/* ------------------------------------------------------------------ calls */
const char* rve_strerror(int code);
const char* rve_last_error(void);
void        rve_default_options(rve_options* opts);

/* Context on one device.  opts may be NULL (defaults).  Fails with
 * RVE_ERR_NO_DEVICE when no sm_103 device is present. */
int rve_create(rve_ctx* out, const rve_options* opts);
int rve_destroy(rve_ctx ctx);
int rve_set_options(rve_ctx ctx, const rve_options* opts);
int rve_get_options(rve_ctx ctx, rve_options* opts);

/* Tetrahedral RVE mesh with hierarchic H1 basis of order p (Sec. 1, Sec. 7):
 *   xyz [nv][3] vertex coordinates, tets [nt][4] vertex indices (any orientation),
 *   phase [nt] 0 = matrix, 1 = yarn, fibre_dir [nt][3] yarn axis (need not be
 *   normalised; ignored for matrix tets; NULL = x axis), p in 1..3.
 * The box must be axis aligned with matching opposite faces if the periodic
 * BC is used later.  The default BC is periodic. */
int rve_mesh_load(rve_ctx ctx, const double* xyz, int64_t nv, const int32_t* tets, int64_t nt,
                  const uint8_t* phase, const double* fibre_dir, int p, rve_mesh* out);
int rve_mesh_free(rve_ctx ctx, rve_mesh mesh);
int rve_mesh_info(rve_ctx ctx, rve_mesh mesh, rve_mesh_stats* out);

/* Constituent properties and the degradation state (T_C, c_wt, t_h) of the
 * macro point this RVE serves (Sec. 4, Sec. 5).  deg may be NULL: paper
 * constants, matrix only.  Fails with RVE_ERR_NOT_SPD for non-physical
 * constants. */
int rve_set_materials(rve_ctx ctx, rve_mesh mesh, const rve_matrix_props* matrix,
                      const rve_yarn_props* yarn, double T_C, double c_wt, double t_h,
                      const rve_degradation* deg);

/* Boundary condition switch of the unified constraint approach (Sec. 2). */
int rve_set_bc(rve_ctx ctx, rve_mesh mesh, int bc);

/* Solve the 6 mechanical and 3 + 3 transport unit cell problems (Eq. Eq_C_stress
 * and its scalar counterpart) and return C (row-major 6x6), K and D (3x3).
 * Any output pointer may be NULL; stats may be NULL.  Returns
 * RVE_ERR_NOT_CONVERGED (outputs still written) if rtol was not reached. */
int rve_homogenise(rve_ctx ctx, rve_mesh mesh, double* C, double* K, double* D, rve_stats* stats);

/* The paper's own route to the homogenised tensors (Sec. 2): after the cell
 * problems are solved (as rve_homogenise, whose energy-form tensors are written
 * to C_energy, K_energy, D_energy), the constraint rows C of the boundary
 * condition are written out (Eqs. eq_RVE_disc_Eqs, eq_mat_C_and_D: one row per
 * boundary DOF for linear Dirichlet; u_image - u_master per image DOF of the
 * unfolded mesh for periodic; the uniform-traction rows plus the rigid-mode rows
 * for Neumann), D = C X with X the nodal interpolant of the unit macro fields,
 * the Lagrange multipliers lambda recovered from the equilibrium of the total
 * field, K u + C^T lambda = 0, and sigma_bar = -D^T lambda / V
 * (Eq. eq_homo_stress) returned as C (6x6, column j = load case j), K and D
 * (3x3).  They equal the energy-form tensors up to the solver tolerance and
 * are not symmetrised.  Any output may be NULL.  Errors as rve_homogenise. */
int rve_homogenise_weak(rve_ctx ctx, rve_mesh mesh, double* C, double* K, double* D, double* C_energy,
                        double* K_energy, double* D_energy, rve_stats* stats);

/* Batched FE^2 evaluation (Sec. 5): for G macro Gauss points with states
 * (T_C[g], c_wt[g], t_h[g]) and RVE meshes[mesh_id[g]] (each with materials and
 * BC already set; the per-point state replaces the mesh's own), write
 * C[g*36..], K[g*9..], D[g*9..] and status[g] (RVE_OK or a negative code).
 * Points sharing a mesh are solved together, `batch` RVEs per device pass.
 * Host arrays; the copy in and out is part of the call. */
int macro_update_gauss_points(rve_ctx ctx, const rve_mesh* meshes, int n_meshes, int64_t G,
                              const double* T_C, const double* c_wt, const double* t_h,
                              const int32_t* mesh_id, double* C, double* K, double* D,
                              int32_t* status, int mode, rve_stats* stats);

/* Same with device-resident inputs and outputs (all pointers on the context's
 * device); mesh_id_host is the host copy of mesh_id used for scheduling. */
int macro_update_gauss_points_dev(rve_ctx ctx, const rve_mesh* meshes, int n_meshes, int64_t G,
                                  const double* T_C_dev, const double* c_wt_dev,
                                  const double* t_h_dev, const int32_t* mesh_id_host,
                                  double* C_dev, double* K_dev, double* D_dev,
                                  int32_t* status_dev, int mode, rve_stats* stats);

/* The same batched evaluation for points whose degradation factor 1 - omega is
 * already known (Sec. 5: the macro time loop integrates the degradation
 * parameter at every macro Gauss point and hands it to the RVE, whose matrix
 * modulus it scales).  W[g] in (0, 1] replaces the degradation law at
 * (T, c, t), so a point is handed over exactly whatever its moisture history
 * (a point that degraded and then dried out keeps its W).  The mesh's
 * apply_to_yarn choice still applies.  Fails with RVE_ERR_INVALID_ARGUMENT when
 * some W[g] lies outside (0, 1] or is NaN; otherwise as
 * macro_update_gauss_points.  Host arrays; _dev takes W and the outputs on the
 * context's device (mesh_id_host on the host, for scheduling). */
int macro_update_gauss_points_w(rve_ctx ctx, const rve_mesh* meshes, int n_meshes, int64_t G,
                                const double* W, const int32_t* mesh_id, double* C, double* K, double* D,
                                int32_t* status, int mode, rve_stats* stats);
int macro_update_gauss_points_w_dev(rve_ctx ctx, const rve_mesh* meshes, int n_meshes, int64_t G,
                                    const double* W_dev, const int32_t* mesh_id_host, double* C_dev,
                                    double* K_dev, double* D_dev, int32_t* status_dev, int mode,
                                    rve_stats* stats);

/* Batch-size autotuner for one mesh (scheduling; no counterpart in the paper).
 * Solves the n sample states (host arrays, all on mesh m) once untimed, then
 * twice per candidate batch size (candidates: n_cand sizes, or NULL / 0 for
 * {8, 16, 32, 64, 128, 256}), times each pass on the host clock (the faster of
 * a candidate's two passes counts), and keeps the
 * smallest candidate within 6 % of the fastest (a call runs several meshes at
 * once, which fill the GPU between them, so a larger batch gains less there
 * than alone): later calls with options.batch == 0 solve this mesh in batches of
 * *best.  rates (optional, n_cand or 6 entries) receives each candidate's
 * homogenisations per second (0 for one that failed).  The sample should
 * follow the distribution of the states the mesh will see: the warm starts
 * make the rate depend on how densely the degradation factors fall.  Fails
 * with RVE_ERR_STATE before rve_set_materials; a candidate that does not fit
 * in device memory ends the search with RVE_ERR_OUT_OF_MEMORY. */
int rve_autotune_batch(rve_ctx ctx, rve_mesh m, int64_t n, const double* T_C, const double* c_wt,
                       const double* t_h, const int32_t* candidates, int n_cand, int32_t* best,
                       double* rates);

/* Sharding of one batch of macro Gauss points over n_ranks processes, one GPU
 * each (scheduling; the paper runs its RVEs on distributed-memory HPC, Secs. 1
 * and 8).  cost[g] > 0 is an estimate of point g's solve cost (e.g. the DOFs
 * of its RVE times its expected PCG iterations).  Writes offsets[n_ranks + 1]:
 * rank r takes the contiguous points [offsets[r], offsets[r + 1]).  The
 * boundaries minimise the largest block cost (the linear-partition optimum,
 * found by bisection to 1e-12 of the total); imbalance (optional) receives
 * the largest block cost over the mean.  Host computation only: no context,
 * no device. */
int rve_partition_blocks(int64_t G, const double* cost, int n_ranks, int64_t* offsets, double* imbalance);

/* Schedule autotuner for one mesh (no counterpart in the paper): times every
 * pair of a batch size from batches[n_batch] and an operator kernel from
 * kernels[n_kernel] (RVE_KERNEL_CUDA_CORE, RVE_KERNEL_TENSOR) as
 * rve_autotune_batch does, on the n sample states, and keeps, of the pairs
 * within 6 % of the fastest, the smallest batch (then the faster kernel):
 * later calls with options.batch == 0 and options.operator_kernel ==
 * RVE_KERNEL_AUTO use that pair for this mesh.  rates (optional,
 * [n_kernel][n_batch]) receives homogenisations per second of each pair.
 * The tensor kernel applies to the mechanics at p = 2, 3 in MIXED precision;
 * elsewhere both candidates run the same kernel. */
int rve_autotune_schedule(rve_ctx ctx, rve_mesh m, int64_t n, const double* T_C, const double* c_wt,
                          const double* t_h, const int32_t* batches, int n_batch, const int32_t* kernels,
                          int n_kernel, int32_t* best_batch, int32_t* best_kernel, double* rates);

/* ------------------------------------------------------- learned surrogate
 * No counterpart in the paper: an ensemble of MLPs (8 features -> 4 x 256
 * SiLU -> 33 Cholesky-factor entries of the normalised C, K, D, diagonals
 * through softplus, so every prediction is SPD), trained on the GPU from
 * cell solves of this library, BF16 weights and activations with FP32
 * accumulation on the tensor cores, FP32 master weights and Adam.  The
 * ensemble spread max_e |T_e - mean| / |mean| decides when a point falls back
 * to the plain batched PCG. */
typedef struct rve_surrogate_s* rve_surrogate;

/* Ensemble of `members` (1..16) randomly initialised networks (seeded). */
int rve_surrogate_create(rve_ctx ctx, int members, uint64_t seed, rve_surrogate* out);
int rve_surrogate_free(rve_ctx ctx, rve_surrogate s);

/* The 8 features of G macro points on a mesh with materials set: (T, c_wt,
 * log10 t_h, matrix E (1-omega), yarn E1, E2, G12 (degraded if apply_to_yarn),
 * matrix k); the degradation factor runs on the device (Sec. 4).  Host arrays,
 * feat [G][8]. */
int rve_gauss_point_features(rve_ctx ctx, rve_mesh mesh, int64_t G, const double* T_C,
                             const double* c_wt, const double* t_h, double* feat);

/* Train every member on n samples (features [n][8], tensors C [n][36], K, D
 * [n][9], host) for `epochs` epochs of minibatch Adam (batch a multiple of 64,
 * n >= 64); normalisation is fitted to the data.  loss_history [epochs] may be
 * NULL. */
int rve_surrogate_train(rve_ctx ctx, rve_surrogate s, int64_t n, const double* feat,
                        const double* C, const double* K, const double* D, int epochs, int batch,
                        double lr, uint64_t seed, double* loss_history);

/* One forward/backward pass of one member on n rows (multiple of 64) without
 * updating it: target_factors [n][33] are factor entries in the network's
 * normalised units; grads receives the parameter gradient in the layout of
 * rve_surrogate_get_params (after its header); loss the mean squared error. */
int rve_surrogate_gradients(rve_ctx ctx, rve_surrogate s, int member, int n, const double* feat,
                            const float* target_factors, float* grads, double* loss);

/* Ensemble mean tensors (SI units) and spread for n feature rows (host). */
int rve_surrogate_predict(rve_ctx ctx, rve_surrogate s, int64_t n, const double* feat, double* C,
                          double* K, double* D, double* spread);

/* Inference path of rve_surrogate_predict[_dev] and the surrogate route: fused = 1
 * (default) evaluates every member's five layers for 128-row tiles in one kernel
 * with the activations kept in shared memory (ensembles of up to 4 members; larger
 * ones use the other path); fused = 0 launches one tensor-core GEMM per member and
 * layer.  Both compute the same products in the same order. */
int rve_surrogate_set_fused(rve_ctx ctx, rve_surrogate s, int fused);

/* The same on the device: feat_dev [n][8], outputs C_dev [n][36], K_dev [n][9],
 * D_dev [n][9] (SI units) and spread_dev [n], all on the context's device;
 * enqueued on the context's stream (the caller synchronises).  Uses library-owned
 * work buffers sized for chunks of 65,536 points (allocated on first use). */
int rve_surrogate_predict_dev(rve_ctx ctx, rve_surrogate s, int64_t n, const double* feat_dev, double* C_dev,
                              double* K_dev, double* D_dev, double* spread_dev);

/* Save / load: a float array [52 + members * n_params] (feature mean and std,
 * output scales, reference tensor scales, then each member's FP32 weights and
 * biases layer by layer, weights [in][out]).  With buf NULL, get_params writes
 * the required length. */
int rve_surrogate_get_params(rve_ctx ctx, rve_surrogate s, float* buf, int64_t* len);
int rve_surrogate_set_params(rve_ctx ctx, rve_surrogate s, const float* buf, int64_t len);

/* Batched FE^2 evaluation with the surrogate: points whose ensemble spread is
 * at most tau take the surrogate's mean tensors (fallback[g] = 0); the others,
 * and every point of a mesh whose surrogate is NULL, are solved by the plain
 * batched PCG of macro_update_gauss_points (fallback[g] = 1).  Host arrays. */
int macro_update_gauss_points_surrogate(rve_ctx ctx, const rve_mesh* meshes,
                                        const rve_surrogate* surrogates, int n_meshes, double tau,
                                        int64_t G, const double* T_C, const double* c_wt,
                                        const double* t_h, const int32_t* mesh_id, double* C,
                                        double* K, double* D, int32_t* status, uint8_t* fallback,
                                        rve_stats* stats);

/* ------------------------------------------------------ coupled macro step
 * The macro level of the paper's framework (Secs. 3, 4 and 5): heat and
 * moisture transport through the structure with the homogenised conductivity
 * and diffusivity (Eq. Eq_field, discretised with linear tetrahedra as
 * Eq. Eq_field_disc, consistent capacity matrix), advanced by one implicit
 * (backward Euler) step at a time, with one exposed face held at a prescribed
 * temperature and moisture content and zero flux elsewhere; then, at the four
 * Gauss points of every tetrahedron, the degradation field 1 - omega advanced
 * by backward Euler of the rate form (Eq. Eq_Model_RateForm) at the new T and c.
 * Each Gauss point is handed to the RVE path as (T, c, t_eq), t_eq being the
 * exposure time for which the closed form (Eq. Eq_Model_final1) at the point's
 * current T and c gives its 1 - omega, so that macro_update_gauss_points[_dev]
 * or the surrogate refresh its C, K, D.  A point with no moisture now (the
 * consistent-capacity transport undershoots slightly ahead of the front) gets
 * t_eq = 0, i.e. is handed over undegraded; the stats count such points that
 * had degraded and report the largest 1 - omega missed.  Nodes: xyz [nv][3] in m; tets
 * [nt][4] with positive orientation.  Temperatures in deg C, moisture in wt%,
 * time in hours.  FP64 throughout. */
typedef struct rve_macro_s* rve_macro;

typedef struct rve_macro_stats {
    int32_t iterations_T;       /* PCG iterations of the heat solve */
    int32_t iterations_c;       /* PCG iterations of the moisture solve */
    int32_t converged;          /* 1 if both reached rtol */
    int32_t gauss_points_unencodable; /* points with 1 - omega < 1 but no moisture now: t_eq = 0 hands
                                         them over as undegraded */
    double  rel_residual_T, rel_residual_c;
    double  seconds;
    double  handover_max_err;   /* largest 1 - omega among those points (the hand-over error) */
} rve_macro_stats;

/* Copies the mesh and its geometry to the device.  RVE_ERR_BAD_MESH for an
 * out-of-range index or a non-positive tetrahedron volume. */
int rve_macro_create(rve_ctx ctx, const double* xyz, int64_t nv, const int32_t* tets, int64_t nt,
                     rve_macro* out);
int rve_macro_free(rve_ctx ctx, rve_macro m);

/* Homogenised thermal conductivity K_T [3][3] (W/mK) with volumetric heat
 * capacity rho_cp (J/m^3K), and moisture diffusivity D_c [3][3] (m^2/s, unit
 * capacity).  RVE_ERR_NOT_SPD unless both are symmetric positive definite. */
int rve_macro_set_transport(rve_ctx ctx, rve_macro m, const double K_T[9], double rho_cp, const double D_c[9]);

/* The exposed face: node_mask[nv] (non-zero = held) and its temperature and
 * moisture content. */
int rve_macro_set_face(rve_ctx ctx, rve_macro m, const uint8_t* node_mask, double T_C, double c_wt);

/* Held nodes with their own values: values[node * 2 + field] (field 0 temperature,
 * 1 moisture) for the nodes with node_mask != 0.  Replaces set_face. */
int rve_macro_set_held(rve_ctx ctx, rve_macro m, const uint8_t* node_mask, const double* values);

/* Uniform initial temperature and moisture; 1 - omega = 1 at every Gauss point. */
int rve_macro_reset(rve_ctx ctx, rve_macro m, double T0_C, double c0_wt);

/* One coupled step of dt_h hours: both transport solves (Jacobi PCG to the
 * relative preconditioned residual rtol, at most max_iter iterations), then
 * the Gauss-point states.  deg NULL = paper constants.  RVE_ERR_STATE before
 * set_transport, set_face and reset; RVE_ERR_NOT_CONVERGED (fields still
 * advanced) if rtol was not reached. */
int rve_macro_step(rve_ctx ctx, rve_macro m, double dt_h, const rve_degradation* deg, double rtol, int max_iter,
                   rve_macro_stats* stats);

/* The steady problem K psi = 0 with the held values (both fields), no time
 * derivative and no degradation update: the potential solve of the yarn
 * directions below, or a macro steady state.  Same convergence rule as a step. */
int rve_macro_solve_steady(rve_ctx ctx, rve_macro m, double rtol, int max_iter, rve_macro_stats* stats);

/* Gradient of one field (0 temperature / potential, 1 moisture) per tetrahedron
 * [nt][3] (host array), constant on each linear element. */
int rve_macro_gradients(rve_ctx ctx, rve_macro m, int field, double* grad);

/* Yarn directions from potential flow (Sec. 6): for each yarn y the Laplace
 * problem grad^2 phi = 0 is solved on its own tetrahedra (yarn_of_tet[e] == y;
 * -1 = matrix), with phi = 0 on the nodes at the yarn's lower end along its
 * axis yarn_axis[y] (0 x, 1 y, 2 z), phi = 1 at its upper end and zero flux on
 * its lateral surface (linear tetrahedra, the GPU PCG of the macro step to rtol).
 * dir[e][3] (host, in/out) receives grad phi / |grad phi| for every yarn
 * tetrahedron; matrix tetrahedra, and any with zero gradient, keep their input
 * value.  The result can be passed as fibre_dir to rve_mesh_load. */
int rve_fibre_directions(rve_ctx ctx, const double* xyz, int64_t nv, const int32_t* tets, int64_t nt,
                         const int32_t* yarn_of_tet, int n_yarn, const int32_t* yarn_axis, double rtol,
                         double* dir);

/* Checkpoint / resume of the macro time loop: restores a state saved with
 * rve_macro_get (nodal T and c [nv], Gauss-point 1 - omega [nt * 4], host
 * arrays) in place of rve_macro_reset, and recomputes the Gauss-point T, c
 * and t_eq from it (deg NULL = paper constants; 1 - omega is not advanced).
 * Continuing with rve_macro_step then follows the run that saved the state.
 * RVE_ERR_INVALID_ARGUMENT for a 1 - omega outside (0, 1] or a non-finite
 * nodal value. */
int rve_macro_set_state(rve_ctx ctx, rve_macro m, const double* T_nodal, const double* c_nodal, const double* W_gp,
                        const rve_degradation* deg);

/* Device pointers to the Gauss-point arrays [nt * 4] (tet-major): temperature,
 * moisture, 1 - omega and t_eq.  Valid until the next step or free; any output
 * may be NULL.  They can be passed straight to macro_update_gauss_points_dev. */
int rve_macro_gauss_dev(rve_ctx ctx, rve_macro m, const double** T_gp, const double** c_gp, const double** W_gp,
                        const double** t_eq_gp);

/* Host copies of the nodal fields [nv] and the Gauss-point arrays [nt * 4];
 * any output may be NULL. */
int rve_macro_get(rve_ctx ctx, rve_macro m, double* T_nodal, double* c_nodal, double* T_gp, double* c_gp,
                  double* W_gp, double* t_eq_gp);

/* ------------------------------------------------- macro mechanics (FE^2)
 * The macro mechanical problem of the fully nested FE^2 step (Sec. 5): linear
 * elasticity on the macro mesh of rve_macro_create with the homogenised
 * stiffness C_bar of every macro Gauss point.  Linear tetrahedra, 3 DOFs per
 * node (u[node * 3 + component], m), K = sum over tetrahedra and Gauss points
 * of |T| / 4 B^T C_g B, FP64 Jacobi PCG on the device. */

typedef struct rve_macro_mech_stats {
    int32_t iterations;         /* PCG iterations */
    int32_t converged;          /* 1 if rtol was reached */
    double  rel_residual;       /* sqrt((r, M^-1 r) / max((f, M^-1 f), (r0, M^-1 r0))), free DOFs */
    double  seconds;
} rve_macro_mech_stats;

/* Prescribed displacements: fixed[nv * 3] (host; non-zero = held DOF) at
 * values[nv * 3] (host, m; NULL = 0, e.g. symmetry rollers).  The first call
 * also sets the starting displacement to zero. */
int rve_macro_mech_set_bc(rve_ctx ctx, rve_macro m, const uint8_t* fixed, const double* values);

/* The displacement the next solve starts from: u[nv * 3] (host, m), NULL =
 * zero.  A restart from a saved state, or a solve from rest. */
int rve_macro_mech_set_u(rve_ctx ctx, rve_macro m, const double* u);

/* The load: a uniform traction t[3] (Pa) on every element face whose three
 * vertices are all marked in face_nodes[nv] (host); each of those vertices
 * receives t |F| / 3 (the consistent nodal force).  Only boundary faces may
 * have all three vertices marked (a plane face of the body, say).  add = 0
 * replaces the load, add = 1 adds to it (several loaded faces). */
int rve_macro_mech_set_traction(rve_ctx ctx, rve_macro m, const uint8_t* face_nodes, const double t[3], int add);

/* Solves K u = f with the held DOFs at their values, starting from the
 * previous solution (a warm start across macro time steps), then forms the
 * Gauss-point stresses sigma_g = C_g B u.  C_gp[nt * 4][6][6] (Pa) is tet-major
 * in the Gauss-point order of rve_macro_gauss_dev, Voigt [xx, yy, zz, xy, yz,
 * zx] with engineering shear as the C output of macro_update_gauss_points*;
 * on the device if C_on_device (read during the call only), else a host array.
 * Each C_g enters by its symmetric part.  RVE_ERR_STATE before set_bc and
 * set_traction; RVE_ERR_NOT_CONVERGED (u and stresses still written) if rtol
 * was not reached within max_iter. */
int rve_macro_mech_solve(rve_ctx ctx, rve_macro m, const double* C_gp, int C_on_device, double rtol, int max_iter,
                         rve_macro_mech_stats* stats);

/* Host copies of u[nv * 3], the Gauss-point stresses [nt * 4][6] (Pa, Voigt
 * as above) and the nodal load [nv * 3] (N); any output may be NULL.
 * RVE_ERR_STATE for an output that has not been set or solved yet. */
int rve_macro_mech_get(rve_ctx ctx, rve_macro m, double* u, double* stress_gp, double* load);

/* ---------------------------------------------------- inspection entry points
 * These expose single steps of the path for parity tests. */

/* Degradation factor 1 - omega for n states, computed on the device by the
 * same kernel the batched path uses (Sec. 4, Eq. Model_final1).  deg NULL =
 * paper constants. */
int rve_degradation_factor(rve_ctx ctx, int64_t n, const double* T_C, const double* c_wt,
                           const double* t_h, const rve_degradation* deg, double* out);

/* Per-tet constituent tensors after rve_set_materials, as built on the device
 * (FP64): stiffness [nt][6][6] (Voigt, Pa), conductivity [nt][3][3],
 * diffusivity [nt][3][3].  Any output may be NULL. */
int rve_mesh_get_tensors(rve_ctx ctx, rve_mesh mesh, double* stiffness, double* conductivity,
                         double* diffusivity);

/* Apply the assembled-free operator y = K x of one field on the mesh's DOF
 * numbering (the current BC's; no constraint applied).  field 0 = mechanics
 * (x, y [n_scalar_dofs][3][ncols]), 1 = thermal, 2 = moisture
 * ([n_scalar_dofs][ncols]); units of the current materials; FP64. */
int rve_apply_operator(rve_ctx ctx, rve_mesh mesh, int field, int ncols, const double* x,
                       double* y);

/* The FP32 operator of the mixed-precision inner solve of the mechanics
 * (Eq. RVE_Eq_var_final, as the PCG applies it): y = sum_e s(col, phase_e) K_e x_e
 * for the active columns, with s = scale[col][phase] (phase 0 matrix, 1 yarn;
 * NULL: all ones) and energy[col] = x_col . y_col accumulated element by
 * element (NULL: not returned).  kernel 0: the tensor-core kernel (p = 2 or 3
 * only); 1: the matrix-free CUDA-core kernel.  x, y: host [n_scalar_dofs][3]
 * [ncols] in SI units (x rounded to FP32 on the way in), ncols a positive
 * multiple of 6; active (NULL: all) [ncols] nonzero for the columns to apply,
 * the others come back as zero.  Diagnostic entry point: it allocates and
 * frees its own device buffers.  RVE_ERR_TIMEOUT if a bounded device wait
 * gave up. */
int rve_apply_operator_mixed(rve_ctx ctx, rve_mesh mesh, int kernel, int ncols, const double* x,
                             const double* scale, const int32_t* active, double* y, double* energy);

/* Allocation-free variant of the operator apply, for callers that cannot
 * allocate device memory while they run: for example a host application that
 * owns all GPU memory through its own pre-sized pool and forbids further
 * cudaMalloc/cudaFree (which can also synchronise the device), or a real-time
 * loop that must not allocate.  This call allocates nothing: the caller passes
 * device buffers, and the only scratch (per-block energy partials and column
 * scales) lives in a file-scope __device__ array of about 0.9 MB that every
 * GPU loading librve holds until the process exits.  The mesh must already be
 * loaded and have materials (its device data is allocated by rve_mesh_load).
 * The paper has no counterpart of this call; it computes the same operator as
 * rve_apply_operator.
 *   field 0: mechanics, x_dev / y_dev [n_scalar_dofs][3][ncols];
 *   field 1: scalar fields, x_dev / y_dev [n_scalar_dofs][ncols], where column
 *            c uses the conductivity when c % 6 < 3 and the diffusivity otherwise.
 *   ncols must be a positive multiple of 6 and at most 96; larger values are
 *   rejected with RVE_ERR_INVALID_ARGUMENT.
 * Writes y_dev = K x_dev and energy_dev[c] = x_c . K x_c (SI units), enqueued on
 * the context's stream; the caller synchronises.  The first call on a device
 * looks up the scratch address (cudaGetSymbolAddress); make that first call
 * before any stream capture.  All calls share the one scratch array, which keeps
 * the last call's contents: calls that overlap on the GPU (different streams or
 * contexts on one device) race on it and must be serialised by the caller. */
int rve_operator_energy_noalloc(rve_ctx ctx, rve_mesh mesh, int field, int ncols,
                                const double* x_dev, double* y_dev, double* energy_dev);

/* Hierarchic DOF map of the current BC: edofs [nt][n_local] scalar DOF index of
 * each local function (4 vertex, then 6 quadratic edge, 6 cubic edge, 4 face
 * functions as p allows) and the vertex order used by each tet [nt][4]. */
int rve_mesh_get_dofmap(rve_ctx ctx, rve_mesh mesh, int32_t* edofs, int32_t* local_vertices);

/* Element colouring of the current DOF map (used by the deterministic mode):
 * colour_of[nt] (may be NULL) receives each element's colour; returns the number
 * of colours in *n_colours.  No two elements of one colour share a DOF. */
int rve_mesh_get_colouring(rve_ctx ctx, rve_mesh mesh, int32_t* colour_of, int32_t* n_colours);

/* ---------------------------------------------------------------- debugging
 * The library can be built as a checking build (RVE_BOUNDS_CHECK=1): the
 * operator, the double-float residual and the diagonal kernels then test every
 * element's DOF indices against the map's DOF count and its column against the
 * column count before any gather or scatter, count the violations, record the
 * first (element, column) and skip that element.  rve_homogenise and
 * macro_update_gauss_points[_w][_dev] then return RVE_ERR_BOUNDS when a
 * violation was counted during the call.  A release build compiles the checks out.
 *
 * rve_debug_bounds: *checking_build = 1 in a checking build; *violations, the
 * first element and column since the last reset (-1 when none); reset != 0 clears
 * the count afterwards.  Any pointer may be NULL. */
int rve_debug_bounds(rve_ctx ctx, int32_t* checking_build, int64_t* violations, int64_t* first_element,
                     int32_t* first_column, int reset);

/* Test hook of the checking build: the kernels of this mesh compare DOF indices
 * against n_nodes instead of the map's own count (0 restores it).  With a bound
 * below the count, the elements touching higher DOFs are reported and skipped,
 * while every access that does run stays inside the mesh's arrays. */
int rve_debug_set_node_bound(rve_ctx ctx, rve_mesh mesh, int64_t n_nodes);

/* The small solve of the energy-optimal warm start (warm_start = 4): the energy
 * minimisation of Sec. 2 restricted to the span of n previous solutions gives
 * G c = g with G_pk = x_p . A x_k and g_p = x_p . b.  c = G^+ g for the symmetric part
 * of G (n x n, row-major), by cyclic Jacobi rotations, with the eigenvalues at or
 * below rel times the largest dropped.  Host only: needs no context and no device.
 * RVE_ERR_INVALID_ARGUMENT for n outside [1, 8], a null pointer or rel < 0;
 * RVE_ERR_NUMERIC (c untouched) when G has a non-finite entry, no positive
 * eigenvalue, or the result is not finite. */
int rve_debug_galerkin_solve(int n, const double* G, const double* g, double rel, double* c);

#ifdef __cplusplus
}
#endif

#endif /* RVE_H */
