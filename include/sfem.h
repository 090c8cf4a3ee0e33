/*
 * sfem.h — C ABI of the GB300 FS-FEM-T4 library (libsfem.so).
 *
 * Face-based smoothed FEM with 4-node tetrahedra for 3D linear elasticity
 * (Section 2.1, STEP 1-5): per-tet volumes and shape gradients (Eq. 1,
 * Eq. 10), face smoothing domains (Fig. 1; V_k = (V_i + V_j)/4 on interior
 * faces, V_i/4 on exterior faces), smoothed gradients (Eq. 4-7), the
 * smoothed stiffness K = sum_k V_k Bbar_k^T c Bbar_k (Eq. 9), its CSR
 * assembly (the COO/CSC route of Section 3.3, Eq. 12), and iterative solves
 * of K d = f (Eq. 8) with essential conditions imposed by elimination
 * (STEP 5).  All compute runs in sm_103a CUDA kernels on the stream passed
 * to sfem_mesh_setup; there is no CPU fallback.
 *
 * Conventions (all entry points):
 *   - node and tet ids are 0-based; DOF = 3*node + component (x, y, z);
 *   - vectors of nrhs load cases are stored one after another (ndof each);
 *   - strain/stress order is Voigt (xx, yy, zz, yz, zx, xy), engineering
 *     shears (Eq. 4, Eq. 6); the material matrix is isotropic (E, nu);
 *   - every call returns an sfem_status; the library never aborts and never
 *     traps on the device.  On error, sfem_last_error() gives a message for
 *     the calling thread;
 *   - input arrays are borrowed and copied; the caller keeps ownership;
 *   - device memory is owned by the context and freed by sfem_destroy.
 */
#ifndef SFEM_H
#define SFEM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SFEM_API_VERSION 1

typedef enum sfem_status {
  SFEM_OK = 0,
  SFEM_EINVAL = -1,      /* bad argument (null pointer, size, option) */
  SFEM_EMESH = -2,       /* invalid mesh: node id out of range, degenerate or
                            non-finite tet, face shared by more than 2 tets,
                            node in more tets than the library supports */
  SFEM_ENOMEM = -3,      /* device allocation failed */
  SFEM_ENOCONV = -4,     /* iteration limit reached above the tolerance */
  SFEM_EBREAKDOWN = -5,  /* CG breakdown: p^T A p <= 0 or non-finite scalar */
  SFEM_ECUDA = -6,       /* CUDA runtime error */
  SFEM_ETIMEOUT = -7     /* a bounded device-side wait gave up */
} sfem_status;

typedef struct sfem_ctx sfem_ctx;

/* Optional device allocator (e.g. a framework's caching allocator).  When
 * alloc is NULL the library uses cudaMallocAsync/cudaFreeAsync on the
 * context stream.  alloc returns NULL on failure. */
typedef void *(*sfem_alloc_fn)(size_t bytes, void *stream, void *user);
typedef void (*sfem_free_fn)(void *ptr, size_t bytes, void *stream, void *user);

typedef struct sfem_opts {
  int inputs_on_device;  /* 1: xyz, tets, dir_*, trac_* are device pointers */
  int nrhs;              /* load cases in trac (>= 1; 0 is read as 1) */
  sfem_alloc_fn alloc;
  sfem_free_fn free;
  void *alloc_user;
  int reserved[8];       /* must be zero */
} sfem_opts;

typedef struct sfem_mesh_info {
  int64_t n_nodes, n_tets, ndof;
  int64_t n_faces, n_interior, n_boundary;   /* N_f = N_i + N_b */
  int64_t n_dir, nrhs;
  int64_t nnz;             /* scalar non-zeros of K (0 until sfem_assemble) */
  int64_t n_slivers;       /* tets with quality 6 sqrt(2) V / l_rms^3 < 1e-3 */
  int64_t n_bad_tets;      /* degenerate (V <= 1e-14 l_rms^3) or non-finite */
  int64_t n_bad_faces;     /* faces shared by more than two tets */
  int64_t max_tets_per_node;
  double min_quality, min_volume, max_volume;
  double setup_ms;         /* device time of the last setup */
} sfem_mesh_info;

/* Device CSR of the unconstrained K, owned by the context (valid until
 * sfem_destroy).  Rows and columns are DOFs; column indices ascend within a
 * row; every DOF pair of two nodes sharing a face stencil is present, even
 * when its value is numerically zero. */
typedef struct sfem_csr {
  int64_t n_rows;
  int64_t nnz;
  const int64_t *row_ptr;  /* n_rows + 1 */
  const int32_t *col;      /* nnz */
  const double *val;       /* nnz */
} sfem_csr;

/* Operators for sfem_apply and for the FP64 steps of sfem_solve. */
enum {
  SFEM_OP_CSR64 = 0,    /* assembled CSR, FP64 (needs sfem_assemble) */
  SFEM_OP_MF64 = 1,     /* matrix-free, FP64 */
  SFEM_OP_MF32 = 2,     /* matrix-free, FP32 (FP64 geometry rounded once) */
  SFEM_OP_MF32_F64 = 3, /* the FP32 matrix-free arithmetic on FP64 vectors (the operator
                           of SFEM_SOLVE_IR32_64's inner iterations) */
  SFEM_OP_NS64 = 4,     /* NS-FEM-T4 (node-based smoothing domains, one of the S-FEM models
                           of Sec. 2.1), matrix-free, FP64: V_n = sum of V_e / 4 over the
                           node's tets, eps_n their V_e-weighted strain average,
                           K = sum_n V_n Bbar_n^T c Bbar_n.  sfem_apply, and sfem_solve
                           with SFEM_SOLVE_PCG64 (op64 = SFEM_OP_NS64, precond 0, bc 0;
                           Jacobi scaling by the FS-FEM diagonal) */
  SFEM_OP_ES64 = 5      /* ES-FEM-T4 (edge-based smoothing domains, Sec. 2.1): a sixth of
                           every tet around an edge; otherwise as SFEM_OP_NS64.  The edge
                           table is built on first use (SFEM_EMESH if a node has more
                           than 96 higher-numbered neighbours) */
};

/* Solver kinds. */
enum {
  SFEM_SOLVE_PCG64 = 0,        /* Jacobi-PCG, all FP64 */
  SFEM_SOLVE_IR32_64 = 1,      /* FP64 residual/update around FP32 Jacobi-PCG */
  SFEM_SOLVE_FPCG_LEARNED = 2, /* flexible PCG with a learned coarse correction */
  SFEM_SOLVE_FCG_CNET = 3      /* truncated flexible CG with the learned coarse solve of an
                                  sfem_cnet model (opts.learned; NULL: Jacobi-PCG) */
};

typedef struct sfem_solve_opts {
  int kind;            /* SFEM_SOLVE_* */
  int op64;            /* operator of FP64 steps: SFEM_OP_CSR64 or SFEM_OP_MF64 (FS-FEM);
                          SFEM_OP_NS64 / SFEM_OP_ES64 solve the NS-FEM / ES-FEM system
                          instead (PCG64 only) */
  int rhs;             /* load case to solve (0 .. nrhs-1) */
  int u_on_device;     /* 1: u is a device pointer */
  int warm_start;      /* 1: u holds an initial guess (Dirichlet DOFs are reset) */
  int max_iter;        /* total CG iterations (0: 200000) */
  double tol;          /* relative true residual ||b - A u|| / ||b|| (0: 1e-8) */
  double inner_tol;    /* IR: FP32 residual reduction that triggers a reliable update (0: 0.1) */
  int max_outer;       /* IR: reliable updates at most (0: 200) */
  int check_every;     /* iterations between host convergence checks (0: 32) */
  const void *learned; /* FPCG_LEARNED: an sfem_learned handle (NULL: flexible CG with
                          the Jacobi preconditioner alone) */
  int fp32_vectors;    /* IR vectors: 0 FP64 p, q, r (default); 1 all FP32; 2 FP32 p, q and FP64 r;
                          3 FP32 r, p, q with a double-float correction (two FP32 words,
                          updated by compensated FP32 arithmetic; with precond 1, the
                          choice for the two-level solve: as many iterations as 0, half
                          the traffic, no FP64 arithmetic per DOF) */
  int learned_window;  /* FPCG_LEARNED stagnation guard: the correction is switched off for
                          the rest of the solve when ||r|| has not fallen 10% below its best
                          value for this many iterations (0: 100) */
  int learned_pace;    /* FPCG_LEARNED pace guard: the Jacobi-PCG iteration count to keep
                          pace with (e.g. measured on the training loads); the correction
                          is switched off when ||r|| lies more than 30x above the
                          log-linear line from ||r_0|| to the tolerance over this many
                          iterations (0: no pace guard) */
  int precond;         /* PCG64 and IR32_64 (fp32_vectors 0 or 3): 0 Jacobi; 1 Jacobi plus the
                          Galerkin coarse correction of sfem_coarse_setup */
  int bc;              /* Dirichlet conditions: 0 masked elimination, A = P K P + (I - P),
                          b = P (f - K g) + (I - P) g (default); 1 the penalty method of
                          STEP 5 (Sec. 3.3), A = K + alpha S, b = f + alpha S g with S the
                          prescribed DOFs (PCG64 with precond 0 only; SFEM_EINVAL otherwise).
                          The relative residual is then measured on this system; the
                          penalty rows cancel in the recursive residual, so tolerances
                          much below 1e-9 may end in SFEM_ENOCONV. */
  int penalty_exp;     /* bc 1: alpha = 10^penalty_exp x max_i K_ii (0: 8; at most 15) */
} sfem_solve_opts;

typedef struct sfem_solve_info {
  int status;              /* sfem_status of the solve */
  int iterations;          /* CG iterations (inner iterations for IR) */
  int outer_iterations;    /* IR refinement steps / true-residual restarts */
  int fallbacks;           /* FPCG: iterations that fell back to Jacobi; IR and
                              batch: 1 if the FP32-operator CG stagnated and FP64
                              PCG finished the solve */
  double true_relres;      /* ||b - A u||_2 / ||b||_2 in FP64, after exit */
  double bnorm;            /* ||b||_2 */
  double solve_ms;         /* device time of the solve */
  int learned_iterations;  /* FPCG: iterations run with the learned correction active */
  int reserved[3];
} sfem_solve_info;

/* sfem_mesh_setup — geometry, topology, smoothing domains, loads, BCs.
 *
 * Computes on the device, in FP64: tet volumes by Eq. 10 (absolute value)
 * and shape gradients (Eq. 1), mesh checks, the tet-neighbour and face
 * tables (the Face_in/Face_out information of Section 3.2, Fig. 7, built
 * from the tets instead of a TetGen face file), the smoothing-domain
 * volumes V_k (Fig. 1), the nodal loads of piecewise-constant tractions
 * (t * A / 3 per triangle node, A by Eq. 11; "nodal load" of Section 3.3
 * STEP 5), the Dirichlet mask and the Jacobi diagonal of A.
 *
 *   xyz       n_nodes x 3 FP64, row-major
 *   tets      n_tets x 4 int32, node ids (either orientation)
 *   E, nu     Young's modulus (> 0) and Poisson ratio (-1 < nu < 0.5)
 *   dir_dofs  n_dir DOFs with prescribed values dir_vals (may be 0 / NULL)
 *   trac_tris n_tri x 3 node ids of boundary triangles
 *   trac      nrhs x n_tri x 3 FP64 traction vectors (Pa), constant per triangle
 *   opts      may be NULL (host inputs, nrhs = 1, default allocator)
 *   stream    cudaStream_t for all work of this context (NULL: legacy stream)
 *
 * Returns SFEM_EMESH (with counts in sfem_get_info) for invalid meshes.
 * The context is created on the current CUDA device. */
int sfem_mesh_setup(sfem_ctx **out, const double *xyz, int64_t n_nodes,
                    const int32_t *tets, int64_t n_tets, double E, double nu,
                    const int32_t *dir_dofs, const double *dir_vals, int64_t n_dir,
                    const int32_t *trac_tris, const double *trac, int64_t n_tri,
                    const sfem_opts *opts, void *stream);

/* sfem_assemble — CSR of the unconstrained smoothed stiffness (Eq. 9).
 * Sums the 12x12 (exterior) and 15x15 (interior) face matrices
 * V_k Bbar_k^T c Bbar_k (Section 3.3, STEP 1-5; Eq. 12 counts their
 * entries) directly into canonical CSR.  FP64.  The arrays in *out are
 * device pointers owned by the context. */
int sfem_assemble(sfem_ctx *ctx, sfem_csr *out);

/* sfem_apply — y = A u with A = P K P + (I - P) (STEP 5 by elimination;
 * P masks the free DOFs).  u and y are device pointers of nrhs * ndof
 * entries: double for SFEM_OP_CSR64 / SFEM_OP_MF64 / SFEM_OP_MF32_F64, float for
 * SFEM_OP_MF32.
 * The matrix-free operators evaluate Eq. 9 as: per tet strain
 * eps_e = B_e u_e, per face eps_k = (V_i eps_i + V_j eps_j) / (V_i + V_j)
 * (Eq. 2-3 with V_k = (V_i+V_j)/4), stress c eps_k, scattered back through
 * the smoothed gradients. */
int sfem_apply(sfem_ctx *ctx, const void *u, void *y, int op, int nrhs);

/* sfem_solve — solve A u = b, b = P (f - K g) + (I - P) g (Eq. 8 with
 * STEP 5; f from the tractions plus f_extra, g the prescribed values).
 * f_extra: NULL or ndof FP64 nodal forces (host unless u_on_device).
 * u: ndof FP64, output (and input for warm_start).  Stops on the FP64 true
 * relative residual <= tol.  Returns SFEM_ENOCONV / SFEM_EBREAKDOWN with
 * the final residual in info. */
int sfem_solve(sfem_ctx *ctx, const double *f_extra, double *u,
               const sfem_solve_opts *opts, sfem_solve_info *info);

/* sfem_batch_solve — solve every load case of every context together (the
 * batched form of sfem_solve's SFEM_SOLVE_IR32_64; no counterpart in the
 * paper, which solves one model at a time).  Each round is one persistent
 * cooperative launch running FP32-operator CG iterations (FP64 vectors and
 * reductions) for all active systems, followed by the FP64 refresh (u += d,
 * true residual f - K u, convergence test, residual replacement) of the
 * systems that stopped; rounds are captured once as a CUDA graph and
 * replayed until every system has converged.
 *   ctxs  n contexts on the current device (any sizes, nrhs each); the
 *         work runs on ctxs[0]'s stream
 *   u     n pointers, u[i] holding nrhs_i x ndof_i FP64 (host, or device if
 *         opts->u_on_device); input with warm_start, output always
 *   infos sum(nrhs_i) entries (may be NULL), in context then load-case order
 *   stats may be NULL
 * Returns SFEM_OK when every system converged, else the first failure;
 * SFEM_ETIMEOUT if a bounded grid barrier gave up. */
typedef struct sfem_batch_opts {
  double tol;            /* relative true residual per system (0: 1e-8) */
  double inner_tol;      /* reliable-update trigger (0: 0.1) */
  int max_iter;          /* CG iterations per system (0: 200000) */
  int max_rounds;        /* rounds at most (0: 400) */
  int iters_per_launch;  /* CG iterations per persistent launch at most (0: 2000) */
  int u_on_device;
  int warm_start;
  int autotune;          /* 1: time 1..max CTAs per SM on the first rounds (cached per shape) */
  int use_graph;         /* 1: capture a round as a CUDA graph */
  int precond;           /* 0: the persistent Jacobi solve of all systems together; 1: each
                            system by the two-level mixed solve of its context (coarse space
                            built on first use where possible, see patch_nodes; inner_tol 0:
                            0.03);
                            2: the persistent solve of all systems together with the two-level
                            preconditioner of each context inside the launch (restriction,
                            coarse product and prolongation as phases of the persistent
                            kernel; coarse spaces built on first use, see patch_nodes,
                            and kept by the contexts; a beam without one runs Jacobi;
                            inner_tol 0: 0.03) */
  int patch_nodes;       /* precond 1 and 2: patch width (node spacings) of the coarse spaces
                            the batch builds for contexts that have none (0: 6; the library's
                            default grid if that setup fails); -1: no coarse space is built,
                            contexts without one run Jacobi (inside the launch with precond 2) */
  int reserved[3];
} sfem_batch_opts;

typedef struct sfem_batch_stats {
  int rounds;             /* persistent launches */
  int ctas_per_sm;        /* launch shape chosen by the autotuner (or 1) */
  int graph;              /* 1 if the rounds ran as a CUDA graph */
  int n_systems;
  long long total_iterations;  /* CG iterations summed over systems */
  double ms;              /* device time of the whole batch */
  int fallback_systems;   /* systems that stagnated on the FP32 operator (three
                             refreshes in a row improving the true residual by
                             less than 10%) and were finished by FP64 PCG (with the
                             two-level preconditioner where a coarse space exists) */
  int launch_iterations;  /* iterations of the persistent launches (each steps every
                             active system once), summed over launches */
  float fallback_ms;      /* device time of the FP64 PCG fallbacks (part of ms) */
  int reserved[1];
} sfem_batch_stats;

int sfem_batch_solve(sfem_ctx *const *ctxs, int n, double *const *u, const sfem_batch_opts *opts,
                     sfem_solve_info *infos, sfem_batch_stats *stats);

/* ---- two-level preconditioner (no counterpart in the paper) --------------
 *
 * M^-1 = D^-1 + Pi A_c^-1 Pi^T with A_c = Pi^T A Pi (Galerkin).  Pi holds one
 * trilinear function per patch centre and displacement component on a
 * d0 x d1 x d2 grid of centres over the mesh's bounding box (centre i at
 * lo + (i + 1/2) ext / d), masked by P.  sfem_coarse_setup builds Pi and
 * A_c with the FP32 matrix-free operator (tile by tile, or by probing with
 * 3 x prod(min(5, d_a)) applies), factors A_c by a banded blocked Cholesky
 * (FP32 or FP64, see factor) and keeps C = A_c^-1 in FP32 on the device
 * (3P <= 8192; patches at least 2.5 node spacings wide where d_a >= 5).
 * Solves use it with sfem_solve_opts.precond = 1.  Returns SFEM_EBREAKDOWN
 * if A_c is not positive definite. */
typedef struct sfem_coarse_opts {
  int patch_dims[3];   /* centres per axis (0: about patch_nodes nodes per patch axis) */
  int patch_nodes;     /* 0: 8, widened (9, 10, ...) while the axes left at 0 give more than
                          8192 coarse DOFs */
  int assembly;        /* A_c: 0 tile by tile (each tile applies its part of the operator to
                          the coarse functions of the cells it touches; probing is used for
                          a tile that touches more than 4 cells on an axis); 1 probing with
                          the whole operator in colour classes */
  int factor;          /* Cholesky of A_c: 0 FP32 (C is FP32 in any case; cond(A_c) ~ 1e5 on
                          the 2M-tet beam), switching to FP64 on a non-positive pivot;
                          1 FP64 */
  int reserved[6];
} sfem_coarse_opts;

int sfem_coarse_setup(sfem_ctx *ctx, const sfem_coarse_opts *opts);
int sfem_coarse_info(const sfem_ctx *ctx, int *patch_dims /* 3 */, int *n_coarse, int *probes,
                     double *setup_ms);
/* z = D^-1 r + P Pi C Pi^T r for one masked residual r (device, ndof FP64). */
int sfem_coarse_apply(sfem_ctx *ctx, const double *r, double *z);

/* ---- learned coarse correction (no counterpart in the paper) -------------
 *
 * A small network maps the residual, pooled over a regular grid of patches,
 * to a coarse displacement correction used inside flexible PCG
 * (SFEM_SOLVE_FPCG_LEARNED):
 *   patches   a d0 x d1 x d2 grid of boxes over the mesh's bounding box; a
 *             node belongs to the box holding it;
 *   pooling   mean nodal residual per patch (3 values);
 *   inputs    per patch 84 values: the pooled residuals of its 3x3x3 patch
 *             neighbourhood (zero outside the grid), k-major over the offsets
 *             (-1,0,1)^3 and then the component, divided by the RMS of all
 *             pooled values; then the patch centre normalised to [0,1]^3;
 *   network   84 -> 128 -> GELU -> 128 -> GELU -> 3 (GELU with the exact
 *             error function); parameters are one FP32 vector in the order
 *             W1 (84 x 128, row-major, input-major), b1, W2 (128 x 128), b2,
 *             W3 (128 x 3), b3 (n_params = 27523); inference uses BF16 copies
 *             of the parameters (round to nearest even) for the weights, FP32
 *             biases and FP32 accumulation;
 *   prolong   trilinear interpolation of the patch outputs between patch
 *             centres (clamped to the outermost centres), masked by P: c;
 *   z         D^-1 r + alpha c with alpha = c.r / c.A c (c.A c by the FP32
 *             matrix-free operator); an unusable c (c.A c <= 0, non-finite
 *             alpha or z.r) gives z = D^-1 r for that iteration.
 * Training targets are the pooled errors u* - x of the same snapshots,
 * divided by their RMS; the loss is sum((y - T)^2) / rows.  A model is bound
 * to the mesh, device and stream of the context it was created on. */
typedef struct sfem_learned sfem_learned;

typedef struct sfem_learned_opts {
  int patch_dims[3];   /* patch grid (0: about patch_nodes nodes per patch axis) */
  int patch_nodes;     /* 0: 8 */
  uint64_t seed;       /* initial parameters: He-normal weights by a counter-based
                          generator (splitmix64 + Box-Muller), zero biases */
  int reserved[6];
} sfem_learned_opts;

/* Create a model on ctx's mesh with freshly initialised parameters. */
int sfem_learned_create(sfem_learned **out, sfem_ctx *ctx, const sfem_learned_opts *opts);
void sfem_learned_destroy(sfem_learned *m);
int sfem_learned_info(const sfem_learned *m, int *patch_dims /* 3, may be NULL */,
                      int *n_patches, int *n_params);
/* FP32 master parameters from / to HOST memory (n = n_params); setting them
 * resets the Adam state. */
int sfem_learned_set_params(sfem_learned *m, const float *theta, int64_t n);
int sfem_learned_get_params(sfem_learned *m, float *theta, int64_t n);
/* Versioned blob (HOST memory): 8 int32 (magic, version 1, 84, 128, 3,
 * patch dims) then the FP32 parameters.  export with buf = NULL only
 * reports the size. */
int sfem_learned_export(sfem_learned *m, void *buf, size_t cap, size_t *size);
int sfem_learned_import(sfem_learned *m, const void *buf, size_t size);
/* Y (rows x 3) = network(X (rows x 84)) with the BF16 inference path;
 * device pointers. */
int sfem_learned_forward(sfem_learned *m, const float *X, float *Y, int64_t rows);
/* Features X (n_patches x 84) of the residual r and, if e is not NULL,
 * targets T (n_patches x 3) = pooled e / RMS; device pointers (r, e: ndof
 * FP64). */
int sfem_learned_sample(sfem_learned *m, sfem_ctx *ctx, const double *r, const double *e,
                        float *X, float *T);
/* z = D^-1 r + alpha c for one residual (device FP64, ndof); alpha to host. */
int sfem_learned_correction(sfem_learned *m, sfem_ctx *ctx, const double *r, double *z,
                            double *alpha);
/* Run the flexible PCG of opts (kind SFEM_SOLVE_FPCG_LEARNED, opts->learned
 * NULL for a Jacobi-PCG trajectory or m for the model's own) on ctx and
 * write one training sample per snapshot (before the first iteration and
 * every opts->check_every iterations): features of r into X and targets of
 * u_star - x into T (device; n_patches rows each) while rows fit in
 * cap_rows.  u_star: device FP64 reference solution.  *rows: rows written. */
int sfem_learned_collect(sfem_learned *m, sfem_ctx *ctx, const sfem_solve_opts *opts,
                         const double *u_star, float *X, float *T, int64_t cap_rows,
                         int64_t *rows, sfem_solve_info *info);
/* Loss and gradient (FP32 forward and backward with the FP32 master
 * parameters) of rows samples; grad: device, n_params floats (may be NULL);
 * loss: host (may be NULL). */
int sfem_learned_loss_grad(sfem_learned *m, const float *X, const float *T, int64_t rows,
                           float *grad, double *loss);
/* One Adam step (Kingma & Ba, bias-corrected) with grad (device; NULL: the
 * gradient of the last loss_grad). */
int sfem_learned_adam(sfem_learned *m, const float *grad, float lr, float b1, float b2, float eps);
/* epochs of mini-batch Adam (b1 0.9, b2 0.999, eps 1e-8) over rows samples
 * (device X, T), each epoch visiting rows in the order r -> (a r + b) mod
 * rows with a, b drawn from seed; loss (host, may be NULL): mean loss over
 * all rows afterwards. */
int sfem_learned_train(sfem_learned *m, const float *X, const float *T, int64_t rows,
                       int64_t batch_rows, int epochs, float lr, uint64_t seed, double *loss);

/* Learned coarse solve (no counterpart in the paper, which solves directly;
 * the spec addition of a network that maps a pooled residual to a
 * coarse displacement correction).  The model works on the coarse space of
 * sfem_coarse_setup (trilinear functions of a grid of patch centres, n_c =
 * 3 x centres coarse DOFs):
 *   input     x = r_c / RMS(r_c), r_c = Pi^T r (restriction = weighted
 *             pooling of the residual over the cells around each centre);
 *   network   n_c -> hidden -> GELU -> hidden -> GELU -> n_c (GELU with
 *             the exact erf), BF16 weights, FP32 biases and accumulation at
 *             inference, FP32 master weights for training;
 *   correction z = D^-1 r + alpha P Pi y, alpha = y.r_c / y.A_c y (the
 *             A-optimal step along the correction, formed on the coarse level
 *             with the FP32 A_c kept by sfem_coarse_setup; 0, and counted in
 *             info.fallbacks, when y.A_c y <= 0 or alpha is not finite);
 *   targets   t = A_c^-1 r_c / RMS: the Galerkin coarse solution, whose
 *             prolongation is the A-orthogonal projection of the error onto the
 *             coarse space; training rows (x, t) are collected from the
 *             library's own solves (sfem_cnet_solve);
 *   solver    flexible CG with each new direction A-orthogonalised against the
 *             last `window` directions (SFEM_SOLVE_FCG_CNET); with the Jacobi
 *             preconditioner alone (model NULL) it is Jacobi-PCG.
 * Parameters are one FP32 vector: W1 (n_c x hidden, input-major), b1, W2
 * (hidden x hidden), b2, W3 (hidden x n_c), b3.  A model is bound to the
 * context (device, stream, mesh, coarse space) it was created on. */
typedef struct sfem_cnet sfem_cnet;

typedef struct sfem_cnet_opts {
  int hidden;     /* hidden width (0: 128; a multiple of 32, at most 256) */
  uint64_t seed;  /* initial parameters: He-normal weights by a counter-based generator
                     (splitmix64 + Box-Muller), zero biases */
  int reserved[6];
} sfem_cnet_opts;

/* Training-row collection and direction window of sfem_cnet_solve. */
typedef struct sfem_cnet_run {
  int window;          /* directions the new one is A-orthogonalised against (0: 5; 1 .. 8) */
  int snap_every;      /* a training row every this many iterations (0: none) */
  float *X, *T;        /* DEVICE row buffers, cap_rows x n_c floats each */
  int64_t cap_rows;
  int64_t rows;        /* in: rows already in the buffers; out: rows after the solve */
  int reserved[4];
} sfem_cnet_run;

/* Create a model on ctx (after sfem_coarse_setup) with fresh parameters;
 * SFEM_EINVAL without a coarse space or with a bad width. */
int sfem_cnet_create(sfem_cnet **out, sfem_ctx *ctx, const sfem_cnet_opts *opts);
void sfem_cnet_destroy(sfem_cnet *m);
int sfem_cnet_info(const sfem_cnet *m, int *n_coarse, int *hidden, int64_t *n_params);
/* FP32 parameters from / to HOST memory (n = n_params); set resets Adam. */
int sfem_cnet_set_params(sfem_cnet *m, const float *theta, int64_t n);
int sfem_cnet_get_params(sfem_cnet *m, float *theta, int64_t n);
/* Y[r] = network(X[r] / RMS(X[r])) by the inference path (BF16 weights);
 * DEVICE X, Y (rows x n_c). */
int sfem_cnet_forward(sfem_cnet *m, sfem_ctx *ctx, const float *X, float *Y, int64_t rows);
/* Loss sum((y - T)^2) / rows (FP32 master weights) and its gradient (DEVICE
 * grad, n_params, may be NULL); loss to host. */
int sfem_cnet_loss_grad(sfem_cnet *m, const float *X, const float *T, int64_t rows, float *grad, double *loss);
/* epochs of mini-batch Adam (0.9, 0.999, 1e-8), rows visited in the order
 * r -> (a r + b) mod rows with a, b drawn from seed; loss: mean of the last
 * epoch (host, may be NULL). */
int sfem_cnet_train(sfem_cnet *m, const float *X, const float *T, int64_t rows, int64_t batch_rows, int epochs,
                    float lr, uint64_t seed, double *loss);
/* Rows first .. first + count - 1 of the DEVICE buffers X, T (n_c floats
 * each): x standard normal (counter-based generator of (seed, entry)), t =
 * A_c^-1 x by the coarse setup's FP32 inverse, both divided by their RMS.
 * Rows that teach the network the coarse solve in every direction, beside
 * the rows of the solver's own residuals. */
int sfem_cnet_random_rows(sfem_cnet *m, sfem_ctx *ctx, float *X, float *T, int64_t first, int64_t count,
                          uint64_t seed);
/* z = D^-1 r + alpha P Pi y for one residual (DEVICE r, z: ndof FP64); alpha
 * to host. */
int sfem_cnet_correction(sfem_cnet *m, sfem_ctx *ctx, const double *r, double *z, double *alpha);
/* A solve of opts (rhs, tol, max_iter, op64 CSR64 or MF64, u_on_device,
 * warm_start) by truncated flexible CG with the model (m NULL: Jacobi),
 * appending training rows to run (may be NULL).  Status as sfem_solve. */
int sfem_cnet_solve(sfem_cnet *m, sfem_ctx *ctx, const sfem_solve_opts *opts, double *u, sfem_cnet_run *run,
                    sfem_solve_info *info);

int sfem_get_info(const sfem_ctx *ctx, sfem_mesh_info *info);

/* Copies of setup results to HOST buffers (for checks and post-processing). */
int sfem_get_geometry(sfem_ctx *ctx, double *vol /* n_tets */,
                      double *grad /* n_tets x 4 x 3 */);
int sfem_get_neighbors(sfem_ctx *ctx, int32_t *nbr /* n_tets x 4, -1 exterior */);
/* Faces in library order: nodes (a, b, c, d0, d1) with d1 = -1 on exterior
 * faces (a < b < c), adjacent tets (t0, t1 = -1 exterior), and V_k. */
int sfem_get_faces(sfem_ctx *ctx, int32_t *nodes /* n_faces x 5 */,
                   int32_t *tets /* n_faces x 2 */, double *Vk /* n_faces */);
int sfem_get_rhs(sfem_ctx *ctx, double *b /* ndof */, int rhs);

/* sfem_recover — strain and stress recovery for output (post-processing,
 * Sec. 3.4: strain and stress from the nodal displacements, written with the
 * mesh for visualisation).
 *   u            DEVICE pointer, ndof doubles (a displacement field, e.g. the
 *                solution of sfem_solve);
 *   face_strain  DEVICE, n_faces x 6 or NULL: the smoothed strain
 *                eps_k = Bbar_k u_k of every face (Eq. 5-7) in the order of
 *                sfem_get_faces, Voigt (xx, yy, zz, yz, zx, xy) with
 *                engineering shear strains (Eq. 4);
 *   face_stress  DEVICE, n_faces x 6 or NULL: sigma_k = D eps_k;
 *   node_strain, node_stress  DEVICE, n_nodes x 6 or NULL: the means of
 *                eps_k and sigma_k over the faces whose triangle contains
 *                the node, weighted by V_k;
 *   node_vm      DEVICE, n_nodes or NULL: von Mises stress of node_stress.
 * FP64.  The nodal sums are accumulated by atomics (rounding order not
 * fixed).  Output pointers may be NULL; the call synchronises the context
 * stream.  Returns SFEM_EINVAL for a context without setup or a NULL u. */
int sfem_recover(sfem_ctx *ctx, const double *u, double *face_strain, double *face_stress, double *node_strain,
                 double *node_stress, double *node_vm);
int sfem_get_diag(sfem_ctx *ctx, double *diag /* ndof, diagonal of A */);

/* sfem_apply_noalloc — y = A u like sfem_apply(ctx, u, y, SFEM_OP_MF64, 1),
 * but allocating no device memory (the paper has no counterpart).  For
 * callers that must not allocate per call: an application whose memory pool
 * (another framework's caching allocator) already holds the device memory,
 * and latency-bound loops that apply the operator thousands of times, where
 * an allocation or a free may synchronise the device.
 *   u, y   device pointers, ndof doubles each (one load case);
 *   limit  meshes of at most 131072 tets (SFEM_EINVAL beyond, with a message);
 *   scratch a fixed 8 MiB array inside the library, held by every GPU that
 *          loads it until the process exits, shared by all calls: calls that
 *          overlap on the GPU (several streams or contexts) race on it.
 * The first call on a device looks up the scratch address (with the
 * context's device current) and keeps it for the life of the process; make
 * that first call before any stream capture.  A device reset
 * (cudaDeviceReset) ends every context of this library and also the
 * validity of that kept address: the entry point is not usable after one.
 * Work runs on the context stream.  No cudaMalloc/cudaFree is called. */
int sfem_apply_noalloc(sfem_ctx *ctx, const double *u, double *y);

/* Measurement helpers (no counterpart in the paper).
 * sfem_time_operator: launches the raw operator y = K u (no masking) of
 * `op` `reps` times on library-owned scratch vectors (u: deterministic
 * values in [-1, 1), y accumulating), exactly as the solvers launch it,
 * between CUDA events on the context stream; writes the mean device time
 * per application in milliseconds.
 * sfem_launch_count: kernels launched by this process through the library
 * so far (graph launches count their kernel nodes; captures do not count). */
int sfem_time_operator(sfem_ctx *ctx, int op, int reps, double *ms_per_apply);

/* sfem_selftest_barrier — diagnostic (no counterpart in the paper): runs the
 * bounded wait of the batched solver's grid barrier in a state where it
 * cannot complete (one block, the arrival count offset by one), so that the
 * wait runs out as it would if a block of the persistent kernel never
 * arrived.  *status receives SFEM_ETIMEOUT when the barrier gave up and
 * reported it (the expected outcome), SFEM_OK if it did not; *wait_ms (may
 * be NULL) the device time of the wait (a few seconds).  The context stays
 * usable.  Returns SFEM_EINVAL for a context without setup or a NULL status. */
int sfem_selftest_barrier(sfem_ctx *ctx, int *status, double *wait_ms);
int64_t sfem_launch_count(void);

/* sfem_gemm_f32 — diagnostic (no counterpart in the paper): the FP32 GEMM
 * that trains both learned corrections, alone.  C = op(A) op(B), row-major,
 * M x N with inner dimension K; op(A) = A^T when ta != 0 (A stored K x M,
 * leading dimension lda), else A (M x K); op(B) = B^T when tb != 0 (B stored
 * N x K), else B (K x N).  All three are DEVICE pointers of the current
 * device (not overlapping C); the call runs on its legacy default stream,
 * synchronises, and writes the GEMM's device time to *ms (may be NULL).
 * K = 0 writes zeros (A and B may then be NULL).
 * Tensor cores (tcgen05, TF32 operands split in three products for FP32
 * accuracy, FP32 accumulation), split over K when the output has fewer
 * 128 x 128 tiles than the device has SMs.  Returns SFEM_EINVAL for bad
 * sizes, leading dimensions or NULL pointers, SFEM_ETIMEOUT if a CTA gave up waiting for its
 * MMAs (C is then incomplete), SFEM_ECUDA on a CUDA error. */
int sfem_gemm_f32(int M, int N, int K, const float *A, int lda, int ta, const float *B, int ldb, int tb, float *C,
                  int ldc, double *ms);

/* sfem_tile_info — diagnostic (no counterpart in the paper): the layout of
 * the FP32 tiled operator of a context.  Writes up to n of, in order:
 *   [0] tiles, [1] largest halo (tets), [2] largest node list, [3] length of
 *   a tile's force-slot arrays, [4] total halo tets, [5] total tile nodes,
 *   [6] shared memory of the one-CTA-per-tile kernel (bytes), [7] shared
 *   memory of the persistent prefetching kernel for FP32 vectors (bytes),
 *   [8] its grid (0: the one-CTA-per-tile kernel runs instead), [9] its
 *   threads per CTA.
 * Returns SFEM_EINVAL for a context without setup, a NULL out or n < 1. */
int sfem_tile_info(sfem_ctx *ctx, int64_t *out, int n);

void sfem_destroy(sfem_ctx *ctx);
const char *sfem_strerror(int status);
const char *sfem_last_error(void);
int sfem_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SFEM_H */
