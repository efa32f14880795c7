/*
 * md.h -- C ABI of the GB300 library for the neural-preconditioned solve of
 * the discretised 3D-1D coupled elliptic problem (arXiv 2505.08491).
 *
 * The problem (Section 2, eq. (problem)) couples Q1 diffusion on the unit
 * cube Omega to a P1 problem on an embedded 1D graph Lambda through the
 * cross-section average T_Lambda.  Its Galerkin discretisation is the block
 * system of eq. (mainsys),
 *
 *     A u = b,   A = K + beta M,   u = [u0 ; u1],
 *
 * u0: Q1 nodal values on the (N+1)^3 grid of the unit cube (x fastest),
 * u1: P1 nodal values on the 1D mesh of the graph.  The solve is flexible
 * GMRES (Section 4) right-preconditioned by the block upper-triangular
 * preconditioner of eq. (twosteps): an exact 1D solve followed by a
 * convolutional network standing in for the inverse of the 3D block
 * C = K00 + beta M00 (eq. (decoupled_3d_problem), (matrixC)).  Variants
 * declared below: the block lower-triangular order, Jacobi pre- and
 * post-smoothing around the network (Section 5), and the 3D solve as inner
 * FGMRES steps with the network as their preconditioner (Section 6).
 *
 * Conventions shared by every entry point
 *   - Vectors are DEVICE pointers owned by the caller, laid out as
 *     [u0 (n3 entries, grid node (i,j,k) at i + (N+1)(j + (N+1)k)) ; u1 (n1)].
 *   - Handles (md_op, md_cnn, md_batch) own their device memory; only the
 *     matching *_destroy frees it.
 *   - md_stream is a cudaStream_t passed as void*.  Calls are asynchronous on
 *     that stream unless stated; scalar outputs written to host memory are
 *     valid when the call returns (those calls synchronise the stream).
 *   - Every call returns an md_status; md_last_error() gives a thread-local
 *     message for the last failure.  No exception crosses the ABI.  There is
 *     no CPU fallback: without a usable GPU the calls return MD_ERR_CUDA.
 *   - Calls on one handle must not overlap on the GPU (a handle keeps scratch
 *     buffers); order them on one stream or synchronise between streams.
 */
#ifndef MD_H
#define MD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef void* md_stream;
typedef struct md_op md_op;
typedef struct md_cnn md_cnn;
typedef struct md_batch md_batch;

typedef enum {
    MD_OK = 0,
    MD_NOT_CONVERGED = 1,       /* solve ended at maxit above tol; x holds the last iterate */
    MD_ERR_ARG = -1,            /* invalid argument (sizes, null pointers, graph not a forest ...) */
    MD_ERR_OOM = -2,            /* device allocation failed */
    MD_ERR_CUDA = -3,           /* a CUDA runtime call failed (no GPU, launch error ...) */
    MD_ERR_TIMEOUT = -4,        /* a bounded device-side wait ran out */
    MD_ERR_NAN = -5,            /* non-finite value where a finite one is required */
    MD_ERR_IO = -6,             /* file missing, short, or failed checksum */
    MD_ERR_UNIMPLEMENTED = -7
} md_status;

typedef enum { MD_FP32 = 0, MD_FP64 = 1 } md_prec;

/* The 1D graph Lambda (Section 2): straight segments between nodes.  The
 * graph must be a forest (no cycles).  Every edge is split into
 * elems_per_edge P1 elements of equal length.  Host pointers. */
typedef struct {
    int n_nodes;
    const double* xyz;          /* n_nodes * 3 coordinates inside (0,1)^3 */
    int n_edges;
    const int* edges;           /* n_edges * 2 node ids */
    int elems_per_edge;         /* >= 1 */
} md_graph;

/* Coefficients and boundary conditions of eq. (problem).  NULL selects
 * k_omega = 1, sigma_omega = 0, k_lambda = 1, homogeneous Dirichlet
 * conditions on the cube faces and natural conditions at every graph end.
 * The 1D diffusion coefficient used is k_lambda * pi R^2 (the |D| weight of
 * a_Lambda, eq. (alambda)).
 *   natural_boundary = 1: the natural (Neumann) condition of eq. (problem)
 *     on the cube faces: every grid node is an unknown (sigma_omega > 0 or a
 *     1D Dirichlet node keeps A positive definite);
 *   dirichlet_1d: graph node ids on the part dLambda_D of the graph boundary
 *     where u_Lambda = u_d (eq. (problem)); those unknowns are eliminated
 *     symmetrically -- identity rows and columns of the 1D block, no
 *     coupling columns -- and their value enters the load vector (md_rhs). */
typedef struct {
    double k_omega;
    double sigma_omega;
    double k_lambda;
    int natural_boundary;
    int n_dirichlet_1d;
    const int* dirichlet_1d;     /* host, n_dirichlet_1d graph node ids */
    double u_d;
} md_params;

/* Sizes of an assembled instance. */
typedef struct {
    int N;                      /* Q1 elements per cube edge */
    int n3;                     /* (N+1)^3 grid nodes */
    int n1;                     /* 1D mesh nodes */
    int nq;                     /* 1D quadrature points (2 per element) */
    int n_touch;                /* grid nodes reached by the averaging operator */
    long long n;                /* n3 + n1 */
    double alpha;               /* ||diag(C_II)||_2 / sqrt(#interior nodes), Section 5.1 */
    double beta;
} md_op_info_t;

/* ---- assembly ------------------------------------------------------------
 * md_assemble -- eq. (mainsys), Section 2.1.  Builds, for grid N (>= 2) and
 * the graph with radius R (> 0) and coupling beta (>= 0; the factor 2 pi eps
 * of eq. (mainsys)):
 *   K00: the Q1 stiffness (+ sigma mass) of a_Omega, applied matrix-free as a
 *        27-point stencil, homogeneous Dirichlet rows/columns on the cube
 *        boundary (identity there);
 *   Pi:  the cross-section average at 2 Gauss points per 1D element, each
 *        the mean of the trilinear interpolant at 8 circle points;
 *   W, Psi, K1 and the tree LDL^T factorisation of B11 = kappa K1 + beta
 *        Psi^T W Psi; the distance field d_h (Section 2.1) on the grid.
 * Host geometry runs in FP64 on the CPU; d_h and diag(A) are computed on the
 * GPU.  Synchronous.  *out receives a handle freed by md_op_destroy. */
md_status md_assemble(int N, const md_graph* g, double radius, double beta,
                      const md_params* p, md_op** out);
void md_op_destroy(md_op* op);
md_status md_op_get_info(const md_op* op, md_op_info_t* info);
/* Copy the device distance field d_h (n3 floats) into a device buffer. */
md_status md_op_distance(const md_op* op, float* d, md_stream s);

/* md_rhs -- the load vector of eq. (problem_weak): b0 = M_Omega f (Q1 mass
 * times nodal values f, device FP64, n3 entries, NULL for f = 0) with b0 = 0
 * on Dirichlet nodes, b1_i = g * int_Lambda psi_i ds; with 1D Dirichlet nodes
 * (md_params) b1 = u_d on them, and their value's columns moved to the right
 * (b0 += beta Pi^T W Psi_D u_d, b1 -= B11[:, D] u_d).  b: device FP64, n. */
md_status md_rhs(const md_op* op, const double* f, double g, double* b, md_stream s);

/* md_apply -- y = A u, eq. (mainsys), matrix-free.  prec selects FP32 (u, y
 * float*) or FP64 (double*).  u and y must not alias.  Asynchronous. */
md_status md_apply(const md_op* op, md_prec prec, const void* u, void* y, md_stream s);

/* md_apply_noalloc -- the same y = A u as md_apply, for callers that must not
 * allocate device memory or write the operator's own scratch (an application
 * that reserves all device memory at start-up, or several users sharing one
 * read-only operator handle).  The paper has no counterpart: this is a
 * deployment variant of md_apply.  Its scratch (the quadrature-point values
 * and a copy of the instance descriptor) is one static device array of the
 * library, sized for MD_NOALLOC_MAX_NQ quadrature points (about 129 KB),
 * which every GPU that loads the library keeps until the process exits.
 * Operators with more quadrature points are rejected with MD_ERR_ARG.
 * Nothing is allocated: the first call on a device (made with that device
 * current) looks up the array's address once; make that first call before any
 * stream capture.  All calls share the array and it keeps the last call's
 * contents, so calls that overlap on the GPU race with each other: order them
 * on one stream or synchronise.  Asynchronous on s. */
#define MD_NOALLOC_MAX_NQ 16384
md_status md_apply_noalloc(const md_op* op, md_prec prec, const void* u, void* y, md_stream s);

/* ---- the network -----------------------------------------------------------
 * Six 3x3x3 'same' convolutions 3->32->32->32->32->32->1 with bias, GELU
 * (x Phi(x)) after layers 1-5 (the fully convolutional hypothesis space of
 * Section 4.2; channel pattern of this library).  Weights BF16, biases FP32,
 * FP32 accumulation.
 * Parameter layout (host float array, MD_CNN_NPARAMS entries): for each layer
 * l, the weights W[co][ci][kz][ky][kx] (cross-correlation orientation,
 * Y(p) = b + sum_q W(q) X(p+q), q in {-1,0,1}^3 at index q+1) followed by the
 * biases b[co].  Weights are rounded to BF16 (nearest even) on upload. */
#define MD_CNN_LAYERS 6
#define MD_CNN_NPARAMS 114209
md_status md_cnn_create(const float* host_params, long long n_params, md_cnn** out);
/* Engine of the convolutions: 0 = 5th-gen tensor cores (tcgen05 implicit
 * GEMM, the default), 1 = CUDA cores (same arithmetic: BF16 operands, FP32
 * accumulation; kept as the cross-check of the tensor-core path).
 * Takes effect at the next launch that builds its work (a new md_batch). */
md_status md_cnn_set_engine(md_cnn* c, int engine);
md_status md_cnn_get_params(const md_cnn* c, float* host_params, long long n_params);
void md_cnn_destroy(md_cnn* c);
/* File: magic "MDCNN001", int64 count, count FP32 values, uint64 FNV-1a
 * checksum of the value bytes.  MD_ERR_IO on a short file or bad checksum. */
md_status md_cnn_save(const md_cnn* c, const char* path);
md_status md_cnn_load(const char* path, md_cnn** out);

/* md_cnn_forward -- raw network pass on `batch` grids of (n+1)^3 nodes:
 * X: device float, batch * 3 * (n+1)^3, channel-major per sample
 * (sample, channel, z, y, x); Y: device float, batch * (n+1)^3.  The input
 * is rounded to BF16 like the preconditioner's.  Asynchronous. */
md_status md_cnn_forward(const md_cnn* c, int n_nodes_edge, int batch, const float* X, float* Y, md_stream s);

/* md_cnn_backward -- gradients of sum(dY * Y) for the pass above: dparams
 * (device float, MD_CNN_NPARAMS, overwritten) and optionally dX (device
 * float, like X, nullable).  Recomputes the forward activations. */
md_status md_cnn_backward(const md_cnn* c, int n_nodes_edge, int batch, const float* X,
                          const float* dY, float* dparams, float* dX, md_stream s);

/* ---- The paper's U-net U3 (Section 4.2, the U3 table of Section 5.1) ----
 * Encoder conv3 2->32 | maxpool2 + conv3 32->64 | maxpool2 + conv3 64->128,
 * bottleneck conv3 128->128, decoder [up2 128->64 | skip] + conv3 128->64,
 * [up2 64->32 | skip] + conv3 64->32, output conv3 32->1; GELU x Phi(x)
 * after every conv3 but the last.  conv3: 3x3x3 zero 'same' padding with
 * bias; maxpool2: 2x2x2 windows at even offsets (an odd size's last plane
 * dropped); up2: transposed 2x2x2 convolution with stride 2, zero planes
 * appended up to the skip's size.  FP32 throughout, CUDA cores.
 * Parameter layout (host float array, md_unet_num_params() entries): the
 * seven conv3 layers in the order above, then the two up2 layers; each its
 * weights (conv3: c_out, c_in, 3, 3, 3 in the cross-correlation orientation
 * of md_cnn; up2: c_in, c_out, 2, 2, 2) then its biases. */
typedef struct md_unet md_unet;
long long md_unet_num_params(void);
md_status md_unet_create(const float* host_params, long long n_params, md_unet** out);
void md_unet_destroy(md_unet* u);
/* md_unet_forward -- Y = U3(X) on `batch` grids of n^3 nodes (4 <= n <= 1024):
 * X: device float, batch * 2 * n^3, (sample, channel, z, y, x); Y: device
 * float, batch * n^3.  The first call for a larger (n, batch) allocates the
 * workspace (synchronising the stream); calls on one handle must not
 * overlap.  Asynchronous otherwise.  MD_ERR_ARG on a bad size. */
md_status md_unet_forward(md_unet* u, int n, int batch, const float* X, float* Y, md_stream s);
/* md_unet_backward -- gradients of sum(dY * Y) for the pass above, summed over
 * the batch: dparams (device float, md_unet_num_params(), overwritten) and
 * optionally dX (device float, like X, nullable).  Recomputes the forward
 * activations (workspace as md_unet_forward, larger).  Weight gradients are
 * accumulated with atomic additions: their summation order, and so their
 * last bits, vary from call to call. */
md_status md_unet_backward(md_unet* u, int n, int batch, const float* X, const float* dY, float* dparams,
                           float* dX, md_stream s);
/* Parameters: set from host (on_device = 0) or device memory, asynchronous on
 * s; get to host (synchronous). */
md_status md_unet_set_params(md_unet* u, const float* params, int on_device, md_stream s);
md_status md_unet_get_params(const md_unet* u, float* host_params, long long n_params);
/* md_unet_train_loss -- md_train_loss with the U-net as the network: per
 * sample the input X = [b0 / s, d_h] (the U-net's two channels: the 3D block's
 * right-hand side b0 = r0 + l of eq. (twosteps) scaled by s = ||b0||, and the
 * distance field), z0 = (s / alpha) U(X), loss ||C z0 - b0||^2 / ||b0||^2
 * over the unknown 3D rows, averaged over the samples; dparams (device float,
 * md_unet_num_params(), nullable) its gradient.  Samples share a grid size;
 * with 1D parts zero (the block lower-triangular order) b0 = r0. */
md_status md_unet_train_loss(md_unet* u, int count, const md_op* const* ops, const float* const* r,
                             double* loss, float* dparams, md_stream s);
/* md_unet_opt_step -- one AdamW step on the U-net's parameters (decoupled
 * weight decay on the weights, not the biases); the first step allocates the
 * moment buffers. */
md_status md_unet_opt_step(md_unet* u, const float* grad, double lr, double beta1, double beta2, double eps,
                           double weight_decay, md_stream s);

/* md_precondition -- z = Q~ r, eq. (twosteps) with the network as the 3D
 * solve (eq. (decoupled_3d_problem)):
 *   z1 = B11^{-1} r1;  l = beta Pi^T W Psi z1;  b0 = r0 + l;  s = ||b0||;
 *   z0 = (s / alpha) N([r0/s, l/s, d_h]) on interior nodes, z0 = r0 on
 *   Dirichlet nodes.
 * cnn == NULL gives the Jacobi preconditioner z = diag(A)^{-1} r.
 * r, z: device float, n.  Asynchronous. */
md_status md_precondition(const md_op* op, const md_cnn* cnn, const float* r, float* z, md_stream s);

/* md_precondition_lower -- the block lower-triangular order of the same
 * preconditioner (the other reading of how the network and the 1D solve are
 * composed in eq. (twosteps)): the network first on [r0/s, 0, d_h] with
 * s = ||r0||, z0 = (s / alpha) N(X) on interior nodes and r0 on Dirichlet
 * nodes; then z1 = B11^{-1} (r1 + beta Psi^T W Pi z0).  Arguments as
 * md_precondition; cnn must not be NULL.  Asynchronous. */
md_status md_precondition_lower(const md_op* op, const md_cnn* cnn, const float* r, float* z, md_stream s);

/* md_precondition_smoothed -- the network preconditioner with Jacobi pre- and
 * post-smoothing around its 3D solve (Section 5, 'Effect of pre- and
 * post-smoothing', the relaxation S_J(C, b0, x0, nu)): with b0 the right-hand
 * side of the 3D solve (r0 + l in the upper order, r0 in the lower one) and
 * D^{-1} = diag(rho_i / c_ii), rho_i = min(1, 2 c_ii / S_i), S_i = sum_j |K00_ij|
 * + beta sum_j (Pi^T W Pi)_ij (Jacobi on stencil rows; on rows the coupling
 * makes heavy, the scaling that keeps every sweep with omega < 1 contracting),
 *     x  = nu damped Jacobi sweeps x <- x + omega D^{-1} (b0 - C x) from 0,
 *     x += N(b0 - C x)   (network input [(b0 - C x - l)/s, l/s, d_h],
 *                         s = ||b0 - C x||, output (s / alpha) N(X),
 *                         b0 - C x itself on Dirichlet nodes),
 *     z0 = nu more sweeps from x,
 * and z1 as in md_precondition (lower = 0) or md_precondition_lower
 * (lower = 1).  nu in [0, 8] (0 gives the unsmoothed preconditioner),
 * 0 < omega < 2, else MD_ERR_ARG.  cnn must not be NULL.  r, z: device
 * float, n.  Uses the operator's cached solver scratch: calls on one
 * operator must be ordered.  Asynchronous. */
md_status md_precondition_smoothed(const md_op* op, const md_cnn* cnn, int lower, int nu, double omega,
                                   const float* r, float* z, md_stream s);

/* md_precondition_inner -- the network preconditioner whose 3D block solve is
 * m steps of flexible GMRES on C z0 = b0 from z0 = 0, right-preconditioned by
 * the network (Section 6: the 3D solve of the block preconditioner as '3
 * steps of P-FGMRES'): v_0 = b0 / ||b0||, z_0 the network on the block's own
 * input [r0/s, l/s, d_h] scaled by 1/||b0||, later z_j the network on
 * [v_j, 0, d_h]; w = C z_j orthogonalised against v_0..v_j (two classical
 * Gram-Schmidt passes, FP64 sums), v_{j+1} = w / ||w||; then
 * z0 = sum_j y_j z_j with y the FP64 least-squares solution of
 * min ||b0|| e_1 - H y||.  z1 as in md_precondition (lower = 0) or
 * md_precondition_lower (lower = 1).  m in [0, 4] (0: one network
 * application), else MD_ERR_ARG; cnn must not be NULL.  r, z: device float,
 * n.  Uses the operator's cached solver scratch (allocated at the first call):
 * calls on one operator must be ordered.  Asynchronous. */
md_status md_precondition_inner(const md_op* op, const md_cnn* cnn, int lower, int m, const float* r, float* z,
                                md_stream s);

/* md_lift -- the 1D part of the preconditioner on its own (Section 3 eqs.
 * (matrixC), (setB)): z1 = B11^{-1} r1 (tree factorisation) and its forcing on
 * the 3D problem l = -beta M01 z1 = beta Pi^T W Psi z1.  With r1 the 1D load
 * this is an element of the set B the training set is built from (Section 4.1).
 * r: device float, n (only the 1D part r1 is read); z1: device float, n1
 * (nullable); l: device float, n3 (zero on nodes the averaging does not
 * reach).  Asynchronous. */
md_status md_lift(const md_op* op, const float* r, float* z1, float* l, md_stream s);

/* ---- solves -----------------------------------------------------------------
 * md_solve -- solve A x = b to ||b - A x||_2 / ||b||_2 <= tol.
 *   cnn != NULL: flexible GMRES(restart) (Section 4, Saad 1993), right-
 *     preconditioned by md_precondition; Krylov vectors FP32, Hessenberg and
 *     Givens in FP64, and at every restart x += Z y and r = b - A x in FP64.
 *     Safeguard (not in the paper): an instance whose network gives no
 *     usable direction, a non-finite one, or a restart cycle of 10 or more
 *     iterations that does not halve the true residual continues with the
 *     Jacobi preconditioner (counted in md_batch_stats_t.fallback_instances).
 *   cnn == NULL: conjugate gradients with the Jacobi preconditioner in FP64.
 * b: device FP64 (n); x: device FP64 (n), in: initial guess, out: solution.
 * maxit bounds the total iterations.  *iters and *relres (host) receive the
 * iterations done and the final true relative residual.  Synchronises s.
 * Returns MD_NOT_CONVERGED when maxit is reached above tol.  b = 0: the
 * relative residual is taken as 0 and the solve returns at once with x as
 * given (the zero solution when started from x = 0). */
md_status md_solve(const md_op* op, const md_cnn* cnn, const double* b, double* x,
                   double tol, int restart, int maxit, int* iters, double* relres, md_stream s);

typedef enum {
    MD_SOLVER_FGMRES_CNN = 0,      /* FGMRES + block preconditioner with the network */
    MD_SOLVER_FGMRES_JACOBI = 1,   /* FGMRES + diag(A)^{-1} */
    MD_SOLVER_CG_JACOBI = 2        /* Jacobi-CG, FP64 */
} md_solver;

/* md_batch -- many instances solved together, one launch per kernel across
 * all instances (the ensembled stacking of Section 5.7); instances stop
 * independently on their own convergence.  A solve is one launch of a CUDA
 * graph captured at the first solve (again when the network, block order,
 * smoothing, inner steps or profiling change): its restart cycles run under
 * a conditional WHILE node decided on the device, so the host waits once per
 * solve; the kernels of an iteration slot return at once for instances that
 * have left the cycle.
 * Vectors of the batch are concatenated: instance i occupies
 * [offset[i], offset[i] + n_i) of a batched vector.
 * The batch borrows ops and cnn: they must not be destroyed before the
 * batch (its captured graph reads their device buffers at every solve). */
md_status md_batch_create(int n_ops, const md_op* const* ops, const md_cnn* cnn, md_solver solver,
                          int restart, md_batch** out);
void md_batch_destroy(md_batch* b);
/* host array of n_ops + 1 offsets (the last is the total length) */
md_status md_batch_offsets(const md_batch* b, long long* offsets);
/* b_all, x_all: device FP64 batched vectors; x_all in: initial guesses.
 * iters, relres: host arrays of n_ops (nullable).  Synchronises s. */
md_status md_batch_solve(md_batch* b, const double* b_all, double* x_all, double tol, int maxit,
                         int* iters, double* relres, md_stream s);
/* Per-instance device timestamps (ns, globaltimer) of convergence for the
 * last md_batch_solve, relative to its start; host array of n_ops. */
md_status md_batch_times(const md_batch* b, double* seconds);

/* Instrumentation.  With profiling on, the solve graph takes device
 * timestamps (the global nanosecond timer, from one-thread kernels between
 * the sections) around each preconditioner application, around its four
 * hidden 32->32 convolutions, around the operator apply, around the
 * Arnoldi/Givens kernels and around each restart; md_batch_stats returns
 * totals since the last reset (device time, ms, summed over the slots that
 * ran), the kernels the solves ran and their graph launches.  The timestamp
 * kernels add no work to the others. */
typedef struct {
    long long kernel_launches;   /* kernels run by md_batch_solve calls (graph nodes executed) */
    long long cycles;            /* restart cycles (CG: chunks of 25 iterations) */
    long long iterations;        /* sum over instances of Krylov iterations */
    long long precond_nodes;     /* sum over instances of network-preconditioned iterations x grid nodes */
    double prec_ms;              /* preconditioner applications (iteration slots) */
    double conv_hidden_ms;       /* the 4 hidden convolution launches per application */
    long long conv_hidden_launches;
    double apply_ms;             /* A z in FP32 */
    double arnoldi_ms;           /* dots, updates, Givens */
    double restart_ms;           /* least squares, x update, FP64 residual */
    long long fallback_instances; /* network solves whose instance switched to Jacobi */
    long long graph_launches;    /* host launches: one graph per md_batch_solve */
    long long slot_gating;       /* 2: one graph launch per solve, its restart cycles under a conditional
                                    WHILE node, every iteration slot launched (its kernels return at
                                    once for instances out of the cycle); 3: the host-driven loop of
                                    md_batch_set_host_loop */
} md_batch_stats_t;
md_status md_batch_set_profiling(md_batch* b, int enable);
/* enable = 1: solves run as a set-up graph and one graph per restart cycle
 * (every iteration slot launched), the host reading the count of finished
 * instances after each cycle; the same kernels as the device-driven solve,
 * for kernel profilers, which cannot profile the kernels of graphs with
 * conditional nodes.  0 (default): one graph launch per solve. */
md_status md_batch_set_host_loop(md_batch* b, int enable);
/* lower = 1: the network-preconditioned batch uses md_precondition_lower's
 * block order; 0 (default): the paper's upper-triangular order. */
md_status md_batch_set_prec_order(md_batch* b, int lower);
/* nu > 0: the network-preconditioned batch smooths its 3D solve with nu
 * damped Jacobi sweeps (damping omega) before and after the network, as
 * md_precondition_smoothed; 0 (default): no smoothing.  Limits and errors as
 * md_precondition_smoothed. */
md_status md_batch_set_smoothing(md_batch* b, int nu, double omega);
/* m > 0: the network-preconditioned batch solves its 3D block by m inner
 * FGMRES steps, as md_precondition_inner (buffers of 9 vectors of the batch's
 * length are allocated at the first call); 0 (default): one network
 * application.  Not combined with smoothing (MD_ERR_ARG). */
md_status md_batch_set_inner_iters(md_batch* b, int m);
/* md_batch_set_unet -- the 3D block solve of a network-preconditioned FGMRES
 * batch by the U-net u instead of the batch's md_cnn (u NULL: back to it):
 * z0 = (s / alpha) U([b0 / s, d_h]) on the unknown nodes, v0 on Dirichlet
 * nodes, in either block order (b0 = r0 + l upper, r0 lower).  The instances
 * must share the grid size; not combined with smoothing or inner steps
 * (MD_ERR_ARG).  The batch borrows u.  The first call runs one U-net pass to
 * size its workspace (synchronising the device): call it before any capture. */
md_status md_batch_set_unet(md_batch* b, md_unet* u);
md_status md_batch_stats(const md_batch* b, md_batch_stats_t* out);

/* Autotuning.  A network- or Jacobi-preconditioned FGMRES batch of at least
 * 10^6 unknowns times its launch choices on the GPU when it is created and
 * keeps the fastest: the elements per block of its Krylov vector kernels
 * (candidates 4096-32768, timed on Gram-Schmidt steps over the whole batch)
 * and the 128-row tiles per plane step of its tensor-core convolutions (1 or
 * 2, timed on a forward pass over every grid).  Smaller batches keep the
 * defaults (8192 elements, 2 tiles; CG batches 2048 elements).
 * md_batch_tuning reports the choices and the timings (microseconds). */
typedef struct {
    int tuned;                   /* 1 if the choices below were timed */
    int vec_chunk;               /* elements per block of the Krylov vector kernels */
    int n_vec;
    int vec_candidates[8];
    double vec_us[8];            /* Gram-Schmidt steps at basis lengths 6, 14, 22, 30 (those below
                                    the restart length), summed, with each candidate */
    int conv_tps;                /* 128-row tiles per plane step of the convolutions (0: no network) */
    double conv_us[2];           /* one forward pass with 1 and 2 tiles per step */
} md_tuning_t;
md_status md_batch_tuning(const md_batch* b, md_tuning_t* out);
md_status md_batch_reset_stats(md_batch* b);

/* md_solve_batched -- one-shot form: create, solve (per-instance device
 * pointers given as host arrays), destroy. */
md_status md_solve_batched(int n, const md_op* const* ops, const md_cnn* cnn, const double* const* b,
                           double* const* x, double tol, int restart, int maxit, int* iters,
                           double* relres, md_stream s);

/* ---- training ----------------------------------------------------------------
 * md_train -- unsupervised training of the network (Section 3.2 eq. (risk),
 * (trained_preconditioner); the loss of Section 5.1):
 *   per sample (instance op_k, residual r = [r0; r1]):
 *     b0 = r0 + beta Pi^T W Psi B11^{-1} r1,  s = ||b0||,
 *     L = || C z0 - b0 ||^2 / ||b0||^2,  z0 = (s / alpha) N([r0/s, l/s, d_h]),
 *   mean over a minibatch, AdamW, cosine learning-rate decay from lr to lr_min.
 * Samples of one minibatch share a grid size (the sampler groups them).
 * cnn: in/out network (trained in place).  Synchronous. */
typedef struct {
    int n_ops;
    const md_op* const* ops;       /* training instances (host array) */
    int n_samples;
    const int* sample_op;          /* host, n_samples: index into ops */
    const float* const* sample_r;  /* host array of device pointers: residual of length n of its op */
    int epochs;
    int batch;
    double lr, lr_min, beta1, beta2, weight_decay, eps;
    uint64_t seed;                 /* shuffling */
    double* loss_history;          /* host, epochs entries (mean loss per epoch), nullable */
} md_train_cfg;
md_status md_train(md_cnn* cnn, const md_train_cfg* cfg);

/* md_train_loss -- the loss above and optionally its gradient for `count`
 * samples (mean), without updating the network.  dparams: device float
 * MD_CNN_NPARAMS or NULL.  *loss written on return (synchronises s). */
md_status md_train_loss(const md_cnn* cnn, int count, const md_op* const* ops, const float* const* r,
                        double* loss, float* dparams, md_stream s);

/* md_krylov_basis -- the Krylov augmentation of the training set (Section
 * 4.1.1): an orthonormal basis q_0 = b/||b||, q_1, ..., q_m of the Krylov space
 * K_{m+1}(C, b) of the 3D block C = K00 + beta Pi^T W Pi (C q is the 3D part of
 * A [q; 0]), each new vector orthogonalised by two passes of modified
 * Gram-Schmidt, in FP64.  b: device float n3 (nonzero); Q: device float,
 * (m+1) x n3, row j = q_j.  m in [1, 16], else MD_ERR_ARG.  Allocates its FP64
 * work vectors; synchronises s. */
md_status md_krylov_basis(const md_op* op, const float* b, int m, float* Q, md_stream s);

/* md_opt -- AdamW state (FP32 master weights copied from the network, first
 * and second moments) for training loops driven by the caller, one step per
 * call with a gradient the caller provides (the mean-loss gradient of
 * md_train_loss, or its average over processes in data-parallel training,
 * where every process applies the same step to its copy of the network).
 * The update is md_train's: m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
 * w -= lr wd w on weights (not biases), w -= lr m^ / (sqrt(v^) + eps) with
 * the bias-corrected moments of step t.  grad: device float MD_CNN_NPARAMS.
 * md_opt_step writes the new weights into cnn (its parameters and BF16
 * images) and synchronises s; MD_ERR_NAN if a weight became non-finite. */
typedef struct md_opt md_opt;
md_status md_opt_create(const md_cnn* cnn, md_opt** out);
md_status md_opt_step(md_opt* opt, md_cnn* cnn, const float* grad, double lr, double beta1, double beta2,
                      double eps, double weight_decay, md_stream s);
void md_opt_destroy(md_opt* opt);

const char* md_last_error(void);
const char* md_version(void);

#ifdef __cplusplus
}
#endif
#endif /* MD_H */
