/*
 * sg.h -- C ABI of the GB300 stochastic-Galerkin domain-decomposition wave solver.
 *
 * The library advances the intrusive stochastic Galerkin (Hermite chaos) semi-discretisation
 * of the 2-D acoustic wave equation with a log-normal squared wave speed
 *     u_tt + eta u_t - div(c_s(x, xi) grad u) = f          (Sec. 4, Eq. acous_sto)
 * with Newmark-beta (gamma = 1/2, zeta = 1/4, Sec. 2).  Each time step solves the transient
 * system K~ U_{n+1} = F~_{n+1} (Eq. K_T_Sto) by PCG on the non-overlapping domain
 * decomposition interface (Schur complement, Eq. Sto_Schur) preconditioned by the
 * probabilistic two-level Neumann-Neumann preconditioner (Eq. NNCP2).  All per-step work runs
 * in the library's own CUDA kernels on one GPU.
 *
 * Conventions
 *   - Every entry point returns SG_OK (0) or a negative SG_E* code; sg_strerror() names it.
 *   - Caller-owned input structs are read during the call only; nothing is retained.
 *   - A handle owns all of its device memory (allocated in sg_setup, released in sg_destroy).
 *   - All device work of a handle is issued on the CUDA stream given to sg_setup (NULL means
 *     the legacy default stream); the calls below synchronise that stream before returning
 *     unless stated otherwise.
 *   - A handle is not thread-safe: one host thread at a time.
 *   - Field layout for sg_get_field / sg_get_state / sg_set_state (handles of sg_setup; for
 *     sg_setup_mesh handles see there): node-major over the free
 *     nodes (x index fastest, then y; node (i, j) for 1 <= i, j <= N-1), PCE mode fastest:
 *     value(i, j, k) is element ((j-1) (N-1) + (i-1)) * P + k.  PCE modes follow the graded
 *     multi-index order (total degree, then descending lexicographic), orthonormal basis.
 *
 * Environment switches.  They select between complete implementations of the same step and never
 * skip work.  Set them before sg_setup and keep them set while the handle steps: the set-up reads
 * some, and the launch shapes read the others when the step graph is captured at the first sg_step
 * (and at every launch in the host-driven mode).  Each is "on"
 * when set, whatever its value (except SG_FORCE_NODS).
 *   SG_EAGER        sg_step enqueues the step's kernels from the host instead of launching the
 *                   captured graph: the same kernels, visible to profilers that cannot enter
 *                   conditional graph nodes (same as sg_set_enqueue_mode(h, 1)).
 *   SG_PDL          programmatic dependent launch between the FP32 inner-loop kernels.
 *   SG_NO_MMA       FP32 subdomain CG preconditioned by the line sweeps of the mean operator
 *                   instead of its dense BF16 inverse on the tensor cores.
 *   SG_NO_GFIX      FP32 and FP64 operator applies with the runtime triple-product table instead of
 *                   the table compiled for (M, p, p_in).
 *   SG_FP64_RT      FP64 operator applies with the runtime triple-product table (FP32 keeps the
 *                   compiled one).
 *   SG_APPLY_FP64   FP64 arithmetic in the outer-loop operator applies of the mixed-precision path
 *                   (effective load, residual corrections) instead of float-float pairs of FP32
 *                   values (about 1e-13 relative; used when the compiled table applies).
 *   SG_APPLY_LINES  grid lines per block of the compiled-table operator apply (1 .. L, when the tile
 *                   fits shared memory), in place of the built-in choice.
 *   SG_LINE_OLD     mean-operator line sweeps of subdomains at least 41 nodes wide by the block kernel
 *                   with the factor staged line by line, instead of the register-tiled kernel.
 *   SG_FORCE_NODS   apply without staged edge differences at every size; the value 2 also reads the
 *                   triple-product table from global memory (the variants of the widest subdomains).
 *   SG_FORCE_GLINE  line sweep reading the factor and residual from global memory at every size.
 *   SG_A6_SOLVE     mixed precision recovers the interior unknowns by an explicit Dirichlet solve
 *                   (Alg. 1) instead of accumulating them along the interface PCG.
 */
#ifndef SG_H
#define SG_H

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define SG_OK         0
#define SG_EINVAL    -1   /* invalid argument (sizes, pointers, parameters)                 */
#define SG_ENOMEM    -2   /* device or host allocation failed                               */
#define SG_ECUDA     -3   /* a CUDA runtime call failed (the message is kept per handle)    */
#define SG_ENOTCONV  -4   /* PCG reached max_iter before ||r||/||G|| <= tol                 */
#define SG_ENUMERIC  -5   /* NaN/Inf or loss of positive definiteness detected              */
#define SG_ETIMEOUT  -6   /* a bounded device-side wait expired                             */
#define SG_ENOTSUP   -7   /* configuration outside what this build supports                 */

/* ---- precision modes (sg_params.precision) ----
 * The outer interface PCG (Schur matvec, dot products, residual recurrence, coarse solve) is FP64 in
 * every mode; the modes differ in the subdomain solves of its matvec and preconditioner (Secs. 3, 5). */
#define SG_FP64      0    /* every kernel computes in FP64                                  */
#define SG_MIXED     1    /* FP32 subdomain CG with one FP64 residual correction per Dirichlet
                             solve; its mean-operator preconditioner is the BF16 tensor-core
                             product where that applies (subdomains of at most 40 x 40 nodes,
                             P <= 32) and the FP32 line sweeps elsewhere                     */
#define SG_FP32      2    /* as SG_MIXED with the FP32 line sweeps at every size (no BF16)   */
#define SG_BF16      3    /* as SG_MIXED with the BF16 tensor-core preconditioner required: the
                             dense inverse up to 40 x 40 nodes (P <= 32), the line sweeps with
                             their per-line products on the tensor cores for 41 .. 65 nodes per
                             side; SG_ENOTSUP elsewhere                                        */

/* ---- interface preconditioner (sg_params.precond) ---- */
#define SG_PC_NN2     0   /* probabilistic two-level Neumann-Neumann (Eq. NNCP2; the method)     */
#define SG_PC_NN1     1   /* one-level Neumann-Neumann, sum R^T D S_s^{-1} D R (comparison of
                             Sec. 6.1; local Neumann solves with the whole interface free)     */
#define SG_PC_LUMPED  2   /* lumped, sum R^T D K~_GG D R (comparison of Sec. 6.1)              */

/* ---- warm start (sg_params.warm) ---- */
#define SG_WARM_PREV     0   /* previous step's interface solution (Alg. 1)                 */
#define SG_WARM_LEARNED  1   /* Newmark predictor plus a learned estimate of its error
                                (extension of the method)                                    */

/* ---- sources (sg_source.kind) ---- */
#define SG_SRC_NONE    0
#define SG_SRC_PULSE   1  /* u0 = amp exp(-((x-x0)^2 + (y-y0)^2) / width^2), v0 = 0 (Eq. initial_2Dwave) */
#define SG_SRC_RICKER  2  /* f = amp r(t) delta(x - (x0, y0)), r Ricker of peak frequency freq      */

typedef struct sg_handle_s* sg_handle;

/* Structured grid: N x N cells on the unit square, each cell split along (i,j)->(i+1,j+1),
 * homogeneous Dirichlet boundary; partition into nsub_x x nsub_y equal subdomains
 * (N divisible by both). */
typedef struct { int N; int nsub_x; int nsub_y; } sg_grid;

/* Gaussian field g = g0 + sum_n sigma sqrt(lambda_n) phi_n(x) xi_n with covariance
 * sigma^2 exp(-|dx|/bx - |dy|/by) (Sec. 4, Eqs. CovarKer2D, KLE); M random variables.
 * modes == NULL: the analytic eigenpairs of that separable kernel (top M by lambda).  Otherwise the
 * caller's KL: modes[n * n_elem + e] = phi_n at the centroid of element e (n < M, n_elem = 2 N^2;
 * element e = 2 (j N + i) + t of cell (i, j), t = 0 the triangle (i,j),(i+1,j),(i+1,j+1) with centroid
 * ((i + 2/3) h, (j + 1/3) h), t = 1 the triangle (i,j),(i+1,j+1),(i,j+1), centroid ((i + 1/3) h,
 * (j + 2/3) h)) and lambdas[n] > 0; bx, by are then unused.  Both arrays are read during sg_setup only.
 * Errors: SG_EINVAL if modes is given without lambdas, or a lambda is not positive, or a value is not
 * finite. */
typedef struct {
  int M;
  double sigma;
  double bx;
  double by;
  double g0;
  const double* modes;    /* M x n_elem values, or NULL */
  const double* lambdas;  /* M values (with modes)        */
} sg_kl;

/* Output PCE order p (P = C(M+p, p) terms) and input (coefficient) order p_in. */
typedef struct { int p; int p_in; } sg_pce;

typedef struct {
  double dt;          /* time step                                                          */
  double tol;         /* outer PCG: stop when ||r||_2 / ||G_Gamma||_2 <= tol                */
  double alpha0;      /* Rayleigh damping C = alpha0 M + alpha1 K (Rayleigh appendix)       */
  double alpha1;
  int    max_iter;    /* outer PCG iteration cap (SG_ENOTCONV beyond)                       */
  int    precision;   /* SG_FP64, SG_MIXED, SG_FP32 or SG_BF16                              */
  int    warm;        /* SG_WARM_PREV or SG_WARM_LEARNED                                    */
  double inner_tol;   /* subdomain solves: relative residual target (0 = automatic: 1e-14 in
                         FP64; in FP32 sqrt(0.1 tol) within [1e-6, 1e-4], since a corrected
                         solve is two FP32 solves whose tolerances multiply)                  */
  int    inner_max_iter; /* subdomain solves: iteration cap (0 = automatic)                 */
  int    autotune;    /* 1: time candidate tile shapes of the hot kernels at set-up and keep the
                         fastest per problem shape (process-wide table); 0: built-in heuristics */
  int    warm_train_steps; /* SG_WARM_LEARNED: steps of online training (0 = 20)              */
  double warm_lr;          /* SG_WARM_LEARNED: Adam learning rate (0 = 1e-3)                  */
  int    precond;          /* SG_PC_NN2 (default), SG_PC_NN1 or SG_PC_LUMPED                  */
} sg_params;

typedef struct { int kind; double x0, y0, width, freq, amp; } sg_source;

/* Per-call statistics of sg_step. */
typedef struct {
  int    steps;           /* steps advanced by this call                                    */
  int    step_index;      /* time-step counter of the handle after the call                 */
  int    iters_last;      /* outer PCG iterations of the last step                          */
  long long iters_total;  /* outer PCG iterations summed over this call's steps              */
  long long inner_total;  /* subdomain-solver iterations summed over this call's steps       */
  double relres_last;     /* final ||r|| / ||G_Gamma|| of the last step                      */
  double ms;              /* wall time of the call measured with CUDA events on the stream  */
} sg_stats;

/* Problem sizes, for allocating caller buffers. */
typedef struct {
  int N, nsub, P, P_in, n_free, n_gamma, n_corner, n_sub_nodes;
  long long device_bytes;  /* device memory owned by the handle                              */
  int fp32_precond;        /* FP32 subdomain-CG preconditioner: 0 line sweeps of the mean
                              operator, 1 its dense BF16 inverse on the tensor cores            */
  int compiled_apply;      /* 1 when the triple-product table of (M, p, p_in) is compiled into
                              the FP32 operator apply, 0 for the runtime-table kernel          */
} sg_sizes;

/* Launch plan of the per-step kernels for one problem, as sg_setup chooses it (sg_plan_query).
 * Tile choices that an autotuned sg_setup earlier in the process recorded for the same sizes are
 * taken into account, as sg_setup does.  Index [0]: the FP64 kernels; [1]: the FP32 kernels (used
 * by SG_MIXED). */
typedef struct {
  int L, P, P_in, nsub, nnz_G;  /* subdomain nodes per side, PCE terms, nonzero triple products */
  int apply_variant[2];     /* SG operator apply (Sec. 4, Eq. stoksub): 0 triple-product table
                               staged in shared memory, 1 the same without staged edge differences,
                               2 table read from global memory, 3 table compiled into the kernel  */
  int apply_lines[2];       /* grid lines per block                                               */
  int apply_tiles[2];       /* blocks per subdomain problem                                       */
  long long apply_smem[2];  /* dynamic shared memory per block, bytes                             */
  int line_kind[2];         /* mean-operator line solve: 0 block kernel with the factor staged,
                               1 warp-team kernel, 2 factor and residual read from global memory,
                               3 register-tiled kernel, 4 per-line products on the tensor cores   */
  int line_modes[2];        /* PCE modes per block                                                */
  int line_groups[2];       /* blocks per subdomain problem                                       */
  int line_block[2][3];     /* block shape                                                        */
  long long line_smem[2];   /* dynamic shared memory per block, bytes                             */
  int mma;                  /* 1: dense BF16 inverse of the mean operator on the tensor cores    */
  int mma_kp;               /* rows of that inverse per subdomain, L^2 rounded up to 128          */
  int mma_nc, mma_mt;       /* 64-node chunks and 128-row tiles per subdomain                     */
  int mma_nb;               /* PCE rows of the residual image (16 or 32)                          */
  long long mma_smem;       /* dynamic shared memory of the product kernel, bytes                 */
  int fits;                 /* 1 when the kernels of this precision fit their shared-memory
                               limits, i.e. sg_setup would not return SG_ENOTSUP for the size     */
} sg_plan;

/* Host-only query: builds the problem on the host (no device memory, no CUDA call; works without
 * a GPU) and writes the launch plan sg_setup would use to *out.  params->precision selects the
 * kernels that `fits` covers; the source is irrelevant to the plan and not taken.  Errors as
 * sg_setup: SG_EINVAL for invalid sizes or parameters (message in sg_last_error(NULL)),
 * SG_ENOTSUP for subdomains wider than 255 cells or fewer than 2 x 2 subdomains. */
int sg_plan_query(const sg_grid* grid, const sg_kl* kl, const sg_pce* pce, const sg_params* params,
                  sg_plan* out);

/* Build the solver: KL eigenpairs (analytic, separable exponential kernel), log-normal PCE of
 * c_s at element centroids (Eqs. c0pce, LNL0), Hermite triple products G_ijk, subdomain
 * operators, mean-operator line factorisations, coarse basis and F_cc^{-1} (Eq. Fcc_2), and the
 * initial state (u0, v0 = 0, consistent a0).  `stream` is a cudaStream_t or NULL.
 * Errors: SG_EINVAL for invalid sizes/parameters, SG_ENOMEM, SG_ECUDA, SG_ENUMERIC if a
 * factorisation meets a non-positive pivot.  On error *out is NULL. */
int sg_setup(const sg_grid* grid, const sg_kl* kl, const sg_pce* pce, const sg_params* params,
             const sg_source* src, void* stream, sg_handle* out);

/* Unstructured triangle mesh of the unit square with an element partition (Sec. 3: any partition
 * into non-overlapping subdomains; Sec. 6: unstructured meshes).  Arrays are caller-owned and read
 * during sg_setup_mesh only. */
typedef struct {
  int nv;                          /* vertices                                                      */
  const double* xy;                /* nv x 2 coordinates, row-major                                 */
  const unsigned char* dirichlet;  /* nv flags: 1 marks a homogeneous Dirichlet vertex (eliminated) */
  int ne;                          /* triangles                                                     */
  const int* tri;                  /* ne x 3 vertex ids (either orientation)                        */
  const int* part;                 /* ne subdomain ids 0 .. nsub - 1, every id used                 */
} sg_mesh;

/* Build the solver on a general partition of a triangle mesh: the same per-step method as sg_setup
 * (SG operator of Eq. K_T_Sto, interface PCG on Eq. Sto_Schur, two-level preconditioner Eq. NNCP2
 * or the comparison preconditioners of Sec. 6.1) with
 *   - vertex classes by the corner reading of Sec. 3: an interface vertex is a free vertex of
 *     triangles of two or more subdomains; it is a corner when it lies in three or more subdomains,
 *     or in exactly two subdomains A, B without exactly two A|B interface edges (an edge whose two
 *     triangles lie in A and B): the end points of interface curves;
 *   - P1 mass and stiffness of each subdomain's own triangles (coefficient: the log-normal PCE at
 *     the triangle centroids, Eqs. c0pce, LNL0), applied as sparse rows;
 *   - subdomain solves by CG preconditioned by the dense inverse of the subdomain's mean operator
 *     (FP64 in SG_FP64, FP32 in SG_MIXED / SG_FP32, where the operator applies of the outer loop
 *     stay FP64); SG_BF16 applies that inverse as a BF16 product on the tensor cores in the FP32
 *     Dirichlet and Neumann solves (P <= 32, at most 1600 free vertices per subdomain).
 * kl->modes, when given, holds phi_n at the triangle centroids in the mesh's triangle order
 * (modes[n * ne + e]).  The source: a pulse is evaluated at the free vertices; a point source uses
 * the P1 values at (x0, y0) in the first triangle (in the given order) that contains it.  Fields of
 * a mesh handle (sg_get_field, sg_get_state, sg_set_state, sg_step_host, sg_sample_field) list the
 * free vertices (not Dirichlet and in at least one triangle; a vertex of no triangle carries no
 * unknown) in ascending vertex id, PCE mode fastest.  sg_sizes.N is 0 for a mesh handle.
 * Errors: SG_EINVAL for invalid meshes, partitions or parameters (vertex ids out of range, an edge in
 * more than two triangles, unused subdomain ids, a degenerate triangle, a source outside the mesh),
 * SG_ENOTSUP for SG_BF16 beyond its limits, fewer than two subdomains or a subdomain with more than 4096
 * free vertices (the dense mean-operator inverse), SG_ENUMERIC if a mean operator is not
 * positive definite, SG_ENOMEM, SG_ECUDA.  On error *out is NULL. */
int sg_setup_mesh(const sg_mesh* mesh, const sg_kl* kl, const sg_pce* pce, const sg_params* params,
                  const sg_source* src, void* stream, sg_handle* out);

/* Element partition of a triangle mesh for sg_setup_mesh by recursive coordinate bisection (host only,
 * no CUDA call): the triangles of a part that is to become k subdomains are ordered by centroid along
 * the part's longer extent (ties by the other coordinate, then by triangle index) and cut after
 * floor(n floor(k/2) / k) of its n triangles into floor(k/2) and k - floor(k/2) subdomains.  xy: nv x 2,
 * tri: ne x 3 vertex ids; part (caller-owned, ne ints) receives ids 0 .. nparts - 1, every id used.
 * Errors: SG_EINVAL (null arrays, nparts outside 1 .. ne, a vertex id out of range). */
int sg_partition_rcb(int nv, const double* xy, int ne, const int* tri, int nparts, int* part);

/* Sizes and device-memory needs of a mesh problem, from the host set-up of sg_setup_mesh alone (no
 * device memory, no CUDA call; works without a GPU): to choose a partition that fits before building
 * the solver.  Byte counts are the large device arrays sg_setup_mesh allocates for params->precision
 * and params->precond. */
typedef struct {
  int nsub, n_free, n_gamma, n_corner;  /* subdomains, free vertices, interface vertices, corners     */
  int P, P_in, nnz_G;                   /* PCE terms (output, input), nonzero triple products        */
  int n_sub_nodes;                      /* free vertices of the largest subdomain (local layout rows) */
  int max_owners;                       /* most subdomains sharing one interface vertex              */
  int max_corners;                      /* most corners of one subdomain                             */
  int max_gamma;                        /* most interface vertices of one subdomain                  */
  long long row_entries;                /* sparse-row entries of all subdomains                      */
  long long coarse_dim;                 /* n_corner * P: order of the coarse matrix F_cc             */
  long long bytes_rows;                 /* sparse rows (FP64 and FP32 values)                        */
  long long bytes_inverses;             /* dense mean-operator inverses (+ the BF16 image for SG_BF16) */
  long long bytes_coarse_basis;         /* local coarse bases of the two-level preconditioner        */
  long long bytes_coarse_matrix;        /* dense FP64 inverse of F_cc                                */
  long long bytes_vectors;              /* state, step and subdomain-solve vectors                   */
  int mma;                              /* 1: SG_BF16's tensor-core product applies                  */
  int fits;                             /* 1: sg_setup_mesh accepts the sizes (at most 4096 free
                                           vertices per subdomain; SG_BF16 within its limits)        */
} sg_mesh_plan;

/* Errors as sg_setup_mesh's host checks (SG_EINVAL with a message in sg_last_error(NULL)). */
int sg_mesh_plan_query(const sg_mesh* mesh, const sg_kl* kl, const sg_pce* pce, const sg_params* params,
                       sg_mesh_plan* out);

/* Advance nsteps Newmark steps (Alg. 1 loop, stochastic form of Sec. 5): effective load
 * (Eqs. fparts, UmCm), condensed RHS G_Gamma, PCG with M_NNC^{-1}, interior recovery, Newmark
 * update.  stats may be NULL.  Returns SG_ENOTCONV (state still advanced) if a step hit
 * max_iter, SG_ENUMERIC on NaN/Inf. */
int sg_step(sg_handle h, int nsteps, sg_stats* stats);

/* Advance nsteps steps of every handle in hs[0..n) (independent problems of any sizes);
 * out_n[i] receives handle i's statistics (may be NULL).  Handles must share one stream. */
int sg_solve_batch(sg_handle* hs, int n, int nsteps, sg_stats* out_n);

/* Copy the displacement PCE coefficients U_n.  mode = -1: all P modes (n_free * P values,
 * layout above); 0 <= mode < P: that mode only (n_free values).  dst is device memory when
 * on_device != 0, else host memory. */
int sg_get_field(sg_handle h, int mode, double* dst, int on_device);

/* Mean (mode 0) and variance (sum over k >= 1 of U_k^2, orthonormal basis) of U_n on the free
 * nodes into host or device arrays of n_free doubles each; either pointer may be NULL. */
int sg_get_moments(sg_handle h, double* mean, double* var, int on_device);

/* Capacity of sg_get_moments_noalloc: free nodes of the largest handle it accepts. */
#define SG_NOALLOC_MAX_FREE (1 << 20)

/* Same results as sg_get_moments(h, mean, var, 0) for callers that cannot allocate device memory:
 * for example a host application whose own allocator owns the whole device and would fail or lose
 * track of a cudaMalloc made behind its back, or a latency-critical loop that must not pay for
 * cudaMalloc / cudaFree, which can synchronise the whole device.  mean / var are host arrays of
 * n_free doubles; either may be NULL, not both (SG_EINVAL).  Instead of handle-owned memory, the
 * device staging buffer is one fixed array inside the library: 2 x SG_NOALLOC_MAX_FREE doubles
 * (16 MiB), held by every GPU that loads the library until the process exits.  Handles with more
 * than SG_NOALLOC_MAX_FREE free nodes get SG_EINVAL.  The device current at the call must be the
 * one the handle was set up on (else SG_EINVAL).  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress) with that device current.  All calls share the array and
 * it keeps the last call's values: calls whose device work overlaps in time race and may read
 * each other's values.  The call allocates nothing and synchronises the handle's stream.  The
 * paper has no counterpart: this entry point exists only for allocation-restricted callers. */
int sg_get_moments_noalloc(sg_handle h, double* mean, double* var);

/* Samples of the PCE surrogate of U_n (statistics and PDFs of the SG solution, Sec. 6.2): for each of
 * nsamp draws xi_s (row s of xi: M values, standard normal for the method's measure) and each of npts
 * free nodes nodes[j] (free-node index in the layout above),
 *     out[s * npts + j] = sum_k U_k(x_j) Psi_k(xi_s),
 * Psi_k the orthonormal multivariate Hermite polynomial of the k-th multi-index.  The caller draws xi,
 * so the samples are reproducible.  xi, nodes and out are device arrays when on_device != 0, else host
 * arrays (staged through handle-owned device buffers that grow to the largest call).  Errors:
 * SG_EINVAL for empty sizes, null pointers or (host input) a node out of range (device input: NaN is
 * written for such a node); SG_ENOTSUP for M > 12 or p > 10.  Synchronises the handle's stream. */
int sg_sample_field(sg_handle h, int nsamp, const double* xi, int npts, const int* nodes, double* out,
                    int on_device);

/* Checkpoint: state = [U | V | A] (3 * n_free * P doubles, layout above) followed by one
 * double holding the step index.  sg_set_state restores it (the PCG warm start is reset to the
 * interface restriction of U). */
int sg_get_state(sg_handle h, double* dst, int on_device);
int sg_set_state(sg_handle h, const double* src, int on_device);

/* Host-buffer entry point for end-to-end use: for each of nsteps steps, copies that step's
 * deterministic nodal load (n_free doubles from f_host + s * n_free, added to mode 0 of the
 * built-in source term) host->device, advances one step, and copies the step's mean field
 * (n_free doubles to u_host + s * n_free) device->host.  f_host may be NULL (no extra load);
 * u_host may be NULL.  Host buffers should be pinned for asynchronous copies. */
int sg_step_host(sg_handle h, int nsteps, const double* f_host, double* u_host, sg_stats* stats);

int sg_get_sizes(sg_handle h, sg_sizes* out);

/* Per-step outer iteration counts of the last sg_step call (up to cap entries); returns the
 * number written or a negative code. */
int sg_get_iters(sg_handle h, int* iters, double* relres, int cap);

/* Learned warm start (extension of the paper's method; with warm = SG_WARM_LEARNED).  The PCG
 * starts from the Newmark predictor p = u^n + dt v^n + dt^2/2 a^n of the interface solution plus a
 * learned estimate of the predictor's error: per interface (dof, mode) row a 4-32-32-1 tanh MLP
 * (BF16 weights, FP32 arithmetic) maps the normalised history [e^n, e^{n-1}, e^{n-2}, e^{n-3}] / s of
 * the predictor's errors e^k = u^k - p^k (s their RMS) to c; the guess is p + s c.  The network
 * trains online (Adam, hand-written kernels) on the first warm_train_steps steps; until it has
 * trained, and for rows without history, the guess is p.  The PCG still stops at the same relative
 * residual.  Weights: NN_NP = 1249 floats, order W1 (32x4, row-major), b1 (32), W2 (32x32), b2 (32),
 * W3 (32), b3 (1).
 * sg_warm_weights copies the FP32 master weights out (get_host) and/or in (set_host, which also
 * marks the network as trained, ends its online training and resets Adam); n must be 1249. */
int sg_warm_weights(sg_handle h, float* get_host, const float* set_host, int n);
int sg_warm_status(sg_handle h, int* trained, int* train_left, float* loss);

/* Network evaluation on caller device buffers (for gradient checks): X rows x 4, t rows, theta the
 * 1249 FP32 parameters (rounded to BF16 as in the solver).  Writes y (rows, optional) and, when t
 * and grad are given, grad (1249 floats) of the mean squared error and the loss (host double).
 * Allocates and frees its own scratch; synchronises the device. */
int sg_mlp_eval(int rows, const float* X, const float* t, const float* theta, float* y, float* grad, double* loss);

/* Enqueue mode of sg_step: 0 (default) launches one captured CUDA graph per step whose inner
 * and outer loops are conditional nodes; 1 enqueues the same kernels from the host with the
 * loop conditions read back each iteration (for per-kernel profiling and debugging). */
int sg_set_enqueue_mode(sg_handle h, int eager);

/* Per-kernel CUDA-event timing in the host-driven mode: returns the accumulated device time and
 * launch count of the kernel class selected by the previous call, then selects `which` and
 * resets the totals.  which: 0 none, 1 preconditioner step of the FP32/FP64 subdomain CG (line
 * sweeps with the fused CG update, or CG update + residual pack + tensor-core product), 2 fused
 * SG operator apply, 3 the tensor-core product kernel alone, 4 the operator applies with FP64
 * inputs and outputs (effective load and residual corrections; float-float arithmetic in the
 * mixed path).  On a mesh handle, class 1 is the dense mean-operator product (or the pack and
 * tensor-core product with SG_BF16) and class 2 the sparse-row apply of the subdomain CG; class 4
 * times its FP64 applies.  Events are recorded on the stream the kernel is launched on. */
int sg_kernel_timing(sg_handle h, int which, double* total_ms, long long* launches);

/* Kernels launched by this library in this process so far (all handles), counted on the device
 * by the first thread of every kernel; returns a negative code on error. */
long long sg_launch_count(sg_handle h);

int sg_destroy(sg_handle h);
const char* sg_strerror(int code);
/* Message of the last CUDA failure seen by h (or by sg_setup when h is NULL). */
const char* sg_last_error(sg_handle h);

#ifdef __cplusplus
}
#endif
#endif /* SG_H */
