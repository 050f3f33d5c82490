/*
 * nlfem — GB300 (sm_103a) assembly of 2D nonlocal finite element operators.
 *
 * C ABI of libnlfem.so. All pointers are plain host or device pointers; sizes are
 * element counts. Every function returns an int status: 0 (NLFEM_OK) or a negative
 * NLFEM_ERR_* code; nlfem_last_error() then holds a message for the calling thread.
 * No function aborts, traps or exits the process.
 *
 * The operator (arXiv 2207.03921, Sec. 2): for a kernel Psi with horizon delta, the
 * approximate bilinear form (eq. biFormApprox)
 *     A_h^#(phi_j, phi_i) = sum_k sum_l int_{E_k} int_{E_l} 1_{B^#(x)}(y)
 *                           (phi_i(x) - phi_i(y))^T Psi(x,y) (phi_j(x) - phi_j(y)) dy dx
 * over all ordered element pairs of the base domain, with P1 continuous or discontinuous
 * basis functions (Sec. 2.2), the ball approximations nocaps / approxcaps (Defs. 2.1, 2.2)
 * or the infinity-norm ball, and the quadrature of Alg. 1 and Tab. 1 (Sec. 2.3).
 */
#ifndef NLFEM_H
#define NLFEM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define NLFEM_OK 0
#define NLFEM_ERR_INVALID_ARG (-1)  /* a NULL handle, negative size, unknown enum, delta <= 0 ... */
#define NLFEM_ERR_BAD_MESH (-2)     /* degenerate triangle, vertex index out of range */
#define NLFEM_ERR_OOM (-3)          /* a device allocation failed */
#define NLFEM_ERR_BUDGET (-4)       /* the assembly would exceed params.mem_budget_bytes */
#define NLFEM_ERR_CUDA (-5)         /* a CUDA runtime call failed */
#define NLFEM_ERR_NOT_CONVERGED (-6)/* nlfem_solve reached max_iter */
#define NLFEM_ERR_TIMEOUT (-7)      /* a bounded device wait ran out */
#define NLFEM_ERR_UNSUPPORTED (-8)  /* a size limit of this implementation was exceeded, or a
                                       combination it does not provide (the singular rule for
                                       peridynamics or a tabulated kernel, a discontinuous mesh
                                       with s > 1/2, an FP64 item where FP32 bulk is required) */

/* kernels of Sec. 3 */
#define NLFEM_KERNEL_CONSTANT 0     /* gamma = c, c = 4 / (pi delta^4) by default */
#define NLFEM_KERNEL_FRACTIONAL 1   /* gamma = c |x-y|^(-2-2s), c = (2-2s)/(pi delta^(2-2s)) (eq. fractional-scaling) */
#define NLFEM_KERNEL_PERIDYNAMIC 2  /* Psi = c (x-y)(x-y)^T / |x-y|^3, c = 3 / delta^3 (eq. ker:peridynamics), 2 dofs per node */
#define NLFEM_KERNEL_TABULATED 3    /* user-defined radial kernel gamma = c g(|x-y|) (the Conclusion's user kernels):
                                       g given by params.kernel_table at r_i = i delta / (n - 1), linear
                                       in between, held at g(delta) beyond; c = kconst, default 1;
                                       bounded kernels only: intersecting pairs take the standard rule */

/* ball approximations of the Euclidean ball (Sec. 2.2) */
#define NLFEM_BALL_NOCAPS 0         /* Def. 2.1 */
#define NLFEM_BALL_APPROXCAPS 1     /* Def. 2.2 */
#define NLFEM_BALL_INFINITY 2       /* the infinity norm ball |x - y|_inf <= delta, cut exactly (Sec. 2.2);
                                       constant kernel default c = 3 / (4 delta^4) (Sec. 3.3) */

/* rule on intersecting element pairs (Tab. 1) */
#define NLFEM_CLOSE_AUTO 0          /* club for 0 < s < 1, diamond for -1 < s <= 0 and peridynamics, heart otherwise */
#define NLFEM_CLOSE_DUFFY 1         /* regularising transforms to (0,1)^4 with a tensor Gauss rule */
#define NLFEM_CLOSE_NOZERODIV 2     /* truncation rule, dropping point pairs with x_p = y_q */
#define NLFEM_CLOSE_STANDARD 3      /* truncation rule as on disjoint pairs */

/* arithmetic of the separated-pair quadrature */
#define NLFEM_PREC_FP64 0           /* everything in FP64 */
#define NLFEM_PREC_FP32_BULK 1      /* truncation quadrature in FP32, the singular rule and the cut
                                       geometry as selected by
                                       singular_precision and geometry_precision, sums over pairs in
                                       exact fixed point, FP64 result; within 1e-5 relative
                                       (Frobenius) of the FP64 result */

/* FP32 bulk: arithmetic of the singular rule on intersecting pairs (Tab. 1 club) */
#define NLFEM_SINGULAR_FP64 0       /* default: transform points, kernel values and sums in FP64, each
                                       pair's block added to the fixed-point sums from FP64 */
#define NLFEM_SINGULAR_FP32 1       /* points and sums in FP32 (a relative error of a few 1e-7) */

/* FP32 bulk: arithmetic of the polygon E_l cut by the ball of an outer point (Defs. 2.1, 2.2) */
#define NLFEM_GEOMETRY_FP32 0       /* default: positions in FP32 relative to x_p. Euclidean balls: every
                                       decision (vertex in the ball, crossings of an edge, caps) equals
                                       the FP64 one; near a tie the outer point is cut in FP64. Infinity
                                       ball: FP32 Sutherland-Hodgman passes, decisions equal to the FP64
                                       ones except for the constant kernel, whose result depends on the
                                       cut region only: there a decision within rounding of a side may
                                       differ, which moves a polygon edge by a rounding-sized sliver */
#define NLFEM_GEOMETRY_FP64 1       /* every cut outer point is cut in FP64 (decisions, crossings, cap
                                       centres), the polygon rounded once to FP32 relative to x_p */

typedef struct nlfem_mesh_s* nlfem_mesh_t;
typedef struct nlfem_system_s* nlfem_system_t;
typedef struct nlfem_batch_s* nlfem_batch_t;

typedef struct {
    int kernel;              /* NLFEM_KERNEL_* */
    double delta;            /* horizon, > 0 */
    double s;                /* fractional order s in (0,1) for NLFEM_KERNEL_FRACTIONAL; ignored otherwise */
    double kconst;           /* kernel constant; NaN selects the constant of Sec. 3 for the kernel
                                (constant kernel: 4/(pi delta^4), on the infinity ball 3/(4 delta^4);
                                tabulated kernel: 1) */
    int ball;                /* NLFEM_BALL_* */
    int quad_outer;          /* 7 (Sec. 3.1 rule) or 16 (degree-7 conical product rule) */
    int quad_inner;          /* 7 or 16 */
    int duffy_gauss;         /* Gauss points per direction of the singular rule, 1..32 (5 in Sec. 3.1) */
    int close_rule;          /* NLFEM_CLOSE_* */
    int precision;           /* NLFEM_PREC_* */
    int64_t mem_budget_bytes;/* 0 = unlimited; else the assembly fails with NLFEM_ERR_BUDGET beyond it */
    /* label-dependent kernel (Sec. 1, interface problems): with n_materials > 0 the kernel on
     * E_k x E_l is multiplied by material_scale[m_k * n_materials + m_l], m the material labels
     * of nlfem_mesh_set_materials. The table (host memory, n_materials^2 doubles, read during
     * the call) must be symmetric so that A stays symmetric. 0 / NULL = no labels. */
    int n_materials;         /* 0..16 */
    const double* material_scale;
    /* NLFEM_KERNEL_TABULATED: table_size (2..1024) values of g, host memory, read during the call */
    int table_size;
    const double* kernel_table;
    /* FP32 bulk only (ignored by NLFEM_PREC_FP64, which does everything in FP64) */
    int singular_precision;  /* NLFEM_SINGULAR_* (0 = FP64) */
    int geometry_precision;  /* NLFEM_GEOMETRY_* (0 = FP32) */
} nlfem_params;

typedef struct {
    int64_t npairs;          /* ordered interacting element pairs, (k,k) included */
    int64_t pairs_identical, pairs_edge, pairs_vertex, pairs_separated;
    int64_t nnz;             /* CSR nonzeros (dof level) */
    int64_t device_bytes;    /* device memory held by the mesh handle and the system */
    double ms_pairs;         /* pair search of the last cold assembly (0 when cached) */
    double ms_pattern;       /* CSR pattern and reduction index (0 when cached) */
    double ms_quadrature;    /* pair quadrature kernels */
    double ms_reduce;        /* segmented reduction into CSR */
    int cached;              /* 1 if the pair list / pattern of the mesh handle were reused */
    double ms_whole;         /* FP32 bulk: standard-rule pairs with E_l in the ball of every outer point */
    double ms_cut;           /* FP32 bulk: the other standard-rule pairs (FP64 plain: all pairs) */
    double ms_close;         /* intersecting pairs under the singular or the diamond rule */
    int64_t pairs_whole;     /* standard-rule pairs with E_l in the ball of every point of E_k */
    int64_t n_upper;         /* node-level upper pattern entries (one reduction unit each) */
    int64_t n_contrib;       /* contributions gathered by the ordered reduction (FP64 path; 0 before) */
    double ms_sums;          /* FP32 bulk: per-element ll sums and close-list adds */
} nlfem_assembly_info;

typedef struct {
    int iterations;          /* inner CG iterations, summed over refinement steps */
    int refinements;         /* FP64 residual refinement steps */
    double rel_residual;     /* ||b - A_FF u_F|| / ||b|| in FP64 at exit */
} nlfem_solve_info;

/* Thread-local message of the last failing call on this thread ("" if none). */
const char* nlfem_last_error(void);

/* Library version string. */
const char* nlfem_version(void);

/*
 * Upload a triangle mesh of the base domain (Sec. 2.2): vertices verts [M x 2] (x, y
 * interleaved, FP64) and triangles elems [K x 3] (vertex indices, any orientation; they
 * are made counter-clockwise). elem_label [K]: 1 = element of Omega, 0 = of Omega_D; NULL
 * labels every element Omega (pure Neumann-type base domain). A node is a Dirichlet node
 * iff it is a vertex of an Omega_D element. ndof_per_node: 1 (scalar kernels) or 2
 * (peridynamics). Pointers may be host or device memory; the data are copied, the caller
 * keeps ownership. Work is ordered on stream (a cudaStream_t, NULL = legacy default).
 * The handle is owned by the library until nlfem_mesh_destroy.
 * Errors: INVALID_ARG (NULL pointer, M < 3, K < 1, ndof not 1 or 2), BAD_MESH (index out
 * of range, zero-area triangle), OOM, CUDA.
 */
int nlfem_mesh_create(const double* verts, int64_t M, const int32_t* elems, int64_t K,
                      const int8_t* elem_label, int ndof_per_node, void* stream,
                      nlfem_mesh_t* out);

void nlfem_mesh_destroy(nlfem_mesh_t mesh);

/*
 * Discontinuous P1 ansatz (Sec. 2.2, J = n (d+1) K): the same mesh with every element
 * carrying its own copies of its vertices. Node 3k + a of the handle is vertex a of element k
 * as given in elems (k < K, a < 3), so the handle has 3K nodes: f_nodal, g_nodal and u are
 * given per copy, dof (3k + a) * ndof + c. Pairs are found and classified by the vertices'
 * positions, as for the continuous mesh. Touching pairs under the singular rule take the
 * factored form of eq. case-one-factoredOut (the six dofs of the pair, the same regularising
 * maps with the Gauss rule in every direction), which Tab. 1 admits for s <= 1/2 only: a
 * fractional kernel with s > 1/2 makes nlfem_assemble fail with UNSUPPORTED. The constant,
 * peridynamic and tabulated kernels assemble as usual.
 * Arguments, ownership and errors as nlfem_mesh_create.
 */
int nlfem_mesh_create_dg(const double* verts, int64_t M, const int32_t* elems, int64_t K,
                         const int8_t* elem_label, int ndof_per_node, void* stream, nlfem_mesh_t* out);

/*
 * Material labels of the elements for label-dependent kernels (Sec. 1: the kernel may depend
 * on element labels, which assembles interface problems monolithically). material [K] int8
 * in 0..15, host or device, copied; NULL removes the labels. Independent of the Omega /
 * Omega_D labels of nlfem_mesh_create; the pair list and pattern do not depend on them.
 * Errors: INVALID_ARG (a label outside 0..15), CUDA, OOM.
 */
int nlfem_mesh_set_materials(nlfem_mesh_t mesh, const int8_t* material, void* stream);

/* Fill p with the defaults of Sec. 3.1 for the given kernel: delta = 0.1, nocaps,
 * 7-point rules, 5 Gauss points, automatic close-pair rule, FP64. */
void nlfem_params_default(nlfem_params* p, int kernel);

/*
 * Assemble the stiffness matrix A_h^# of eq. biFormApprox (the pair loop of Alg. 1: for every
 * ordered interacting pair (E_k, E_l) the singular rule if they intersect and the rule of
 * Tab. 1 asks for it, else the truncation rule of eq. discrete-inner on E_l cut by the ball
 * approximation of each outer point; Alg. 2 / eq. graph:interactionEdges define the pairs)
 * over all dofs of the base domain (full Neumann-type
 * matrix, symmetric to the last bit) and the load vector F_i = int_Omega f phi_i computed
 * with the outer rule from the P1 interpolant of f_nodal [M x ndof] (host or device, NULL
 * means f = 0). The interaction graph, CSR pattern and reduction index are built on the
 * first call and cached in the mesh handle for later calls with the same delta, ball,
 * outer rule and close-pair class (see nlfem_assembly_info.cached).
 * Work is ordered on stream; the call returns after the result is complete on the
 * device. The system handle is owned by the library until nlfem_system_destroy.
 * Errors: INVALID_ARG, UNSUPPORTED (more than 32768 partners per element, or a row
 * referring to more than 2^32 / 84 pairs), BUDGET, OOM, CUDA.
 */
int nlfem_assemble(nlfem_mesh_t mesh, const nlfem_params* params, const double* f_nodal,
                   void* stream, nlfem_system_t* out);

/*
 * Persistent batch plan (FP32 bulk only): the systems of n meshes stay on the device and
 * their values are re-assembled in place by replaying one CUDA graph (close lists, pilot,
 * scale, fused bulk launches, ll sums, conversion to CSR, load vectors), so repeated
 * assemblies of many small problems pay no per-kernel launch cost. nlfem_batch_create does
 * the cold work and one assembly, then captures the graph (the load data f_nodal is copied
 * into the plan); nlfem_batch_run replays it on stream (ms, if not NULL, receives its device
 * time); nlfem_batch_system returns system i, owned by the plan (valid until
 * nlfem_batch_destroy; do not pass it to nlfem_system_destroy). Every run gives the same
 * bits as nlfem_assemble. The paper has no counterpart (execution strategy of this
 * implementation). Errors: as nlfem_batch_assemble; UNSUPPORTED for an FP64 item.
 */
int nlfem_batch_create(const nlfem_mesh_t* meshes, const nlfem_params* params, const double* const* f_nodal,
                       int n, void* stream, nlfem_batch_t* out);
int nlfem_batch_run(nlfem_batch_t batch, void* stream, double* ms);
int nlfem_batch_system(nlfem_batch_t batch, int i, nlfem_system_t* out);
void nlfem_batch_destroy(nlfem_batch_t batch);

/*
 * Autotuner of the FP32-bulk launch shape: for the kernel class of params (kernel type,
 * rules, ball) it times the whole-pair and the cut-pair kernels on mesh with every candidate
 * grid size (2 ... 64 resident blocks of 4 warps per SM; each warp takes 32-pair tiles) and,
 * for the cut-pair kernel, every candidate number of outer points per chunk (its full chunk,
 * half of it, 2: the polygons of a chunk are built, then drained one fan triangle per lane),
 * and keeps the fastest for the rest of the process. best receives [0] the blocks per SM of
 * the whole-pair kernel, [1] those of the cut-pair kernel and [2] its outer points per chunk.
 * The results of every assembly are the same bits whatever the shape. The paper has no
 * counterpart. Errors: INVALID_ARG, UNSUPPORTED (FP64), OOM, CUDA.
 */
int nlfem_autotune(nlfem_mesh_t mesh, const nlfem_params* params, void* stream, int32_t best[3]);

/*
 * Set the FP32-bulk launch shape of the kernel class of params without timing (for example a
 * shape nlfem_autotune chose in an earlier process): shape[0] blocks per SM of the whole-pair
 * kernel (1 ... 64), shape[1] of the cut-pair kernel (1 ... 64), shape[2] its outer points per
 * chunk (0 = its full chunk, 8 with approxcaps, 7 otherwise, or fewer). Results do not depend
 * on it. No counterpart in the paper. Errors: INVALID_ARG (NULL, out of range), UNSUPPORTED
 * (FP64).
 */
int nlfem_tune_set(const nlfem_params* params, const int32_t shape[3]);

/*
 * Batched assembly: the same result as n calls of nlfem_assemble (every system is the same
 * bits), with the whole-pair and cut-pair kernels of all FP32-bulk items of one kernel class
 * (kernel type, outer and inner rule, ball) fused into one persistent launch each, so many
 * small meshes keep the GPU busy (a batching of the work of Sec. 3.4 across problems; the
 * paper assembles one problem at a time). meshes: n distinct mesh handles; params: n
 * parameter sets; f_nodal: NULL or n pointers (each NULL, host or device, as for
 * nlfem_assemble); out: n system handles, owned by the caller as for nlfem_assemble. FP64
 * items are assembled one after the other in the same call. The ms_* fields of every
 * system's info describe the whole batch. Errors: INVALID_ARG (NULL, n < 0, a mesh twice),
 * UNSUPPORTED, BUDGET (per item), OOM, CUDA; on error no system is returned.
 */
int nlfem_batch_assemble(const nlfem_mesh_t* meshes, const nlfem_params* params, const double* const* f_nodal,
                         int n, void* stream, nlfem_system_t* out);

/* Borrowed device pointers of the assembled matrix in CSR form, the format in which the
 * paper's library hands the stiffness matrix back to its Python front end for any sparse
 * solver (Sec. 1; Sec. 3.4 sums the per-thread parts into it) (valid until
 * nlfem_system_destroy): row_ptr [nrows + 1] int64, col [nnz] int32 (sorted per row),
 * val [nnz] FP64. Dof d of node m is row m * ndof + d. Errors: INVALID_ARG (NULL). */
int nlfem_system_csr(nlfem_system_t sys, const int64_t** row_ptr, const int32_t** col,
                     const double** val, int64_t* nrows, int64_t* nnz);

/* Borrowed device pointer to the load vector F [nrows]. */
int nlfem_system_rhs(nlfem_system_t sys, const double** F);

/* Borrowed device pointer to the Dirichlet node flags [M] (int8, 1 = Dirichlet). */
int nlfem_system_dirichlet(nlfem_system_t sys, const int8_t** flags);

/* Counts and timings of the assembly that produced sys (nlfem_assembly_info above), copied
 * to the caller's info (host). Errors: INVALID_ARG (NULL). */
int nlfem_system_info(nlfem_system_t sys, nlfem_assembly_info* info);

/* Device pointers to the interaction graph of the cached pair list: k [npairs], l [npairs]
 * (int32, sorted by (k, l)). Valid until the next nlfem_assemble with other parameters
 * or nlfem_mesh_destroy. */
int nlfem_mesh_pairs(nlfem_mesh_t mesh, const int32_t** k, const int32_t** l, int64_t* npairs);

/*
 * Solve the nonlocal Dirichlet problem A_FF u_F = F_F - A_FD g (eq.
 * inhomogeneousDirichletData): F = free dofs, D = dofs of Dirichlet nodes. g_nodal
 * [nrows] holds the Dirichlet data (values at free dofs are ignored; NULL = 0).
 * Conjugate gradients on A_FF in FP32, wrapped in FP64 residual refinement until
 * ||b - A_FF u_F|| <= tol_rel ||b|| (FP64). u_out [nrows], device, caller-owned: on
 * return holds u_F at free dofs and g at Dirichlet dofs. g_nodal may be host or device.
 * Errors: INVALID_ARG, NOT_CONVERGED (max_iter inner iterations reached; u_out holds the
 * last iterate and info the residual), OOM, CUDA.
 */
int nlfem_solve(nlfem_system_t sys, const double* g_nodal, double tol_rel, int max_iter,
                double* u_out, nlfem_solve_info* info, void* stream);

/*
 * Pure Neumann-type problem on the full matrix (every dof unknown, Dirichlet flags
 * ignored). A annihilates its null space N up to rounding: the constants for scalar
 * kernels, the rigid motions (two translations and the rotation (-y, x)) for the
 * peridynamic kernel (Sec. 1 and Rem. 2.4: the symmetrised form keeps N exact). Returns the
 * u orthogonal to N with P A u = P F, P the orthogonal projector onto the complement of N
 * (for an exact null space: the minimum-norm solution of A u = F - (the part of F in N)).
 * Projected FP32 conjugate gradients inside FP64 residual refinement until
 * ||P (F - A u)|| <= tol_rel ||P F||. u_out [nrows], device, caller-owned.
 * Errors: INVALID_ARG, NOT_CONVERGED (u_out holds the last iterate), OOM, CUDA.
 */
int nlfem_solve_neumann(nlfem_system_t sys, double tol_rel, int max_iter, double* u_out,
                        nlfem_solve_info* info, void* stream);

/*
 * Work of the assembly that produced sys, counted on the device with the canonical FP64
 * geometry (for FLOP accounting; it does not change sys). counts[16] receives: [0] kernel
 * evaluations of the truncation quadrature, [1] outer points whose inner element lies
 * fully in the ball, [2] outer points whose inner element was cut and retriangulated,
 * [3] sub-triangles of the cut polygons, [4] kernel evaluations of the singular rule,
 * [5] pairs on the truncation path, [6] pairs on the singular path, [7] outer points
 * with an empty intersection, [8] outer points visited; split by the FP32-bulk kernels:
 * [9] evaluations of the whole-pair kernel, [10] evaluations of the cut-pair kernel,
 * [11] outer points, [12] cut outer points, [13] nonempty outer points and
 * [14] evaluations on sub-triangles of the cut-pair kernel, [15] evaluations of the
 * canonical truncation kernel. The mesh's cached pair list must still be the one sys was
 * assembled on. Errors: INVALID_ARG, CUDA.
 */
int nlfem_system_census(nlfem_system_t sys, int64_t counts[16], void* stream);

void nlfem_system_destroy(nlfem_system_t sys);

/*
 * Interaction graph of a small mesh, computed without allocating any device memory.
 * For callers that cannot call cudaMalloc at the point where they need the pairs: a serving
 * process that reserved the device memory up front for its own arena (an allocation here
 * would take memory the arena already counts as its own, or fail), a host framework whose
 * caching allocator owns the device memory, or a context where an out-of-memory failure
 * must not be possible. The paper has no counterpart; it returns the same pairs as
 * nlfem_mesh_pairs after an nlfem_assemble with the same delta, ball and outer rule.
 * verts [M x 2] FP64, elems [K x 3] int32 (device memory; any orientation), out_k and
 * out_l device int32 arrays of length capacity, owned by the caller; on success they hold
 * the *npairs ordered interacting pairs sorted by (k, l) (host int64 output).
 * Limits: K <= 32768 triangles and M <= 65536 vertices (NLFEM_ERR_UNSUPPORTED beyond).
 * The working data lives in a file-scope device array of 4,981,504 bytes (about 5 MB) that
 * every GPU loading this library holds until the process exits; the first call on a device
 * looks up its address, so make that first call before any stream capture. All calls share
 * that array and it keeps the last call's contents (each call clears what it counts into);
 * calls that overlap on the GPU (other streams or host threads) race and must be serialised.
 * The call synchronises stream: it reads the mesh checks and the pair count back to the
 * host before it writes the pairs.
 * Errors: INVALID_ARG (NULL or host pointers, delta <= 0, unknown ball / rule, capacity
 * too small: *npairs then holds the number needed), UNSUPPORTED, BAD_MESH, CUDA.
 */
int nlfem_pairs_noalloc(const double* verts, int64_t M, const int32_t* elems, int64_t K, double delta,
                        int ball, int quad_outer, int32_t* out_k, int32_t* out_l, int64_t capacity,
                        int64_t* npairs, void* stream);

/* Device memory held by a mesh handle and its cached pair list / pattern, in bytes. */
int64_t nlfem_mesh_device_bytes(nlfem_mesh_t mesh);

/*
 * Working buffers are taken from the current device's default CUDA memory pool, which
 * the library sets to keep freed blocks for reuse (no unmapping at every synchronisation).
 * nlfem_trim_memory synchronises stream and returns every unused block of that pool to
 * the driver. No counterpart in the paper (memory management of this implementation).
 * Errors: CUDA.
 */
int nlfem_trim_memory(void* stream);

#ifdef __cplusplus
}
#endif

#endif /* NLFEM_H */
