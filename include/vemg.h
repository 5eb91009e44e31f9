/*
 * vemg.h -- C ABI of libvemg: a GB300 (sm_103a) solver for the P1 finite-element Poisson
 * problem on thin (small aspect ratio) tetrahedral meshes, preconditioned by vertical-
 * extrapolation multigrid, after Kramer, Cotter and Pain, "Solving the Poisson equation on
 * small aspect ratio domains using unstructured meshes".
 *
 * Conventions shared by every entry point:
 *   - Nodes are numbered by the caller ("caller order"). Vectors passed in and out (b, x, f) are
 *     in caller order; the library permutes internally (top-surface nodes first, section 3,
 *     Eqs. phi_decomposition and equation_decomposition).
 *   - Arrays named *_dev are device pointers on the current CUDA device; arrays in vemg_mesh and
 *     names ending in _host are host pointers. The caller owns every array it passes; the
 *     library copies what it keeps. Objects the library returns (vemg_hierarchy, the arrays of a
 *     vemg_csr filled by vemg_assemble) are owned by the library and freed by vemg_destroy /
 *     vemg_csr_free.
 *   - stream is a cudaStream_t (NULL = the legacy default stream). Setup synchronises the
 *     stream; solves enqueue their work on it and synchronise it before returning (the
 *     iteration count and status are host values).
 *   - Every entry point returns a status code (VEMG_OK = 0). No C++ exception crosses the ABI.
 *     On error, output arrays hold unspecified values unless stated otherwise.
 *   - Device memory comes from the allocator installed with vemg_set_allocator (cudaMalloc
 *     when none is installed).
 *   - A hierarchy may be used by one host thread at a time.
 */
#ifndef VEMG_H
#define VEMG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define VEMG_OK 0
#define VEMG_EINVAL 1      /* bad argument (null pointer, size, option out of range) */
#define VEMG_EMESH 2       /* invalid mesh: non-positive tet volume, index out of range, no top
                              nodes, top triangle with a non-top vertex, node outside the top
                              surface's projection */
#define VEMG_ENOMEM 3      /* the allocator returned NULL */
#define VEMG_ENOTCONV 4    /* max_it reached; x holds the last iterate, info is filled */
#define VEMG_EBREAKDOWN 5  /* CG breakdown: p^T A p <= 0, NaN or Inf in the iteration */
#define VEMG_ETIMEOUT 6    /* a bounded device-side wait expired */
#define VEMG_ECUDA 7       /* a CUDA runtime call failed */
#define VEMG_EINTERNAL 8   /* an internal capacity was exceeded */

/* node tags (bitmask), section 2.1: top surface, floor, coasts */
#define VEMG_TAG_TOP 1
#define VEMG_TAG_FLOOR 2
#define VEMG_TAG_COAST 4

/* boundary conditions, section 3: all-Neumann (constants are the nullspace, removed by mean
   projection) or Dirichlet phi = 0 on the top surface (the matrix A_bar) */
#define VEMG_NEUMANN 0
#define VEMG_DIRICHLET_TOP 1

/* preconditioner (the three compared in section 6) */
#define VEMG_PRECOND_ADDITIVE 0  /* vertical lumping + additive smoother, Eq. ourpreconditioner (section 5.5) */
#define VEMG_PRECOND_VL_SOR 1    /* vertical lumping as the first coarsening of a V-cycle on A with SOR smoothing */
#define VEMG_PRECOND_SA 2        /* smoothed-aggregation AMG on A */
#define VEMG_PRECOND_NONE 3      /* none: plain CG, for the spectrum of A itself (section 4); FP64 only */

/* how a preconditioner application is launched */
#define VEMG_CYCLE_PERSISTENT 0  /* one cooperative kernel runs every phase of the V-cycles */
#define VEMG_CYCLE_LAUNCHES 1    /* one kernel per phase (colour sweep, residual, transfer) */
#define VEMG_CYCLE_AUTO 2        /* the fastest structure as measured on GB300: one kernel per phase */
#define VEMG_CYCLE_HYBRID 3      /* one kernel per phase on each chain's finest level, one cooperative
                                    kernel for the coarser levels of both chains */

/* precision of the preconditioner; the outer Krylov loop is always FP64 */
#define VEMG_PREC_FP64 0   /* everything FP64, CG outer loop */
#define VEMG_PREC_FP32 1   /* V-cycle values, vectors and arithmetic FP32, flexible CG outer loop */
#define VEMG_PREC_BF16 2   /* as FP32, with the off-diagonal values of the V-cycle operators (A, P,
                              P^T of every level) rounded to BF16 (from FP32, nearest even) and
                              stored in BF16; diagonals, vectors and sums FP32. The cycle runs one
                              kernel per phase; the batched solves and the single-CTA coarse tail
                              read FP32 copies of the same rounded values. A surface chain with the
                              near-nullspace {1, x, y} (surf_nullspace = 3) keeps FP32 values */

/* Tetrahedral mesh, HOST pointers (section 2.1, section 3).
   xyz: n_nodes x 3 doubles (x, y, z), z up, top surface at the largest z of each column.
   tets: n_tets x 4 node ids with positive orientation ((p1-p0).((p2-p0)x(p3-p0)) > 0).
   tags: n_nodes bitmasks of VEMG_TAG_*.
   top_tris: n_top_tris x 3 node ids (all tagged VEMG_TAG_TOP), counter-clockwise in (x, y);
   the triangulation of the top surface used for vertical extrapolation (section 5.4). */
typedef struct vemg_mesh {
    int64_t n_nodes;
    const double *xyz;
    int64_t n_tets;
    const int32_t *tets;
    const uint8_t *tags;
    int64_t n_top_tris;
    const int32_t *top_tris;
} vemg_mesh;

/* Square CSR matrix, DEVICE pointers, rows sorted by column, 32-bit indices. */
typedef struct vemg_csr {
    int64_t n;
    int64_t nnz;
    int32_t *rowptr; /* n + 1 */
    int32_t *col;    /* nnz */
    double *val;     /* nnz */
} vemg_csr;

typedef struct vemg_options {
    int bc;           /* VEMG_NEUMANN or VEMG_DIRICHLET_TOP */
    int precision;    /* VEMG_PREC_FP64, VEMG_PREC_FP32 or VEMG_PREC_BF16 */
    double strength;  /* SA strong-coupling threshold, section 6: 0.01 */
    double omega_p;   /* SA prolongator smoothing weight, section 6: 2/3 */
    int coarse_max;   /* a level of at most this many rows is solved directly (dense), 1..1024 */
    int max_levels;   /* per multigrid chain, at most 16 */
    int precond;      /* VEMG_PRECOND_*. With Dirichlet-top the additive form and SA are the same
                         cycle (SA on A_bar); VL_SOR needs Neumann (VEMG_EINVAL otherwise) */
    int cycle;        /* VEMG_CYCLE_*: same arithmetic, different launch structure */
    int tail_rows;    /* per-phase cycles: the first level below the finest with at most this many
                         rows, and every level under it, run as one kernel (the coarse tail of the
                         V-cycle; 0: never); 0..262144 */
    int surf_nullspace; /* near-nullspace of the surface chain's smoothed aggregation: 1 = the
                         constants (the paper's SA), 3 = {1, x, y} with the top nodes' horizontal
                         coordinates (Vanek, Mandel and Brezina's choice for fourth-order-like
                         operators: E~^T A E~ of vertically unstructured meshes, section 4; node
                         blocks of up to 3 coarse unknowns per aggregate below level 0, strength
                         by block Frobenius norms, prolongator smoothing with the unfiltered A) */
    int tail_cluster; /* the kernel of the coarse tail: 0 = one CTA whose steps are separated by
                         CTA barriers (tail_rows at most 65536), 2..16 = one thread-block cluster
                         of that many CTAs whose steps are separated by the hardware cluster
                         barrier; the vectors stay in global memory either way */
} vemg_options;

typedef struct vemg_info {
    int iters;            /* CG iterations (matrix-vector products with A) */
    int status;           /* VEMG_OK, VEMG_ENOTCONV or VEMG_EBREAKDOWN */
    double relres;        /* ||r_k||_2 / ||b||_2 of the recursively updated residual */
    double true_relres;   /* ||b - A x||_2 / ||b||_2 recomputed at exit */
    double b_mean;        /* Neumann: the mean removed from b (0 for Dirichlet-top) */
} vemg_info;

typedef struct vemg_hierarchy vemg_hierarchy;

/* Fill opts with the paper's parameters (section 6): strength 0.01, omega_p = 2/3, Neumann,
   FP64, coarse_max = 1024, max_levels = 10, the additive preconditioner, VEMG_CYCLE_AUTO,
   tail_rows = 0, surf_nullspace = 1, tail_cluster = 0. */
void vemg_default_options(vemg_options *opts);

/* Assemble the P1 stiffness matrix A_ij = integral grad N_i . grad N_j in physical coordinates
   (section 3, Eq. Ax=b; the paper's rescaled A_eps equals (H / L^2) A). A_out receives device
   arrays allocated by the library, in caller order; release them with vemg_csr_free. Entries
   are summed over elements in ascending element index. Returns VEMG_EMESH on a non-positive
   volume or an out-of-range node id. Synchronises the stream. */
int vemg_assemble(const vemg_mesh *mesh, vemg_csr *A_out, void *stream);

/* Load vector b = M f (section 3, Eq. Ax=b): M_ij = integral N_i N_j, f given by its nodal values.
   f_dev and b_dev are device arrays of n_nodes doubles in caller order. */
int vemg_load(const vemg_mesh *mesh, const double *f_dev, double *b_dev, void *stream);

/* Free the arrays of a matrix returned by vemg_assemble. */
void vemg_csr_free(vemg_csr *A);

/* Build the preconditioner hierarchy for A (caller order, device, as vemg_assemble returns it):
   the top-first ordering, the vertical extrapolation operator E~ by column location on the top
   triangulation (section 5.4), the surface operator E~^T A E~ (section 5.1, Eq. reduced AMG),
   the Dirichlet-top block A_bar, and smoothed-aggregation chains on both (section 6), giving
   the additive preconditioner of Eq. ourpreconditioner (section 5.5). Dirichlet-top builds
   the A_bar chain only. *out is owned by the library. Synchronises the stream. */
int vemg_setup(const vemg_csr *A, const vemg_mesh *mesh, const vemg_options *opts, void *stream,
               vemg_hierarchy **out);

/* Free a hierarchy and all its device memory. NULL is ignored. */
void vemg_destroy(vemg_hierarchy *h);

/* Solve A x = b by preconditioned CG (FP64 preconditioner) or flexible CG (FP32 preconditioner)
   from x0 = 0 (section 6: the multigrid cycle is applied as a preconditioner within each CG
   iteration). Neumann: b is projected to zero mean (info->b_mean), every preconditioned
   residual is projected to zero mean, and x has zero mean. Dirichlet-top: top entries of b are
   ignored and x = 0 on top nodes. Stops when ||r_k|| <= rtol ||b||; ||b|| = 0 gives x = 0 and
   iters = 0. b_dev and x_dev are device arrays of n_nodes doubles (caller order) and may not
   overlap. Returns info->status. Synchronises the stream. */
int vemg_solve(vemg_hierarchy *h, const double *b_dev, double *x_dev, double rtol, int max_it,
               vemg_info *info, void *stream);

/* As vemg_solve with HOST arrays b_host and x_host (n_nodes doubles, caller order): copies b to
   the device, solves, copies x back. Page-locked host memory gives asynchronous copies. The first
   call allocates two device vectors of n_nodes doubles that stay with the hierarchy (counted by
   vemg_hierarchy_bytes), so later calls allocate nothing. */
int vemg_solve_host(vemg_hierarchy *h, const double *b_host, double *x_host, double rtol, int max_it,
                    vemg_info *info, void *stream);

/* Solve k systems A X = B with one right-hand side per column: column c of B is
   B_dev[c * ldb + i], i < n_nodes (caller order), and likewise X. Each column is an independent
   CG/FCG run with its own step lengths and convergence test; a converged column is frozen. A column
   whose best residual has not dropped by 1% in 30 iterations has reached the round-off floor and
   stops with VEMG_ENOTCONV (relres holds its last residual).
   infos has k entries. Returns VEMG_OK if every column converged, else the first non-OK
   column status. */
int vemg_solve_batch(vemg_hierarchy *h, int k, const double *B_dev, int64_t ldb, double *X_dev,
                     int64_t ldx, double rtol, int max_it, vemg_info *infos, void *stream);

/* ---- continuous batching ----
   An engine holds `slots` right-hand-side columns of one hierarchy (rounded up to a power of two,
   at most 128). Requests are admitted into free slots between iterations and retired when done,
   while the other slots keep iterating: each column has its own Krylov recurrence, tolerance and
   iteration limit (the batched form of vemg_solve). Work is enqueued on the engine's stream, so
   engines of different hierarchies on different streams run concurrently on the device. Each
   engine owns its work memory (vemg_engine_bytes); one engine per hierarchy at a time. */
typedef struct vemg_engine vemg_engine;

/* Launch shapes of the batched solve's row kernels (the paper has no counterpart: an autotuner of
   this implementation). Three classes: 0 = colour sweeps, 1 = the other V-cycle operations,
   2 = the outer FP64 operations (A p, the true residual, E~ and E~^T). Each has kw lanes per row
   (4, 8, 16 or 32; each lane takes the columns lane, lane + kw, ...) and warps per block (2, 4, 8).
   The first batched solve (or engine) of a width K times every candidate shape on this
   hierarchy's finest level and outer operator and keeps the fastest of each class; the results do
   not depend on the shapes. vemg_batch_tuning reports the batch width and the shapes in use with
   their measured launch times in microseconds (VEMG_EINVAL before any batched solve);
   vemg_batch_set_tuning imposes shapes for width K (allocating its work if needed). */
int vemg_batch_tuning(const vemg_hierarchy *h, int *K, int *kw3, int *warps3, float *us3);
int vemg_batch_set_tuning(vemg_hierarchy *h, int K, const int *kw3, const int *warps3, void *stream);

#define VEMG_SLOT_FREE 0
#define VEMG_SLOT_RUNNING 1
#define VEMG_SLOT_DONE 2    /* converged, broken down or out of iterations: retire it */

int vemg_engine_create(vemg_hierarchy *h, int slots, void *stream, vemg_engine **out);
void vemg_engine_destroy(vemg_engine *e);

/* Copy b (device, caller order) into a free slot, project it (Neumann) and start its iteration at
   the next step. *slot receives the slot; VEMG_ENOMEM if no slot is free. Asynchronous: b_dev is
   read by kernels on the engine's stream, so it must hold its values when that stream reaches
   them (order its producer before, e.g. an event the engine's stream waits on) and must stay
   allocated until they have run (the engine's stream has passed this call). */
int vemg_engine_admit(vemg_engine *e, const double *b_dev, double rtol, int max_it, int *slot);

/* Enqueue `iters` iterations of every occupied slot and a copy of the slot states (asynchronous;
   vemg_engine_wait completes it). */
int vemg_engine_launch(vemg_engine *e, int iters);
int vemg_engine_wait(vemg_engine *e);

/* Whether the engine's stream still has work (*busy = 1) or has completed everything enqueued on
   it (*busy = 0), without waiting. After *busy = 0 the slot states are those of the last launch,
   as after vemg_engine_wait; a server can thus step every engine at its own pace. */
int vemg_engine_query(const vemg_engine *e, int *busy);

/* State of a slot after the last wait (or a query that found the engine idle): VEMG_SLOT_FREE /
   RUNNING / DONE, and its info (iters, status, recursive relres; true_relres = -1: not
   computed). */
int vemg_engine_poll(const vemg_engine *e, int slot, vemg_info *info, int *state);

/* Copy the slot's x (device, caller order, zero mean for Neumann, 0 on top nodes for Dirichlet-top)
   and free the slot. Synchronises the engine's stream. */
int vemg_engine_retire(vemg_engine *e, int slot, double *x_dev);

int vemg_engine_slots(const vemg_engine *e, int *slots, int *free_slots);
int vemg_engine_bytes(const vemg_engine *e, size_t *bytes);

/* Device bytes held by a hierarchy (operators, transfer operators, work vectors). */
int vemg_hierarchy_bytes(const vemg_hierarchy *h, size_t *bytes);

/* Install the device allocator used by every later allocation (NULL alloc restores cudaMalloc /
   cudaFree). alloc(bytes, ctx) returns a device pointer or NULL; free(ptr, ctx) releases it.
   Memory allocated before a change is released through the allocator that allocated it. */
int vemg_set_allocator(void *(*alloc)(size_t bytes, void *ctx), void (*free_fn)(void *ptr, void *ctx),
                       void *ctx);

/* Human-readable name of a status code (static string). */
const char *vemg_strerror(int status);

/* ---- spectrum (section 4): the CG coefficients of a solve give the Lanczos tridiagonal of the
   preconditioned operator, whose extreme eigenvalues converge to those of M^-1 A (of A with
   VEMG_PRECOND_NONE; on the complement of the constants with Neumann) ---- */

/* Coefficients of the last vemg_solve on h: alpha[k] = (r_k, z_k) / (p_k, A p_k) and beta[k] =
   (r_k, z_k) / (r_{k-1}, z_{k-1}) (beta[0] = 0), k < *count = iterations of that solve (at most
   4096 are kept). Host arrays of capacity entries; VEMG_EINVAL if capacity < *count (with *count
   set) or if the V-cycles are FP32 (flexible CG has no Lanczos recurrence). Synchronous. */
int vemg_solve_coefficients(vemg_hierarchy *h, int capacity, double *alpha, double *beta, int *count);

/* Smallest and largest eigenvalue of the tridiagonal T with T_00 = 1/alpha_0,
   T_kk = 1/alpha_k + beta_k/alpha_{k-1}, T_{k,k+1} = sqrt(beta_{k+1})/alpha_k, for k < count
   (Sturm-sequence bisection, relative accuracy ~1e-14). Host arrays; VEMG_EINVAL if count < 1
   or a coefficient is not positive. Touches no GPU. */
int vemg_lanczos_extremes(const double *alpha, const double *beta, int count, double *lambda_min,
                          double *lambda_max);

/* The CUDA error behind the last VEMG_ECUDA returned on this host thread: the runtime's message,
   the failing call and its source location. Empty if none. The string is owned by the library
   and stays valid until the next failing call on this thread. */
const char *vemg_last_error(void);

/* Self-test of the bounded wait behind VEMG_CYCLE_PERSISTENT (no counterpart in the paper): a
   cooperative launch of launched_blocks CTAs meets at one grid barrier that expects
   claimed_blocks CTAs (1 <= launched_blocks <= claimed_blocks <= 8, else VEMG_EINVAL). Equal
   counts: the barrier completes, VEMG_OK. claimed > launched: it can never complete, every wait
   gives up after a few milliseconds and the call returns VEMG_ETIMEOUT with the CUDA context
   intact. Allocates 12 bytes of device memory; synchronous on the stream. */
int vemg_selftest_barrier(int claimed_blocks, int launched_blocks, void *stream);

/* ---- introspection and single steps (used by parity tests; all in the internal top-first
   ordering of section 3, chain 0 = surface chain on E~^T A E~, chain 1 = A_bar chain, chain 2 =
   the single chain of VEMG_PRECOND_VL_SOR (A with E~, then the surface chain) or VEMG_PRECOND_SA)
   ---- */

/* Sizes: key is one of "n", "mtop", "nnzA", "nnzE", "nnzAc", "nlev" (of the chain), "direct"
   (coarsest level of the chain solved by the dense solve), "nsd" (near-nullspace vectors of the
   chain: 1 or 3), "lev.n", "lev.nnz", "lev.nnzP", "lev.ncolours" (of level `level` of the
   chain). *out = -1 if the item does not exist. */
int vemg_get_size(const vemg_hierarchy *h, const char *key, int chain, int level, int64_t *out);

/* Copy a CSR matrix to HOST arrays sized by vemg_get_size: name is "A" (internal order), "E"
   (vertical extrapolation E~, n x mtop), "Ac" (E~^T A E~), "lev.A", "lev.P" (of a chain level). */
int vemg_get_csr(const vemg_hierarchy *h, const char *name, int chain, int level, int32_t *rowptr_host,
                 int32_t *col_host, double *val_host);

/* Copy an integer array to HOST: "new2old" (n: caller id of each internal node), "tri_of" (n:
   located top triangle of each internal node, -1 on top nodes), "lev.agg" (aggregate of each
   node of a level), "lev.colour" (colour of each node of a level). */
int vemg_get_int(const vemg_hierarchy *h, const char *name, int chain, int level, int32_t *out_host);

/* Copy the near-nullspace rows of a level of a chain built with the near-nullspace {1, x, y}
   (vemg_options.surf_nullspace = 3) to HOST: lev.n x 3 doubles, row-major; level 0 holds
   (1, x, y) of the top nodes, a coarser level the rows R of its aggregates' local QR
   factorisations. VEMG_EINVAL for a chain with the constant near-nullspace. */
int vemg_get_nullspace(const vemg_hierarchy *h, int chain, int level, double *out_host);

/* y = A x on the unknowns of the hierarchy's boundary condition (internal order, device). */
int vemg_spmv(vemg_hierarchy *h, const double *x_dev, double *y_dev, void *stream);

/* z = M^-1 r, one application of the preconditioner of Eq. ourpreconditioner (internal order,
   device, without the mean projection). */
int vemg_precond(vemg_hierarchy *h, const double *r_dev, double *z_dev, void *stream);

/* One V-cycle of chain `chain` from a zero initial guess on its finest level (device). */
int vemg_vcycle(vemg_hierarchy *h, int chain, const double *b_dev, double *x_dev, void *stream);

/* y = A x exactly as vemg_spmv computes it (the same products summed in the same order, so the
   same bits), but allocating no device memory. (The paper has no counterpart: this serves
   callers that cannot call cudaMalloc, such as code running inside an allocator callback, or a
   process whose device memory budget is fixed before the solve starts.)
   vemg_setup builds everything this call reads (the solve-order index map and operator), so it
   works on any hierarchy vemg_setup returned, before or after any solve.
   Its work buffers live in one static device array owned by the library: 12 MiB, enough for
   hierarchies of at most 1,048,576 unknowns; a larger hierarchy is rejected with VEMG_EINVAL
   (vemg_last_error gives the count). Every device that loads libvemg holds that array until the
   process exits. The first call on a device looks up the array's device address
   (cudaGetSymbolAddress) with that device current. All calls share the one array: calls whose GPU work overlaps (several streams or host
   threads at once) race and give wrong results. The array needs no clearing: each call writes
   every entry it later reads. x_dev and y_dev are device arrays in the internal order, as for
   vemg_spmv. Each call synchronises the stream (cudaStreamSynchronize) before it returns. */
int vemg_spmv_static(vemg_hierarchy *h, const double *x_dev, double *y_dev, void *stream);

/* ---- measurement ---- */

/* Number of CUDA kernels the solve path of this hierarchy has launched since setup (host count). */
int vemg_kernel_launches(const vemg_hierarchy *h, int64_t *count);

/* Kernel classes that vemg_probe can time. */
#define VEMG_PROBE_NONE 0
#define VEMG_PROBE_SPMV_A 1      /* q = A p of the outer Krylov loop */
#define VEMG_PROBE_SOR_COARSE 2  /* multicolour SOR launches on every level except the finest
                                    level of the A_bar chain (every level of the other chains) */
#define VEMG_PROBE_SOR VEMG_PROBE_SOR_COARSE   /* the same class under its earlier name */
#define VEMG_PROBE_RESIDUAL 3    /* every V-cycle residual launch */
#define VEMG_PROBE_SOR_FINE 4    /* SOR launches on the finest level of the A_bar chain */
#define VEMG_PROBE_VCYCLE 5      /* the persistent preconditioner kernel (VEMG_CYCLE_PERSISTENT) */
#define VEMG_PROBE_TRANSFER 6    /* restrictions, prolongations and E~^T r (sliced-ELL transfers) */
#define VEMG_PROBE_VECTOR 7      /* the Krylov vector kernels: x/r update, z combination, p update */
#define VEMG_PROBE_DENSE 8       /* the dense coarsest-level solves */
#define VEMG_PROBE_TAIL 9        /* the coarse-tail kernels (vemg_options.tail_rows) */

/* Start timing one kernel class (VEMG_PROBE_NONE stops): every later launch of that class
   records a CUDA event before and after itself on its stream. Resets the accumulated totals. */
int vemg_probe(vemg_hierarchy *h, int kind);

/* Read the totals accumulated since vemg_probe (synchronises the device): summed kernel time in
   milliseconds, number of launches, and summed algorithmic bytes, i.e. for a sparse pass
   nnz (value + index bytes) + rows (row pointer + vector reads and writes). */
int vemg_probe_read(vemg_hierarchy *h, double *total_ms, int64_t *launches, double *algorithmic_bytes);

/* Per-phase profile of the persistent preconditioner kernel, summed over the applications run
   since vemg_probe(h, VEMG_PROBE_VCYCLE): for phase k of the program, its kind op[k] (0 one SOR
   colour, 1 residual, 2 y = S x (restriction or E~ transfer), 3 y += S x (prolongation), 4 E~^T r
   of the outer residual, 5 dense coarsest solve), its multigrid level, its CTA group (0 surface,
   1 A_bar; a single chain has group 0 only) and the SM clock cycles from the end of the previous
   phase's barrier to the end of its own, seen by the group's first CTA (the phase's critical
   path). Without a persistent program, the same for the steps of the cluster tails
   (vemg_options.tail_cluster) since vemg_probe(h, VEMG_PROBE_TAIL), timed by the cluster's first
   CTA (group 0 the surface chain's tail, 1 the A_bar chain's). capacity: entries the caller's arrays hold; *count
   receives the number of phases (VEMG_EINVAL, with *count set, if capacity is smaller; 0 phases
   without a persistent program or cluster tail). Synchronises the device. */
int vemg_probe_phases(vemg_hierarchy *h, int capacity, int *count, int *op, int *level, int *group,
                      double *cycles);

#ifdef __cplusplus
}
#endif

#endif /* VEMG_H */
