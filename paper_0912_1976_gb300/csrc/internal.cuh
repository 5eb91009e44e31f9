// internal.cuh -- data structures and helpers shared by the translation units of libvemg.
#pragma once

#include <cuda_runtime.h>
#include <utility>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/vemg.h"

namespace vemg {

constexpr int kMaxLevels = 16;

// ------------------------------------------------------------------------------------------
// errors

struct Error {
    int code;
};

#define VEMG_CHECK_CUDA(call)                                                         \
    do {                                                                             \
        cudaError_t e_ = (call);                                                     \
        if (e_ != cudaSuccess) {                                                     \
            ::vemg::set_last_cuda_error(e_, #call, __FILE__, __LINE__);              \
            throw ::vemg::Error{VEMG_ECUDA};                                         \
        }                                                                            \
    } while (0)

#define VEMG_CHECK_LAUNCH() VEMG_CHECK_CUDA(cudaGetLastError())

void set_last_cuda_error(cudaError_t e, const char *what, const char *file, int line);
const char *last_cuda_error();
void set_last_error_message(const char *msg);   // a library-side reason behind a status code

inline int grid_for(int64_t n, int block) { return (int)((n + block - 1) / block); }

// a * b + c rounded once. The solve kernels that must give the same bits for the same row (the
// per-phase kernels and the cluster tail) spell out every multiply-add with these, so that no
// difference in the compiler's contraction choices can separate them.
__device__ __forceinline__ float fmadd(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmadd(double a, double b, double c) { return __fma_rn(a, b, c); }

// ------------------------------------------------------------------------------------------
// programmatic dependent launch: a kernel launched with pdl_launch may start while the kernel
// before it on the stream finishes; pdl_begin() at its top waits until that kernel has completed
// and its memory is visible, then lets the next kernel start its own launch. Without the launch
// attribute both instructions do nothing.

__device__ __forceinline__ void pdl_begin() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline void pdl_launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t s, Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    VEMG_CHECK_CUDA(cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...));
}

// ------------------------------------------------------------------------------------------
// device memory

void *dev_alloc_raw(size_t bytes);
void dev_free_raw(void *p);

// An owner of device allocations; freed together.
struct Arena {
    std::vector<void *> ptrs;
    size_t bytes = 0;
    template <class T>
    T *alloc(int64_t count) {
        size_t b = (size_t)(count > 0 ? count : 1) * sizeof(T);
        b = (b + 255) & ~(size_t)255;
        void *p = dev_alloc_raw(b);
        ptrs.push_back(p);
        bytes += b;
        return (T *)p;
    }
    void release() {
        for (void *p : ptrs) dev_free_raw(p);
        ptrs.clear();
        bytes = 0;
    }
};

// While one of these lives on a thread (and no caller allocator is installed), that thread's
// Scratch buffers come from the device's memory pool in the order of stream s: releasing one does
// not wait for the whole device, so a setup does not stall behind other streams' work.
struct ScratchStream {
    bool prev_on;
    cudaStream_t prev_s;
    explicit ScratchStream(cudaStream_t s);
    ~ScratchStream();
    ScratchStream(const ScratchStream &) = delete;
    ScratchStream &operator=(const ScratchStream &) = delete;
};
// *ordered: whether the block is stream-ordered (then released on *s)
void *scratch_alloc(size_t bytes, bool *ordered, cudaStream_t *s);
void scratch_free(void *p, bool ordered, cudaStream_t s);

// Temporary device buffer freed at scope exit.
template <class T>
struct Scratch {
    T *p = nullptr;
    bool ordered = false;
    cudaStream_t s = nullptr;
    explicit Scratch(int64_t count) {
        size_t b = (size_t)(count > 0 ? count : 1) * sizeof(T);
        p = (T *)scratch_alloc(b, &ordered, &s);
    }
    ~Scratch() { scratch_free(p, ordered, s); }
    Scratch(const Scratch &) = delete;
    Scratch &operator=(const Scratch &) = delete;
    operator T *() const { return p; }
};

// ------------------------------------------------------------------------------------------
// sparse matrices on the device

struct DCsr {
    int n = 0, m = 0;   // rows, cols
    int nnz = 0;
    int *rp = nullptr, *ci = nullptr;
    double *v = nullptr;
};

// FP32 copy of a level's values (mixed precision)
struct DCsrF {
    float *v = nullptr;
};

struct Level {
    DCsr A;              // level operator, natural ordering of the level
    DCsr P, PT;          // transfer to level + 1 (absent on the coarsest)
    int *agg = nullptr;  // aggregate of each row (absent on the coarsest)
    int ncolours = 0;
    int *colour = nullptr;
    std::vector<int> cptr;  // host: ncolours + 1 offsets into crow
    std::vector<int64_t> cnnz;  // host: matrix entries in the rows of each colour
    int *crow = nullptr;    // rows grouped by colour, ascending within a colour
    double *diag = nullptr;
    double *x = nullptr, *b = nullptr, *r = nullptr;
    // FP32 mirrors for the mixed-precision cycle
    float *Af = nullptr, *Pf = nullptr, *PTf = nullptr, *diagf = nullptr;
    float *xf = nullptr, *bf = nullptr, *rf = nullptr;
    // chains with the near-nullspace {1, x, y}: its rows (n x 3) and, below level 0, the node
    // blocks (the coarse unknowns of one aggregate, consecutive rows bptr[J] .. bptr[J + 1])
    double *B = nullptr;
    int *blk = nullptr, *bptr = nullptr;
    int nblk = 0;
};

// Opt-in timing of one kernel class: CUDA events recorded on the launching stream around each
// launch, plus the algorithmic bytes of each launch (bytes the operation must move at minimum).
enum ProbeKind {
    PROBE_NONE = 0, PROBE_SPMV_A = 1, PROBE_SOR = 2, PROBE_RESIDUAL = 3, PROBE_SOR_FINE = 4, PROBE_VCYCLE = 5,
    PROBE_TRANSFER = 6, PROBE_VECTOR = 7, PROBE_DENSE = 8, PROBE_TAIL = 9
};

struct Probe {
    int kind = PROBE_NONE;
    std::vector<cudaEvent_t> ev;   // pairs
    std::vector<double> bytes;     // per recorded launch
    int used = 0;                  // launches recorded
    double total_ms = 0.0, total_bytes = 0.0;
    int64_t launches = 0;
};

// Sliced ELL with slices of 32 rows (one warp, one thread per row). Entry k of the row in lane
// l of slice s is at off[s] + 32 k + l; unused entries hold value 0 and a column inside the
// matrix. Slices never straddle the row groups given at construction (colours).
struct Sell {
    int n = 0, m = 0;         // rows, columns
    int nslices = 0;
    int *row0 = nullptr;      // first row of each slice
    int *nrow = nullptr;      // rows in each slice (<= 32)
    int *off = nullptr;       // element offset of each slice
    int *width = nullptr;     // stored entries per row of each slice
    int *col = nullptr;
    void *v = nullptr;        // double or float values
    bool fp32 = false;
    int64_t nnz = 0;          // stored (unpadded) entries
    int64_t padded = 0;       // stored entries including padding
    void *vh = nullptr;       // BF16 copy of the FP32 values (BF16 precision), else null
};

// One multigrid level in solve order: rows grouped by colour (colour-major, ascending natural
// index within a colour). Vectors of the level live in this order.
struct SLevel {
    int n = 0, ncolours = 0;
    Sell A;                        // off-diagonal entries (SOR sweeps, residual)
    void *diag = nullptr, *dinv = nullptr;
    std::vector<int> cslice;       // host: slice range of each colour (ncolours + 1)
    std::vector<int> crow;         // host: row range of each colour (ncolours + 1)
    std::vector<int64_t> cnnz;     // host: stored off-diagonal entries of each colour
    Sell P, PT;                    // prolongation (fine rows) and restriction (coarse rows)
    void *x = nullptr, *b = nullptr, *r = nullptr;
};

struct SChain {
    int nlev = 0;
    SLevel lv[kMaxLevels];
    bool direct = false, singular = false, fp32 = false, is_bar = false;
    int nc = 0;
    double *G = nullptr;           // coarsest dense inverse in solve order
    float *Gf = nullptr;           // its FP32 copy (FP32 cycles)
    // the coarse tail (levels tail_level.. as one single-CTA kernel, persist.cu); -1: none
    int tail_level = -1, tail_n = 0;
    const void *tail = nullptr;
    void *ctail = nullptr;         // the tail as one thread-block cluster (persist.cu), host object
    double tail_bytes = 0.0;       // algorithmic bytes of one tail launch
};

struct Chain {
    int nlev = 0;
    Level lv[kMaxLevels];
    bool singular = false;  // constants are the nullspace (Neumann surface chain)
    bool direct = false;    // coarsest level solved by the dense inverse
    int nc = 0;
    double *G = nullptr;    // nc x nc: inverse of the coarsest operator (projected on singular chains)
    bool is_bar = false;    // the A_bar chain (its level 0 is the finest smoother level)
    int nsd = 1;            // near-nullspace vectors: 1 (constants) or 3 ({1, x, y})
    double *nu = nullptr;   // nsd > 1, singular: the coarsest level's nullspace (the coarse constant)
};

struct Graphs;
struct BatchWork;
struct Persist;

}  // namespace vemg

struct vemg_hierarchy {
    vemg::Arena arena;
    int n = 0, mtop = 0, bc = VEMG_NEUMANN, precision = VEMG_PREC_FP64;
    vemg_options opts{};
    int *new2old = nullptr, *old2new = nullptr;  // device
    vemg::DCsr A;                                // internal order (Neumann operator)
    int *tri_of = nullptr;                       // located top triangle per internal node
    double *bary = nullptr;
    vemg::DCsr E, ET, Ac;
    vemg::Chain surf, bar;
    vemg::Chain one;                             // the single chain of VL_SOR / SA
    int precond = VEMG_PRECOND_ADDITIVE;
    // Krylov work vectors (internal order, length n)
    double *x = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr, *b = nullptr;
    double *host_b = nullptr, *host_x = nullptr;  // device copies of vemg_solve_host's buffers (caller order)
    float *rf = nullptr, *zf = nullptr;           // mixed precision preconditioner input / output
    double *red = nullptr;                        // reduction partials
    double *scal = nullptr;                       // device scalars
    int nred = 0;
    // batched solve work (allocated on first use)
    int batch_cap = 0;
    double *bx = nullptr, *br = nullptr, *bz = nullptr, *bp = nullptr, *bq = nullptr, *bb = nullptr;
    double *bscal = nullptr;
    vemg::Probe probe;
    int64_t launches = 0;                         // kernels launched by the solve path
    // ---- solve order (see layout.cu) ----
    int nu = 0;                                   // unknowns: n (Neumann) or n - mtop
    int *caller_of = nullptr;                     // caller id of each solve-order unknown
    int *tops = nullptr;                          // caller ids of the top nodes
    vemg::Sell Aop;                               // outer operator, FP64, diagonal included
    vemg::Sell Enon;                              // E~ rows of non-top nodes (Neumann)
    float *Enon_vf = nullptr;                     // FP32 copy of its values (FP32 V-cycles)
    vemg::Sell ETs;                               // E~^T (surface rows)
    vemg::SChain ssurf, sbar;
    // CUDA graphs of the solve (built on the first solve)
    vemg::Graphs *graphs = nullptr;
    cudaStream_t side = nullptr;                  // second branch of the preconditioner
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_mid = nullptr, ev_coarse = nullptr;
    unsigned *ctr = nullptr;                      // arrival counters of the block reductions
    vemg::BatchWork *batch = nullptr;             // multi-right-hand-side work (batch.cu)
    vemg::Persist *persist = nullptr;             // the persistent preconditioner program (persist.cu)
    double *coef = nullptr;                       // CG coefficients of the last solve (alpha, beta)
};

namespace vemg {
static constexpr int kCoefCap = 8192;   // CG coefficients kept per solve: 4096 iterations
// the preconditioner is one V-cycle of one chain (Dirichlet-top, VL_SOR, SA) rather than the two
// branches of the additive form
inline bool single_chain(const vemg_hierarchy *h) {
    return h->bc == VEMG_DIRICHLET_TOP || h->precond != VEMG_PRECOND_ADDITIVE;
}
inline const Chain &the_chain(const vemg_hierarchy *h) { return h->bc == VEMG_DIRICHLET_TOP ? h->bar : h->one; }
// persist.cu
void build_persist(vemg_hierarchy *h, cudaStream_t s);
void release_persist(vemg_hierarchy *h);
void launch_persist(vemg_hierarchy *h, const double *r, cudaStream_t s);
bool persist_coarse_only(const vemg_hierarchy *h);   // the program holds levels >= 1 only (hybrid)
void persist_reset(vemg_hierarchy *h, cudaStream_t s);
double persist_bytes(const vemg_hierarchy *h);
const int *persist_err(const vemg_hierarchy *h);
int barrier_selftest(int claimed, int launched, cudaStream_t s);
int solve_scalar_iters();   // index of the iteration count among the solve's device scalars
void persist_profile_reset(vemg_hierarchy *h);
void build_tails(vemg_hierarchy *h, cudaStream_t s);
void launch_tail(const SChain &C, cudaStream_t s, bool profile = false);
void release_ctail(SChain &C);
void ctail_profile_reset(SChain &C);
int ctail_profile(const SChain &C, int group, std::vector<int> &op, std::vector<int> &level, std::vector<int> &grp,
                  std::vector<double> &cycles);
double ctail_bytes(const SChain &C);
int persist_profile(vemg_hierarchy *h, int cap, int *count, int *op, int *level, int *group, double *cycles);
// setup.cu
void assemble(const vemg_mesh *mesh, vemg_csr *A_out, cudaStream_t s);
void load_vector(const vemg_mesh *mesh, const double *f, double *b, cudaStream_t s);
void setup(vemg_hierarchy *h, const vemg_csr *A, const vemg_mesh *mesh, cudaStream_t s);
// layout.cu
void build_solve_layout(vemg_hierarchy *h, cudaStream_t s);
// solve.cu
void prepare_solve(vemg_hierarchy *h, cudaStream_t s);
void release_graphs(vemg_hierarchy *h);
// batch.cu
void release_batch(vemg_hierarchy *h);
int solve(vemg_hierarchy *h, const double *b, double *x, double rtol, int max_it, vemg_info *info,
          cudaStream_t s);
int solve_batch(vemg_hierarchy *h, int k, const double *B, int64_t ldb, double *X, int64_t ldx, double rtol,
                int max_it, vemg_info *infos, cudaStream_t s);
void spmv_op(vemg_hierarchy *h, const double *x, double *y, cudaStream_t s);
void precond(vemg_hierarchy *h, const double *r, double *z, cudaStream_t s);
void vcycle(vemg_hierarchy *h, int chain, const double *b, double *x, cudaStream_t s);
void probe_start(vemg_hierarchy *h, int kind);
void probe_read(vemg_hierarchy *h, double *ms, int64_t *launches, double *bytes);
}  // namespace vemg
