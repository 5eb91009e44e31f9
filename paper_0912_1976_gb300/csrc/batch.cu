#include <vector>
// batch.cu -- many right-hand sides in one solve.
//
// K systems A x_c = b_c share one hierarchy. Vectors are interleaved (row-major n x K, K a power
// of two): x[i*K + c], in the natural (internal) ordering of each level. The operators are the
// setup's natural-order CSR matrices: a group of KW = min(K, 32) lanes works on one row, the lanes
// load KW consecutive entries of the row at once and pass them round by warp shuffles, so each
// matrix entry is read once for all columns and the gathers x[j*K + c] are KW consecutive words.
// Natural order keeps a row's neighbours close in memory, so the gathers stay in L2 even when the
// K-column vectors are far larger than L2 (the colour-major order of the one-column solve does
// not: each colour's pass would sweep the whole vector). Colour sweeps walk the level's list of
// rows of each colour. Each column keeps its own Krylov scalars
// (alpha, beta, norms, mean) and its own convergence test; a converged column is frozen (alpha = 0)
// until every column has converged. The iteration runs as CUDA graphs with a WHILE node, like the
// single right-hand-side solve (solve.cu); the V-cycles of the two branches run on two streams.
#include <math.h>

#include <algorithm>

#include <type_traits>

#include "internal.cuh"

namespace vemg {

static constexpr int kBT = 512;        // their threads
static constexpr int kBU = 8;          // entries loaded per round trip in a batched row
static constexpr int kMaxK = 128;      // widest batch
static constexpr int kSellWarps = 4;   // warps per block of the batched row kernels (untuned default)
static constexpr int kMaxWarps = 8;    // most warps per block the autotuner tries
// columns a lane of a batched row kernel takes per pass when the batch is wide enough (K >= that
// many times the lanes per row): 8 with FP32 accumulators, 4 with FP64 ones (8 FP64 accumulators
// spill). Narrower batches take one column per pass: unused accumulator slots cost registers and
// code size, which slowed the 8-column engines of the serving stream by about 2x.
template <class AT>
__host__ __device__ constexpr int cols_per_lane() { return sizeof(AT) == 4 ? 8 : 4; }

static thread_local int64_t *b_count = nullptr;
struct BTune;
static thread_local const BTune *b_tune = nullptr;   // launch shapes of the batch being recorded

struct TuneScope {
    const BTune *saved;
    explicit TuneScope(const BTune *t) : saved(b_tune) { b_tune = t; }
    ~TuneScope() { b_tune = saved; }
};
#define BATCH_LAUNCHED()         \
    do {                         \
        VEMG_CHECK_LAUNCH();     \
        if (b_count) ++*b_count; \
    } while (0)

// per-column scalar slots (sc[slot * K + c])
enum {
    B_RZ = 0, B_PQ, B_ALPHA, B_BETA, B_MU, B_BN, B_RN, B_FLAG, B_ITERS, B_CONV, B_ZERO, B_TRUE, B_BMEAN, B_XMEAN,
    B_TOL, B_MAXIT, B_FRESH, B_BEST, B_LASTIMP, B_STALL, B_COUNT
};

// a column whose best residual has not dropped by 1% in this many iterations has reached the
// round-off floor: it stops (status VEMG_ENOTCONV with its last residual)
static constexpr int kStallIters = 30;
// global scalars after the per-column block (g[slot])
enum { G_TOL = 0, G_MAXIT, G_CONT, G_ITERS, G_COUNT };

// one multigrid level as the batched cycle sees it
struct BLevel {
    int n = 0, ncolours = 0;
    const int *rp = nullptr, *ci = nullptr, *colour = nullptr, *crow = nullptr;
    const void *v = nullptr, *dinv = nullptr;
    std::vector<int> cptr;
    const int *prp = nullptr, *pci = nullptr, *trp = nullptr, *tci = nullptr;
    const void *pv = nullptr, *tv = nullptr;
};

struct BChain {
    int nlev = 0;
    BLevel lv[kMaxLevels];
    bool direct = false;
    int nc = 0;
    const double *G = nullptr;
    const float *Gf = nullptr;   // FP32 copy (FP32 cycles)
};

struct CsrP {
    const int *rp, *ci;
    const void *v;
};

struct BatchGraphs {
    cudaGraph_t g = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphConditionalHandle handle = 0;
    int64_t k_pre = 0, k_body = 0, k_post = 0;
};

// Launch shapes of the batched row kernels, by class: 0 = colour sweeps, 1 = the other V-cycle
// operations (residuals, restrictions, prolongations), 2 = the outer FP64 operations (A p, the
// true residual, E~ and E~^T). kw: lanes per row (each lane takes columns lane, lane + kw, ...),
// warps: warps per block. Chosen per batch width by timing the candidates (autotune below); the
// per-column arithmetic is the same for every shape.
struct BTune {
    int kw[3] = {0, 0, 0}, warps[3] = {0, 0, 0};   // 0: the untuned default
    float us[3] = {0.f, 0.f, 0.f};                  // the chosen shapes' measured launch times
    int tried = 0;                                   // candidate launches timed
};

struct BatchWork {
    BTune tune;
    int K = 0;
    double *X = nullptr, *R = nullptr, *Z = nullptr, *P = nullptr, *Q = nullptr, *B = nullptr;
    void *lx[2][kMaxLevels] = {}, *lb[2][kMaxLevels] = {}, *lr[2][kMaxLevels] = {};
    double *sc = nullptr;      // B_COUNT * K per-column scalars, then G_COUNT globals
    double *part = nullptr;    // reduction partials
    unsigned *ctr = nullptr;
    BatchGraphs *graphs = nullptr;
    Arena arena;
    BChain *bsurf = nullptr, *bbar = nullptr;
    CsrP Aout{};
    const int *caller_of = nullptr;   // caller id of each unknown (internal order)
    // FP32 V-cycles: E~'s values in FP32 (the prolongation z = E~ y_s is formed in FP32) and an
    // FP32 copy of the A_bar part of the outer residual (the finest level's right-hand side,
    // converted once per application instead of on every read)
    float *Ev32 = nullptr, *Rb32 = nullptr;
    ~BatchWork() {
        delete bsurf;
        delete bbar;
    }
};

static double *gsc(BatchWork *w) { return w->sc + B_COUNT * w->K; }

// ------------------------------------------------------------------------------------------
// batched CSR row operations (natural order)

// BOP_SPMV_PLUS: y = b_part + A x, where rows r >= cur start from b[(r - cur) K + c] (and the
// others from 0): z = [0; x_bar] + E~ y_s formed in the accumulator type, converted once
enum { BOP_SPMV = 0, BOP_SPMV_ADD = 1, BOP_SOR = 2, BOP_RES = 3, BOP_SPMV_PLUS = 4 };

__global__ void k_bto_float(int64_t n, const double *__restrict__ a, float *__restrict__ b) {
    pdl_begin();
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) b[i] = (float)a[i];
}

// Rows idx in [0, nrows): row = rows ? rows[idx] : r0 + idx, a group of KW lanes per row, columns
// c = lane % KW + j KW. SOR skips the diagonal entry and, when sweeping from x = 0 (cur >= 0), every
// entry whose column has colour >= cur (not yet visited: zero). RES keeps the diagonal: y = b - A x.
template <int OP, class VT, class XT, class BT, class YT, class AT, int KW, int CPL>
__global__ void __launch_bounds__(32 * kMaxWarps) k_bcsr(int nrows, const int *__restrict__ rows, int r0, CsrP A,
                                                         const VT *__restrict__ dg, const BT *__restrict__ b,
                                                         const XT *x, YT *y, int K, const int *__restrict__ colour,
                                                         int cur) {
    constexpr int RW = 32 / KW;
    int w = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (w * RW >= nrows) {   // warp-uniform
        pdl_begin();
        return;
    }
    int idx = w * RW + lane / KW;
    bool valid = idx < nrows;
    int r = valid ? (rows ? rows[idx] : r0 + idx) : 0;
    int lo = valid ? A.rp[r] : 0, wd = valid ? A.rp[r + 1] - lo : 0;
    const VT *v = (const VT *)A.v;
    const int gl = lane % KW, gb = lane - gl;
    const bool skip_all = OP == BOP_SOR && cur == 0;
    int wmax = __reduce_max_sync(0xffffffffu, (unsigned)wd);
    // the row's first KW entries are setup data: loaded before waiting on the previous kernel
    int cc0 = -1;
    VT vv0 = (VT)0;
    if (!skip_all) {
        cc0 = gl < wd ? __ldg(A.ci + lo + gl) : -1;
        vv0 = gl < wd ? __ldg(v + lo + gl) : (VT)0;
        if (OP == BOP_SOR && cc0 >= 0 && (cc0 == r || (cur > 0 && __ldg(colour + cc0) >= cur))) cc0 = -1;
    }
    pdl_begin();
    // a lane takes the columns c0, c0 + KW, ..., CPL of them per pass, so that each entry of the
    // row issues CPL independent loads of its neighbour's x row. K, KW and CPL are powers of two
    // and K is a multiple of CPL * KW (or CPL = 1), so every column c0 + u KW of a pass exists and
    // every lane of the warp makes the same number of passes (the shuffles need all 32).
    for (int c0 = gl; c0 < K; c0 += CPL * KW) {
        AT acc[CPL];
#pragma unroll
        for (int u = 0; u < CPL; ++u)
            acc[u] = (OP == BOP_SPMV_PLUS && valid && r >= cur) ? (AT)b[(int64_t)(r - cur) * K + c0 + u * KW] : (AT)0;
        if (!skip_all) {
            for (int k0 = 0; k0 < wmax; k0 += KW) {
                int k = k0 + gl;
                int cc = cc0;
                VT vv = vv0;
                if (k0 > 0) {
                    cc = k < wd ? __ldg(A.ci + lo + k) : -1;
                    vv = k < wd ? __ldg(v + lo + k) : (VT)0;
                    if (OP == BOP_SOR && cc >= 0 && (cc == r || (cur > 0 && __ldg(colour + cc) >= cur))) cc = -1;
                }
                int nj = min(KW, wmax - k0);
#pragma unroll
                for (int jj = 0; jj < KW; ++jj) {
                    if (jj < nj) {
                        int cj = __shfl_sync(0xffffffffu, cc, gb + jj);
                        VT vj = __shfl_sync(0xffffffffu, vv, gb + jj);
                        if (cj >= 0) {
                            const XT *xr = x + (int64_t)cj * K;
#pragma unroll
                            for (int u = 0; u < CPL; ++u) acc[u] += (AT)vj * (AT)xr[c0 + u * KW];
                        }
                    }
                }
            }
        }
        if (!valid) continue;
#pragma unroll
        for (int u = 0; u < CPL; ++u) {
            const int c = c0 + u * KW;
            int64_t e = (int64_t)r * K + c;
            if (OP == BOP_SPMV || OP == BOP_SPMV_PLUS) y[e] = (YT)acc[u];
            else if (OP == BOP_SPMV_ADD) y[e] = (YT)((AT)y[e] + acc[u]);
            else if (OP == BOP_SOR) y[e] = (YT)(((AT)b[e] - acc[u]) * (AT)dg[r]);
            else y[e] = (YT)((AT)b[e] - acc[u]);
        }
    }
}

// one lane per row and column group (K = 1, 2): entries loaded kBU at a time
template <int OP, class VT, class XT, class BT, class YT, class AT, int KW>
__global__ void __launch_bounds__(32 * kMaxWarps) k_bcsr_narrow(int nrows, const int *__restrict__ rows, int r0,
                                                                CsrP A, const VT *__restrict__ dg,
                                                                const BT *__restrict__ b, const XT *x, YT *y, int K,
                                                                const int *__restrict__ colour, int cur) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int idx = (int)(t / KW), c = (int)(t % KW);
    if (idx >= nrows) {
        pdl_begin();
        return;
    }
    int r = rows ? rows[idx] : r0 + idx;
    int lo = A.rp[r], hi = A.rp[r + 1];
    const VT *v = (const VT *)A.v;
    pdl_begin();
    AT acc = (OP == BOP_SPMV_PLUS && r >= cur) ? (AT)b[(int64_t)(r - cur) * K + c] : (AT)0;
    if (!(OP == BOP_SOR && cur == 0)) {
        for (int k0 = lo; k0 < hi; k0 += kBU) {
            int cc[kBU];
            VT a[kBU];
#pragma unroll
            for (int u = 0; u < kBU; ++u) {
                int k = k0 + u;
                cc[u] = k < hi ? __ldg(A.ci + k) : -1;
                a[u] = k < hi ? __ldg(v + k) : (VT)0;
                if (OP == BOP_SOR && cc[u] >= 0 && (cc[u] == r || (cur > 0 && __ldg(colour + cc[u]) >= cur))) cc[u] = -1;
            }
#pragma unroll
            for (int u = 0; u < kBU; ++u)
                if (cc[u] >= 0) acc += (AT)a[u] * (AT)x[(int64_t)cc[u] * K + c];
        }
    }
    int64_t e = (int64_t)r * K + c;
    if (OP == BOP_SPMV || OP == BOP_SPMV_PLUS) y[e] = (YT)acc;
    else if (OP == BOP_SPMV_ADD) y[e] = (YT)((AT)y[e] + acc);
    else if (OP == BOP_SOR) y[e] = (YT)(((AT)b[e] - acc) * (AT)dg[r]);
    else y[e] = (YT)((AT)b[e] - acc);
}

// cls: the launch-shape class of the call (BTune); kw, nw > 0 force a shape (autotuning)
template <int OP, class VT, class XT, class BT, class YT, class AT>
static void bcsr(CsrP A, int nrows, const int *rows, int r0, const VT *dg, const BT *b, const XT *x, YT *y, int K,
                 const int *colour, int cur, cudaStream_t s, int cls = 1, int kw = 0, int nw = 0) {
    if (nrows <= 0) return;
    if (kw <= 0 && b_tune && b_tune->kw[cls] > 0) {
        kw = b_tune->kw[cls];
        nw = b_tune->warps[cls];
    }
    int KW = std::min(K, kw > 0 ? kw : 32);
    const int wpb = nw > 0 ? nw : kSellWarps;
    dim3 blk(32 * wpb);
    if (KW < 4) {
        int64_t t = (int64_t)nrows * KW;
        if (KW == 1)
            pdl_launch(k_bcsr_narrow<OP, VT, XT, BT, YT, AT, 1>, grid_for(t, 32 * wpb), blk, s, nrows, rows, r0, A, dg, b, x, y, K, colour, cur);
        else
            pdl_launch(k_bcsr_narrow<OP, VT, XT, BT, YT, AT, 2>, grid_for(t, 32 * wpb), blk, s, nrows, rows, r0, A, dg, b, x, y, K, colour, cur);
        BATCH_LAUNCHED();
        return;
    }
    int RW = 32 / KW;
    int64_t warps = (nrows + RW - 1) / RW;
    int grid = (int)((warps + wpb - 1) / wpb);
    constexpr int C = cols_per_lane<AT>();
    const bool wide = K >= C * KW;   // then K is a multiple of C * KW (both powers of two)
    switch (KW) {
        case 4:
            if (wide) pdl_launch(k_bcsr<OP, VT, XT, BT, YT, AT, 4, C>, grid, blk, s, nrows, rows, r0, A, dg, b, x, y, K, colour, cur);
            else pdl_launch(k_bcsr<OP, VT, XT, BT, YT, AT, 4, 1>, grid, blk, s, nrows, rows, r0, A, dg, b, x, y, K, colour, cur);
            break;
        case 8:
            if (wide) pdl_launch(k_bcsr<OP, VT, XT, BT, YT, AT, 8, C>, grid, blk, s, nrows, rows, r0, A, dg, b, x, y, K, colour, cur);
            else pdl_launch(k_bcsr<OP, VT, XT, BT, YT, AT, 8, 1>, grid, blk, s, nrows, rows, r0, A, dg, b, x, y, K, colour, cur);
            break;
        case 16:
            if (wide) pdl_launch(k_bcsr<OP, VT, XT, BT, YT, AT, 16, C>, grid, blk, s, nrows, rows, r0, A, dg, b, x, y, K, colour, cur);
            else pdl_launch(k_bcsr<OP, VT, XT, BT, YT, AT, 16, 1>, grid, blk, s, nrows, rows, r0, A, dg, b, x, y, K, colour, cur);
            break;
        default:
            if (wide) pdl_launch(k_bcsr<OP, VT, XT, BT, YT, AT, 32, C>, grid, blk, s, nrows, rows, r0, A, dg, b, x, y, K, colour, cur);
            else pdl_launch(k_bcsr<OP, VT, XT, BT, YT, AT, 32, 1>, grid, blk, s, nrows, rows, r0, A, dg, b, x, y, K, colour, cur);
            break;
    }
    BATCH_LAUNCHED();
}

// x = G b on the coarsest level, one thread per (row, column)
template <class XT, class BT>
__global__ void k_bdense(int n, const XT *__restrict__ G, const BT *__restrict__ b, XT *__restrict__ x, int K) {
    pdl_begin();
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)n * K) return;
    int r = (int)(t >> (__ffs(K) - 1)), c = (int)(t & (K - 1));
    XT s = 0;
    for (int j = 0; j < n; ++j) s += G[(int64_t)r * n + j] * (XT)b[(int64_t)j * K + c];
    x[t] = (XT)s;
}

template <class XT, class BT>
static void bsweep(const BLevel &L, const BT *b, XT *x, bool forward, bool from_zero, int K, cudaStream_t s) {
    CsrP A{L.rp, L.ci, L.v};
    for (int cc = 0; cc < L.ncolours; ++cc) {
        int c = forward ? cc : L.ncolours - 1 - cc;
        int nrows = L.cptr[c + 1] - L.cptr[c];
        bcsr<BOP_SOR, XT, XT, BT, XT, XT>(A, nrows, L.crow + L.cptr[c], 0, (const XT *)L.dinv, b, x, x, K, L.colour,
                                         from_zero ? c : -1, s, 0);
    }
}

template <class XT, class BT>
static void bvcycle(const BChain &C, BatchWork *W, int ch, int l, const BT *b, XT *x, cudaStream_t s) {
    const BLevel &L = C.lv[l];
    const int K = W->K;
    if (l == C.nlev - 1) {
        if (C.direct) {
            int64_t t = (int64_t)C.nc * K;
            const XT *G = sizeof(XT) == sizeof(float) ? (const XT *)C.Gf : (const XT *)C.G;
            pdl_launch(k_bdense<XT, BT>, grid_for(t, 256), 256, s, C.nc, G, b, x, K);
            BATCH_LAUNCHED();
            return;
        }
        bsweep<XT, BT>(L, b, x, true, true, K, s);
        bsweep<XT, BT>(L, b, x, false, false, K, s);
        return;
    }
    XT *r = (XT *)W->lr[ch][l];
    XT *nb = (XT *)W->lb[ch][l + 1], *nx = (XT *)W->lx[ch][l + 1];
    const BLevel &N = C.lv[l + 1];
    bsweep<XT, BT>(L, b, x, true, true, K, s);
    bcsr<BOP_RES, XT, XT, BT, XT, XT>(CsrP{L.rp, L.ci, L.v}, L.n, nullptr, 0, (const XT *)nullptr, b, x, r, K,
                                      nullptr, -1, s);
    bcsr<BOP_SPMV, XT, XT, XT, XT, XT>(CsrP{L.trp, L.tci, L.tv}, N.n, nullptr, 0, (const XT *)nullptr,
                                       (const XT *)nullptr, r, nb, K, nullptr, -1, s);
    bvcycle<XT, XT>(C, W, ch, l + 1, (const XT *)nb, nx, s);
    bcsr<BOP_SPMV_ADD, XT, XT, XT, XT, XT>(CsrP{L.prp, L.pci, L.pv}, L.n, nullptr, 0, (const XT *)nullptr,
                                           (const XT *)nullptr, nx, x, K, nullptr, -1, s);
    bsweep<XT, BT>(L, b, x, false, false, K, s);
}

// ------------------------------------------------------------------------------------------
// per-column deterministic reductions in two stages. Stage 1 (streaming kernels): each block
// covers kBT * kBE consecutive elements of the n x K block; thread t always holds column
// t % K (K divides kBT), loads its kBE elements first, and the block writes one partial per
// column and sum. Stage 2 (k_bstage2): one block per column adds the block partials in fixed
// order and applies the scalar step of that column; the last column block sets the globals.

static constexpr int kBE = 8;   // elements per thread in stage 1

static int stage1_blocks(int64_t N) { return (int)((N + (int64_t)kBT * kBE - 1) / ((int64_t)kBT * kBE)); }

template <int NS>
__device__ void bblock_partials(double (&acc)[NS], int K, double *part) {
    __shared__ double sh[kBT];
    const int t = threadIdx.x;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        sh[t] = acc[s];
        __syncthreads();
        if (t < K) {
            double v = 0.0;
            for (int j = t; j < kBT; j += K) v += sh[j];
            part[((int64_t)blockIdx.x * NS + s) * K + t] = v;
        }
        __syncthreads();
    }
}

// stage-1 sums: s0 = sum a*b (or sum a when b is null), s1 = sum c*d (or sum c), ...
struct BSums {
    const double *a[5];
    const double *b[5];
    int ns;
};

template <int NS>
__global__ void __launch_bounds__(kBT) k_bsums(int64_t N, int K, BSums d, double *part) {
    pdl_begin();
    double acc[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) acc[s] = 0.0;
    int64_t base = (int64_t)blockIdx.x * kBT * kBE + threadIdx.x;
    double va[NS][kBE], vb[NS][kBE];
#pragma unroll
    for (int j = 0; j < kBE; ++j) {
        int64_t e = base + (int64_t)j * kBT;
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            va[s][j] = e < N ? d.a[s][e] : 0.0;
            vb[s][j] = (e < N && d.b[s]) ? d.b[s][e] : 1.0;
        }
    }
#pragma unroll
    for (int j = 0; j < kBE; ++j)
#pragma unroll
        for (int s = 0; s < NS; ++s) acc[s] = fma(va[s][j], vb[s][j], acc[s]);
    bblock_partials<NS>(acc, K, part);
}

// the preconditioner's sums over z, r (and q): s0 = sum z, s1 = sum r z, s2 = sum r
// [, s3 = sum z q, s4 = sum q]; each vector is loaded once per element (the generic kernel
// above would load z three times and hold 80 values per thread). Same order of accumulation.
template <int NS>
__global__ void __launch_bounds__(kBT, 2) k_bsums_zrq(int64_t N, int K, const double *__restrict__ z,
                                                      const double *__restrict__ r, const double *__restrict__ q,
                                                      double *part) {
    pdl_begin();
    double acc[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) acc[s] = 0.0;
    int64_t base = (int64_t)blockIdx.x * kBT * kBE + threadIdx.x;
    double vz[kBE], vr[kBE], vq[kBE];
#pragma unroll
    for (int j = 0; j < kBE; ++j) {
        int64_t e = base + (int64_t)j * kBT;
        vz[j] = e < N ? z[e] : 0.0;
        vr[j] = e < N ? r[e] : 0.0;
        vq[j] = (NS == 5 && e < N) ? q[e] : 0.0;
    }
#pragma unroll
    for (int j = 0; j < kBE; ++j) {
        acc[0] += vz[j] * 1.0;
        acc[1] += vr[j] * vz[j];
        acc[2] += vr[j] * 1.0;
        if (NS == 5) {
            acc[3] += vz[j] * vq[j];
            acc[4] += vq[j] * 1.0;
        }
    }
    bblock_partials<NS>(acc, K, part);
}

enum { ST_MEAN_B = 0, ST_BN, ST_ALPHA, ST_RN, ST_BETA, ST_MEAN_X, ST_TRUE };

// stage 2: one block per column
__global__ void __launch_bounds__(256) k_bstage2(int op, int nblk, int ns, int K, const double *__restrict__ part,
                                                double *sc, double inv_n, int neumann, int flexible, int first,
                                                unsigned *ctr, int *active, cudaGraphConditionalHandle handle,
                                                int use_cond) {
    __shared__ double red[256 / 32];
    __shared__ double tot[5];
    const int c = blockIdx.x, t = threadIdx.x;
    for (int s = 0; s < ns; ++s) {
        double v = 0.0;
        for (int k = t; k < nblk; k += 256) v += part[((int64_t)k * ns + s) * K + c];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((t & 31) == 0) red[t >> 5] = v;
        __syncthreads();
        if (t == 0) {
            double w = 0.0;
            for (int i = 0; i < 256 / 32; ++i) w += red[i];
            tot[s] = w;
        }
        __syncthreads();
    }
    double *g = sc + B_COUNT * K;
    if (t == 0) {
        // converged, broken down, or out of iterations: frozen while other columns continue
        bool frozen = sc[B_CONV * K + c] != 0.0 || sc[B_FLAG * K + c] != 0.0 ||
                      sc[B_ITERS * K + c] >= sc[B_MAXIT * K + c] || sc[B_STALL * K + c] != 0.0;
        switch (op) {
            case ST_MEAN_B: sc[B_BMEAN * K + c] = tot[0] * inv_n; break;
            case ST_MEAN_X: sc[B_XMEAN * K + c] = tot[0] * inv_n; break;
            case ST_TRUE: sc[B_TRUE * K + c] = sqrt(tot[0]); break;
            case ST_BN: {
                double bn = sqrt(tot[0]);
                sc[B_BN * K + c] = bn;
                if (bn == 0.0) {
                    sc[B_ZERO * K + c] = 1.0;
                    sc[B_CONV * K + c] = 1.0;
                } else if (sc[B_MAXIT * K + c] > 0.0) {
                    atomicOr(active, 1);
                }
                __threadfence();
                if (atomicAdd(ctr, 1u) == (unsigned)(K - 1)) {
                    g[G_CONT] = atomicAdd(active, 0) ? 1.0 : 0.0;
                    *active = 0;
                    *ctr = 0u;
                }
                break;
            }
            case ST_ALPHA: {
                double pq = tot[0];
                sc[B_PQ * K + c] = pq;
                if (frozen) sc[B_ALPHA * K + c] = 0.0;
                else if (!(pq > 0.0)) {
                    sc[B_FLAG * K + c] = 1.0;
                    sc[B_ALPHA * K + c] = 0.0;
                } else sc[B_ALPHA * K + c] = sc[B_RZ * K + c] / pq;
                break;
            }
            case ST_RN: {
                double rn = sqrt(tot[0]);
                if (!frozen) {
                    sc[B_RN * K + c] = rn;
                    sc[B_ITERS * K + c] += 1.0;
                    if (!(rn == rn)) sc[B_FLAG * K + c] = 1.0;
                    else if (rn <= sc[B_TOL * K + c] * sc[B_BN * K + c]) sc[B_CONV * K + c] = 1.0;
                    double best = sc[B_BEST * K + c];
                    if (best == 0.0 || rn < 0.99 * best) {
                        sc[B_BEST * K + c] = rn;
                        sc[B_LASTIMP * K + c] = sc[B_ITERS * K + c];
                    } else if (sc[B_ITERS * K + c] - sc[B_LASTIMP * K + c] >= kStallIters) {
                        sc[B_STALL * K + c] = 1.0;
                    }
                    if (sc[B_CONV * K + c] == 0.0 && sc[B_FLAG * K + c] == 0.0 && sc[B_STALL * K + c] == 0.0 &&
                        sc[B_ITERS * K + c] < sc[B_MAXIT * K + c])
                        atomicOr(active, 1);
                }
                __threadfence();
                if (atomicAdd(ctr, 1u) == (unsigned)(K - 1)) {
                    // last column: every other column's flag is visible
                    int act = atomicAdd(active, 0);
                    g[G_ITERS] += 1.0;
                    g[G_CONT] = act ? 1.0 : 0.0;
                    if (use_cond) cudaGraphSetConditional(handle, act ? 1u : 0u);
                    *active = 0;
                    *ctr = 0u;
                }
                break;
            }
            case ST_BETA: {
                double mu = neumann ? tot[0] * inv_n : 0.0;
                double rz = tot[1] - mu * tot[2];
                double beta = 0.0;
                const bool fresh = sc[B_FRESH * K + c] != 0.0;
                sc[B_FRESH * K + c] = 0.0;
                if (!fresh && !frozen) {
                    if (flexible) beta = -(tot[3] - mu * tot[4]) / sc[B_PQ * K + c];
                    else beta = rz / sc[B_RZ * K + c];
                    if (!(rz == rz) || !(beta == beta)) sc[B_FLAG * K + c] = 1.0;
                }
                sc[B_MU * K + c] = mu;
                sc[B_BETA * K + c] = frozen ? 0.0 : beta;
                sc[B_RZ * K + c] = rz;
                break;
            }
        }
    }
}

// b -= mean (Neumann), r = b, x = p = 0 (streaming, no reduction)
// rb32 (FP32 V-cycles on two chains): the FP32 copy of r's A_bar part (elements from off32 on),
// the finest A_bar level's right-hand side; every kernel that writes r writes it too
__global__ void k_bprepare(int64_t N, int K, int neumann, double *__restrict__ b, double *__restrict__ r,
                           double *__restrict__ x, double *__restrict__ p, const double *__restrict__ sc,
                           float *__restrict__ rb32, int64_t off32) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= N) return;
    double bi = b[e] - (neumann ? sc[B_BMEAN * K + (int)(e & (K - 1))] : 0.0);
    b[e] = bi;
    r[e] = bi;
    if (rb32 && e >= off32) rb32[e - off32] = (float)bi;
    x[e] = 0.0;
    p[e] = 0.0;
}

// X += alpha P, R -= alpha Q per column, the FP32 copy of R's A_bar part, and the stage-1 sums
// of R * R: the elements of a thread and the order of its sum are those of k_bsums, so the
// partials are the same bits as a separate pass would give
__global__ void __launch_bounds__(kBT) k_bupdate_xr(int64_t N, int K, const double *__restrict__ p,
                                                    const double *__restrict__ q, double *__restrict__ x,
                                                    double *__restrict__ r, const double *__restrict__ sc,
                                                    float *__restrict__ rb32, int64_t off32, double *part) {
    pdl_begin();
    double acc[1] = {0.0};
    const int64_t base = (int64_t)blockIdx.x * kBT * kBE + threadIdx.x;
    const double a = sc[B_ALPHA * K + (int)(base & (K - 1))];   // kBT is a multiple of K: one column
#pragma unroll
    for (int j = 0; j < kBE; ++j) {
        const int64_t e = base + (int64_t)j * kBT;
        double rn = 0.0;
        if (e < N) {
            x[e] = fma(a, p[e], x[e]);
            rn = fma(-a, q[e], r[e]);
            r[e] = rn;
            if (rb32 && e >= off32) rb32[e - off32] = (float)rn;
        }
        acc[0] = fma(rn, rn, acc[0]);
    }
    bblock_partials<1>(acc, K, part);
}

// z += x (assign: z = x)
template <class XT>
__global__ void k_badd(int64_t N, const XT *__restrict__ x, double *__restrict__ z, int assign = 0) {
    pdl_begin();
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= N) return;
    z[e] = assign ? (double)x[e] : z[e] + (double)x[e];
}

// P = (Z - mu) + beta P per column
__global__ void k_bupdate_p(int64_t N, int K, const double *__restrict__ sc, const double *__restrict__ z,
                            double *__restrict__ p) {
    pdl_begin();
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= N) return;
    int c = (int)(e & (K - 1));
    p[e] = (z[e] - sc[B_MU * K + c]) + sc[B_BETA * K + c] * p[e];
}

__global__ void k_bsub_mean(int64_t N, int K, double *__restrict__ x, const double *__restrict__ sc, int slot) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < N) x[e] -= sc[slot * K + (int)(e & (K - 1))];
}


__global__ void k_binit(double *sc, int K, double tol, int maxit) {
    for (int i = 0; i < B_COUNT * K + G_COUNT; ++i) sc[i] = 0.0;
    for (int c = 0; c < K; ++c) {
        sc[B_TOL * K + c] = tol;
        sc[B_MAXIT * K + c] = (double)maxit;
        sc[B_FRESH * K + c] = 1.0;
    }
    double *g = sc + B_COUNT * K;
    g[G_TOL] = tol;
    g[G_MAXIT] = (double)maxit;
}

// gather k caller-order columns (column c at B[c * ldb]) into the interleaved solve-order block
__global__ void k_bgather(int nu, int K, int k, int64_t ldb, const int *__restrict__ caller_of,
                          const double *__restrict__ Bin, double *__restrict__ Bk) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)nu * K) return;
    int i = (int)(t >> (__ffs(K) - 1)), c = (int)(t & (K - 1));
    Bk[t] = c < k ? Bin[(int64_t)c * ldb + caller_of[i]] : 0.0;
}

__global__ void k_bscatter(int nu, int K, int k, int64_t ldx, const int *__restrict__ caller_of,
                           const int *__restrict__ tops, int ntop, const double *__restrict__ Xk,
                           double *__restrict__ Xout) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t nmax = (int64_t)(nu > ntop ? nu : ntop) * k;
    if (t >= nmax) return;
    int i = (int)(t / k), c = (int)(t % k);
    if (i < nu) Xout[(int64_t)c * ldx + caller_of[i]] = Xk[(int64_t)i * K + c];
    if (i < ntop) Xout[(int64_t)c * ldx + tops[i]] = 0.0;
}

__global__ void k_bcond_init(const double *g, cudaGraphConditionalHandle handle) {
    cudaGraphSetConditional(handle, g[G_CONT] != 0.0 ? 1u : 0u);
}

// ------------------------------------------------------------------------------------------
// the batched iteration

template <class XT>
static void bprecond(vemg_hierarchy *h, BatchWork *W, cudaStream_t s) {
    const int K = W->K;
    const bool two = !single_chain(h);
    const int mt = two ? h->mtop : 0;
    XT *xb = (XT *)W->lx[1][0];
    if (two) {
        XT *b0 = (XT *)W->lb[0][0], *x0 = (XT *)W->lx[0][0];
        VEMG_CHECK_CUDA(cudaEventRecord(h->ev_fork, s));
        VEMG_CHECK_CUDA(cudaStreamWaitEvent(h->side, h->ev_fork, 0));
        // surface branch: r_c = E~^T r in FP64, one V-cycle on E~^T A E~
        bcsr<BOP_SPMV, double, double, double, XT, double>(CsrP{h->ET.rp, h->ET.ci, h->ET.v}, h->mtop, nullptr, 0,
                                                           (const double *)nullptr, (const double *)nullptr, W->R,
                                                           b0, K, nullptr, -1, h->side, 2);
        bvcycle<XT, XT>(*W->bsurf, W, 0, 0, (const XT *)b0, x0, h->side);
        VEMG_CHECK_CUDA(cudaEventRecord(h->ev_join, h->side));
        const int64_t nbk = (int64_t)(h->n - mt) * K;
        if (std::is_same<XT, float>::value && W->Rb32) {   // kept current by every writer of r
            bvcycle<XT, XT>(*W->bbar, W, 1, 0, (const XT *)W->Rb32, xb, s);
        } else {
            bvcycle<XT, double>(*W->bbar, W, 1, 0, W->R + (int64_t)mt * K, xb, s);
        }
        VEMG_CHECK_CUDA(cudaStreamWaitEvent(s, h->ev_join, 0));
        // z = E~ y_s + [0; x_bar]: with FP32 V-cycles formed in FP32 from x_bar on and converted
        // once into the FP64 z; with FP64 ones in FP64
        if (std::is_same<XT, float>::value && W->Ev32) {
            bcsr<BOP_SPMV_PLUS, float, XT, XT, double, float>(CsrP{h->E.rp, h->E.ci, W->Ev32}, h->n, nullptr, 0,
                                                             (const float *)nullptr, (const XT *)xb, x0, W->Z, K,
                                                             nullptr, mt, s, 2);
        } else {
            bcsr<BOP_SPMV, double, XT, double, double, double>(CsrP{h->E.rp, h->E.ci, h->E.v}, h->n, nullptr, 0,
                                                               (const double *)nullptr, (const double *)nullptr, x0,
                                                               W->Z, K, nullptr, -1, s, 2);
            pdl_launch(k_badd<XT>, grid_for(nbk, 256), 256, s, nbk, (const XT *)xb, W->Z + (int64_t)mt * K, 0);
            BATCH_LAUNCHED();
        }
    } else {
        bvcycle<XT, double>(*W->bbar, W, 1, 0, W->R, xb, s);
        int64_t N = (int64_t)h->nu * K;
        pdl_launch(k_badd<XT>, grid_for(N, 256), 256, s, N, (const XT *)xb, W->Z, 1);
        BATCH_LAUNCHED();
    }
}

// the first element of r's A_bar part (the FP32 copy covers it)
static int64_t rb32_offset(const vemg_hierarchy *h, const BatchWork *W) {
    return single_chain(h) ? 0 : (int64_t)h->mtop * W->K;
}

// one per-column sum (the wider sums of the preconditioner step are k_bsums_zrq's)
static void bsums(BatchWork *W, int64_t N, const BSums &d, cudaStream_t s) {
    if (d.ns != 1) throw Error{VEMG_EINTERNAL};
    pdl_launch(k_bsums<1>, stage1_blocks(N), kBT, s, N, W->K, d, W->part);
    BATCH_LAUNCHED();
}

static void bstage2(vemg_hierarchy *h, BatchWork *W, int op, int ns, int64_t N, int first, cudaStream_t s,
                    cudaGraphConditionalHandle hd = 0, int use_cond = 0) {
    k_bstage2<<<W->K, 256, 0, s>>>(op, stage1_blocks(N), ns, W->K, W->part, W->sc, 1.0 / (double)h->nu,
                                   h->bc == VEMG_NEUMANN, h->precision != VEMG_PREC_FP64, first, W->ctr,
                                   (int *)(W->ctr + 1), hd, use_cond);
    BATCH_LAUNCHED();
}

static void bprecond_any(vemg_hierarchy *h, BatchWork *W, int first, cudaStream_t s) {
    if (h->precision != VEMG_PREC_FP64) bprecond<float>(h, W, s);   // BF16 hierarchies: FP32 values here
    else bprecond<double>(h, W, s);
    // t0 = sum z, t1 = (r, z), t2 = sum r [, t3 = (z, q), t4 = sum q]
    int64_t N = (int64_t)h->nu * W->K;
    bool flex = h->precision != VEMG_PREC_FP64;
    (void)first;
    const int ns = flex ? 5 : 3;
    if (flex)
        pdl_launch(k_bsums_zrq<5>, stage1_blocks(N), kBT, s, N, W->K, (const double *)W->Z, (const double *)W->R,
                   (const double *)W->Q, W->part);
    else
        pdl_launch(k_bsums_zrq<3>, stage1_blocks(N), kBT, s, N, W->K, (const double *)W->Z, (const double *)W->R,
                   (const double *)nullptr, W->part);
    BATCH_LAUNCHED();
    bstage2(h, W, ST_BETA, ns, N, first, s);
}

// b -= mean (Neumann), r = b, x = p = 0, ||b|| per column; the iterations themselves start in the
// loop body, where every column enters as fresh (first direction p = z - mu)
static void bphase_pre(vemg_hierarchy *h, BatchWork *W, cudaStream_t s) {
    const int K = W->K, nu = h->nu;
    const int64_t N = (int64_t)nu * K;
    const bool neu = h->bc == VEMG_NEUMANN;
    if (neu) {
        BSums d{{W->B}, {nullptr}, 1};
        bsums(W, N, d, s);
        bstage2(h, W, ST_MEAN_B, 1, N, 0, s);
    }
    k_bprepare<<<grid_for(N, 256), 256, 0, s>>>(N, K, neu, W->B, W->R, W->X, W->P, W->sc, W->Rb32, rb32_offset(h, W));
    BATCH_LAUNCHED();
    BSums d{{W->B}, {W->B}, 1};
    bsums(W, N, d, s);
    bstage2(h, W, ST_BN, 1, N, 0, s);
}

static void bphase_step(vemg_hierarchy *h, BatchWork *W, cudaStream_t s, cudaGraphConditionalHandle hd, int use_cond) {
    const int K = W->K;
    const int64_t N = (int64_t)h->nu * K;
    bcsr<BOP_SPMV, double, double, double, double, double>(W->Aout, h->nu, nullptr, 0, (const double *)nullptr,
                                                           (const double *)nullptr, W->P, W->Q, K, nullptr, -1, s, 2);
    {
        BSums d{{W->P}, {W->Q}, 1};
        bsums(W, N, d, s);
        bstage2(h, W, ST_ALPHA, 1, N, 0, s);
    }
    pdl_launch(k_bupdate_xr, stage1_blocks(N), kBT, s, N, K, (const double *)W->P, (const double *)W->Q, W->X, W->R,
               (const double *)W->sc, W->Rb32, rb32_offset(h, W), W->part);
    BATCH_LAUNCHED();
    bstage2(h, W, ST_RN, 1, N, 0, s, hd, use_cond);
}

static void bphase_direction(vemg_hierarchy *h, BatchWork *W, cudaStream_t s) {
    bprecond_any(h, W, 0, s);
    int64_t N = (int64_t)h->nu * W->K;
    pdl_launch(k_bupdate_p, grid_for(N, 256), 256, s, N, W->K, (const double *)W->sc, (const double *)W->Z, W->P);
    BATCH_LAUNCHED();
}

static void bphase_post(vemg_hierarchy *h, BatchWork *W, cudaStream_t s) {
    const int K = W->K, nu = h->nu;
    const int64_t N = (int64_t)nu * K;
    if (h->bc == VEMG_NEUMANN) {
        BSums d{{W->X}, {nullptr}, 1};
        bsums(W, N, d, s);
        bstage2(h, W, ST_MEAN_X, 1, N, 0, s);
        k_bsub_mean<<<grid_for(N, 256), 256, 0, s>>>(N, K, W->X, W->sc, B_XMEAN);
        BATCH_LAUNCHED();
    }
    // true residual into Q
    bcsr<BOP_RES, double, double, double, double, double>(W->Aout, h->nu, nullptr, 0, (const double *)nullptr, W->B,
                                                          W->X, W->Q, K, nullptr, -1, s, 2);
    BSums d{{W->Q}, {W->Q}, 1};
    bsums(W, N, d, s);
    bstage2(h, W, ST_TRUE, 1, N, 0, s);
}

static void release_batch_graphs(BatchWork *W) {
    BatchGraphs *G = W->graphs;
    if (!G) return;
    if (G->exec) cudaGraphExecDestroy(G->exec);
    if (G->g) cudaGraphDestroy(G->g);
    delete G;
    W->graphs = nullptr;
}

static void build_batch_graphs(vemg_hierarchy *h, BatchWork *W) {
    BatchGraphs *G = new BatchGraphs();
    W->graphs = G;
    cudaStream_t cs;
    VEMG_CHECK_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    int64_t *saved = b_count;
    int64_t count = 0;
    b_count = &count;
    try {
        // one graph per solve: the preparation and the kernel that sets the loop condition, a
        // WHILE node whose body is one iteration of every column, then the exit work
        VEMG_CHECK_CUDA(cudaGraphCreate(&G->g, 0));
        VEMG_CHECK_CUDA(cudaGraphConditionalHandleCreate(&G->handle, G->g, 0, cudaGraphCondAssignDefault));
        VEMG_CHECK_CUDA(cudaStreamBeginCaptureToGraph(cs, G->g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        bphase_pre(h, W, cs);
        k_bcond_init<<<1, 1, 0, cs>>>(gsc(W), G->handle);
        BATCH_LAUNCHED();
        G->k_pre = count;
        cudaStreamCaptureStatus st;
        const cudaGraphNode_t *deps = nullptr;
        size_t ndeps = 0;
        VEMG_CHECK_CUDA(cudaStreamGetCaptureInfo(cs, &st, nullptr, nullptr, &deps, nullptr, &ndeps));
        std::vector<cudaGraphNode_t> frontier(deps, deps + ndeps);
        cudaGraph_t captured = G->g;
        VEMG_CHECK_CUDA(cudaStreamEndCapture(cs, &captured));
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = G->handle;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t cnode;
        VEMG_CHECK_CUDA(cudaGraphAddNode(&cnode, G->g, frontier.data(), nullptr, frontier.size(), &cp));
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        count = 0;
        VEMG_CHECK_CUDA(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        bphase_direction(h, W, cs);
        bphase_step(h, W, cs, G->handle, 1);
        VEMG_CHECK_CUDA(cudaStreamEndCapture(cs, &body));
        G->k_body = count;
        count = 0;
        VEMG_CHECK_CUDA(cudaStreamBeginCaptureToGraph(cs, G->g, &cnode, nullptr, 1, cudaStreamCaptureModeThreadLocal));
        bphase_post(h, W, cs);
        captured = G->g;
        VEMG_CHECK_CUDA(cudaStreamEndCapture(cs, &captured));
        G->k_post = count;
        VEMG_CHECK_CUDA(cudaGraphInstantiate(&G->exec, G->g, 0));
    } catch (...) {
        cudaStreamDestroy(cs);
        b_count = saved;
        release_batch_graphs(W);
        throw;
    }
    b_count = saved;
    VEMG_CHECK_CUDA(cudaStreamDestroy(cs));
}

void release_batch(vemg_hierarchy *h) {
    BatchWork *W = h->batch;
    if (!W) return;
    release_batch_graphs(W);
    W->arena.release();
    delete W;
    h->batch = nullptr;
}

__global__ void k_to_f32(int64_t n, const double *__restrict__ a, float *__restrict__ b) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) b[i] = (float)a[i];
}

__global__ void k_recip(int n, const double *__restrict__ d, void *out, int fp32) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double v = 1.0 / d[i];
    if (fp32) ((float *)out)[i] = (float)v;
    else ((double *)out)[i] = v;
}

static const void *values(Arena &ar, const double *v, int64_t n, bool fp32, cudaStream_t s) {
    if (!fp32) return v;
    float *f = ar.alloc<float>(n);
    if (n > 0) {
        k_to_f32<<<grid_for(n, 256), 256, 0, s>>>(n, v, f);
        VEMG_CHECK_LAUNCH();
    }
    return f;
}

static BChain *build_bchain(const Chain &C, bool fp32, Arena &ar, cudaStream_t s) {
    BChain *B = new BChain();
    B->nlev = C.nlev;
    B->direct = C.direct;
    B->nc = C.nc;
    B->G = C.G;
    if (C.direct && fp32) B->Gf = (const float *)values(ar, C.G, (int64_t)C.nc * C.nc, true, s);
    for (int l = 0; l < C.nlev; ++l) {
        const Level &L = C.lv[l];
        BLevel &T = B->lv[l];
        T.n = L.A.n;
        T.ncolours = L.ncolours;
        T.rp = L.A.rp;
        T.ci = L.A.ci;
        T.colour = L.colour;
        T.crow = L.crow;
        T.cptr = L.cptr;
        T.v = values(ar, L.A.v, L.A.nnz, fp32, s);
        void *di = fp32 ? (void *)ar.alloc<float>(L.A.n) : (void *)ar.alloc<double>(L.A.n);
        k_recip<<<grid_for(L.A.n, 256), 256, 0, s>>>(L.A.n, L.diag, di, fp32);
        VEMG_CHECK_LAUNCH();
        T.dinv = di;
        if (l + 1 < C.nlev) {
            T.prp = L.P.rp;
            T.pci = L.P.ci;
            T.pv = values(ar, L.P.v, L.P.nnz, fp32, s);
            T.trp = L.PT.rp;
            T.tci = L.PT.ci;
            T.tv = values(ar, L.PT.v, L.PT.nnz, fp32, s);
        }
    }
    return B;
}

BatchWork *new_batch_work(vemg_hierarchy *h, int K, cudaStream_t s);

static BatchWork *batch_work(vemg_hierarchy *h, int K, cudaStream_t s) {
    if (h->batch && h->batch->K == K) return h->batch;
    VEMG_CHECK_CUDA(cudaStreamSynchronize(s));
    release_batch(h);
    h->batch = new_batch_work(h, K, s);
    return h->batch;
}

// The autotuner: for each class of row kernel, every candidate shape (lanes per row 4, 8, 16, 32
// up to K; 2, 4 or 8 warps per block) is launched on a representative operation of this
// hierarchy at this batch width (class 0: the largest colour of the finest A_bar level swept
// over all its entries; class 1: the residual of that level; class 2: the outer q = A p), one
// warm-up and two timed launches each (CUDA events), and the fastest shape is kept. The vectors
// are the batch's own work buffers (zeroed); the per-column arithmetic does not depend on the shape.
template <class XT>
static void autotune_t(vemg_hierarchy *h, BatchWork *W, cudaStream_t s) {
    const int K = W->K;
    const BLevel &L = W->bbar->lv[0];
    XT *lx = (XT *)W->lx[1][0], *lb = (XT *)W->lb[1][0], *lr = (XT *)W->lr[1][0];
    const size_t vb = sizeof(XT) * (size_t)L.n * K;
    VEMG_CHECK_CUDA(cudaMemsetAsync(lx, 0, vb, s));
    VEMG_CHECK_CUDA(cudaMemsetAsync(lb, 0, vb, s));
    VEMG_CHECK_CUDA(cudaMemsetAsync(W->P, 0, sizeof(double) * (size_t)h->nu * K, s));
    int cbig = 0;
    for (int c = 1; c < L.ncolours; ++c)
        if (L.cptr[c + 1] - L.cptr[c] > L.cptr[cbig + 1] - L.cptr[cbig]) cbig = c;
    const CsrP A{L.rp, L.ci, L.v};
    cudaEvent_t e0, e1;
    VEMG_CHECK_CUDA(cudaEventCreate(&e0));
    VEMG_CHECK_CUDA(cudaEventCreate(&e1));
    int64_t *saved = b_count;
    b_count = nullptr;
    try {
        for (int cls = 0; cls < 3; ++cls) {
            float best = 0.f;
            for (int kw : {4, 8, 16, 32}) {
                if (kw > K) continue;
                for (int wp : {2, 4, 8}) {
                    auto run = [&]() {
                        if (cls == 0)
                            bcsr<BOP_SOR, XT, XT, XT, XT, XT>(A, L.cptr[cbig + 1] - L.cptr[cbig], L.crow + L.cptr[cbig], 0,
                                                               (const XT *)L.dinv, lb, lx, lx, K, L.colour, -1, s, 0,
                                                               kw, wp);
                        else if (cls == 1)
                            bcsr<BOP_RES, XT, XT, XT, XT, XT>(A, L.n, nullptr, 0, (const XT *)nullptr, lb, lx, lr, K,
                                                               nullptr, -1, s, 1, kw, wp);
                        else
                            bcsr<BOP_SPMV, double, double, double, double, double>(
                                W->Aout, h->nu, nullptr, 0, (const double *)nullptr, (const double *)nullptr, W->P,
                                W->Q, K, nullptr, -1, s, 2, kw, wp);
                    };
                    run();
                    VEMG_CHECK_CUDA(cudaEventRecord(e0, s));
                    run();
                    run();
                    VEMG_CHECK_CUDA(cudaEventRecord(e1, s));
                    VEMG_CHECK_CUDA(cudaEventSynchronize(e1));
                    float ms = 0.f;
                    VEMG_CHECK_CUDA(cudaEventElapsedTime(&ms, e0, e1));
                    const float us = 500.f * ms;   // per launch
                    W->tune.tried++;
                    if (W->tune.kw[cls] == 0 || us < best) {
                        best = us;
                        W->tune.kw[cls] = kw;
                        W->tune.warps[cls] = wp;
                        W->tune.us[cls] = us;
                    }
                }
            }
        }
    } catch (...) {
        b_count = saved;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        throw;
    }
    b_count = saved;
    VEMG_CHECK_CUDA(cudaEventDestroy(e0));
    VEMG_CHECK_CUDA(cudaEventDestroy(e1));
}

static void autotune(vemg_hierarchy *h, BatchWork *W, cudaStream_t s) {
    if (W->K < 4) return;   // one lane per row and column: no shape to choose
    if (h->precision != VEMG_PREC_FP64) autotune_t<float>(h, W, s);
    else autotune_t<double>(h, W, s);
}

BatchWork *new_batch_work(vemg_hierarchy *h, int K, cudaStream_t s) {
    BatchWork *W = new BatchWork();
    W->K = K;
    Arena &ar = W->arena;
    int64_t N = (int64_t)h->n * K;
    W->X = ar.alloc<double>(N);
    W->R = ar.alloc<double>(N);
    W->Z = ar.alloc<double>(N);
    W->P = ar.alloc<double>(N);
    W->Q = ar.alloc<double>(N);
    W->B = ar.alloc<double>(N);
    VEMG_CHECK_CUDA(cudaMemsetAsync(W->Q, 0, sizeof(double) * N, s));
    VEMG_CHECK_CUDA(cudaMemsetAsync(W->Z, 0, sizeof(double) * N, s));
    const bool fp32 = h->precision != VEMG_PREC_FP64;
    size_t es = fp32 ? sizeof(float) : sizeof(double);
    const Chain *chains[2] = {&h->surf, single_chain(h) ? &the_chain(h) : &h->bar};
    if (!single_chain(h)) W->bsurf = build_bchain(h->surf, fp32, ar, s);
    W->bbar = build_bchain(*chains[1], fp32, ar, s);
    if (h->bc == VEMG_NEUMANN) {
        W->Aout = CsrP{h->A.rp, h->A.ci, h->A.v};
        W->caller_of = h->new2old;
    } else {
        const DCsr &A0 = h->bar.lv[0].A;
        W->Aout = CsrP{A0.rp, A0.ci, A0.v};
        W->caller_of = h->new2old + h->mtop;
    }
    for (int ch = 0; ch < 2; ++ch)
        for (int l = 0; l < chains[ch]->nlev && (ch == 1 || !single_chain(h)); ++l) {
            int64_t m = (int64_t)chains[ch]->lv[l].A.n * K;
            W->lx[ch][l] = ar.alloc<char>((int64_t)es * m);
            W->lb[ch][l] = ar.alloc<char>((int64_t)es * m);
            W->lr[ch][l] = ar.alloc<char>((int64_t)es * m);
        }
    if (fp32 && !single_chain(h)) {
        W->Ev32 = ar.alloc<float>(h->E.nnz);
        k_bto_float<<<grid_for(h->E.nnz, 256), 256, 0, s>>>(h->E.nnz, (const double *)h->E.v, W->Ev32);
        VEMG_CHECK_LAUNCH();
        W->Rb32 = ar.alloc<float>((int64_t)(h->n - h->mtop) * K);
    }
    W->sc = ar.alloc<double>(B_COUNT * K + G_COUNT);
    W->part = ar.alloc<double>((int64_t)5 * stage1_blocks(N) * K);
    W->ctr = ar.alloc<unsigned>(2);
    VEMG_CHECK_CUDA(cudaMemsetAsync(W->ctr, 0, sizeof(unsigned) * 2, s));
    VEMG_CHECK_CUDA(cudaStreamSynchronize(s));
    try {
        autotune(h, W, s);
    } catch (...) {
        W->arena.release();
        delete W;
        throw;
    }
    VEMG_CHECK_CUDA(cudaStreamSynchronize(s));
    return W;
}

int solve_batch(vemg_hierarchy *h, int k, const double *Bin, int64_t ldb, double *Xout, int64_t ldx, double rtol,
                int max_it, vemg_info *infos, cudaStream_t s) {
    if (k == 0) return VEMG_OK;
    if (k > kMaxK || h->precond == VEMG_PRECOND_NONE) throw Error{VEMG_EINVAL};
    prepare_solve(h, s);
    int K = 1;
    while (K < k) K *= 2;
    BatchWork *W = batch_work(h, K, s);
    TuneScope tune(&W->tune);
    b_count = &h->launches;
    const int nu = h->nu;
    k_binit<<<1, 1, 0, s>>>(W->sc, K, rtol, max_it);
    BATCH_LAUNCHED();
    k_bgather<<<grid_for((int64_t)nu * K, 256), 256, 0, s>>>(nu, K, k, ldb, W->caller_of, Bin, W->B);
    BATCH_LAUNCHED();
    // with a probe on, the same phases are launched on the stream (profilers see every kernel)
    const bool use_graph = h->probe.kind == PROBE_NONE;
    if (!W->graphs) build_batch_graphs(h, W);
    BatchGraphs *G = W->graphs;
    if (use_graph) {
        VEMG_CHECK_CUDA(cudaGraphLaunch(G->exec, s));   // the whole batched solve, one launch
    } else {
        bphase_pre(h, W, s);
        for (;;) {
            double cont = 0.0;
            VEMG_CHECK_CUDA(cudaMemcpyAsync(&cont, gsc(W) + G_CONT, sizeof(double), cudaMemcpyDeviceToHost, s));
            VEMG_CHECK_CUDA(cudaStreamSynchronize(s));
            if (cont == 0.0) break;
            bphase_direction(h, W, s);
            bphase_step(h, W, s, 0, 0);
        }
        bphase_post(h, W, s);
    }
    std::vector<double> hs(B_COUNT * K + G_COUNT);
    VEMG_CHECK_CUDA(cudaMemcpyAsync(hs.data(), W->sc, sizeof(double) * hs.size(), cudaMemcpyDeviceToHost, s));
    int ntop = h->bc == VEMG_DIRICHLET_TOP ? h->mtop : 0;
    int64_t nsc = (int64_t)std::max(nu, ntop) * k;
    k_bscatter<<<grid_for(nsc, 256), 256, 0, s>>>(nu, K, k, ldx, W->caller_of, h->tops, ntop, W->X, Xout);
    BATCH_LAUNCHED();
    VEMG_CHECK_CUDA(cudaStreamSynchronize(s));
    int rounds = (int)hs[B_COUNT * K + G_ITERS];
    if (use_graph) h->launches += G->k_pre + G->k_post + (int64_t)rounds * G->k_body;
    int rc = VEMG_OK;
    for (int c = 0; c < k; ++c) {
        vemg_info &in = infos[c];
        double bn = hs[B_BN * K + c];
        in.iters = (int)hs[B_ITERS * K + c];
        in.relres = bn > 0.0 ? hs[B_RN * K + c] / bn : 0.0;
        in.true_relres = bn > 0.0 ? hs[B_TRUE * K + c] / bn : 0.0;
        in.b_mean = hs[B_BMEAN * K + c];
        if (hs[B_ZERO * K + c] != 0.0) in.status = VEMG_OK;
        else if (hs[B_FLAG * K + c] != 0.0) in.status = VEMG_EBREAKDOWN;
        else if (hs[B_CONV * K + c] != 0.0) in.status = VEMG_OK;
        else in.status = VEMG_ENOTCONV;
        if (in.status != VEMG_OK && rc == VEMG_OK) rc = in.status;
    }
    return rc;
}

}  // namespace vemg

// ------------------------------------------------------------------------------------------
// continuous batching: an engine holds K column slots of one hierarchy. A request is admitted into
// a free slot between iterations (its column is prepared and marked fresh, so its first direction
// is p = z - mu while the other columns continue their own recurrences); every step advances all
// occupied slots by whole iterations; a finished slot is retired (x copied out) and reused.

namespace vemg {

struct Engine {
    vemg_hierarchy *h = nullptr;
    BatchWork *W = nullptr;
    cudaStream_t s = nullptr;
    cudaGraphExec_t step = nullptr;
    cudaGraph_t gstep = nullptr;
    int64_t k_step = 0;
    std::vector<int> used;        // slot occupied
    double *hsc = nullptr;        // pinned copy of the per-column scalars
    double *colpart = nullptr;    // single-column reduction partials
    int ncolblk = 0;
};

static constexpr int kColBlocks = 128;

// sum over rows of column c of a (or of a^2); per-block partials
__global__ void k_col_sum(int n, int K, int c, const double *__restrict__ a, int square, double *part) {
    __shared__ double sh[256];
    double v = 0.0;
    for (int i = blockIdx.x * 256 + threadIdx.x; i < n; i += kColBlocks * 256) {
        double x = a[(int64_t)i * K + c];
        v += square ? x * x : x;
    }
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// admission of column c: after the sum of b (mode 0) or of the projected b squared (mode 1)
__global__ void k_col_admit(int mode, int neumann, double inv_n, int K, int c, const double *__restrict__ part,
                            double *sc, double tol, int maxit) {
    double t = 0.0;
    for (int k = 0; k < kColBlocks; ++k) t += part[k];
    if (mode == 0) {
        sc[B_BMEAN * K + c] = neumann ? t * inv_n : 0.0;
        return;
    }
    double bn = sqrt(t);
    for (int slot = 0; slot < B_COUNT; ++slot)
        if (slot != B_BMEAN) sc[slot * K + c] = 0.0;
    sc[B_BN * K + c] = bn;
    sc[B_TOL * K + c] = tol;
    sc[B_MAXIT * K + c] = (double)maxit;
    sc[B_FRESH * K + c] = 1.0;
    if (bn == 0.0) {
        sc[B_ZERO * K + c] = 1.0;
        sc[B_CONV * K + c] = 1.0;
    }
}

__global__ void k_col_gather(int nu, int K, int c, const int *__restrict__ caller_of, const double *__restrict__ b,
                             double *__restrict__ B) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nu) B[(int64_t)i * K + c] = b[caller_of[i]];
}

// b -= mean, r = b, x = p = z = q = 0 in column c
__global__ void k_col_prepare(int nu, int K, int c, const double *__restrict__ sc, double *B, double *R, double *X,
                              double *P, double *Z, double *Q, float *rb32, int64_t off32) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nu) return;
    int64_t e = (int64_t)i * K + c;
    double bi = B[e] - sc[B_BMEAN * K + c];
    B[e] = bi;
    R[e] = bi;
    if (rb32 && e >= off32) rb32[e - off32] = (float)bi;
    X[e] = 0.0;
    P[e] = 0.0;
    Z[e] = 0.0;
    Q[e] = 0.0;
}

__global__ void k_col_mean(int K, int c, const double *__restrict__ part, double inv_n, double *sc) {
    double t = 0.0;
    for (int k = 0; k < kColBlocks; ++k) t += part[k];
    sc[B_XMEAN * K + c] = t * inv_n;
}

__global__ void k_col_scatter(int nu, int K, int c, int neumann, const int *__restrict__ caller_of,
                              const int *__restrict__ tops, int ntop, const double *__restrict__ sc,
                              const double *__restrict__ X, double *__restrict__ x) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    double mu = neumann ? sc[B_XMEAN * K + c] : 0.0;
    if (i < nu) x[caller_of[i]] = X[(int64_t)i * K + c] - mu;
    if (i < ntop) x[tops[i]] = 0.0;
}

// a retired slot is frozen (zero right-hand side, converged) until it is admitted again
__global__ void k_col_free(int nu, int K, int c, double *sc, double *B, double *R, double *X, double *P, float *rb32,
                           int64_t off32) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nu) {
        int64_t e = (int64_t)i * K + c;
        B[e] = 0.0;
        R[e] = 0.0;
        if (rb32 && e >= off32) rb32[e - off32] = 0.0f;
        X[e] = 0.0;
        P[e] = 0.0;
    }
    if (i == 0) {
        for (int slot = 0; slot < B_COUNT; ++slot) sc[slot * K + c] = 0.0;
        sc[B_ZERO * K + c] = 1.0;
        sc[B_CONV * K + c] = 1.0;
    }
}

__global__ void k_engine_init(double *sc, int K) {
    for (int i = 0; i < B_COUNT * K + G_COUNT; ++i) sc[i] = 0.0;
    for (int c = 0; c < K; ++c) {
        sc[B_ZERO * K + c] = 1.0;
        sc[B_CONV * K + c] = 1.0;
    }
}

BatchWork *new_batch_work(vemg_hierarchy *h, int K, cudaStream_t s);

}  // namespace vemg

using namespace vemg;

struct vemg_engine : vemg::Engine {};

extern "C" {

int vemg_engine_create(vemg_hierarchy *h, int slots, void *stream, vemg_engine **out) {
    if (!h || !out || slots < 1 || slots > kMaxK || h->precond == VEMG_PRECOND_NONE) return VEMG_EINVAL;
    *out = nullptr;
    vemg_engine *e = new vemg_engine();
    try {
        cudaStream_t s = (cudaStream_t)stream;
        prepare_solve(h, s);
        int K = 1;
        while (K < slots) K *= 2;
        e->h = h;
        e->s = s;
        e->W = new_batch_work(h, K, s);
        e->used.assign(K, 0);
        VEMG_CHECK_CUDA(cudaMallocHost(&e->hsc, sizeof(double) * (B_COUNT * K + G_COUNT)));
        e->colpart = e->W->arena.alloc<double>(kColBlocks);
        k_engine_init<<<1, 1, 0, s>>>(e->W->sc, K);
        VEMG_CHECK_LAUNCH();
        // one iteration of every occupied column, as a graph
        TuneScope tune(&e->W->tune);
        cudaStream_t cs;
        VEMG_CHECK_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        int64_t count = 0;
        b_count = &count;
        VEMG_CHECK_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        bphase_direction(h, e->W, cs);
        bphase_step(h, e->W, cs, 0, 0);
        VEMG_CHECK_CUDA(cudaStreamEndCapture(cs, &e->gstep));
        b_count = nullptr;
        e->k_step = count;
        VEMG_CHECK_CUDA(cudaStreamDestroy(cs));
        VEMG_CHECK_CUDA(cudaGraphInstantiate(&e->step, e->gstep, 0));
        VEMG_CHECK_CUDA(cudaStreamSynchronize(s));
    } catch (const Error &err) {
        b_count = nullptr;
        vemg_engine_destroy(e);
        return err.code;
    } catch (...) {
        b_count = nullptr;
        vemg_engine_destroy(e);
        return VEMG_EINTERNAL;
    }
    *out = e;
    return VEMG_OK;
}

void vemg_engine_destroy(vemg_engine *e) {
    if (!e) return;
    if (e->s) cudaStreamSynchronize(e->s);
    if (e->step) cudaGraphExecDestroy(e->step);
    if (e->gstep) cudaGraphDestroy(e->gstep);
    if (e->hsc) cudaFreeHost(e->hsc);
    if (e->W) {
        e->W->arena.release();
        delete e->W;
    }
    delete e;
}

int vemg_engine_admit(vemg_engine *e, const double *b_dev, double rtol, int max_it, int *slot) {
    if (!e || !b_dev || !slot || !(rtol >= 0.0) || max_it < 0) return VEMG_EINVAL;
    int c = -1;
    for (int k = 0; k < (int)e->used.size(); ++k)
        if (!e->used[k]) {
            c = k;
            break;
        }
    if (c < 0) return VEMG_ENOMEM;
    try {
        vemg_hierarchy *h = e->h;
        BatchWork *W = e->W;
        const int nu = h->nu, K = W->K;
        const bool neu = h->bc == VEMG_NEUMANN;
        cudaStream_t s = e->s;
        k_col_gather<<<grid_for(nu, 256), 256, 0, s>>>(nu, K, c, W->caller_of, b_dev, W->B);
        VEMG_CHECK_LAUNCH();
        k_col_sum<<<kColBlocks, 256, 0, s>>>(nu, K, c, W->B, 0, e->colpart);
        VEMG_CHECK_LAUNCH();
        k_col_admit<<<1, 1, 0, s>>>(0, neu, 1.0 / nu, K, c, e->colpart, W->sc, rtol, max_it);
        VEMG_CHECK_LAUNCH();
        k_col_prepare<<<grid_for(nu, 256), 256, 0, s>>>(nu, K, c, W->sc, W->B, W->R, W->X, W->P, W->Z, W->Q, W->Rb32,
                                                        rb32_offset(h, W));
        VEMG_CHECK_LAUNCH();
        k_col_sum<<<kColBlocks, 256, 0, s>>>(nu, K, c, W->B, 1, e->colpart);
        VEMG_CHECK_LAUNCH();
        k_col_admit<<<1, 1, 0, s>>>(1, neu, 1.0 / nu, K, c, e->colpart, W->sc, rtol, max_it);
        VEMG_CHECK_LAUNCH();
        h->launches += 6;
    } catch (const Error &err) {
        return err.code;
    }
    e->used[c] = 1;
    *slot = c;
    return VEMG_OK;
}

int vemg_engine_launch(vemg_engine *e, int iters) {
    if (!e || iters < 0) return VEMG_EINVAL;
    for (int k = 0; k < iters; ++k) {
        cudaError_t err = cudaGraphLaunch(e->step, e->s);
        if (err != cudaSuccess) {
            set_last_cuda_error(err, "cudaGraphLaunch", __FILE__, __LINE__);
            return VEMG_ECUDA;
        }
    }
    e->h->launches += (int64_t)iters * e->k_step;
    const int K = e->W->K;
    cudaError_t err = cudaMemcpyAsync(e->hsc, e->W->sc, sizeof(double) * (B_COUNT * K + G_COUNT),
                                      cudaMemcpyDeviceToHost, e->s);
    if (err != cudaSuccess) {
        set_last_cuda_error(err, "cudaMemcpyAsync", __FILE__, __LINE__);
        return VEMG_ECUDA;
    }
    return VEMG_OK;
}

int vemg_engine_wait(vemg_engine *e) {
    if (!e) return VEMG_EINVAL;
    cudaError_t err = cudaStreamSynchronize(e->s);
    if (err != cudaSuccess) {
        set_last_cuda_error(err, "cudaStreamSynchronize", __FILE__, __LINE__);
        return VEMG_ECUDA;
    }
    return VEMG_OK;
}

int vemg_engine_query(const vemg_engine *e, int *busy) {
    if (!e || !busy) return VEMG_EINVAL;
    cudaError_t err = cudaStreamQuery(e->s);
    if (err == cudaErrorNotReady) {
        *busy = 1;
        return VEMG_OK;
    }
    if (err != cudaSuccess) {
        set_last_cuda_error(err, "cudaStreamQuery", __FILE__, __LINE__);
        return VEMG_ECUDA;
    }
    *busy = 0;
    return VEMG_OK;
}

int vemg_engine_poll(const vemg_engine *e, int slot, vemg_info *info, int *state) {
    if (!e || !state || slot < 0 || slot >= (int)e->used.size()) return VEMG_EINVAL;
    if (!e->used[slot]) {
        *state = VEMG_SLOT_FREE;
        return VEMG_OK;
    }
    const int K = e->W->K;
    const double *sc = e->hsc;
    bool conv = sc[B_CONV * K + slot] != 0.0, flag = sc[B_FLAG * K + slot] != 0.0;
    bool out = sc[B_ITERS * K + slot] >= sc[B_MAXIT * K + slot] || sc[B_STALL * K + slot] != 0.0;
    *state = (conv || flag || out) ? VEMG_SLOT_DONE : VEMG_SLOT_RUNNING;
    if (info) {
        double bn = sc[B_BN * K + slot];
        info->iters = (int)sc[B_ITERS * K + slot];
        info->relres = bn > 0.0 ? sc[B_RN * K + slot] / bn : 0.0;
        info->true_relres = -1.0;
        info->b_mean = sc[B_BMEAN * K + slot];
        info->status = sc[B_ZERO * K + slot] != 0.0 ? VEMG_OK
                       : flag                       ? VEMG_EBREAKDOWN
                       : conv                       ? VEMG_OK
                                                    : VEMG_ENOTCONV;
    }
    return VEMG_OK;
}

int vemg_engine_retire(vemg_engine *e, int slot, double *x_dev) {
    if (!e || !x_dev || slot < 0 || slot >= (int)e->used.size() || !e->used[slot]) return VEMG_EINVAL;
    try {
        vemg_hierarchy *h = e->h;
        BatchWork *W = e->W;
        const int nu = h->nu, K = W->K;
        const bool neu = h->bc == VEMG_NEUMANN;
        cudaStream_t s = e->s;
        if (neu) {
            k_col_sum<<<kColBlocks, 256, 0, s>>>(nu, K, slot, W->X, 0, e->colpart);
            VEMG_CHECK_LAUNCH();
            k_col_mean<<<1, 1, 0, s>>>(K, slot, e->colpart, 1.0 / nu, W->sc);
            VEMG_CHECK_LAUNCH();
        }
        int ntop = neu ? 0 : h->mtop;
        k_col_scatter<<<grid_for(std::max(nu, ntop), 256), 256, 0, s>>>(nu, K, slot, neu, W->caller_of, h->tops, ntop,
                                                                         W->sc, W->X, x_dev);
        VEMG_CHECK_LAUNCH();
        k_col_free<<<grid_for(nu, 256), 256, 0, s>>>(nu, K, slot, W->sc, W->B, W->R, W->X, W->P, W->Rb32,
                                                     rb32_offset(h, W));
        VEMG_CHECK_LAUNCH();
        VEMG_CHECK_CUDA(cudaStreamSynchronize(s));
        h->launches += neu ? 4 : 2;
    } catch (const Error &err) {
        return err.code;
    }
    e->used[slot] = 0;
    return VEMG_OK;
}

int vemg_batch_tuning(const vemg_hierarchy *h, int *K, int *kw, int *warps, float *us) {
    if (!h || !K || !kw || !warps || !us) return VEMG_EINVAL;
    if (!h->batch) return VEMG_EINVAL;
    const BTune &t = h->batch->tune;
    *K = h->batch->K;
    for (int c = 0; c < 3; ++c) {
        kw[c] = t.kw[c];
        warps[c] = t.warps[c];
        us[c] = t.us[c];
    }
    return VEMG_OK;
}

int vemg_batch_set_tuning(vemg_hierarchy *h, int K, const int *kw, const int *warps, void *stream) {
    if (!h || !kw || !warps || K < 1 || K > kMaxK || (K & (K - 1)) || h->precond == VEMG_PRECOND_NONE)
        return VEMG_EINVAL;
    for (int c = 0; c < 3; ++c)
        if (!(kw[c] == 4 || kw[c] == 8 || kw[c] == 16 || kw[c] == 32) || !(warps[c] == 2 || warps[c] == 4 ||
                                                                          warps[c] == 8))
            return VEMG_EINVAL;
    try {
        cudaStream_t s = (cudaStream_t)stream;
        prepare_solve(h, s);
        BatchWork *W = batch_work(h, K, s);
        for (int c = 0; c < 3; ++c) {
            W->tune.kw[c] = kw[c];
            W->tune.warps[c] = warps[c];
            W->tune.us[c] = 0.f;
        }
        release_batch_graphs(W);   // recaptured with the new shapes at the next solve
    } catch (const Error &err) {
        return err.code;
    } catch (...) {
        return VEMG_EINTERNAL;
    }
    return VEMG_OK;
}

int vemg_engine_slots(const vemg_engine *e, int *slots, int *free_slots) {
    if (!e || !slots || !free_slots) return VEMG_EINVAL;
    *slots = (int)e->used.size();
    int f = 0;
    for (int u : e->used) f += !u;
    *free_slots = f;
    return VEMG_OK;
}

int vemg_engine_bytes(const vemg_engine *e, size_t *bytes) {
    if (!e || !bytes) return VEMG_EINVAL;
    *bytes = e->W->arena.bytes;
    return VEMG_OK;
}

}  // extern "C"
