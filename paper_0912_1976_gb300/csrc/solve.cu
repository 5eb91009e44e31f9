#include <vector>
// solve.cu -- the solve phase: preconditioned CG with the additive vertical-extrapolation
// multigrid preconditioner (Kramer, Cotter and Pain, section 5.5, Eq. ourpreconditioner):
//
//   z = E~ V(E~^T A E~)(E~^T r) + [0; I] V(A_bar)([0; I]^T r)
//
// where V(.) is one smoothed-aggregation V-cycle (section 5.1, section 6: one forward SOR sweep
// with omega = 1 before the coarse correction, one backward sweep after it), and CG projects the
// constant nullspace out of every preconditioned residual (section 3). With an FP32 preconditioner
// the outer loop is flexible CG (Notay's FCG(1)), since the preconditioner is then not exactly
// symmetric (section 5.5 on nested inexact inner solves).
//
// Operators are sliced ELL in solve order (layout.cu); one thread per row, 32 rows per warp.
// Reductions are deterministic (fixed grid, fixed order). One solve runs as three CUDA graphs:
// the first iteration, a WHILE conditional node whose body is one further iteration (the
// condition is set on the device from the residual norm), and the exit work.
#include <math.h>

#include <algorithm>

#include <type_traits>

#include <cuda_bf16.h>

#include "internal.cuh"

namespace vemg {

static constexpr int kRedBlocks = 608;  // 4 x 152 SMs
static constexpr int kRedThreads = 256;
static constexpr int kSellBlock = 128;  // 4 slices per block
static constexpr int kRows = 1;         // rows per thread and loop trip in the streaming kernels (1: k_combine fits 4 blocks per SM)
static constexpr int kEmax = 4;         // E~ rows with at most this many entries take the fast path

// ------------------------------------------------------------------------------------------
// launch accounting and opt-in kernel timing

static thread_local int64_t *g_count = nullptr;
static thread_local Probe *g_probe = nullptr;
static constexpr int kProbePairs = 1024;

#define SOLVE_LAUNCHED()         \
    do {                         \
        VEMG_CHECK_LAUNCH();     \
        if (g_count) ++*g_count; \
    } while (0)

static void probe_flush(Probe &p) {
    if (p.used == 0) return;
    for (int i = 0; i < p.used; ++i) {
        // the pairs may sit on two streams (surface and A_bar branches): wait for each one
        VEMG_CHECK_CUDA(cudaEventSynchronize(p.ev[2 * i + 1]));
        float ms = 0.f;
        VEMG_CHECK_CUDA(cudaEventElapsedTime(&ms, p.ev[2 * i], p.ev[2 * i + 1]));
        p.total_ms += ms;
        p.total_bytes += p.bytes[i];
    }
    p.launches += p.used;
    p.used = 0;
}

struct ProbeScope {
    Probe *p = nullptr;
    cudaStream_t s;
    double bytes;
    ProbeScope(int kind, double bytes_, cudaStream_t s_) : s(s_), bytes(bytes_) {
        if (g_probe && g_probe->kind == kind) {
            p = g_probe;
            if ((int)p->ev.size() < 2 * kProbePairs) {
                p->ev.resize(2 * kProbePairs);
                for (auto &e : p->ev) VEMG_CHECK_CUDA(cudaEventCreate(&e));
                p->bytes.resize(kProbePairs);
            }
            VEMG_CHECK_CUDA(cudaEventRecord(p->ev[2 * p->used], s));
        }
    }
    ~ProbeScope() noexcept(false) {
        if (!p) return;
        VEMG_CHECK_CUDA(cudaEventRecord(p->ev[2 * p->used + 1], s));
        p->bytes[p->used] = bytes;
        if (++p->used == kProbePairs) probe_flush(*p);
    }
};

void probe_start(vemg_hierarchy *h, int kind) {
    Probe &p = h->probe;
    if (p.used) probe_flush(p);
    p.kind = kind;
    p.total_ms = p.total_bytes = 0.0;
    p.launches = 0;
}

void probe_read(vemg_hierarchy *h, double *ms, int64_t *launches, double *bytes) {
    Probe &p = h->probe;
    probe_flush(p);
    *ms = p.total_ms;
    *launches = p.launches;
    *bytes = p.total_bytes;
}

// Algorithmic bytes of a sliced-ELL pass: its stored entries (value + column index) once, the
// per-row vector traffic once (x gathers are counted as one read of the x vector).
static double sell_bytes(int64_t nnz, double vb, int64_t rows, double per_row) {
    return (double)nnz * (vb + 4.0) + (double)rows * per_row;
}

// ------------------------------------------------------------------------------------------
// sliced-ELL kernels

// entries of a sliced-ELL row loaded per chunk (before their gathers)
static constexpr int kU = 16;

// the V-cycle kernels' chunk: 8 entries with FP64 values (16 FP64 values and their columns held
// 80 registers and measured 11% slower per FP64-cycle solve), 16 with FP32 or BF16 values
template <class VT>
__host__ __device__ constexpr int cycle_chunk() {
    return sizeof(VT) == sizeof(double) ? 8 : kU;
}

// BF16 values widen to FP32 before they meet the vector; FP32 and FP64 values pass through
__device__ __forceinline__ float float_or_self(__nv_bfloat16 a) { return __bfloat162float(a); }
__device__ __forceinline__ float float_or_self(float a) { return a; }
__device__ __forceinline__ double float_or_self(double a) { return a; }

// The first U entries of a sliced-ELL row (column indices and values), loaded before the
// kernel waits for its predecessor: the operators are setup data that no solve kernel writes,
// so these loads overlap the previous kernel and only the gathers of x remain after the wait.
template <class VT, int U = kU>
struct RowHead {
    int c[U];
    VT a[U];
};

template <class VT, int U>
__device__ __forceinline__ void load_head(RowHead<VT, U> &h, const int *__restrict__ col, const VT *__restrict__ v,
                                          int o, int w) {
#pragma unroll
    for (int u = 0; u < U; ++u) {
        h.c[u] = u < w ? __ldg(col + o + 32 * u) : 0;
        h.a[u] = u < w ? __ldg(v + o + 32 * u) : VT{};
    }
}

// Dot product of one sliced-ELL row with x: the head's entries, then the rest of the row U
// entries at a time (column indices and values first, then the gathers), so that a row costs
// two dependent memory round trips per U entries instead of two per entry. lim >= 0 skips
// columns >= lim. The products are added in the row's stored order whatever U is.
template <class VT, class XT, class AT, int U>
__device__ __forceinline__ AT sell_row(const RowHead<VT, U> &h, const int *__restrict__ col, const VT *__restrict__ v,
                                       int o, int w, const XT *x, int lim) {
    AT acc = 0;
#pragma unroll
    for (int u = 0; u < U; ++u)
        if (u < w && (lim < 0 || h.c[u] < lim)) acc = fmadd((AT)(float_or_self(h.a[u])), (AT)x[h.c[u]], acc);
    for (int k0 = U; k0 < w; k0 += U) {
        int c[U];
        VT a[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            int k = k0 + u;
            c[u] = k < w ? __ldg(col + o + 32 * k) : 0;
            a[u] = k < w ? __ldg(v + o + 32 * k) : VT{};
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (k0 + u < w && (lim < 0 || c[u] < lim)) acc = fmadd((AT)(float_or_self(a[u])), (AT)x[c[u]], acc);
    }
    return acc;
}

template <class VT, class XT, class AT, int U = kU>
__device__ __forceinline__ AT sell_row(const int *__restrict__ col, const VT *__restrict__ v, int o, int w,
                                       const XT *x, int lim) {
    RowHead<VT, U> h;
    load_head(h, col, v, o, w);
    return sell_row<VT, XT, AT, U>(h, col, v, o, w, x, lim);
}

// y = A x (add: y += A x) over the slices [s0, s1); accumulation in AT. With x0: the restriction
// into a level whose V-cycle starts with a sweep from x = 0 also does that sweep's first colour
// (rows below lim0): x0_i = y_i / A_ii, the same product the colour's own launch would form.
template <class VT, class XT, class YT, class AT>
__global__ void __launch_bounds__(kSellBlock) k_sell_spmv(int s0, int s1, const int *__restrict__ row0,
                                                          const int *__restrict__ nrow, const int *__restrict__ off,
                                                          const int *__restrict__ width, const int *__restrict__ col,
                                                          const VT *__restrict__ v, const XT *__restrict__ x,
                                                          YT *__restrict__ y, int add, const YT *__restrict__ dinv0,
                                                          YT *__restrict__ x0, int lim0) {
    int s = s0 + (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    int lane = threadIdx.x & 31;
    const bool active = s < s1 && lane < nrow[s];
    constexpr int U = cycle_chunk<VT>();
    RowHead<VT, U> h;
    int o = 0, w = 0, r = 0;
    YT d0 = 0;
    if (active) {
        o = off[s] + lane;
        w = width[s];
        r = row0[s] + lane;
        if (x0 && r < lim0) d0 = dinv0[r];
        load_head(h, col, v, o, w);
    }
    pdl_begin();
    if (!active) return;
    AT acc = sell_row<VT, XT, AT, U>(h, col, v, o, w, x, -1);
    YT yr = add ? (YT)((AT)y[r] + acc) : (YT)acc;
    y[r] = yr;
    if (x0 && r < lim0) x0[r] = yr * d0;
}

// SOR (omega = 1) on the rows of one colour (slices [s0, s1)):
// x_i = (b_i - sum_{j != i} A_ij x_j) / A_ii. lim >= 0: sweep from x = 0, entries with column
// >= lim (colours not yet visited) are zero and skipped; lim == 0 needs no entries at all.
template <class VT, class XT, class BT>
__global__ void __launch_bounds__(kSellBlock) k_sell_sor(int s0, int s1, const int *__restrict__ row0,
                                                         const int *__restrict__ nrow, const int *__restrict__ off,
                                                         const int *__restrict__ width, const int *__restrict__ col,
                                                         const VT *__restrict__ v, const XT *__restrict__ dinv,
                                                         const BT *__restrict__ b, XT *x, int lim) {
    int s = s0 + (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    int lane = threadIdx.x & 31;
    const bool active = s < s1 && lane < nrow[s];
    constexpr int U = cycle_chunk<VT>();
    RowHead<VT, U> h;
    int o = 0, w = 0, r = 0;
    XT di = 0;
    if (active) {
        o = off[s] + lane;
        w = lim == 0 ? 0 : width[s];
        r = row0[s] + lane;
        di = dinv[r];
        load_head(h, col, v, o, w);
    }
    pdl_begin();
    if (!active) return;
    XT acc = sell_row<VT, XT, XT, U>(h, col, v, o, w, x, lim);
    x[r] = ((XT)b[r] - acc) * di;
}

// r = b - D x - (A - D) x over all slices
template <class VT, class XT, class BT>
__global__ void __launch_bounds__(kSellBlock) k_sell_residual(int nsl, const int *__restrict__ row0,
                                                              const int *__restrict__ nrow, const int *__restrict__ off,
                                                              const int *__restrict__ width, const int *__restrict__ col,
                                                              const VT *__restrict__ v, const XT *__restrict__ diag,
                                                              const BT *__restrict__ b, const XT *__restrict__ x,
                                                              XT *__restrict__ r) {
    int s = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    int lane = threadIdx.x & 31;
    const bool active = s < nsl && lane < nrow[s];
    constexpr int U = cycle_chunk<VT>();
    RowHead<VT, U> h;
    int o = 0, w = 0, i = 0;
    XT dg = 0;
    if (active) {
        o = off[s] + lane;
        w = width[s];
        i = row0[s] + lane;
        dg = diag[i];
        load_head(h, col, v, o, w);
    }
    pdl_begin();
    if (!active) return;
    XT acc = fmadd(dg, x[i], sell_row<VT, XT, XT, U>(h, col, v, o, w, x, -1));
    r[i] = (XT)b[i] - acc;
}

// x = G b for the dense coarsest inverse (one warp per row; G and the sums in the cycle's
// precision)
template <class XT, class BT>
__global__ void k_dense_mv(int n, const XT *__restrict__ Gm, const BT *__restrict__ b, XT *__restrict__ x) {
    pdl_begin();
    int row = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32, lane = threadIdx.x % 32;
    if (row >= n) return;
    XT s = 0;
    for (int k = lane; k < n; k += 32) s = fmadd(Gm[(int64_t)row * n + k], (XT)b[k], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) x[row] = (XT)s;
}

// ------------------------------------------------------------------------------------------
// launch wrappers

template <class VT, class XT, class YT, class AT>
static void sell_spmv(const Sell &S, const XT *x, YT *y, int add, cudaStream_t s, const SLevel *first = nullptr) {
    if (S.nslices == 0) return;
    int64_t threads = (int64_t)S.nslices * 32;
    // first: the level y feeds, whose from-zero sweep's first colour this launch also does
    const YT *d0 = first ? (const YT *)first->dinv : nullptr;
    YT *x0 = first ? (YT *)first->x : nullptr;
    const int lim0 = first ? first->crow[1] : 0;
    // stored entries, y written (and read when adding), x read once; the fused first colour reads
    // its inverse diagonal and writes its x
    const double vb = S.vh ? 2.0 : (double)(S.fp32 ? 4 : 8);
    ProbeScope ps(PROBE_TRANSFER,
                  sell_bytes(S.nnz, vb, S.n, (add ? 2.0 : 1.0) * sizeof(YT)) + (double)sizeof(XT) * S.m +
                      2.0 * sizeof(YT) * lim0,
                  s);
    if (S.vh)   // BF16 values (FP32 vectors)
        pdl_launch(k_sell_spmv<__nv_bfloat16, XT, YT, AT>, grid_for(threads, kSellBlock), kSellBlock, s, 0,
                   S.nslices, S.row0, S.nrow, S.off, S.width, S.col, (const __nv_bfloat16 *)S.vh, x, y, add, d0, x0,
                   lim0);
    else
        pdl_launch(k_sell_spmv<VT, XT, YT, AT>, grid_for(threads, kSellBlock), kSellBlock, s, 0, S.nslices,
                   S.row0, S.nrow, S.off, S.width, S.col, (const VT *)S.v, x, y, add, d0, x0, lim0);
    SOLVE_LAUNCHED();
}

// bytes of one stored value of S as the per-phase kernels read it
template <class XT>
static double value_bytes(const Sell &S) {
    return S.vh ? 2.0 : (double)sizeof(XT);
}

// skip0: a from-zero sweep whose first colour the restriction into this level already did
template <class XT, class BT>
static void sor_sweep(const SLevel &L, const BT *b, XT *x, bool forward, bool from_zero, bool fine, cudaStream_t s,
                      bool skip0 = false) {
    for (int cc = skip0 ? 1 : 0; cc < L.ncolours; ++cc) {
        int c = forward ? cc : L.ncolours - 1 - cc;
        int s0 = L.cslice[c], s1 = L.cslice[c + 1];
        if (s1 == s0) continue;
        int lim = from_zero ? L.crow[c] : -1;
        int rows = L.crow[c + 1] - L.crow[c];
        // stored entries of the colour (none when lim == 0), b / dinv / x-write per row, and one
        // read of the level's x shared among the sweep's colours
        double bytes = sell_bytes(lim == 0 ? 0 : L.cnnz[c], value_bytes<XT>(L.A), rows, 3.0 * sizeof(XT)) +
                       (double)sizeof(XT) * L.n / L.ncolours;
        ProbeScope ps(fine ? PROBE_SOR_FINE : PROBE_SOR, bytes, s);
        int64_t threads = (int64_t)(s1 - s0) * 32;
        if (L.A.vh)
            pdl_launch(k_sell_sor<__nv_bfloat16, XT, BT>, grid_for(threads, kSellBlock), kSellBlock, s, s0, s1,
                       L.A.row0, L.A.nrow, L.A.off, L.A.width, L.A.col, (const __nv_bfloat16 *)L.A.vh,
                       (const XT *)L.dinv, b, x, lim);
        else
            pdl_launch(k_sell_sor<XT, XT, BT>, grid_for(threads, kSellBlock), kSellBlock, s, s0, s1, L.A.row0,
                       L.A.nrow, L.A.off, L.A.width, L.A.col, (const XT *)L.A.v, (const XT *)L.dinv, b, x, lim);
        SOLVE_LAUNCHED();
    }
}

template <class XT, class BT>
static void residual(const SLevel &L, const BT *b, const XT *x, XT *r, cudaStream_t s) {
    ProbeScope ps(PROBE_RESIDUAL, sell_bytes(L.A.nnz, value_bytes<XT>(L.A), L.n, 5.0 * sizeof(XT)), s);
    int64_t threads = (int64_t)L.A.nslices * 32;
    if (L.A.vh)
        pdl_launch(k_sell_residual<__nv_bfloat16, XT, BT>, grid_for(threads, kSellBlock), kSellBlock, s,
                   L.A.nslices, L.A.row0, L.A.nrow, L.A.off, L.A.width, L.A.col, (const __nv_bfloat16 *)L.A.vh,
                   (const XT *)L.diag, b, x, r);
    else
        pdl_launch(k_sell_residual<XT, XT, BT>, grid_for(threads, kSellBlock), kSellBlock, s, L.A.nslices,
                   L.A.row0, L.A.nrow, L.A.off, L.A.width, L.A.col, (const XT *)L.A.v, (const XT *)L.diag, b, x, r);
    SOLVE_LAUNCHED();
}

// whether the restriction into level l does the first colour of its from-zero sweep (levels
// swept one kernel per colour: not the dense coarsest level, not a single-CTA tail)
static bool fused_first(const SChain &C, int l) {
    if (l >= C.nlev || C.lv[l].ncolours < 1) return false;
    if (l == C.nlev - 1 && C.direct) return false;
    return !(l > 0 && l == C.tail_level);
}

// V-cycle with a zero initial guess (section 5.1); b of level 0 may be FP64 (the outer residual).
// first_done: the first colour of the pre-smoothing sweep was done by the restriction into l.
template <class XT, class BT>
static void vcycle_level(const SChain &C, int l, const BT *b, XT *x, cudaStream_t s, bool first_done = false) {
    const SLevel &L = C.lv[l];
    const bool fine = C.is_bar && l == 0;
    if (l > 0 && l == C.tail_level) {
        // the coarse tail: every level from here down and back up in one kernel (one CTA, or one
        // thread-block cluster); it reads b and writes x in this level's own buffers
        ProbeScope ps(PROBE_TAIL, ctail_bytes(C), s);
        launch_tail(C, s, g_probe && g_probe->kind == PROBE_TAIL);
        SOLVE_LAUNCHED();
        return;
    }
    if (l == C.nlev - 1) {
        if (C.direct) {
            const XT *G = sizeof(XT) == sizeof(float) ? (const XT *)C.Gf : (const XT *)C.G;
            ProbeScope ps(PROBE_DENSE, (double)sizeof(XT) * C.nc * (C.nc + 1.0) + (double)sizeof(BT) * C.nc, s);
            pdl_launch(k_dense_mv<XT, BT>, grid_for(C.nc, 8), 256, s, C.nc, G, b, x);
            SOLVE_LAUNCHED();
            return;
        }
        // coarsening stalled above the direct-solve size: one symmetric SOR pass
        sor_sweep<XT, BT>(L, b, x, true, true, fine, s, first_done);
        sor_sweep<XT, BT>(L, b, x, false, false, fine, s);
        return;
    }
    sor_sweep<XT, BT>(L, b, x, true, true, fine, s, first_done);
    residual<XT, BT>(L, b, x, (XT *)L.r, s);
    const SLevel &N = C.lv[l + 1];
    const bool fuse = fused_first(C, l + 1);
    sell_spmv<XT, XT, XT, XT>(L.PT, (const XT *)L.r, (XT *)N.b, 0, s, fuse ? &N : nullptr);
    vcycle_level<XT, XT>(C, l + 1, (const XT *)N.b, (XT *)N.x, s, fuse);
    sell_spmv<XT, XT, XT, XT>(L.P, (const XT *)N.x, x, 1, s);
    sor_sweep<XT, BT>(L, b, x, false, false, fine, s);
}

// The finest level of a V-cycle split around its coarse correction (the hybrid launch
// structure): down = pre-smoothing, residual, restriction into level 1; up = prolongation of
// level 1's x and post-smoothing. The same launches as vcycle_level's, in the same order.
template <class XT, class BT>
static void vcycle_down(const SChain &C, const BT *b, XT *x, cudaStream_t s) {
    const SLevel &L = C.lv[0];
    sor_sweep<XT, BT>(L, b, x, true, true, C.is_bar, s);
    residual<XT, BT>(L, b, x, (XT *)L.r, s);
    sell_spmv<XT, XT, XT, XT>(L.PT, (const XT *)L.r, (XT *)C.lv[1].b, 0, s);
}

template <class XT, class BT>
static void vcycle_up(const SChain &C, const BT *b, XT *x, cudaStream_t s) {
    const SLevel &L = C.lv[0];
    sell_spmv<XT, XT, XT, XT>(L.P, (const XT *)C.lv[1].x, x, 1, s);
    sor_sweep<XT, BT>(L, b, x, false, false, C.is_bar, s);
}

// ------------------------------------------------------------------------------------------
// deterministic block reductions: every block writes its partial sums, the last block to finish
// adds them in block order (fixed grid, fixed order: the same bits on every run)

enum {
    S_RZ = 0, S_PQ, S_ALPHA, S_BETA, S_MU, S_BN, S_RN, S_FLAG, S_TOL, S_MAXIT, S_ITERS, S_CONT, S_ZERO, S_TRUE,
    S_BMEAN, S_XMEAN, S_COUNT
};
enum { C_SPMV = 0, C_XR, C_Z, C_SUMB, C_PREP, C_SUMX, C_TRUE, C_COUNT };

int solve_scalar_iters() { return S_ITERS; }

template <int NS>
__device__ bool finish_block(double (&acc)[NS], double *part, unsigned *counter, double (&tot)[NS]) {
    __shared__ double sh[NS][kRedThreads / 32];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        double v = acc[s];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) sh[s][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < NS) {
        double v = 0.0;
        for (int w = 0; w < kRedThreads / 32; ++w) v += sh[threadIdx.x][w];
        part[threadIdx.x * kRedBlocks + blockIdx.x] = v;
        __threadfence();
    }
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(counter, 1u) == (unsigned)(kRedBlocks - 1);
    __syncthreads();
    if (!last) return false;
    __threadfence();
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        double v = 0.0;
        for (int k = threadIdx.x; k < kRedBlocks; k += kRedThreads) v += __ldcg(part + s * kRedBlocks + k);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        __syncthreads();
        if (lane == 0) sh[s][warp] = v;
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        double v = 0.0;
        for (int w = 0; w < kRedThreads / 32; ++w) v += sh[s][w];
        tot[s] = v;
    }
    if (threadIdx.x == 0) *counter = 0u;
    return true;
}

struct SellArgs {
    int nsl;
    const int *row0, *nrow, *off, *width, *col;
    const double *v;
};

static SellArgs sargs(const Sell &S) {
    return SellArgs{S.nslices, S.row0, S.nrow, S.off, S.width, S.col, (const double *)S.v};
}

// q = A p over all slices and (p, q); the last block sets alpha = rz / pq. At most 64 registers:
// the whole grid (kRedBlocks = 4 per SM) is resident at once.
__global__ void __launch_bounds__(kRedThreads, kRedBlocks / 152) k_spmv_pq(SellArgs A, const double *__restrict__ p,
                                                         double *__restrict__ q, double *sc, double *part,
                                                         unsigned *ctr, double *coef) {
    pdl_begin();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double acc[1] = {0.0};
    for (int s = blockIdx.x * (kRedThreads / 32) + warp; s < A.nsl; s += kRedBlocks * (kRedThreads / 32)) {
        if (lane < A.nrow[s]) {
            int r = A.row0[s] + lane;
            double qv = sell_row<double, double, double>(A.col, A.v, A.off[s] + lane, A.width[s], p, -1);
            q[r] = qv;
            acc[0] += p[r] * qv;
        }
    }
    double tot[1];
    if (!finish_block<1>(acc, part, ctr, tot) || threadIdx.x != 0) return;
    double pq = tot[0];
    sc[S_PQ] = pq;
    if (sc[S_ZERO] != 0.0) sc[S_ALPHA] = 0.0;
    else if (!(pq > 0.0)) {
        sc[S_FLAG] = 1.0;
        sc[S_ALPHA] = 0.0;
    } else sc[S_ALPHA] = sc[S_RZ] / pq;
    // CG coefficient history: alpha_k at 2k (k = iterations completed so far)
    const int k = (int)sc[S_ITERS];
    if (2 * k < kCoefCap) coef[2 * k] = sc[S_ALPHA];
}

// x += alpha p, r -= alpha q; the last block sets ||r||, the iteration count and the continuation
// test (and, inside the solve graph, the WHILE condition)
__global__ void __launch_bounds__(kRedThreads) k_update_xr(int n, const double *__restrict__ p,
                                                           const double *__restrict__ q, double *__restrict__ x,
                                                           double *__restrict__ r, double *sc, double *part,
                                                           unsigned *ctr, cudaGraphConditionalHandle handle,
                                                           int use_cond) {
    pdl_begin();
    double a = sc[S_ALPHA];
    double acc[1] = {0.0};
    constexpr int stride = kRedBlocks * kRedThreads;
    for (int i0 = blockIdx.x * kRedThreads + threadIdx.x; i0 < n; i0 += kRows * stride) {
        double pv[kRows], qv[kRows], xv[kRows], rv[kRows];
#pragma unroll
        for (int u = 0; u < kRows; ++u) {
            int i = i0 + u * stride;
            bool ok = i < n;
            pv[u] = ok ? p[i] : 0.0;
            qv[u] = ok ? q[i] : 0.0;
            xv[u] = ok ? x[i] : 0.0;
            rv[u] = ok ? r[i] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < kRows; ++u) {
            int i = i0 + u * stride;
            if (i < n) {
                x[i] = xv[u] + a * pv[u];
                double ri = rv[u] - a * qv[u];
                r[i] = ri;
                acc[0] += ri * ri;
            }
        }
    }
    double tot[1];
    if (!finish_block<1>(acc, part, ctr, tot) || threadIdx.x != 0) return;
    double rn = sqrt(tot[0]);
    sc[S_RN] = rn;
    double it = sc[S_ZERO] != 0.0 ? 0.0 : sc[S_ITERS] + 1.0;
    sc[S_ITERS] = it;
    if (!(rn == rn)) sc[S_FLAG] = 1.0;
    bool cont = sc[S_ZERO] == 0.0 && sc[S_FLAG] == 0.0 && rn > sc[S_TOL] * sc[S_BN] && it < sc[S_MAXIT];
    sc[S_CONT] = cont ? 1.0 : 0.0;
    if (use_cond) cudaGraphSetConditional(handle, cont ? 1u : 0u);
}

// z from the two branches (Neumann: top rows z = y_s, other rows z = E~ y_s + x_bar; Dirichlet-
// top: z = x_bar) and the sums t0 = sum z, t1 = (r, z), t2 = sum r, t3 = (z, q), t4 = sum q.
// The last block sets mu (mean of z), rz = (r, z - mu) and beta: first direction 0, CG
// rz'/rz, FCG -(z - mu, q) / (p, q).
template <class XT>
__global__ void __launch_bounds__(kRedThreads) k_combine(int nu, int mtop, SellArgs E, const float *__restrict__ evf,
                                                         const XT *__restrict__ ys, const XT *__restrict__ xb,
                                                         double *__restrict__ z, const double *__restrict__ r,
                                                         const double *__restrict__ q, int neumann, int flexible,
                                                         int first, double inv_n, double *sc, double *part,
                                                         unsigned *ctr, const int *__restrict__ perr, double *coef) {
    pdl_begin();
    // FP32 V-cycles with an FP32 copy of E~ (evf): z_i = x_bar_i + sum_k e_k y_s(c_k) is formed in
    // FP32 and converted once (FP64 instructions are scarce on this GPU); otherwise in FP64
    using ZT = typename std::conditional<std::is_same<XT, float>::value, float, double>::type;
    const bool lowz = std::is_same<XT, float>::value && evf != nullptr;
    double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    constexpr int stride = kRedBlocks * kRedThreads;
    const bool dots_q = flexible && !first;
    for (int i0 = blockIdx.x * kRedThreads + threadIdx.x; i0 < nu; i0 += kRows * stride) {
        double zv[kRows], rv[kRows], qv[kRows];
        ZT zl[kRows];
        // loads of every row first (the E~ row entries, x_bar, r, q), then the gathers of y_s
        int ec[kRows][kEmax];
        double ev[kRows][kEmax];
        ZT el[kRows][kEmax];
#pragma unroll
        for (int u = 0; u < kRows; ++u) {
            int i = i0 + u * stride;
            zv[u] = 0.0;
            zl[u] = (ZT)0;
            rv[u] = 0.0;
            qv[u] = 0.0;
#pragma unroll
            for (int k = 0; k < kEmax; ++k) { ec[u][k] = -1; ev[u][k] = 0.0; el[u][k] = (ZT)0; }
            if (i >= nu) continue;
            rv[u] = r[i];
            if (dots_q) qv[u] = q[i];
            if (i < mtop) continue;
            if (mtop == 0) { zv[u] = (double)xb[i]; continue; }
            int qq = i - mtop, sl = qq >> 5, ln = qq & 31;
            int o = E.off[sl] + ln, w = E.width[sl];
            if (lowz) zl[u] = (ZT)xb[qq];
            else zv[u] = (double)xb[qq];
            if (w <= kEmax) {
#pragma unroll
                for (int k = 0; k < kEmax; ++k)
                    if (k < w) {
                        ec[u][k] = __ldg(E.col + o + 32 * k);
                        if (lowz) el[u][k] = (ZT)__ldg(evf + o + 32 * k);
                        else ev[u][k] = __ldg(E.v + o + 32 * k);
                    }
            } else if (lowz) {
                zl[u] += (ZT)sell_row<float, XT, float>(E.col, evf, o, w, ys, -1);
            } else {
                zv[u] += sell_row<double, XT, double>(E.col, E.v, o, w, ys, -1);
            }
        }
#pragma unroll
        for (int u = 0; u < kRows; ++u) {
            int i = i0 + u * stride;
            if (i >= nu) continue;
            double zi;
            if (lowz && i >= mtop && mtop > 0) {
                ZT zf = zl[u];
#pragma unroll
                for (int k = 0; k < kEmax; ++k)
                    if (ec[u][k] >= 0) zf += el[u][k] * (ZT)ys[ec[u][k]];
                zi = (double)zf;
            } else {
                zi = zv[u];
                if (i < mtop) zi = (double)ys[i];
#pragma unroll
                for (int k = 0; k < kEmax; ++k)
                    if (ec[u][k] >= 0) zi += ev[u][k] * (double)ys[ec[u][k]];
            }
            z[i] = zi;
            acc[0] += zi;
            acc[1] += rv[u] * zi;
            acc[2] += rv[u];
            if (dots_q) {
                acc[3] += zi * qv[u];
                acc[4] += qv[u];
            }
        }
    }
    double tot[5];
    if (!finish_block<5>(acc, part, ctr, tot) || threadIdx.x != 0) return;
    double mu = neumann ? tot[0] * inv_n : 0.0;
    double rz = tot[1] - mu * tot[2];
    double beta;
    if (first) beta = 0.0;
    else if (flexible) beta = -(tot[3] - mu * tot[4]) / sc[S_PQ];
    else beta = rz / sc[S_RZ];
    sc[S_MU] = mu;
    sc[S_BETA] = beta;
    sc[S_RZ] = rz;
    if (!(rz == rz) || !(beta == beta)) sc[S_FLAG] = 1.0;
    if (perr && *(const volatile int *)perr) sc[S_FLAG] = 2.0;   // the persistent cycle gave up waiting
    // CG coefficient history: beta_k at 2k - 1 (k = iterations completed so far, k >= 1)
    const int k = (int)sc[S_ITERS];
    if (!first && k >= 1 && 2 * k - 1 < kCoefCap) coef[2 * k - 1] = beta;
}

// p = (z - mu) + beta p
__global__ void k_update_p(int n, const double *__restrict__ sc, const double *__restrict__ z, double *__restrict__ p) {
    pdl_begin();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    double mu = sc[S_MU], beta = sc[S_BETA];
    if (i < n) p[i] = (z[i] - mu) + beta * p[i];
}

// sum of a vector; the last block stores the mean in sc[slot]
__global__ void __launch_bounds__(kRedThreads) k_mean(int n, const double *__restrict__ a, double inv_n, int slot,
                                                      double *sc, double *part, unsigned *ctr) {
    pdl_begin();
    double acc[1] = {0.0};
    constexpr int stride = kRedBlocks * kRedThreads;
    for (int i0 = blockIdx.x * kRedThreads + threadIdx.x; i0 < n; i0 += kRows * stride) {
        double v[kRows];
#pragma unroll
        for (int u = 0; u < kRows; ++u) v[u] = i0 + u * stride < n ? a[i0 + u * stride] : 0.0;
#pragma unroll
        for (int u = 0; u < kRows; ++u) acc[0] += v[u];
    }
    double tot[1];
    if (!finish_block<1>(acc, part, ctr, tot) || threadIdx.x != 0) return;
    sc[slot] = tot[0] * inv_n;
}

// b -= mean (Neumann), r = b, x = 0, p = 0, ||b||; the last block sets ||b|| and the zero flag
__global__ void __launch_bounds__(kRedThreads) k_prepare(int n, int neumann, double *__restrict__ b,
                                                         double *__restrict__ r, double *__restrict__ x,
                                                         double *__restrict__ p, double *sc, double *part,
                                                         unsigned *ctr) {
    pdl_begin();
    double mu = neumann ? sc[S_BMEAN] : 0.0;
    double acc[1] = {0.0};
    constexpr int stride = kRedBlocks * kRedThreads;
    for (int i0 = blockIdx.x * kRedThreads + threadIdx.x; i0 < n; i0 += kRows * stride) {
        double v[kRows];
#pragma unroll
        for (int u = 0; u < kRows; ++u) v[u] = i0 + u * stride < n ? b[i0 + u * stride] : 0.0;
#pragma unroll
        for (int u = 0; u < kRows; ++u) {
            int i = i0 + u * stride;
            if (i < n) {
                double bi = v[u] - mu;
                b[i] = bi;
                r[i] = bi;
                x[i] = 0.0;
                p[i] = 0.0;
                acc[0] += bi * bi;
            }
        }
    }
    double tot[1];
    if (!finish_block<1>(acc, part, ctr, tot) || threadIdx.x != 0) return;
    double bn = sqrt(tot[0]);
    sc[S_BN] = bn;
    if (bn == 0.0) {
        sc[S_ZERO] = 1.0;
        sc[S_CONT] = 0.0;
    }
}

__global__ void k_sub_scalar(int n, double *__restrict__ a, const double *__restrict__ sc, int slot) {
    pdl_begin();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] -= sc[slot];
}

// ||b - A x|| (true residual); the last block stores it
__global__ void __launch_bounds__(kRedThreads) k_true_res(SellArgs A, const double *__restrict__ x,
                                                          const double *__restrict__ b, double *sc, double *part,
                                                          unsigned *ctr) {
    pdl_begin();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double acc[1] = {0.0};
    for (int s = blockIdx.x * (kRedThreads / 32) + warp; s < A.nsl; s += kRedBlocks * (kRedThreads / 32)) {
        if (lane < A.nrow[s]) {
            int r = A.row0[s] + lane;
            double d = b[r] - sell_row<double, double, double>(A.col, A.v, A.off[s] + lane, A.width[s], x, -1);
            acc[0] += d * d;
        }
    }
    double tot[1];
    if (!finish_block<1>(acc, part, ctr, tot) || threadIdx.x != 0) return;
    sc[S_TRUE] = sqrt(tot[0]);
}

// ------------------------------------------------------------------------------------------
// the preconditioner: two independent V-cycles (the additive form of Eq. ourpreconditioner)
// on two streams, joined by the kernel that forms z

template <class XT>
static void precond_t(vemg_hierarchy *h, const double *r, double *z, int first, cudaStream_t s) {
    const SChain &B = h->sbar;
    const bool neu = h->bc == VEMG_NEUMANN, flex = h->precision != VEMG_PREC_FP64;
    const bool two = !single_chain(h);
    const int mt = two ? h->mtop : 0;
    const XT *ys = nullptr;
    // probes of the per-phase kernel classes time the launch-per-phase cycle
    const int pk = h->probe.kind;
    const bool persist = h->persist && pk != PROBE_SOR && pk != PROBE_SOR_FINE && pk != PROBE_RESIDUAL &&
                         pk != PROBE_TRANSFER && pk != PROBE_DENSE && pk != PROBE_TAIL;
    const bool none = h->precond == VEMG_PRECOND_NONE;
    const bool hybrid = persist && persist_coarse_only(h);
    if (none) {
        // no preconditioner (plain CG): z = r, formed by k_combine below
    } else if (hybrid) {
        // finest levels one kernel per phase (surface on the side stream), the coarser levels of
        // both chains in one cooperative kernel between the two halves of the finest levels
        const SChain &S = h->ssurf;
        const bool sc = two && S.nlev >= 2, bc = B.nlev >= 2;
        if (two) {
            VEMG_CHECK_CUDA(cudaEventRecord(h->ev_fork, s));
            VEMG_CHECK_CUDA(cudaStreamWaitEvent(h->side, h->ev_fork, 0));
            sell_spmv<double, double, XT, double>(h->ETs, r, (XT *)S.lv[0].b, 0, h->side);
            if (sc) vcycle_down<XT, XT>(S, (const XT *)S.lv[0].b, (XT *)S.lv[0].x, h->side);
            else vcycle_level<XT, XT>(S, 0, (const XT *)S.lv[0].b, (XT *)S.lv[0].x, h->side);
            VEMG_CHECK_CUDA(cudaEventRecord(h->ev_mid, h->side));
            ys = (const XT *)S.lv[0].x;
        }
        if (bc) vcycle_down<XT, double>(B, r + mt, (XT *)B.lv[0].x, s);
        else vcycle_level<XT, double>(B, 0, r + mt, (XT *)B.lv[0].x, s);
        if (two) VEMG_CHECK_CUDA(cudaStreamWaitEvent(s, h->ev_mid, 0));
        {
            ProbeScope ps(PROBE_VCYCLE, persist_bytes(h), s);
            launch_persist(h, r, s);
            SOLVE_LAUNCHED();
        }
        if (two) {
            VEMG_CHECK_CUDA(cudaEventRecord(h->ev_coarse, s));
            VEMG_CHECK_CUDA(cudaStreamWaitEvent(h->side, h->ev_coarse, 0));
            if (sc) vcycle_up<XT, XT>(S, (const XT *)S.lv[0].b, (XT *)S.lv[0].x, h->side);
            VEMG_CHECK_CUDA(cudaEventRecord(h->ev_join, h->side));
        }
        if (bc) vcycle_up<XT, double>(B, r + mt, (XT *)B.lv[0].x, s);
        if (two) VEMG_CHECK_CUDA(cudaStreamWaitEvent(s, h->ev_join, 0));
    } else if (persist) {
        // both branches (or the single chain) in one cooperative kernel
        {
            ProbeScope ps(PROBE_VCYCLE, persist_bytes(h), s);
            launch_persist(h, r, s);
            SOLVE_LAUNCHED();
        }
        if (two) ys = (const XT *)h->ssurf.lv[0].x;
    } else if (two) {
        const SChain &S = h->ssurf;
        VEMG_CHECK_CUDA(cudaEventRecord(h->ev_fork, s));
        VEMG_CHECK_CUDA(cudaStreamWaitEvent(h->side, h->ev_fork, 0));
        // surface branch: r_c = E~^T r accumulated in FP64, one V-cycle on E~^T A E~
        const bool fuse = fused_first(S, 0);
        sell_spmv<double, double, XT, double>(h->ETs, r, (XT *)S.lv[0].b, 0, h->side, fuse ? &S.lv[0] : nullptr);
        vcycle_level<XT, XT>(S, 0, (const XT *)S.lv[0].b, (XT *)S.lv[0].x, h->side, fuse);
        VEMG_CHECK_CUDA(cudaEventRecord(h->ev_join, h->side));
        ys = (const XT *)S.lv[0].x;
    }
    if (!persist && !none) {   // one kernel per phase
        // additive smoother: one V-cycle on A_bar with the trailing part of r
        vcycle_level<XT, double>(B, 0, r + mt, (XT *)B.lv[0].x, s);
        if (two) VEMG_CHECK_CUDA(cudaStreamWaitEvent(s, h->ev_join, 0));
    }
    const XT *xb = none ? (const XT *)r : (const XT *)B.lv[0].x;   // none: XT is double
    // r, z (and q) per row, x_bar per non-top row, the E~ entries and one read of y_s
    ProbeScope ps(PROBE_VECTOR,
                  (double)h->nu * (16.0 + (flex && !first ? 8.0 : 0.0)) + (double)(h->nu - mt) * sizeof(XT) +
                      (two ? sell_bytes(h->Enon.nnz, h->Enon_vf && sizeof(XT) == 4 ? 4.0 : 8.0, 0, 0.0) +
                                 (double)sizeof(XT) * mt
                           : 0.0),
                  s);
    pdl_launch(k_combine<XT>, kRedBlocks, kRedThreads, s, h->nu, mt, sargs(h->Enon), (const float *)h->Enon_vf, ys, xb, z, r,
                                                     h->q, neu, flex, first, 1.0 / (double)h->nu, h->scal,
                                                     h->red + 5 * kRedBlocks * C_Z, h->ctr + C_Z,
                                                     persist ? persist_err(h) : nullptr, h->coef);
    SOLVE_LAUNCHED();
}

static void precond_solve_order(vemg_hierarchy *h, const double *r, double *z, int first, cudaStream_t s) {
    if (h->precision != VEMG_PREC_FP64) precond_t<float>(h, r, z, first, s);
    else precond_t<double>(h, r, z, first, s);
}

// q = A p of the outer loop, with (p, q) and alpha
static void spmv_outer(vemg_hierarchy *h, const double *x, double *y, cudaStream_t s) {
    ProbeScope ps(PROBE_SPMV_A, sell_bytes(h->Aop.nnz, 8.0, h->Aop.n, 24.0), s);   // p read twice, q write
    pdl_launch(k_spmv_pq, kRedBlocks, kRedThreads, s, sargs(h->Aop), x, y, h->scal, h->red + 5 * kRedBlocks * C_SPMV,
                                                 h->ctr + C_SPMV, h->coef);
    SOLVE_LAUNCHED();
}

__global__ void k_init_scalars(double *sc, double tol, int maxit) {
    for (int i = 0; i < S_COUNT; ++i) sc[i] = 0.0;
    sc[S_TOL] = tol;
    sc[S_MAXIT] = (double)maxit;
    sc[S_CONT] = maxit > 0 ? 1.0 : 0.0;
}

__global__ void k_gather(int n, const int *__restrict__ idx, const double *__restrict__ src, double *__restrict__ dst) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = src[idx[i]];
}

__global__ void k_scatter_out(int nu, const int *__restrict__ caller_of, const int *__restrict__ tops, int ntop,
                              const double *__restrict__ src, double *__restrict__ dst) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nu) dst[caller_of[i]] = src[i];
    if (i < ntop) dst[tops[i]] = 0.0;
}

// before the WHILE node of the solve graph: continue only if the first iteration asked for more
__global__ void k_cond_init(const double *sc, cudaGraphConditionalHandle handle) {
    cudaGraphSetConditional(handle, sc[S_CONT] != 0.0 ? 1u : 0u);
}

// ------------------------------------------------------------------------------------------
// the iteration, shared by the plain stream path and graph capture

struct Graphs {
    cudaGraph_t g = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphConditionalHandle handle = 0;
    int64_t k_pre = 0, k_body = 0, k_post = 0;
};

static double *part_of(vemg_hierarchy *h, int c) { return h->red + 5 * kRedBlocks * c; }

static void phase_pre(vemg_hierarchy *h, cudaStream_t s) {
    const bool neu = h->bc == VEMG_NEUMANN;
    const int nu = h->nu;
    if (neu) {
        pdl_launch(k_mean, kRedBlocks, kRedThreads, s, nu, h->b, 1.0 / (double)nu, S_BMEAN, h->scal, part_of(h, C_SUMB),
                                                  h->ctr + C_SUMB);
        SOLVE_LAUNCHED();
    }
    pdl_launch(k_prepare, kRedBlocks, kRedThreads, s, nu, neu, h->b, h->r, h->x, h->p, h->scal, part_of(h, C_PREP),
                                                 h->ctr + C_PREP);
    SOLVE_LAUNCHED();
    precond_solve_order(h, h->r, h->z, 1, s);
    {
        ProbeScope ps(PROBE_VECTOR, 24.0 * nu, s);   // z, p read; p written
        pdl_launch(k_update_p, grid_for(nu, 256), 256, s, nu, h->scal, h->z, h->p);
        SOLVE_LAUNCHED();
    }
}

// q = A p, alpha, x and r updates, ||r||, continuation
static void phase_step(vemg_hierarchy *h, cudaStream_t s, cudaGraphConditionalHandle hd, int use_cond) {
    spmv_outer(h, h->p, h->q, s);
    ProbeScope ps(PROBE_VECTOR, 48.0 * h->nu, s);   // p, q, x, r read; x, r written
    pdl_launch(k_update_xr, kRedBlocks, kRedThreads, s, h->nu, h->p, h->q, h->x, h->r, h->scal, part_of(h, C_XR),
                                                   h->ctr + C_XR, hd, use_cond);
    SOLVE_LAUNCHED();
}

// new preconditioned residual and search direction
static void phase_direction(vemg_hierarchy *h, cudaStream_t s) {
    precond_solve_order(h, h->r, h->z, 0, s);
    ProbeScope ps(PROBE_VECTOR, 24.0 * h->nu, s);   // z, p read; p written
    pdl_launch(k_update_p, grid_for(h->nu, 256), 256, s, h->nu, h->scal, h->z, h->p);
    SOLVE_LAUNCHED();
}

static void phase_post(vemg_hierarchy *h, cudaStream_t s) {
    const bool neu = h->bc == VEMG_NEUMANN;
    const int nu = h->nu;
    if (neu) {
        pdl_launch(k_mean, kRedBlocks, kRedThreads, s, nu, h->x, 1.0 / (double)nu, S_XMEAN, h->scal, part_of(h, C_SUMX),
                                                  h->ctr + C_SUMX);
        SOLVE_LAUNCHED();
        pdl_launch(k_sub_scalar, grid_for(nu, 256), 256, s, nu, h->x, h->scal, S_XMEAN);
        SOLVE_LAUNCHED();
    }
    pdl_launch(k_true_res, kRedBlocks, kRedThreads, s, sargs(h->Aop), h->x, h->b, h->scal, part_of(h, C_TRUE),
                                                  h->ctr + C_TRUE);
    SOLVE_LAUNCHED();
}

static void build_graphs(vemg_hierarchy *h) {
    Graphs *G = new Graphs();
    h->graphs = G;
    cudaStream_t cs;
    VEMG_CHECK_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    Probe *saved = g_probe;
    g_probe = nullptr;
    int64_t *saved_count = g_count;
    int64_t count = 0;
    g_count = &count;
    try {
        // One graph per solve: the first iteration and the kernel that sets the loop condition,
        // then a WHILE node whose body is one further iteration, then the exit work.
        VEMG_CHECK_CUDA(cudaGraphCreate(&G->g, 0));
        VEMG_CHECK_CUDA(cudaGraphConditionalHandleCreate(&G->handle, G->g, 0, cudaGraphCondAssignDefault));
        VEMG_CHECK_CUDA(cudaStreamBeginCaptureToGraph(cs, G->g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        phase_pre(h, cs);
        phase_step(h, cs, 0, 0);
        k_cond_init<<<1, 1, 0, cs>>>(h->scal, G->handle);
        SOLVE_LAUNCHED();
        G->k_pre = count;
        // the nodes the WHILE node follows: the capture's current frontier
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
        phase_direction(h, cs);
        phase_step(h, cs, G->handle, 1);
        VEMG_CHECK_CUDA(cudaStreamEndCapture(cs, &body));
        G->k_body = count;
        // exit work, after the WHILE node
        count = 0;
        VEMG_CHECK_CUDA(cudaStreamBeginCaptureToGraph(cs, G->g, &cnode, nullptr, 1, cudaStreamCaptureModeThreadLocal));
        phase_post(h, cs);
        captured = G->g;
        VEMG_CHECK_CUDA(cudaStreamEndCapture(cs, &captured));
        G->k_post = count;
        VEMG_CHECK_CUDA(cudaGraphInstantiate(&G->exec, G->g, 0));
    } catch (...) {
        cudaStreamDestroy(cs);
        g_probe = saved;
        g_count = saved_count;
        release_graphs(h);
        throw;
    }
    g_probe = saved;
    g_count = saved_count;
    VEMG_CHECK_CUDA(cudaStreamDestroy(cs));
}

void release_graphs(vemg_hierarchy *h) {
    Graphs *G = h->graphs;
    if (G) {
        if (G->exec) cudaGraphExecDestroy(G->exec);
        if (G->g) cudaGraphDestroy(G->g);
        delete G;
        h->graphs = nullptr;
    }
    if (h->side) cudaStreamDestroy(h->side);
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    if (h->ev_mid) cudaEventDestroy(h->ev_mid);
    if (h->ev_coarse) cudaEventDestroy(h->ev_coarse);
    h->side = nullptr;
    h->ev_fork = h->ev_join = h->ev_mid = h->ev_coarse = nullptr;
}

void prepare_solve(vemg_hierarchy *h, cudaStream_t s) {
    if (h->x) return;
    Arena &ar = h->arena;
    int n = h->n;
    build_solve_layout(h, s);
    h->x = ar.alloc<double>(n);
    h->r = ar.alloc<double>(n);
    h->z = ar.alloc<double>(n);
    h->p = ar.alloc<double>(n);
    h->q = ar.alloc<double>(n);
    h->b = ar.alloc<double>(n);
    h->red = ar.alloc<double>(5 * kRedBlocks * C_COUNT);
    h->scal = ar.alloc<double>(S_COUNT);
    h->ctr = ar.alloc<unsigned>(C_COUNT);
    h->coef = ar.alloc<double>(kCoefCap);
    VEMG_CHECK_CUDA(cudaMemsetAsync(h->ctr, 0, sizeof(unsigned) * C_COUNT, s));
    h->tops = ar.alloc<int>(h->mtop);
    // caller ids of the top nodes (written as 0 by Dirichlet-top solves)
    VEMG_CHECK_CUDA(cudaMemcpyAsync(h->tops, h->new2old, sizeof(int) * h->mtop, cudaMemcpyDeviceToDevice, s));
    VEMG_CHECK_CUDA(cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking));
    VEMG_CHECK_CUDA(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
    VEMG_CHECK_CUDA(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
    VEMG_CHECK_CUDA(cudaEventCreateWithFlags(&h->ev_mid, cudaEventDisableTiming));
    VEMG_CHECK_CUDA(cudaEventCreateWithFlags(&h->ev_coarse, cudaEventDisableTiming));
    VEMG_CHECK_CUDA(cudaStreamSynchronize(s));
    if ((h->opts.cycle == VEMG_CYCLE_PERSISTENT || h->opts.cycle == VEMG_CYCLE_HYBRID) &&
        h->precond != VEMG_PRECOND_NONE)
        build_persist(h, s);
    build_tails(h, s);
}

int solve(vemg_hierarchy *h, const double *b_in, double *x_out, double rtol, int max_it, vemg_info *info,
          cudaStream_t s) {
    prepare_solve(h, s);
    const int nu = h->nu, B = 256;
    const bool use_graph = h->probe.kind == PROBE_NONE;
    g_probe = &h->probe;
    g_count = &h->launches;
    k_init_scalars<<<1, 1, 0, s>>>(h->scal, rtol, max_it);
    SOLVE_LAUNCHED();
    k_gather<<<grid_for(nu, B), B, 0, s>>>(nu, h->caller_of, b_in, h->b);
    SOLVE_LAUNCHED();
    double hs[S_COUNT];
    if (use_graph) {
        if (!h->graphs) build_graphs(h);
        Graphs *G = h->graphs;
        VEMG_CHECK_CUDA(cudaGraphLaunch(G->exec, s));   // the whole solve, one launch
        VEMG_CHECK_CUDA(cudaMemcpyAsync(hs, h->scal, sizeof(double) * S_COUNT, cudaMemcpyDeviceToHost, s));
        VEMG_CHECK_CUDA(cudaStreamSynchronize(s));
        int it = (int)hs[S_ITERS];
        h->launches += G->k_pre + G->k_post + (it > 1 ? (int64_t)(it - 1) * G->k_body : 0);
    } else {
        phase_pre(h, s);
        phase_step(h, s, 0, 0);
        for (;;) {
            double cont = 0.0;
            VEMG_CHECK_CUDA(cudaMemcpyAsync(&cont, h->scal + S_CONT, sizeof(double), cudaMemcpyDeviceToHost, s));
            VEMG_CHECK_CUDA(cudaStreamSynchronize(s));
            if (cont == 0.0) break;
            phase_direction(h, s);
            phase_step(h, s, 0, 0);
        }
        phase_post(h, s);
        VEMG_CHECK_CUDA(cudaMemcpyAsync(hs, h->scal, sizeof(double) * S_COUNT, cudaMemcpyDeviceToHost, s));
        VEMG_CHECK_CUDA(cudaStreamSynchronize(s));
    }
    int ntop = h->bc == VEMG_DIRICHLET_TOP ? h->mtop : 0;
    k_scatter_out<<<grid_for(std::max(nu, ntop), B), B, 0, s>>>(nu, h->caller_of, h->tops, ntop, h->x, x_out);
    SOLVE_LAUNCHED();
    VEMG_CHECK_CUDA(cudaStreamSynchronize(s));
    info->iters = (int)hs[S_ITERS];
    info->relres = hs[S_BN] > 0.0 ? hs[S_RN] / hs[S_BN] : 0.0;
    info->true_relres = hs[S_BN] > 0.0 ? hs[S_TRUE] / hs[S_BN] : 0.0;
    info->b_mean = hs[S_BMEAN];
    int status;
    if (hs[S_ZERO] != 0.0) status = VEMG_OK;
    else if (hs[S_FLAG] == 2.0) status = VEMG_ETIMEOUT;
    else if (hs[S_FLAG] != 0.0) status = VEMG_EBREAKDOWN;
    else if (hs[S_RN] <= hs[S_TOL] * hs[S_BN]) status = VEMG_OK;
    else status = VEMG_ENOTCONV;
    info->status = status;
    if (status == VEMG_ETIMEOUT) {
        persist_reset(h, s);
        VEMG_CHECK_CUDA(cudaStreamSynchronize(s));
    }
    return status;
}

// ------------------------------------------------------------------------------------------
// single steps in the internal (top-first) order, for the parity tests

__global__ void k_perm_in(int n, const int *__restrict__ s2i, const double *__restrict__ a, double *__restrict__ b) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = a[s2i[i]];
}

__global__ void k_perm_out(int n, const int *__restrict__ s2i, const double *__restrict__ a, double *__restrict__ b) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[s2i[i]] = a[i];
}

// solve index -> internal index of the unknowns
__global__ void k_solve_to_internal(int n, int off, const int *__restrict__ caller_of, const int *__restrict__ old2new,
                                    int *out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = old2new[caller_of[i]] - off;
}

void spmv_op(vemg_hierarchy *h, const double *x, double *y, cudaStream_t s) {
    prepare_solve(h, s);
    g_probe = &h->probe;
    g_count = &h->launches;
    int nu = h->nu, off = h->bc == VEMG_DIRICHLET_TOP ? h->mtop : 0;
    Scratch<int> s2i(nu);
    k_solve_to_internal<<<grid_for(nu, 256), 256, 0, s>>>(nu, off, h->caller_of, h->old2new, s2i);
    SOLVE_LAUNCHED();
    Scratch<double> xs(nu), ys(nu);
    k_perm_in<<<grid_for(nu, 256), 256, 0, s>>>(nu, s2i, x, xs);
    SOLVE_LAUNCHED();
    spmv_outer(h, xs, ys, s);
    k_perm_out<<<grid_for(nu, 256), 256, 0, s>>>(nu, s2i, ys, y);
    SOLVE_LAUNCHED();
    VEMG_CHECK_CUDA(cudaStreamSynchronize(s));
}

void precond(vemg_hierarchy *h, const double *r, double *z, cudaStream_t s) {
    prepare_solve(h, s);
    g_probe = &h->probe;
    g_count = &h->launches;
    int nu = h->nu, off = h->bc == VEMG_DIRICHLET_TOP ? h->mtop : 0;
    Scratch<int> s2i(nu);
    k_solve_to_internal<<<grid_for(nu, 256), 256, 0, s>>>(nu, off, h->caller_of, h->old2new, s2i);
    SOLVE_LAUNCHED();
    Scratch<double> rs(nu), zs(nu);
    k_perm_in<<<grid_for(nu, 256), 256, 0, s>>>(nu, s2i, r, rs);
    SOLVE_LAUNCHED();
    precond_solve_order(h, rs, zs, 1, s);
    k_perm_out<<<grid_for(nu, 256), 256, 0, s>>>(nu, s2i, zs, z);
    SOLVE_LAUNCHED();
    VEMG_CHECK_CUDA(cudaStreamSynchronize(s));
}

__global__ void k_perm_in_x(int n, const int *__restrict__ s2n, const double *__restrict__ a, void *b, int fp32) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (fp32) ((float *)b)[i] = (float)a[s2n[i]];
    else ((double *)b)[i] = a[s2n[i]];
}

__global__ void k_perm_out_x(int n, const int *__restrict__ s2n, const void *a, double *b, int fp32) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    b[s2n[i]] = fp32 ? (double)((const float *)a)[i] : ((const double *)a)[i];
}

void vcycle(vemg_hierarchy *h, int chain, const double *b, double *x, cudaStream_t s) {
    prepare_solve(h, s);
    g_probe = &h->probe;
    g_count = &h->launches;
    const Chain &C = chain == 0 ? h->surf : chain == 2 ? h->one : h->bar;
    // the solve layout holds the chain the preconditioner uses: surface and A_bar chains of the
    // additive form, or the single chain
    bool have = single_chain(h) ? (chain == 2 || (chain == 1 && h->bc == VEMG_DIRICHLET_TOP)) : chain != 2;
    if (C.nlev == 0 || !have) throw Error{VEMG_EINVAL};
    const SChain &S = chain == 0 ? h->ssurf : h->sbar;
    int n = C.lv[0].A.n;
    bool f = S.fp32;
    Scratch<char> bs((int64_t)n * 8), xs((int64_t)n * 8);
    k_perm_in_x<<<grid_for(n, 256), 256, 0, s>>>(n, C.lv[0].crow, b, bs, f);
    SOLVE_LAUNCHED();
    if (f) vcycle_level<float, float>(S, 0, (const float *)bs.p, (float *)xs.p, s);
    else vcycle_level<double, double>(S, 0, (const double *)bs.p, (double *)xs.p, s);
    k_perm_out_x<<<grid_for(n, 256), 256, 0, s>>>(n, C.lv[0].crow, xs, x, f);
    SOLVE_LAUNCHED();
    VEMG_CHECK_CUDA(cudaStreamSynchronize(s));
}

}  // namespace vemg
