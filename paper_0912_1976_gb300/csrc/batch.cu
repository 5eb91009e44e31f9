// batch.cu -- many right-hand sides in one solve.
//
// K systems A x_c = b_c share one hierarchy. Vectors are interleaved (row-major n x K, K a power
// of two): x[i*K + c]. In every sliced-ELL pass a group of KW = min(K, 32) lanes works on one row,
// so each matrix entry is loaded once per warp and used for KW (or K) columns, and the gathers
// x[j*K + c] of one entry are KW consecutive words. Each column keeps its own Krylov scalars
// (alpha, beta, norms, mean) and its own convergence test; a converged column is frozen (alpha = 0)
// until every column has converged. The iteration runs as CUDA graphs with a WHILE node, like the
// single right-hand-side solve (solve.cu); the V-cycles of the two branches run on two streams.
#include <math.h>

#include <algorithm>

#include "internal.cuh"

namespace vemg {

static constexpr int kBB = 304;        // blocks of the batched streaming / reduction kernels (2 per SM)
static constexpr int kBT = 512;        // their threads
static constexpr int kBU = 8;          // entries loaded per round trip in a batched row
static constexpr int kMaxK = 128;      // widest batch
static constexpr int kSellWarps = 4;   // warps per block in the batched sliced-ELL kernels

static thread_local int64_t *b_count = nullptr;
#define BATCH_LAUNCHED()         \
    do {                         \
        VEMG_CHECK_LAUNCH();     \
        if (b_count) ++*b_count; \
    } while (0)

// per-column scalar slots (sc[slot * K + c])
enum {
    B_RZ = 0, B_PQ, B_ALPHA, B_BETA, B_MU, B_BN, B_RN, B_FLAG, B_ITERS, B_CONV, B_ZERO, B_TRUE, B_BMEAN, B_XMEAN,
    B_COUNT
};
// global scalars after the per-column block (g[slot])
enum { G_TOL = 0, G_MAXIT, G_CONT, G_ITERS, G_COUNT };
enum { BC_SPMV = 0, BC_XR, BC_Z, BC_SUMB, BC_PREP, BC_SUMX, BC_TRUE, BC_COUNT };

struct BatchGraphs {
    cudaGraph_t gpre = nullptr, gloop = nullptr, gpost = nullptr;
    cudaGraphExec_t pre = nullptr, loop = nullptr, post = nullptr;
    cudaGraphConditionalHandle handle = 0;
    int64_t k_pre = 0, k_body = 0, k_post = 0;
};

struct BatchWork {
    int K = 0;
    double *X = nullptr, *R = nullptr, *Z = nullptr, *P = nullptr, *Q = nullptr, *B = nullptr;
    void *lx[2][kMaxLevels] = {}, *lb[2][kMaxLevels] = {}, *lr[2][kMaxLevels] = {};
    double *sc = nullptr;      // B_COUNT * K per-column scalars, then G_COUNT globals
    double *part = nullptr;    // reduction partials
    unsigned *ctr = nullptr;
    BatchGraphs *graphs = nullptr;
    Arena arena;
};

static double *gsc(BatchWork *w) { return w->sc + B_COUNT * w->K; }

// ------------------------------------------------------------------------------------------
// batched sliced-ELL row operations

struct SellP {
    const int *row0, *nrow, *off, *width, *col;
    const void *v;
};

static SellP sp(const Sell &S) { return SellP{S.row0, S.nrow, S.off, S.width, S.col, S.v}; }

enum { BOP_SPMV = 0, BOP_SPMV_ADD = 1, BOP_SOR = 2, BOP_RES = 3 };

// rows of the slices [s0, s1); KW lanes per row, columns c = lane % KW + j KW
template <int OP, class VT, class XT, class BT, class YT, class AT, int KW>
__global__ void __launch_bounds__(32 * kSellWarps) k_bsell(int s0, int s1, SellP A, const VT *__restrict__ dg,
                                                          const BT *__restrict__ b, const XT *x, YT *y, int K,
                                                          int lim) {
    constexpr int RW = 32 / KW;   // rows per warp
    int w = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    int s = s0 + w / KW;
    if (s >= s1) return;
    int ls = (w % KW) * RW + lane / KW;
    if (ls >= A.nrow[s]) return;
    int r = A.row0[s] + ls, o = A.off[s] + ls, wd = A.width[s];
    const VT *v = (const VT *)A.v;
    for (int c = lane % KW; c < K; c += KW) {
        AT acc = 0;
        if (!(OP == BOP_SOR && lim == 0)) {
            for (int k0 = 0; k0 < wd; k0 += kBU) {
                int cc[kBU];
                VT a[kBU];
#pragma unroll
                for (int u = 0; u < kBU; ++u) {
                    int k = k0 + u;
                    cc[u] = k < wd ? __ldg(A.col + o + 32 * k) : 0;
                    a[u] = k < wd ? __ldg(v + o + 32 * k) : (VT)0;
                }
#pragma unroll
                for (int u = 0; u < kBU; ++u)
                    if (k0 + u < wd && (lim < 0 || cc[u] < lim)) acc += (AT)a[u] * (AT)x[(int64_t)cc[u] * K + c];
            }
        }
        int64_t e = (int64_t)r * K + c;
        if (OP == BOP_SPMV) y[e] = (YT)acc;
        else if (OP == BOP_SPMV_ADD) y[e] = (YT)((AT)y[e] + acc);
        else if (OP == BOP_SOR) y[e] = (YT)(((AT)b[e] - acc) * (AT)dg[r]);
        else y[e] = (YT)((AT)b[e] - ((AT)dg[r] * (AT)x[e] + acc));
    }
}

template <int OP, class VT, class XT, class BT, class YT, class AT>
static void bsell(const Sell &S, int s0, int s1, const VT *dg, const BT *b, const XT *x, YT *y, int K, int lim,
                  cudaStream_t s) {
    if (s1 <= s0) return;
    int KW = std::min(K, 32);
    int64_t warps = (int64_t)(s1 - s0) * KW;
    int grid = (int)((warps + kSellWarps - 1) / kSellWarps);
    dim3 blk(32 * kSellWarps);
    SellP a = sp(S);
    switch (KW) {
        case 1: k_bsell<OP, VT, XT, BT, YT, AT, 1><<<grid, blk, 0, s>>>(s0, s1, a, dg, b, x, y, K, lim); break;
        case 2: k_bsell<OP, VT, XT, BT, YT, AT, 2><<<grid, blk, 0, s>>>(s0, s1, a, dg, b, x, y, K, lim); break;
        case 4: k_bsell<OP, VT, XT, BT, YT, AT, 4><<<grid, blk, 0, s>>>(s0, s1, a, dg, b, x, y, K, lim); break;
        case 8: k_bsell<OP, VT, XT, BT, YT, AT, 8><<<grid, blk, 0, s>>>(s0, s1, a, dg, b, x, y, K, lim); break;
        case 16: k_bsell<OP, VT, XT, BT, YT, AT, 16><<<grid, blk, 0, s>>>(s0, s1, a, dg, b, x, y, K, lim); break;
        default: k_bsell<OP, VT, XT, BT, YT, AT, 32><<<grid, blk, 0, s>>>(s0, s1, a, dg, b, x, y, K, lim); break;
    }
    BATCH_LAUNCHED();
}

// x = G b on the coarsest level, one thread per (row, column)
template <class XT, class BT>
__global__ void k_bdense(int n, const double *__restrict__ G, const BT *__restrict__ b, XT *__restrict__ x, int K) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)n * K) return;
    int r = (int)(t >> (__ffs(K) - 1)), c = (int)(t & (K - 1));
    double s = 0.0;
    for (int j = 0; j < n; ++j) s += G[(int64_t)r * n + j] * (double)b[(int64_t)j * K + c];
    x[t] = (XT)s;
}

template <class XT, class BT>
static void bsweep(const SLevel &L, const BT *b, XT *x, bool forward, bool from_zero, int K, cudaStream_t s) {
    for (int cc = 0; cc < L.ncolours; ++cc) {
        int c = forward ? cc : L.ncolours - 1 - cc;
        int lim = from_zero ? L.crow[c] : -1;
        bsell<BOP_SOR, XT, XT, BT, XT, XT>(L.A, L.cslice[c], L.cslice[c + 1], (const XT *)L.dinv, b, x, x, K, lim, s);
    }
}

template <class XT, class BT>
static void bvcycle(const SChain &C, BatchWork *W, int ch, int l, const BT *b, XT *x, cudaStream_t s) {
    const SLevel &L = C.lv[l];
    const int K = W->K;
    if (l == C.nlev - 1) {
        if (C.direct) {
            int64_t t = (int64_t)C.nc * K;
            k_bdense<XT, BT><<<grid_for(t, 256), 256, 0, s>>>(C.nc, C.G, b, x, K);
            BATCH_LAUNCHED();
            return;
        }
        bsweep<XT, BT>(L, b, x, true, true, K, s);
        bsweep<XT, BT>(L, b, x, false, false, K, s);
        return;
    }
    XT *r = (XT *)W->lr[ch][l];
    XT *nb = (XT *)W->lb[ch][l + 1], *nx = (XT *)W->lx[ch][l + 1];
    bsweep<XT, BT>(L, b, x, true, true, K, s);
    bsell<BOP_RES, XT, XT, BT, XT, XT>(L.A, 0, L.A.nslices, (const XT *)L.diag, b, x, r, K, -1, s);
    bsell<BOP_SPMV, XT, XT, XT, XT, XT>(L.PT, 0, L.PT.nslices, nullptr, (const XT *)nullptr, r, nb, K, -1, s);
    bvcycle<XT, XT>(C, W, ch, l + 1, (const XT *)nb, nx, s);
    bsell<BOP_SPMV_ADD, XT, XT, XT, XT, XT>(L.P, 0, L.P.nslices, nullptr, (const XT *)nullptr, nx, x, K, -1, s);
    bsweep<XT, BT>(L, b, x, false, false, K, s);
}

// ------------------------------------------------------------------------------------------
// per-column deterministic reductions: each thread accumulates for column c = tid % K (K divides
// the block size); blocks write per-column partials; the last block adds them in block order.

template <int NS>
__device__ bool bfinish(double (&acc)[NS], int K, double *part, unsigned *counter) {
    __shared__ double sh[kBT];
    __shared__ bool last;
    const int t = threadIdx.x;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        sh[t] = acc[s];
        __syncthreads();
        if (t < K) {
            double v = 0.0;
            for (int j = t; j < kBT; j += K) v += sh[j];
            part[((int64_t)s * kBB + blockIdx.x) * K + t] = v;
        }
        __syncthreads();
    }
    __threadfence();
    __syncthreads();
    if (t == 0) last = atomicAdd(counter, 1u) == (unsigned)(kBB - 1);
    __syncthreads();
    if (!last) return false;
    __threadfence();
    return true;
}

// in the last block: total of sum slot s for column c
__device__ double btotal(const double *part, int s, int c, int K) {
    double v = 0.0;
#pragma unroll 8
    for (int k = 0; k < kBB; ++k) v += __ldcg(part + ((int64_t)s * kBB + k) * K + c);
    return v;
}

// mean of each column; stored in sc[slot * K + c]
__global__ void __launch_bounds__(kBT) k_bmean(int n, int K, const double *__restrict__ a, double inv_n, int slot,
                                              double *sc, double *part, unsigned *ctr) {
    double acc[1] = {0.0};
    int64_t N = (int64_t)n * K;
    for (int64_t e = blockIdx.x * (int64_t)kBT + threadIdx.x; e < N; e += (int64_t)kBB * kBT) acc[0] += a[e];
    if (!bfinish<1>(acc, K, part, ctr)) return;
    for (int c = threadIdx.x; c < K; c += kBT) sc[slot * K + c] = btotal(part, 0, c, K) * inv_n;
    __syncthreads();
    if (threadIdx.x == 0) *ctr = 0u;
}

// b -= mean (Neumann), r = b, x = p = 0; per-column ||b||, zero columns are converged at once
__global__ void __launch_bounds__(kBT) k_bprepare(int n, int K, int neumann, double *__restrict__ b,
                                                 double *__restrict__ r, double *__restrict__ x,
                                                 double *__restrict__ p, double *sc, double *part, unsigned *ctr) {
    double acc[1] = {0.0};
    int64_t N = (int64_t)n * K;
    for (int64_t e = blockIdx.x * (int64_t)kBT + threadIdx.x; e < N; e += (int64_t)kBB * kBT) {
        int c = (int)(e & (K - 1));
        double bi = b[e] - (neumann ? sc[B_BMEAN * K + c] : 0.0);
        b[e] = bi;
        r[e] = bi;
        x[e] = 0.0;
        p[e] = 0.0;
        acc[0] += bi * bi;
    }
    if (!bfinish<1>(acc, K, part, ctr)) return;
    for (int c = threadIdx.x; c < K; c += kBT) {
        double bn = sqrt(btotal(part, 0, c, K));
        sc[B_BN * K + c] = bn;
        if (bn == 0.0) {
            sc[B_ZERO * K + c] = 1.0;
            sc[B_CONV * K + c] = 1.0;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) *ctr = 0u;
}

// Q = A P over all slices of the FP64 outer operator with per-column (p, q); alpha per column
template <int KW>
__global__ void __launch_bounds__(kBT) k_bspmv_pq(int nsl, SellP A, int K, const double *__restrict__ p,
                                                 double *__restrict__ q, double *sc, double *part, unsigned *ctr) {
    constexpr int RW = 32 / KW;
    constexpr int JK_MAX = kMaxK / 32 > 0 ? kMaxK / 32 : 1;
    const int lane = threadIdx.x & 31;
    const double *v = (const double *)A.v;
    double accj[JK_MAX];
#pragma unroll
    for (int j = 0; j < JK_MAX; ++j) accj[j] = 0.0;
    int nw_total = kBB * (kBT / 32);
    for (int w = blockIdx.x * (kBT / 32) + (threadIdx.x >> 5); w < nsl * KW; w += nw_total) {
        int s = w / KW, ls = (w % KW) * RW + lane / KW;
        if (ls >= A.nrow[s]) continue;
        int r = A.row0[s] + ls, o = A.off[s] + ls, wd = A.width[s];
        int j = 0;
        for (int c = lane % KW; c < K; c += KW, ++j) {
            double acc = 0.0;
            for (int k0 = 0; k0 < wd; k0 += kBU) {
                int cc[kBU];
                double a[kBU];
#pragma unroll
                for (int u = 0; u < kBU; ++u) {
                    int k = k0 + u;
                    cc[u] = k < wd ? __ldg(A.col + o + 32 * k) : 0;
                    a[u] = k < wd ? __ldg(v + o + 32 * k) : 0.0;
                }
#pragma unroll
                for (int u = 0; u < kBU; ++u)
                    if (k0 + u < wd) acc += a[u] * p[(int64_t)cc[u] * K + c];
            }
            int64_t e = (int64_t)r * K + c;
            q[e] = acc;
            accj[j] += p[e] * acc;
        }
    }
    // per-thread accumulators belong to columns lane % KW + j KW; fold them into the layout
    // bfinish expects (column = tid % K) through shared memory
    __shared__ double sh[kBT];
    double tot_thread = 0.0;
    if (K <= 32) {
        // tid % K == lane % KW here (KW == K, 32 % K == 0)
        tot_thread = accj[0];
        double acc1[1] = {tot_thread};
        if (!bfinish<1>(acc1, K, part, ctr)) return;
    } else {
        // K > 32: each lane holds columns lane + 32 j; write them to a (block, column) scratch row
        double colsum[1] = {0.0};
        (void)colsum;
        for (int j = 0; j < K / 32; ++j) {
            sh[threadIdx.x] = accj[j];
            __syncthreads();
            // column c = lane + 32 j: sum over the block's warps
            if (threadIdx.x < 32) {
                double vv = 0.0;
                for (int ww = 0; ww < kBT / 32; ++ww) vv += sh[ww * 32 + threadIdx.x];
                part[(int64_t)blockIdx.x * K + threadIdx.x + 32 * j] = vv;
            }
            __syncthreads();
        }
        __shared__ bool last;
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) last = atomicAdd(ctr, 1u) == (unsigned)(kBB - 1);
        __syncthreads();
        if (!last) return;
        __threadfence();
    }
    for (int c = threadIdx.x; c < K; c += kBT) {
        double pq = btotal(part, 0, c, K);
        sc[B_PQ * K + c] = pq;
        if (sc[B_CONV * K + c] != 0.0 || sc[B_FLAG * K + c] != 0.0) sc[B_ALPHA * K + c] = 0.0;
        else if (!(pq > 0.0)) {
            sc[B_FLAG * K + c] = 1.0;
            sc[B_ALPHA * K + c] = 0.0;
        } else sc[B_ALPHA * K + c] = sc[B_RZ * K + c] / pq;
    }
    __syncthreads();
    if (threadIdx.x == 0) *ctr = 0u;
}

// X += alpha P, R -= alpha Q per column, per-column ||r||, convergence, WHILE condition
__global__ void __launch_bounds__(kBT) k_bupdate_xr(int n, int K, const double *__restrict__ p,
                                                   const double *__restrict__ q, double *__restrict__ x,
                                                   double *__restrict__ r, double *sc, double *part, unsigned *ctr,
                                                   cudaGraphConditionalHandle handle, int use_cond) {
    double acc[1] = {0.0};
    int64_t N = (int64_t)n * K;
    for (int64_t e = blockIdx.x * (int64_t)kBT + threadIdx.x; e < N; e += (int64_t)kBB * kBT) {
        int c = (int)(e & (K - 1));
        double a = sc[B_ALPHA * K + c];
        x[e] += a * p[e];
        double ri = r[e] - a * q[e];
        r[e] = ri;
        acc[0] += ri * ri;
    }
    if (!bfinish<1>(acc, K, part, ctr)) return;
    __shared__ int active;
    if (threadIdx.x == 0) active = 0;
    __syncthreads();
    double *g = sc + B_COUNT * K;
    for (int c = threadIdx.x; c < K; c += kBT) {
        double rn = sqrt(btotal(part, 0, c, K));
        if (sc[B_CONV * K + c] == 0.0 && sc[B_FLAG * K + c] == 0.0) {
            sc[B_RN * K + c] = rn;
            sc[B_ITERS * K + c] += 1.0;
            if (!(rn == rn)) sc[B_FLAG * K + c] = 1.0;
            else if (rn <= g[G_TOL] * sc[B_BN * K + c]) sc[B_CONV * K + c] = 1.0;
            if (sc[B_CONV * K + c] == 0.0 && sc[B_FLAG * K + c] == 0.0 && sc[B_ITERS * K + c] < g[G_MAXIT])
                atomicOr(&active, 1);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        g[G_ITERS] += 1.0;
        g[G_CONT] = active ? 1.0 : 0.0;
        if (use_cond) cudaGraphSetConditional(handle, active ? 1u : 0u);
        *ctr = 0u;
    }
}

// Z from the two branches and per-column t0 = sum z, t1 = (r, z), t2 = sum r, t3 = (z, q),
// t4 = sum q; then per column mu, rz = (r, z - mu), beta (0 on the first direction and on frozen
// columns; CG: rz'/rz; FCG: -(z - mu, q) / (p, q))
template <class XT>
__global__ void __launch_bounds__(kBT) k_bcombine(int nu, int K, int mtop, SellP E, const XT *__restrict__ ys,
                                                 const XT *__restrict__ xb, double *__restrict__ z,
                                                 const double *__restrict__ r, const double *__restrict__ q,
                                                 int neumann, int flexible, int first, double inv_n, double *sc,
                                                 double *part, unsigned *ctr) {
    double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    const bool dq = flexible && !first;
    const double *ev = (const double *)E.v;
    int64_t N = (int64_t)nu * K;
    for (int64_t e = blockIdx.x * (int64_t)kBT + threadIdx.x; e < N; e += (int64_t)kBB * kBT) {
        int i = (int)(e >> (__ffs(K) - 1)), c = (int)(e & (K - 1));
        double zi;
        if (i < mtop) zi = (double)ys[e];
        else if (mtop > 0) {
            int qq = i - mtop, sl = qq >> 5, ln = qq & 31;
            int o = E.off[sl] + ln, w = E.width[sl];
            zi = (double)xb[(int64_t)qq * K + c];
            for (int k = 0; k < w; ++k) zi += ev[o + 32 * k] * (double)ys[(int64_t)E.col[o + 32 * k] * K + c];
        } else zi = (double)xb[e];
        z[e] = zi;
        double ri = r[e];
        acc[0] += zi;
        acc[1] += ri * zi;
        acc[2] += ri;
        if (dq) {
            double qi = q[e];
            acc[3] += zi * qi;
            acc[4] += qi;
        }
    }
    if (!bfinish<5>(acc, K, part, ctr)) return;
    for (int c = threadIdx.x; c < K; c += kBT) {
        double t0 = btotal(part, 0, c, K), t1 = btotal(part, 1, c, K), t2 = btotal(part, 2, c, K);
        double mu = neumann ? t0 * inv_n : 0.0;
        double rz = t1 - mu * t2;
        double beta = 0.0;
        bool frozen = sc[B_CONV * K + c] != 0.0 || sc[B_FLAG * K + c] != 0.0;
        if (!first && !frozen) {
            if (flexible) beta = -(btotal(part, 3, c, K) - mu * btotal(part, 4, c, K)) / sc[B_PQ * K + c];
            else beta = rz / sc[B_RZ * K + c];
            if (!(rz == rz) || !(beta == beta)) sc[B_FLAG * K + c] = 1.0;
        }
        sc[B_MU * K + c] = mu;
        sc[B_BETA * K + c] = frozen ? 0.0 : beta;
        sc[B_RZ * K + c] = rz;
    }
    __syncthreads();
    if (threadIdx.x == 0) *ctr = 0u;
}

// P = (Z - mu) + beta P per column
__global__ void k_bupdate_p(int64_t N, int K, const double *__restrict__ sc, const double *__restrict__ z,
                            double *__restrict__ p) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= N) return;
    int c = (int)(e & (K - 1));
    p[e] = (z[e] - sc[B_MU * K + c]) + sc[B_BETA * K + c] * p[e];
}

__global__ void k_bsub_mean(int64_t N, int K, double *__restrict__ x, const double *__restrict__ sc, int slot) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < N) x[e] -= sc[slot * K + (int)(e & (K - 1))];
}

// per-column ||b - A x|| (true residual), one thread per (row, column) group of the outer operator
template <int KW>
__global__ void __launch_bounds__(kBT) k_btrue(int nsl, SellP A, int K, const double *__restrict__ x,
                                              const double *__restrict__ b, double *sc, double *part, unsigned *ctr) {
    // reuses the layout of k_bspmv_pq: columns lane % KW + j KW
    constexpr int RW = 32 / KW;
    constexpr int JK_MAX = kMaxK / 32 > 0 ? kMaxK / 32 : 1;
    const int lane = threadIdx.x & 31;
    const double *v = (const double *)A.v;
    double accj[JK_MAX];
#pragma unroll
    for (int j = 0; j < JK_MAX; ++j) accj[j] = 0.0;
    for (int w = blockIdx.x * (kBT / 32) + (threadIdx.x >> 5); w < nsl * KW; w += kBB * (kBT / 32)) {
        int s = w / KW, ls = (w % KW) * RW + lane / KW;
        if (ls >= A.nrow[s]) continue;
        int r = A.row0[s] + ls, o = A.off[s] + ls, wd = A.width[s];
        int j = 0;
        for (int c = lane % KW; c < K; c += KW, ++j) {
            double acc = 0.0;
            for (int k = 0; k < wd; ++k) acc += __ldg(v + o + 32 * k) * x[(int64_t)__ldg(A.col + o + 32 * k) * K + c];
            double d = b[(int64_t)r * K + c] - acc;
            accj[j] += d * d;
        }
    }
    __shared__ double sh[kBT];
    if (K <= 32) {
        double acc1[1] = {accj[0]};
        if (!bfinish<1>(acc1, K, part, ctr)) return;
    } else {
        for (int j = 0; j < K / 32; ++j) {
            sh[threadIdx.x] = accj[j];
            __syncthreads();
            if (threadIdx.x < 32) {
                double vv = 0.0;
                for (int ww = 0; ww < kBT / 32; ++ww) vv += sh[ww * 32 + threadIdx.x];
                part[(int64_t)blockIdx.x * K + threadIdx.x + 32 * j] = vv;
            }
            __syncthreads();
        }
        __shared__ bool last;
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) last = atomicAdd(ctr, 1u) == (unsigned)(kBB - 1);
        __syncthreads();
        if (!last) return;
        __threadfence();
    }
    for (int c = threadIdx.x; c < K; c += kBT) sc[B_TRUE * K + c] = sqrt(btotal(part, 0, c, K));
    __syncthreads();
    if (threadIdx.x == 0) *ctr = 0u;
}

__global__ void k_binit(double *sc, int K, double tol, int maxit) {
    for (int i = 0; i < B_COUNT * K + G_COUNT; ++i) sc[i] = 0.0;
    double *g = sc + B_COUNT * K;
    g[G_TOL] = tol;
    g[G_MAXIT] = (double)maxit;
    g[G_CONT] = maxit > 0 ? 1.0 : 0.0;
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
static void bprecond(vemg_hierarchy *h, BatchWork *W, int first, cudaStream_t s) {
    const int K = W->K;
    const bool neu = h->bc == VEMG_NEUMANN, flex = h->precision != VEMG_PREC_FP64;
    const int mt = neu ? h->mtop : 0;
    const SChain &B = h->sbar;
    const XT *ys = nullptr;
    if (neu) {
        const SChain &S = h->ssurf;
        VEMG_CHECK_CUDA(cudaEventRecord(h->ev_fork, s));
        VEMG_CHECK_CUDA(cudaStreamWaitEvent(h->side, h->ev_fork, 0));
        XT *b0 = (XT *)W->lb[0][0], *x0 = (XT *)W->lx[0][0];
        bsell<BOP_SPMV, double, double, double, XT, double>(h->ETs, 0, h->ETs.nslices, nullptr, (const double *)nullptr,
                                                            W->R, b0, K, -1, h->side);
        bvcycle<XT, XT>(S, W, 0, 0, (const XT *)b0, x0, h->side);
        VEMG_CHECK_CUDA(cudaEventRecord(h->ev_join, h->side));
        ys = x0;
    }
    XT *xb = (XT *)W->lx[1][0];
    bvcycle<XT, double>(B, W, 1, 0, W->R + (int64_t)mt * K, xb, s);
    if (neu) VEMG_CHECK_CUDA(cudaStreamWaitEvent(s, h->ev_join, 0));
    k_bcombine<XT><<<kBB, kBT, 0, s>>>(h->nu, K, mt, sp(h->Enon), ys, xb, W->Z, W->R, W->Q, neu, flex, first,
                                       1.0 / (double)h->nu, W->sc, W->part + (int64_t)5 * kBB * K * BC_Z,
                                       W->ctr + BC_Z);
    BATCH_LAUNCHED();
}

static void bprecond_any(vemg_hierarchy *h, BatchWork *W, int first, cudaStream_t s) {
    if (h->precision == VEMG_PREC_FP32) bprecond<float>(h, W, first, s);
    else bprecond<double>(h, W, first, s);
}

static double *bpart(BatchWork *W, int c) { return W->part + (int64_t)5 * kBB * W->K * c; }

static void bspmv_pq(vemg_hierarchy *h, BatchWork *W, cudaStream_t s) {
    const int K = W->K, KW = std::min(K, 32);
    SellP A = sp(h->Aop);
    int nsl = h->Aop.nslices;
    switch (KW) {
        case 1: k_bspmv_pq<1><<<kBB, kBT, 0, s>>>(nsl, A, K, W->P, W->Q, W->sc, bpart(W, BC_SPMV), W->ctr + BC_SPMV); break;
        case 2: k_bspmv_pq<2><<<kBB, kBT, 0, s>>>(nsl, A, K, W->P, W->Q, W->sc, bpart(W, BC_SPMV), W->ctr + BC_SPMV); break;
        case 4: k_bspmv_pq<4><<<kBB, kBT, 0, s>>>(nsl, A, K, W->P, W->Q, W->sc, bpart(W, BC_SPMV), W->ctr + BC_SPMV); break;
        case 8: k_bspmv_pq<8><<<kBB, kBT, 0, s>>>(nsl, A, K, W->P, W->Q, W->sc, bpart(W, BC_SPMV), W->ctr + BC_SPMV); break;
        case 16: k_bspmv_pq<16><<<kBB, kBT, 0, s>>>(nsl, A, K, W->P, W->Q, W->sc, bpart(W, BC_SPMV), W->ctr + BC_SPMV); break;
        default: k_bspmv_pq<32><<<kBB, kBT, 0, s>>>(nsl, A, K, W->P, W->Q, W->sc, bpart(W, BC_SPMV), W->ctr + BC_SPMV); break;
    }
    BATCH_LAUNCHED();
}

static void btrue(vemg_hierarchy *h, BatchWork *W, cudaStream_t s) {
    const int K = W->K, KW = std::min(K, 32);
    SellP A = sp(h->Aop);
    int nsl = h->Aop.nslices;
    switch (KW) {
        case 1: k_btrue<1><<<kBB, kBT, 0, s>>>(nsl, A, K, W->X, W->B, W->sc, bpart(W, BC_TRUE), W->ctr + BC_TRUE); break;
        case 2: k_btrue<2><<<kBB, kBT, 0, s>>>(nsl, A, K, W->X, W->B, W->sc, bpart(W, BC_TRUE), W->ctr + BC_TRUE); break;
        case 4: k_btrue<4><<<kBB, kBT, 0, s>>>(nsl, A, K, W->X, W->B, W->sc, bpart(W, BC_TRUE), W->ctr + BC_TRUE); break;
        case 8: k_btrue<8><<<kBB, kBT, 0, s>>>(nsl, A, K, W->X, W->B, W->sc, bpart(W, BC_TRUE), W->ctr + BC_TRUE); break;
        case 16: k_btrue<16><<<kBB, kBT, 0, s>>>(nsl, A, K, W->X, W->B, W->sc, bpart(W, BC_TRUE), W->ctr + BC_TRUE); break;
        default: k_btrue<32><<<kBB, kBT, 0, s>>>(nsl, A, K, W->X, W->B, W->sc, bpart(W, BC_TRUE), W->ctr + BC_TRUE); break;
    }
    BATCH_LAUNCHED();
}

static void bphase_pre(vemg_hierarchy *h, BatchWork *W, cudaStream_t s) {
    const int K = W->K, nu = h->nu;
    const bool neu = h->bc == VEMG_NEUMANN;
    if (neu) {
        k_bmean<<<kBB, kBT, 0, s>>>(nu, K, W->B, 1.0 / (double)nu, B_BMEAN, W->sc, bpart(W, BC_SUMB), W->ctr + BC_SUMB);
        BATCH_LAUNCHED();
    }
    k_bprepare<<<kBB, kBT, 0, s>>>(nu, K, neu, W->B, W->R, W->X, W->P, W->sc, bpart(W, BC_PREP), W->ctr + BC_PREP);
    BATCH_LAUNCHED();
    bprecond_any(h, W, 1, s);
    int64_t N = (int64_t)nu * K;
    k_bupdate_p<<<grid_for(N, 256), 256, 0, s>>>(N, K, W->sc, W->Z, W->P);
    BATCH_LAUNCHED();
}

static void bphase_step(vemg_hierarchy *h, BatchWork *W, cudaStream_t s, cudaGraphConditionalHandle hd, int use_cond) {
    bspmv_pq(h, W, s);
    k_bupdate_xr<<<kBB, kBT, 0, s>>>(h->nu, W->K, W->P, W->Q, W->X, W->R, W->sc, bpart(W, BC_XR), W->ctr + BC_XR, hd,
                                     use_cond);
    BATCH_LAUNCHED();
}

static void bphase_direction(vemg_hierarchy *h, BatchWork *W, cudaStream_t s) {
    bprecond_any(h, W, 0, s);
    int64_t N = (int64_t)h->nu * W->K;
    k_bupdate_p<<<grid_for(N, 256), 256, 0, s>>>(N, W->K, W->sc, W->Z, W->P);
    BATCH_LAUNCHED();
}

static void bphase_post(vemg_hierarchy *h, BatchWork *W, cudaStream_t s) {
    const int K = W->K, nu = h->nu;
    if (h->bc == VEMG_NEUMANN) {
        k_bmean<<<kBB, kBT, 0, s>>>(nu, K, W->X, 1.0 / (double)nu, B_XMEAN, W->sc, bpart(W, BC_SUMX), W->ctr + BC_SUMX);
        BATCH_LAUNCHED();
        int64_t N = (int64_t)nu * K;
        k_bsub_mean<<<grid_for(N, 256), 256, 0, s>>>(N, K, W->X, W->sc, B_XMEAN);
        BATCH_LAUNCHED();
    }
    btrue(h, W, s);
}

static void release_batch_graphs(BatchWork *W) {
    BatchGraphs *G = W->graphs;
    if (!G) return;
    if (G->pre) cudaGraphExecDestroy(G->pre);
    if (G->loop) cudaGraphExecDestroy(G->loop);
    if (G->post) cudaGraphExecDestroy(G->post);
    if (G->gpre) cudaGraphDestroy(G->gpre);
    if (G->gloop) cudaGraphDestroy(G->gloop);
    if (G->gpost) cudaGraphDestroy(G->gpost);
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
        VEMG_CHECK_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        bphase_pre(h, W, cs);
        bphase_step(h, W, cs, 0, 0);
        VEMG_CHECK_CUDA(cudaStreamEndCapture(cs, &G->gpre));
        G->k_pre = count;
        count = 0;
        VEMG_CHECK_CUDA(cudaGraphCreate(&G->gloop, 0));
        VEMG_CHECK_CUDA(cudaGraphConditionalHandleCreate(&G->handle, G->gloop, 0, cudaGraphCondAssignDefault));
        VEMG_CHECK_CUDA(cudaStreamBeginCaptureToGraph(cs, G->gloop, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        k_bcond_init<<<1, 1, 0, cs>>>(gsc(W), G->handle);
        BATCH_LAUNCHED();
        cudaGraph_t captured = G->gloop;
        VEMG_CHECK_CUDA(cudaStreamEndCapture(cs, &captured));
        cudaGraphNode_t init_node;
        size_t nn = 1;
        VEMG_CHECK_CUDA(cudaGraphGetNodes(G->gloop, &init_node, &nn));
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = G->handle;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t cnode;
        VEMG_CHECK_CUDA(cudaGraphAddNode(&cnode, G->gloop, &init_node, nullptr, 1, &cp));
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        VEMG_CHECK_CUDA(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        bphase_direction(h, W, cs);
        bphase_step(h, W, cs, G->handle, 1);
        VEMG_CHECK_CUDA(cudaStreamEndCapture(cs, &body));
        G->k_body = count - 1;
        G->k_pre += 1;
        count = 0;
        VEMG_CHECK_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        bphase_post(h, W, cs);
        VEMG_CHECK_CUDA(cudaStreamEndCapture(cs, &G->gpost));
        G->k_post = count;
        VEMG_CHECK_CUDA(cudaGraphInstantiate(&G->pre, G->gpre, 0));
        VEMG_CHECK_CUDA(cudaGraphInstantiate(&G->loop, G->gloop, 0));
        VEMG_CHECK_CUDA(cudaGraphInstantiate(&G->post, G->gpost, 0));
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

static BatchWork *batch_work(vemg_hierarchy *h, int K, cudaStream_t s) {
    if (h->batch && h->batch->K == K) return h->batch;
    VEMG_CHECK_CUDA(cudaStreamSynchronize(s));
    release_batch(h);
    BatchWork *W = new BatchWork();
    h->batch = W;
    W->K = K;
    Arena &ar = W->arena;
    int64_t N = (int64_t)h->n * K;
    W->X = ar.alloc<double>(N);
    W->R = ar.alloc<double>(N);
    W->Z = ar.alloc<double>(N);
    W->P = ar.alloc<double>(N);
    W->Q = ar.alloc<double>(N);
    W->B = ar.alloc<double>(N);
    size_t es = h->precision == VEMG_PREC_FP32 ? sizeof(float) : sizeof(double);
    const SChain *chains[2] = {&h->ssurf, &h->sbar};
    for (int ch = 0; ch < 2; ++ch)
        for (int l = 0; l < chains[ch]->nlev; ++l) {
            int64_t m = (int64_t)chains[ch]->lv[l].n * K;
            W->lx[ch][l] = ar.alloc<char>((int64_t)es * m);
            W->lb[ch][l] = ar.alloc<char>((int64_t)es * m);
            W->lr[ch][l] = ar.alloc<char>((int64_t)es * m);
        }
    W->sc = ar.alloc<double>(B_COUNT * K + G_COUNT);
    W->part = ar.alloc<double>((int64_t)5 * kBB * K * BC_COUNT);
    W->ctr = ar.alloc<unsigned>(BC_COUNT);
    VEMG_CHECK_CUDA(cudaMemsetAsync(W->ctr, 0, sizeof(unsigned) * BC_COUNT, s));
    VEMG_CHECK_CUDA(cudaStreamSynchronize(s));
    return W;
}

int solve_batch(vemg_hierarchy *h, int k, const double *Bin, int64_t ldb, double *Xout, int64_t ldx, double rtol,
                int max_it, vemg_info *infos, cudaStream_t s) {
    if (k == 0) return VEMG_OK;
    if (k > kMaxK) throw Error{VEMG_EINVAL};
    prepare_solve(h, s);
    int K = 1;
    while (K < k) K *= 2;
    BatchWork *W = batch_work(h, K, s);
    b_count = &h->launches;
    const int nu = h->nu;
    k_binit<<<1, 1, 0, s>>>(W->sc, K, rtol, max_it);
    BATCH_LAUNCHED();
    k_bgather<<<grid_for((int64_t)nu * K, 256), 256, 0, s>>>(nu, K, k, ldb, h->caller_of, Bin, W->B);
    BATCH_LAUNCHED();
    if (!W->graphs) build_batch_graphs(h, W);
    BatchGraphs *G = W->graphs;
    VEMG_CHECK_CUDA(cudaGraphLaunch(G->pre, s));
    VEMG_CHECK_CUDA(cudaGraphLaunch(G->loop, s));
    VEMG_CHECK_CUDA(cudaGraphLaunch(G->post, s));
    std::vector<double> hs(B_COUNT * K + G_COUNT);
    VEMG_CHECK_CUDA(cudaMemcpyAsync(hs.data(), W->sc, sizeof(double) * hs.size(), cudaMemcpyDeviceToHost, s));
    int ntop = h->bc == VEMG_DIRICHLET_TOP ? h->mtop : 0;
    int64_t nsc = (int64_t)std::max(nu, ntop) * k;
    k_bscatter<<<grid_for(nsc, 256), 256, 0, s>>>(nu, K, k, ldx, h->caller_of, h->tops, ntop, W->X, Xout);
    BATCH_LAUNCHED();
    VEMG_CHECK_CUDA(cudaStreamSynchronize(s));
    int rounds = (int)hs[B_COUNT * K + G_ITERS];
    h->launches += G->k_pre + G->k_post + (rounds > 1 ? (int64_t)(rounds - 1) * G->k_body : 0);
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
