// One preconditioner application as a single persistent kernel.
//
// The V-cycles of Eq. ourpreconditioner (section 5.5) are a long chain of small dependent steps:
// every colour of every multicolour SOR sweep, the residual, the restriction and prolongation of
// each level, the dense coarsest solve. Launched one kernel per step, the cycle is bound by launch
// latency (about 100 dependent launches per cycle on the 2.2M-node workload). Here the steps are
// written once, at the first solve, into a phase program; one cooperative launch runs the whole
// program, with a barrier between dependent phases instead of a kernel boundary.
//
// The CTAs are split into groups, one per chain: the surface branch (E~^T r, then one V-cycle on
// E~^T A E~) and the A_bar branch run side by side, each group with its own barrier. The per-row
// arithmetic is that of the launch-per-phase kernels in solve.cu.
//
// Barrier: one 64-bit arrival counter per group that only grows (release add to arrive, acquire
// loads to wait); barrier k of a launch waits for base + k * nblocks arrivals, base being the
// counter at launch rounded down to a multiple of nblocks. Every wait is bounded; a wait that runs
// out, or sees another CTA's error, sets the error word and every CTA returns. The host turns the
// error word into VEMG_ETIMEOUT and resets the counters.
//
// Latency: a phase reads operator data (slice metadata, column indices, values, diagonals) that
// the kernel never writes. A CTA arrives at the barrier after its phase, then loads that data
// for the first slice it owns in the next phase, then waits: the loads overlap the barrier.
// After the barrier only the gathers of x and the right-hand side remain.
//
// Coherence: data a phase writes is read by other CTAs in later phases of the same kernel, so
// every such read goes to L2 (ld.global.cg) and every such write is an st.global.cg; operators
// and the outer residual, which the kernel never writes, go through the read-only path.
#include <map>

#include "internal.cuh"

namespace vemg {

static constexpr int kPThreads = 256;
static constexpr int kPU = 16;            // entries loaded per batch in a row
static constexpr long kSpinLimit = 1L << 24;

enum : int { PH_SOR = 0, PH_RES, PH_SPMV, PH_SPMV_ADD, PH_RESTRICT_F64, PH_DENSE };

struct PPhase {
    int op;
    int s0, s1;          // slice range (sliced-ELL phases)
    int lim;             // SOR from zero: first row of the colour (columns >= lim are zero); else -1
    int b_outer;         // the right-hand side is the FP64 outer residual r + b_off
    int b_off;
    int n;               // PH_DENSE: rows of the dense inverse
    int level;           // multigrid level of the phase (for profiles)
    const int4 *meta;    // per slice: first row, rows, element offset, width
    const int *col;
    const void *v;       // values (XT; double for PH_RESTRICT_F64; the dense inverse for PH_DENSE)
    const void *d;       // PH_SOR: inverse diagonal; PH_RES: diagonal
    const void *b;       // right-hand side (PH_SOR, PH_RES, PH_DENSE) or SpMV input
    void *x;             // PH_SOR: solution; PH_RES: iterate; SpMV / dense: output
    void *r;             // PH_RES: residual output
};

struct Persist {
    PPhase *phases = nullptr;      // device
    int4 *groups = nullptr;        // device: {first CTA, end CTA, first phase, end phase}
    unsigned long long *bar = nullptr;   // device: arrival counter per group (own 128-byte line)
    int *err = nullptr;            // device
    int ngroups = 0, grid = 0;
    double bytes = 0.0;            // algorithmic bytes of one application
    int nphases = 0;
    bool fp32 = false;
    bool coarse = false;           // levels >= 1 of the chains only (the hybrid structure)
    unsigned long long *cycles = nullptr;   // device: per phase, SM clock cycles summed over launches
    std::vector<int> op, level, group;      // host copies for profiles
};

// ------------------------------------------------------------------------------------------
// device side

static constexpr int kBarStride = 16;   // counters 128 bytes apart
static constexpr int kPhaseWords = (int)(sizeof(PPhase) / sizeof(int));
static_assert(sizeof(PPhase) % sizeof(int) == 0, "phase descriptor is copied as words");
static_assert(kPhaseWords <= kPThreads, "one thread per descriptor word");

__device__ __forceinline__ int ld_volatile(const int *p) { return *(const volatile int *)p; }
__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void red_release(unsigned long long *p, unsigned long long v) {
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

template <class T>
__device__ __forceinline__ T ldcg(const T *p) { return __ldcg(p); }
template <class T>
__device__ __forceinline__ void stcg(T *p, T v) { __stcg(p, v); }

// Arrival: every thread of the CTA has finished the phase (bar.sync), then one release add.
__device__ __forceinline__ void bar_arrive(unsigned long long *ctr) {
    __syncthreads();
    if (threadIdx.x == 0) red_release(ctr, 1ull);
}

// Wait until `target` arrivals; false if the wait ran out or another CTA failed.
__device__ bool bar_wait(const unsigned long long *ctr, unsigned long long target, int *err, long limit) {
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        int ok = 1;
        long spins = 0;
        while (ld_acquire(ctr) < target) {
            if (++spins > limit || ((spins & 255) == 0 && ld_volatile(err))) {
                atomicExch(err, 1);
                ok = 0;
                break;
            }
        }
        if (ok && ld_volatile(err)) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// the operator data of one row's first kPU entries, loaded ahead of the phase
template <class XT>
struct Pre {
    int s;          // slice, or -1
    int i, o, w;    // row, element offset of the row, stored entries
    int c[kPU];
    XT a[kPU];
    XT d;           // inverse diagonal (SOR) or diagonal (residual)
    double bo;      // outer right-hand side entry, when the phase reads the outer residual
};

template <class XT>
__device__ __forceinline__ bool sell_op(int op) {
    return op == PH_SOR || op == PH_RES || op == PH_SPMV || op == PH_SPMV_ADD;
}

template <class XT>
__device__ __forceinline__ void prefetch(const PPhase &p, const double *__restrict__ r, int gw, int lane,
                                         Pre<XT> &q) {
    // every field is written on every path, so nothing of the previous phase stays live
    int s = p.s0 + gw;
    int4 m = make_int4(0, 0, 0, 0);
    bool on = sell_op<XT>(p.op) && s < p.s1;
    if (on) m = __ldg(p.meta + s);
    on = on && lane < m.y;
    q.s = on ? s : -1;
    q.i = m.x + lane;
    q.o = m.z + lane;
    q.w = on ? m.w : 0;
    const XT *v = (const XT *)p.v;
#pragma unroll
    for (int u = 0; u < kPU; ++u) {
        q.c[u] = u < q.w ? __ldg(p.col + q.o + 32 * u) : 0;
        q.a[u] = u < q.w ? __ldg(v + q.o + 32 * u) : (XT)0;
    }
    q.d = on && (p.op == PH_SOR || p.op == PH_RES) ? __ldg((const XT *)p.d + q.i) : (XT)0;
    q.bo = on && p.b_outer && (p.op == PH_SOR || p.op == PH_RES) ? __ldg(r + p.b_off + q.i) : 0.0;
}

// entries [k0, w) of a row dotted with x (x through L2), continuing the sum acc
template <class VT, class XT, class AT, int B>
__device__ __forceinline__ AT prow_from(AT acc, const int *__restrict__ col, const VT *__restrict__ v, int o, int w,
                                        const XT *x, int lim, int k0) {
    for (; k0 < w; k0 += B) {
        int c[B];
        VT a[B];
#pragma unroll
        for (int u = 0; u < B; ++u) {
            int k = k0 + u;
            c[u] = k < w ? __ldg(col + o + 32 * k) : 0;
            a[u] = k < w ? __ldg(v + o + 32 * k) : (VT)0;
        }
#pragma unroll
        for (int u = 0; u < B; ++u)
            if (k0 + u < w && (lim < 0 || c[u] < lim)) acc = fmadd((AT)a[u], (AT)ldcg(x + c[u]), acc);
    }
    return acc;
}

template <class XT>
__device__ __forceinline__ XT rhs(const PPhase &p, const double *__restrict__ r, int i) {
    return p.b_outer ? (XT)__ldg(r + p.b_off + i) : ldcg((const XT *)p.b + i);
}

// one row of a sliced-ELL phase; `first` holds its first kPU entries when pre != nullptr
template <class XT>
__device__ __forceinline__ void sell_row_op(const PPhase &p, const double *__restrict__ r, int i, int o, int w,
                                            const Pre<XT> *pre) {
    const XT *v = (const XT *)p.v;
    const XT *x = (const XT *)(p.op == PH_SPMV || p.op == PH_SPMV_ADD ? p.b : p.x);
    const int lim = p.op == PH_SOR ? p.lim : -1;
    XT acc = (XT)0;
    if (!(p.op == PH_SOR && lim == 0)) {
        if (pre) {
#pragma unroll
            for (int u = 0; u < kPU; ++u)
                if (u < w && (lim < 0 || pre->c[u] < lim)) acc = fmadd(pre->a[u], ldcg(x + pre->c[u]), acc);
            if (w > kPU) acc = prow_from<XT, XT, XT, 8>(acc, p.col, v, o, w, x, lim, kPU);
        } else {
            acc = prow_from<XT, XT, XT, kPU>(acc, p.col, v, o, w, x, lim, 0);
        }
    }
    switch (p.op) {
        case PH_SOR: {
            XT d = pre ? pre->d : __ldg((const XT *)p.d + i);
            XT b = pre && p.b_outer ? (XT)pre->bo : rhs<XT>(p, r, i);
            stcg((XT *)p.x + i, (b - acc) * d);
            break;
        }
        case PH_RES: {
            XT d = pre ? pre->d : __ldg((const XT *)p.d + i);
            XT b = pre && p.b_outer ? (XT)pre->bo : rhs<XT>(p, r, i);
            XT t = fmadd(d, ldcg((const XT *)p.x + i), acc);
            stcg((XT *)p.r + i, b - t);
            break;
        }
        case PH_SPMV: stcg((XT *)p.x + i, acc); break;
        case PH_SPMV_ADD: stcg((XT *)p.x + i, ldcg((const XT *)p.x + i) + acc); break;
        default: break;
    }
}

// PRE: the warp's first slice of the phase was prefetched into `pre` (the grid kernel); the
// single-CTA tail kernel runs without prefetch
template <class XT, bool PRE>
__device__ void run_phase(const PPhase &p, const double *__restrict__ r, int gw, int nw, int lane,
                          const Pre<XT> &pre) {
    if (sell_op<XT>(p.op)) {
        int s = p.s0 + gw;
        if (PRE && s < p.s1 && pre.s == s) {
            sell_row_op<XT>(p, r, pre.i, pre.o, pre.w, &pre);
            s += nw;
        } else if (PRE && s < p.s1) {
            // no prefetched row for this lane (a short slice): nothing to do in this slice
            s += nw;
        }
        for (; s < p.s1; s += nw) {
            int4 m = __ldg(p.meta + s);
            if (lane >= m.y) continue;
            sell_row_op<XT>(p, r, m.x + lane, m.z + lane, m.w, nullptr);
        }
        return;
    }
    if (p.op == PH_RESTRICT_F64) {   // E~^T r of the outer FP64 residual, accumulated in FP64
        const double *v = (const double *)p.v;
        XT *y = (XT *)p.x;
        for (int s = p.s0 + gw; s < p.s1; s += nw) {
            int4 m = __ldg(p.meta + s);
            if (lane >= m.y) continue;
            double acc = 0.0;
            int o = m.z + lane, w = m.w;
            for (int k0 = 0; k0 < w; k0 += kPU) {
                int c[kPU];
                double a[kPU];
#pragma unroll
                for (int u = 0; u < kPU; ++u) {
                    int k = k0 + u;
                    c[u] = k < w ? __ldg(p.col + o + 32 * k) : 0;
                    a[u] = k < w ? __ldg(v + o + 32 * k) : 0.0;
                }
#pragma unroll
                for (int u = 0; u < kPU; ++u)
                    if (k0 + u < w) acc = fmadd(a[u], __ldg(r + c[u]), acc);
            }
            stcg(y + m.x + lane, (XT)acc);
        }
        return;
    }
    if (p.op == PH_DENSE) {   // x = G b, one warp per row, G and sums in XT
        const XT *G = (const XT *)p.v;
        XT *x = (XT *)p.x;
        for (int row = gw; row < p.n; row += nw) {
            XT s = 0;
            for (int k = lane; k < p.n; k += 32) s = fmadd(__ldg(G + (int64_t)row * p.n + k), rhs<XT>(p, r, k), s);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) stcg(x + row, (XT)s);
        }
    }
}

template <class XT>
__global__ void __launch_bounds__(kPThreads, 3) k_precond_persistent(const PPhase *__restrict__ phases,
                                                                      const int4 *__restrict__ groups, int ngroups,
                                                                      const double *__restrict__ r,
                                                                      unsigned long long *bar, int *err,
                                                                      unsigned long long *cycles) {
    __shared__ PPhase sp[2];
    int g = 0;
    while (g + 1 < ngroups && (int)blockIdx.x >= __ldg(&groups[g].y)) ++g;
    const int4 G = groups[g];
    const unsigned nblocks = (unsigned)(G.y - G.x);
    const int warps = kPThreads / 32;
    const int gw = ((int)blockIdx.x - G.x) * warps + (int)(threadIdx.x >> 5);
    const int nw = (int)nblocks * warps;
    const int lane = threadIdx.x & 31;
    unsigned long long *ctr = bar + kBarStride * g;
    if (ld_volatile(err) || G.z >= G.w) return;
    // every CTA reads the counter before it first arrives, and barrier 1 needs every CTA: the
    // values seen all lie in [base, base + nblocks)
    const unsigned long long base = ld_acquire(ctr) / nblocks * nblocks;
    if (threadIdx.x < kPhaseWords) ((int *)&sp[0])[threadIdx.x] = __ldg((const int *)(phases + G.z) + threadIdx.x);
    __syncthreads();
    Pre<XT> pre;
    prefetch<XT>(sp[0], r, gw, lane, pre);
    unsigned long long nbar = 0;
    // profile: the first CTA of the group times each phase up to the end of its barrier (the
    // phase's critical path across the group)
    const bool timer = cycles && (int)blockIdx.x == G.x && threadIdx.x == 0;
    long long t0 = timer ? clock64() : 0;
    for (int k = G.z; k < G.w; ++k) {
        const int cur = (k - G.z) & 1;
        const bool more = k + 1 < G.w;
        if (more && threadIdx.x < kPhaseWords)
            ((int *)&sp[cur ^ 1])[threadIdx.x] = __ldg((const int *)(phases + k + 1) + threadIdx.x);
        run_phase<XT, true>(sp[cur], r, gw, nw, lane, pre);
        if (!more) {
            if (timer) atomicAdd(cycles + k, (unsigned long long)(clock64() - t0));
            break;
        }
        bar_arrive(ctr);                     // also makes the next descriptor visible in the CTA
        prefetch<XT>(sp[cur ^ 1], r, gw, lane, pre);
        ++nbar;
        if (!bar_wait(ctr, base + nbar * nblocks, err, kSpinLimit)) return;
        if (timer) {
            long long t1 = clock64();
            atomicAdd(cycles + k, (unsigned long long)(t1 - t0));
            t0 = t1;
        }
    }
}

// The coarse tail of one chain (every level from a small one down, and back up) in one CTA: the
// phases are separated by __syncthreads() instead of kernel boundaries. Launched on the stream of
// the launch-per-phase cycle in place of the tail's dozens of small dependent launches. Every
// phase descriptor sits in shared memory, and each warp loads the operator data of its first row
// of the next phase (slice metadata, first entries, diagonal: setup data) before the barrier, so
// after it only the gathers of x remain; phase 0's is loaded before the wait on the previous
// kernel. (A thread-block cluster of 8 CTAs with the hardware cluster barrier, tried for larger
// tails, was slower than the launches it replaced.)
static constexpr int kTailThreads = 512;
static constexpr int kTailMaxPhases = 160;

template <class XT>
__global__ void __launch_bounds__(kTailThreads, 1) k_tail(const PPhase *__restrict__ phases, int nphases) {
    __shared__ PPhase sp[kTailMaxPhases];
    const int gw = (int)(threadIdx.x >> 5), nw = kTailThreads / 32, lane = threadIdx.x & 31;
    for (int q = threadIdx.x; q < nphases * kPhaseWords; q += kTailThreads)
        ((int *)sp)[q] = __ldg((const int *)phases + q);
    __syncthreads();
    Pre<XT> pre;
    prefetch<XT>(sp[0], nullptr, gw, lane, pre);
    pdl_begin();
    for (int k = 0; k < nphases; ++k) {
        run_phase<XT, true>(sp[k], nullptr, gw, nw, lane, pre);
        if (k + 1 < nphases) prefetch<XT>(sp[k + 1], nullptr, gw, lane, pre);
        __syncthreads();   // the phase's writes are visible to the CTA
    }
}

// The coarse tail in one thread-block cluster: the program of the single-CTA tail, its steps
// spread over every warp of the cluster and separated by the hardware cluster barrier (release /
// acquire at cluster scope) instead of __syncthreads. The vectors stay in global memory and are
// read and written through L2 (ld.global.cg / st.global.cg), which the barrier orders; remote
// shared-memory gathers measured slower than L2 hits on this GPU. Each warp loads the operator
// data of its first row of the next step between arriving at the barrier and waiting on it. The
// barrier is hardware over CTAs that are co-scheduled by construction: no wait here spins, and
// every thread of every CTA reaches every barrier.
static constexpr int kClusterThreads = 512;

__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.release;" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire;" ::: "memory"); }

template <class XT>
__global__ void __launch_bounds__(kClusterThreads, 1) k_tail_cluster(const PPhase *__restrict__ phases, int nphases,
                                                                      unsigned long long *cycles) {
    // step descriptors, three deep: the one of step k + 2 is written during step k, so that the
    // barrier ending step k - 1 has made those of steps k and k + 1 visible to the whole CTA
    __shared__ PPhase sp[3];
    unsigned rank;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(rank));
    // slices go round-robin over the CTAs (slice j of a step to CTA j mod ncta), so that the gathers
    // of a small step, whose cost is bound by each SM's load pipeline, spread over every SM
    const int warps = kClusterThreads / 32, lane = threadIdx.x & 31;
    const int gw = (int)(threadIdx.x >> 5) * (int)gridDim.x + (int)rank, nw = (int)gridDim.x * warps;
    for (int q = 0; q < 2 && q < nphases; ++q)
        if (threadIdx.x < kPhaseWords) ((int *)&sp[q])[threadIdx.x] = __ldg((const int *)(phases + q) + threadIdx.x);
    __syncthreads();
    Pre<XT> pre;
    prefetch<XT>(sp[0], nullptr, gw, lane, pre);
    asm volatile("griddepcontrol.wait;" ::: "memory");   // b of the tail level comes from the previous kernel
    // profile: CTA 0 times each step up to the end of its barrier (the step's critical path)
    const bool timer = cycles && rank == 0 && threadIdx.x == 0;
    long long t0 = timer ? clock64() : 0;
    for (int k = 0; k < nphases; ++k) {
        const bool more = k + 1 < nphases;
        if (k + 2 < nphases && threadIdx.x < kPhaseWords)
            ((int *)&sp[(k + 2) % 3])[threadIdx.x] = __ldg((const int *)(phases + k + 2) + threadIdx.x);
        if (!more) asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
        run_phase<XT, true>(sp[k % 3], nullptr, gw, nw, lane, pre);
        if (more) {
            cluster_arrive();
            prefetch<XT>(sp[(k + 1) % 3], nullptr, gw, lane, pre);
            cluster_wait();
        }
        if (timer) {
            long long t1 = clock64();
            atomicAdd(cycles + k, (unsigned long long)(t1 - t0));
            t0 = t1;
        }
    }
}

// Self-test of the bounded wait: launched CTAs meet at one barrier that expects `claimed` CTAs.
// With claimed > launched the barrier can never complete; every waiting CTA gives up after
// `limit` polls and the error word is set.
__global__ void k_barrier_selftest(unsigned long long *ctr, int *err, unsigned claimed, long limit) {
    const unsigned long long base = ld_acquire(ctr) / claimed * claimed;
    bar_arrive(ctr);
    bar_wait(ctr, base + claimed, err, limit);
}

int barrier_selftest(int claimed, int launched, cudaStream_t s) {
    if (claimed < 1 || claimed > 8 || launched < 1 || launched > claimed) return VEMG_EINVAL;
    Scratch<unsigned long long> ctr(1);
    Scratch<int> err(1);
    VEMG_CHECK_CUDA(cudaMemsetAsync(ctr, 0, sizeof(unsigned long long), s));
    VEMG_CHECK_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)launched);
    cfg.blockDim = dim3(32);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    // 2^16 polls of the counter (about half a microsecond each): a few tens of milliseconds
    VEMG_CHECK_CUDA(cudaLaunchKernelEx(&cfg, k_barrier_selftest, (unsigned long long *)ctr, (int *)err,
                                       (unsigned)claimed, (long)(1L << 16)));
    int h_err = 0;
    VEMG_CHECK_CUDA(cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    VEMG_CHECK_CUDA(cudaStreamSynchronize(s));
    return h_err ? VEMG_ETIMEOUT : VEMG_OK;
}

// ------------------------------------------------------------------------------------------
// host side: the program

__global__ void k_pack_meta(int ns, const int *__restrict__ row0, const int *__restrict__ nrow,
                            const int *__restrict__ off, const int *__restrict__ width, int4 *meta) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < ns) meta[s] = make_int4(row0[s], nrow[s], off[s], width[s]);
}

namespace {

struct Builder {
    Arena &ar;
    cudaStream_t st;
    std::vector<PPhase> ph;
    std::map<const int *, const int4 *> metas;
    double bytes = 0.0;
    size_t xs = 8;

    Builder(Arena &a, cudaStream_t s) : ar(a), st(s) {}

    const int4 *meta_of(const Sell &S) {
        auto it = metas.find(S.row0);
        if (it != metas.end()) return it->second;
        int4 *m = ar.alloc<int4>(std::max(S.nslices, 1));
        if (S.nslices > 0) {
            k_pack_meta<<<grid_for(S.nslices, 256), 256, 0, st>>>(S.nslices, S.row0, S.nrow, S.off, S.width, m);
            VEMG_CHECK_LAUNCH();
        }
        metas[S.row0] = m;
        return m;
    }
    PPhase sell_phase(int op, const Sell &S, int s0, int s1) {
        PPhase p{};
        p.op = op;
        p.s0 = s0;
        p.s1 = s1;
        p.lim = -1;
        p.meta = meta_of(S);
        p.col = S.col;
        p.v = S.v;
        return p;
    }
    void set_b(PPhase &p, const void *b, int outer_off) {
        if (outer_off >= 0) {
            p.b_outer = 1;
            p.b_off = outer_off;
        } else {
            p.b = b;
        }
    }
    // b: level right-hand side (XT) or, with outer_off >= 0, the outer FP64 residual at that offset
    int lev = 0;
    void sweep(const SLevel &L, const void *b, int outer_off, void *x, bool forward, bool from_zero) {
        for (int cc = 0; cc < L.ncolours; ++cc) {
            int c = forward ? cc : L.ncolours - 1 - cc;
            int s0 = L.cslice[c], s1 = L.cslice[c + 1];
            if (s1 == s0) continue;
            PPhase p = sell_phase(PH_SOR, L.A, s0, s1);
            p.lim = from_zero ? L.crow[c] : -1;
            p.d = L.dinv;
            set_b(p, b, outer_off);
            p.x = x;
            p.level = lev;
            ph.push_back(p);
            int rows = L.crow[c + 1] - L.crow[c];
            bytes += (p.lim == 0 ? 0.0 : (double)L.cnnz[c] * (xs + 4.0)) + (double)rows * 3.0 * xs +
                     (double)xs * L.n / L.ncolours;
        }
    }
    void spmv(const Sell &S, const void *in, void *out, bool add) {
        if (S.nslices == 0) return;
        PPhase p = sell_phase(add ? PH_SPMV_ADD : PH_SPMV, S, 0, S.nslices);
        p.b = in;
        p.x = out;
        p.level = lev;
        ph.push_back(p);
        bytes += (double)S.nnz * (xs + 4.0) + (double)S.n * xs * (add ? 3.0 : 2.0);
    }
    void vcycle(const SChain &C, int l, const void *b, int outer_off, void *x) {
        const SLevel &L = C.lv[l];
        lev = l;
        if (l == C.nlev - 1) {
            if (C.direct) {
                PPhase p{};
                p.op = PH_DENSE;
                p.n = C.nc;
                p.v = C.fp32 ? (const void *)C.Gf : (const void *)C.G;
                set_b(p, b, outer_off);
                p.x = x;
                p.level = l;
                ph.push_back(p);
                bytes += xs * C.nc * (double)C.nc + 2.0 * xs * C.nc;
                return;
            }
            sweep(L, b, outer_off, x, true, true);
            sweep(L, b, outer_off, x, false, false);
            return;
        }
        sweep(L, b, outer_off, x, true, true);
        PPhase p = sell_phase(PH_RES, L.A, 0, L.A.nslices);
        p.d = L.diag;
        set_b(p, b, outer_off);
        p.x = x;
        p.r = L.r;
        p.level = l;
        ph.push_back(p);
        bytes += (double)L.A.nnz * (xs + 4.0) + (double)L.n * 5.0 * xs;
        const SLevel &N = C.lv[l + 1];
        spmv(L.PT, L.r, N.b, false);
        vcycle(C, l + 1, N.b, -1, N.x);
        lev = l;
        spmv(L.P, N.x, x, true);
        sweep(L, b, outer_off, x, false, false);
    }
};

}  // namespace

template <class XT>
static int max_blocks_per_sm() {
    int nb = 0;
    VEMG_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_precond_persistent<XT>, kPThreads, 0));
    return nb;
}

void build_persist(vemg_hierarchy *h, cudaStream_t s) {
    if (h->persist) return;
    const bool fp32 = h->precision != VEMG_PREC_FP64;
    const bool coarse = h->opts.cycle == VEMG_CYCLE_HYBRID;
    bool two = !single_chain(h);
    Builder B(h->arena, s);
    B.xs = fp32 ? 4 : 8;
    std::vector<int2> ranges;   // phase ranges per group
    if (coarse) {
        // levels >= 1 of each chain that has them; the finest levels run one kernel per phase
        const SChain *cs[2] = {two ? &h->ssurf : nullptr, &h->sbar};
        int with = 0;
        for (const SChain *C : cs) {
            if (!C || C->nlev < 2) continue;
            int p0 = (int)B.ph.size();
            B.vcycle(*C, 1, C->lv[1].b, -1, C->lv[1].x);
            ranges.push_back({p0, (int)B.ph.size()});
            ++with;
        }
        if (with == 0) return;   // no coarse levels: the hybrid cycle is the per-phase one
        two = with == 2;
    } else {
        if (two) {
            const SChain &S = h->ssurf;
            int p0 = (int)B.ph.size();
            PPhase p = B.sell_phase(PH_RESTRICT_F64, h->ETs, 0, h->ETs.nslices);
            p.x = S.lv[0].b;
            B.ph.push_back(p);
            B.bytes += (double)h->ETs.nnz * 12.0 + (double)h->ETs.n * B.xs + 8.0 * h->n;
            B.vcycle(S, 0, S.lv[0].b, -1, S.lv[0].x);
            ranges.push_back({p0, (int)B.ph.size()});
        }
        int p0 = (int)B.ph.size();
        B.vcycle(h->sbar, 0, nullptr, two ? h->mtop : 0, h->sbar.lv[0].x);
        ranges.push_back({p0, (int)B.ph.size()});
    }
    int dev = 0, nsm = 0;
    VEMG_CHECK_CUDA(cudaGetDevice(&dev));
    VEMG_CHECK_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    int per_sm = fp32 ? max_blocks_per_sm<float>() : max_blocks_per_sm<double>();
    if (per_sm < 1) throw Error{VEMG_EINTERNAL};
    int grid = nsm * per_sm;
    std::vector<int4> groups;
    if (two) {
        // the surface group: about 1/16 of the CTAs (its operators hold ~3% of the bytes, but it
        // has as many dependent phases as the A_bar chain)
        int gs = std::max(per_sm, grid / 16);
        groups.push_back({0, gs, ranges[0].x, ranges[0].y});
        groups.push_back({gs, grid, ranges[1].x, ranges[1].y});
    } else {
        groups.push_back({0, grid, ranges[0].x, ranges[0].y});
    }
    auto P = new Persist();
    try {
        Arena &ar = h->arena;
        P->nphases = (int)B.ph.size();
        P->phases = ar.alloc<PPhase>(std::max(P->nphases, 1));
        P->groups = ar.alloc<int4>((int)groups.size());
        P->bar = ar.alloc<unsigned long long>(kBarStride * (int)groups.size());
        P->err = ar.alloc<int>(1);
        P->cycles = ar.alloc<unsigned long long>(std::max(P->nphases, 1));
        // every copy on the caller's stream (which may not order itself after the legacy stream)
        VEMG_CHECK_CUDA(cudaMemsetAsync(P->cycles, 0, sizeof(unsigned long long) * std::max(P->nphases, 1), s));
        for (size_t g = 0; g < groups.size(); ++g)
            for (int k = groups[g].z; k < groups[g].w; ++k) {
                P->op.push_back(B.ph[k].op);
                P->level.push_back(B.ph[k].level);
                P->group.push_back((int)g);
            }
        VEMG_CHECK_CUDA(cudaMemcpyAsync(P->phases, B.ph.data(), sizeof(PPhase) * B.ph.size(), cudaMemcpyHostToDevice, s));
        VEMG_CHECK_CUDA(cudaMemcpyAsync(P->groups, groups.data(), sizeof(int4) * groups.size(), cudaMemcpyHostToDevice, s));
        VEMG_CHECK_CUDA(cudaMemsetAsync(P->bar, 0, sizeof(unsigned long long) * kBarStride * groups.size(), s));
        VEMG_CHECK_CUDA(cudaMemsetAsync(P->err, 0, sizeof(int), s));
        VEMG_CHECK_CUDA(cudaStreamSynchronize(s));   // the host vectors are read before they go
        P->ngroups = (int)groups.size();
        P->grid = grid;
        P->bytes = B.bytes;
        P->fp32 = fp32;
        P->coarse = coarse;
    } catch (...) {
        delete P;
        throw;
    }
    h->persist = P;
}

// Coarse tails: the first level below the finest with at most tail_rows rows starts a tail. A
// colour of such a level has about one row per thread of the tail CTA, so a phase costs one
// memory round trip plus a CTA barrier instead of a kernel launch; one SM's bandwidth and FP
// rate bound the size that pays.
struct ClusterTail {
    int ncta = 0;
    unsigned long long *cycles = nullptr;   // device: per step, SM cycles summed over launches
    std::vector<int> op, level;
};

template <class XT>
static bool cluster_schedulable(int ncta) {
    VEMG_CHECK_CUDA(cudaFuncSetAttribute(k_tail_cluster<XT>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)ncta);
    cfg.blockDim = dim3(kClusterThreads);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)ncta;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k_tail_cluster<XT>, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return n >= 1;
}

// ncta == 0: the single-CTA tail (at most kTailMaxPhases steps); 2..16: one cluster of ncta CTAs
static void build_tail(Arena &ar, SChain &C, bool fp32, int tail_rows, int ncta, cudaStream_t s) {
    C.tail_level = -1;
    if (ncta > 0 && !(fp32 ? cluster_schedulable<float>(ncta) : cluster_schedulable<double>(ncta))) return;
    int l0 = -1;
    for (int l = 1; l < C.nlev; ++l)
        if (C.lv[l].n <= tail_rows) {
            l0 = l;
            break;
        }
    if (l0 < 0) return;
    Builder B(ar, s);
    B.xs = fp32 ? 4 : 8;
    for (;;) {   // the single-CTA tail starts deeper while its phases do not fit in shared memory
        B.ph.clear();
        B.vcycle(C, l0, C.lv[l0].b, -1, C.lv[l0].x);
        if (ncta > 0 || (int)B.ph.size() <= kTailMaxPhases) break;
        if (++l0 >= C.nlev) return;
    }
    PPhase *d = ar.alloc<PPhase>((int)B.ph.size());
    VEMG_CHECK_CUDA(cudaMemcpyAsync(d, B.ph.data(), sizeof(PPhase) * B.ph.size(), cudaMemcpyHostToDevice, s));
    VEMG_CHECK_CUDA(cudaStreamSynchronize(s));
    C.tail = d;
    C.tail_n = (int)B.ph.size();
    C.tail_bytes = B.bytes;
    C.tail_level = l0;
    if (ncta > 0) {
        auto T = new ClusterTail();
        T->ncta = ncta;
        try {
            T->cycles = ar.alloc<unsigned long long>(C.tail_n);
            VEMG_CHECK_CUDA(cudaMemsetAsync(T->cycles, 0, sizeof(unsigned long long) * C.tail_n, s));
            VEMG_CHECK_CUDA(cudaStreamSynchronize(s));
        } catch (...) {
            delete T;
            throw;
        }
        for (const PPhase &p : B.ph) {
            T->op.push_back(p.op);
            T->level.push_back(p.level);
        }
        C.ctail = T;
    }
}

void release_ctail(SChain &C) {
    delete (ClusterTail *)C.ctail;   // device memory belongs to the hierarchy's arena
    C.ctail = nullptr;
}

void ctail_profile_reset(SChain &C) {
    auto T = (ClusterTail *)C.ctail;
    if (!T) return;
    // ordered before any later launch on any stream
    VEMG_CHECK_CUDA(cudaMemset(T->cycles, 0, sizeof(unsigned long long) * C.tail_n));
    VEMG_CHECK_CUDA(cudaDeviceSynchronize());
}

// the cluster tail's steps with the persistent program's op codes
int ctail_profile(const SChain &C, int group, std::vector<int> &op, std::vector<int> &level, std::vector<int> &grp,
                  std::vector<double> &cycles) {
    auto T = (const ClusterTail *)C.ctail;
    if (!T) return 0;
    std::vector<unsigned long long> c(C.tail_n);
    VEMG_CHECK_CUDA(cudaDeviceSynchronize());
    VEMG_CHECK_CUDA(cudaMemcpy(c.data(), T->cycles, sizeof(unsigned long long) * c.size(), cudaMemcpyDeviceToHost));
    for (int k = 0; k < C.tail_n; ++k) {
        op.push_back(T->op[k]);
        level.push_back(T->level[k]);
        grp.push_back(group);
        cycles.push_back((double)c[k]);
    }
    return C.tail_n;
}

double ctail_bytes(const SChain &C) { return C.tail_bytes; }

void build_tails(vemg_hierarchy *h, cudaStream_t s) {
    const bool fp32 = h->precision != VEMG_PREC_FP64;
    if (h->precond == VEMG_PRECOND_NONE) return;
    SChain *cs[2] = {single_chain(h) ? nullptr : &h->ssurf, &h->sbar};
    for (SChain *C : cs)
        if (C) build_tail(h->arena, *C, fp32, h->opts.tail_rows, h->opts.tail_cluster, s);
}

void launch_tail(const SChain &C, cudaStream_t s, bool profile) {
    const PPhase *ph = (const PPhase *)C.tail;
    if (C.ctail) {
        auto T = (const ClusterTail *)C.ctail;
        unsigned long long *cyc = profile ? T->cycles : nullptr;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)T->ncta);
        cfg.blockDim = dim3(kClusterThreads);
        cfg.stream = s;
        cudaLaunchAttribute attr[2];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)T->ncta;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[1].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 2;
        if (C.fp32) VEMG_CHECK_CUDA(cudaLaunchKernelEx(&cfg, k_tail_cluster<float>, ph, C.tail_n, cyc));
        else VEMG_CHECK_CUDA(cudaLaunchKernelEx(&cfg, k_tail_cluster<double>, ph, C.tail_n, cyc));
        return;
    }
    if (C.fp32)
        pdl_launch(k_tail<float>, 1, kTailThreads, s, ph, C.tail_n);
    else
        pdl_launch(k_tail<double>, 1, kTailThreads, s, ph, C.tail_n);
}

void release_persist(vemg_hierarchy *h) {
    delete h->persist;   // device memory belongs to the hierarchy's arena
    h->persist = nullptr;
}

double persist_bytes(const vemg_hierarchy *h) { return h->persist ? h->persist->bytes : 0.0; }
bool persist_coarse_only(const vemg_hierarchy *h) { return h->persist && h->persist->coarse; }
const int *persist_err(const vemg_hierarchy *h) { return h->persist ? h->persist->err : nullptr; }

// reset the barrier words and the error word after a failed application
void persist_reset(vemg_hierarchy *h, cudaStream_t s) {
    Persist *P = h->persist;
    if (!P) return;
    VEMG_CHECK_CUDA(cudaMemsetAsync(P->bar, 0, sizeof(unsigned long long) * kBarStride * P->ngroups, s));
    VEMG_CHECK_CUDA(cudaMemsetAsync(P->err, 0, sizeof(int), s));
}

// one cooperative launch of the program: every CTA is resident at once, so the group barriers
// cannot wait on a CTA that has not started
void persist_profile_reset(vemg_hierarchy *h) {
    Persist *P = h->persist;
    if (!P) return;
    // ordered before any later launch on any stream
    VEMG_CHECK_CUDA(cudaMemset(P->cycles, 0, sizeof(unsigned long long) * std::max(P->nphases, 1)));
    VEMG_CHECK_CUDA(cudaDeviceSynchronize());
}

int persist_profile(vemg_hierarchy *h, int cap, int *count, int *op, int *level, int *group, double *cycles) {
    Persist *P = h->persist;
    if (!P) {
        *count = 0;
        return VEMG_OK;
    }
    *count = P->nphases;
    if (cap < P->nphases) return VEMG_EINVAL;
    std::vector<unsigned long long> c(P->nphases);
    VEMG_CHECK_CUDA(cudaDeviceSynchronize());
    VEMG_CHECK_CUDA(cudaMemcpy(c.data(), P->cycles, sizeof(unsigned long long) * P->nphases, cudaMemcpyDeviceToHost));
    for (int k = 0; k < P->nphases; ++k) {
        op[k] = P->op[k];
        level[k] = P->level[k];
        group[k] = P->group[k];
        cycles[k] = (double)c[k];
    }
    return VEMG_OK;
}

void launch_persist(vemg_hierarchy *h, const double *r, cudaStream_t s) {
    Persist *P = h->persist;
    unsigned long long *cyc = h->probe.kind == PROBE_VCYCLE ? P->cycles : nullptr;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)P->grid);
    cfg.blockDim = dim3(kPThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const PPhase *ph = P->phases;
    const int4 *gr = P->groups;
    if (P->fp32)
        VEMG_CHECK_CUDA(cudaLaunchKernelEx(&cfg, k_precond_persistent<float>, ph, gr, P->ngroups, r, P->bar, P->err, cyc));
    else
        VEMG_CHECK_CUDA(cudaLaunchKernelEx(&cfg, k_precond_persistent<double>, ph, gr, P->ngroups, r, P->bar, P->err, cyc));
}

}  // namespace vemg
