// layout.cu -- the solve-phase layout of the hierarchy.
//
// The setup builds every operator in the natural ordering of its level (the ordering the
// method's definitions use). The solve reorders each multigrid level colour by colour, so that
// one colour of a multicolour SOR sweep is a contiguous range of rows, and stores every operator
// of the solve as a sliced ELL matrix (32 rows per slice, one thread per row, entries of a slice
// interleaved so that the 32 threads read consecutive words). The fine ordering of the outer
// Krylov vectors is [top nodes in the colour order of the surface level 0; non-top nodes in the
// colour order of A_bar's level 0], so that the A_bar branch of the preconditioner reads its
// right-hand side as the trailing part of r with no gather.
#include <algorithm>
#include <cstring>

#include <cuda_bf16.h>

#include "internal.cuh"

namespace vemg {

__global__ void k_inverse_perm(int n, const int *__restrict__ s2n, int *n2s) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) n2s[s2n[i]] = i;
}

__global__ void k_sell_width(int nslices, const int *__restrict__ row0, const int *__restrict__ nrow,
                             const int *__restrict__ s2n, const int *__restrict__ rp, int split, int *width) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nslices) return;
    int w = 0;
    for (int l = 0; l < nrow[s]; ++l) {
        int r = row0[s] + l;
        int i = s2n ? s2n[r] : r;
        w = max(w, rp[i + 1] - rp[i] - split);
    }
    width[s] = max(w, 0);
}

__global__ void k_scale32(int n, const int *__restrict__ w, int *o) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) o[i] = 32 * w[i];
}

template <class VT>
__global__ void k_sell_fill(int nslices, const int *__restrict__ row0, const int *__restrict__ nrow,
                            const int *__restrict__ off, const int *__restrict__ width, const int *__restrict__ s2n,
                            const int *__restrict__ n2s, const int *__restrict__ rp, const int *__restrict__ ci,
                            const double *__restrict__ v, int split, int *col, VT *val, VT *diag, VT *dinv) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int s = (int)(t / 32), lane = (int)(t % 32);
    if (s >= nslices) return;
    int o = off[s] + lane, w = width[s];
    int k = 0;
    if (lane < nrow[s]) {
        int r = row0[s] + lane;
        int i = s2n ? s2n[r] : r;
        for (int e = rp[i]; e < rp[i + 1]; ++e) {
            int c = ci[e];
            if (split && c == i) {
                diag[r] = (VT)v[e];
                dinv[r] = (VT)(1.0 / v[e]);
                continue;
            }
            col[o + 32 * k] = n2s ? n2s[c] : c;
            val[o + 32 * k] = (VT)v[e];
            ++k;
        }
    }
    for (; k < w; ++k) {
        col[o + 32 * k] = 0;
        val[o + 32 * k] = (VT)0;
    }
}

static int scan_i32(const int *in, int *out, int n, cudaStream_t s) {
    // small host-side scan (slice tables have at most a few hundred thousand entries)
    std::vector<int> h(n), o(n + 1);
    VEMG_CHECK_CUDA(cudaMemcpyAsync(h.data(), in, sizeof(int) * n, cudaMemcpyDeviceToHost, s));
    VEMG_CHECK_CUDA(cudaStreamSynchronize(s));
    int64_t acc = 0;
    for (int i = 0; i < n; ++i) {
        o[i] = (int)acc;
        acc += h[i];
    }
    if (acc > 0x7fffffffLL) throw Error{VEMG_EINTERNAL};
    o[n] = (int)acc;
    VEMG_CHECK_CUDA(cudaMemcpyAsync(out, o.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice, s));
    VEMG_CHECK_CUDA(cudaStreamSynchronize(s));
    return (int)acc;
}

// Build the sliced ELL of the rows s2n[0..n) of the CSR matrix A (natural order), columns mapped
// through n2s (null: identity). groups: row boundaries (solve order) that slices do not straddle.
// split: the diagonal goes to diag / dinv instead of the slices.
static Sell build_sell(Arena &ar, const DCsr &A, int n, const int *s2n, const int *n2s, int ncols,
                       const std::vector<int> &groups, bool split, bool fp32, void **diag, void **dinv,
                       std::vector<int> *gslice, cudaStream_t s) {
    Sell S;
    S.n = n;
    S.m = ncols;
    S.fp32 = fp32;
    std::vector<int> row0, nrow;
    if (gslice) gslice->assign(1, 0);
    for (size_t g = 0; g + 1 < groups.size(); ++g) {
        for (int r = groups[g]; r < groups[g + 1]; r += 32) {
            row0.push_back(r);
            nrow.push_back(std::min(32, groups[g + 1] - r));
        }
        if (gslice) gslice->push_back((int)row0.size());
    }
    S.nslices = (int)row0.size();
    S.row0 = ar.alloc<int>(S.nslices);
    S.nrow = ar.alloc<int>(S.nslices);
    S.width = ar.alloc<int>(S.nslices);
    S.off = ar.alloc<int>(S.nslices + 1);
    if (S.nslices) {
        VEMG_CHECK_CUDA(cudaMemcpyAsync(S.row0, row0.data(), sizeof(int) * S.nslices, cudaMemcpyHostToDevice, s));
        VEMG_CHECK_CUDA(cudaMemcpyAsync(S.nrow, nrow.data(), sizeof(int) * S.nslices, cudaMemcpyHostToDevice, s));
        k_sell_width<<<grid_for(S.nslices, 128), 128, 0, s>>>(S.nslices, S.row0, S.nrow, s2n, A.rp, split ? 1 : 0,
                                                              S.width);
        VEMG_CHECK_LAUNCH();
    }
    Scratch<int> w32(S.nslices + 1);
    if (S.nslices) {
        k_scale32<<<grid_for(S.nslices, 256), 256, 0, s>>>(S.nslices, S.width, w32);
        VEMG_CHECK_LAUNCH();
    }
    int total = scan_i32(w32, S.off, S.nslices, s);
    S.padded = total;
    S.col = ar.alloc<int>(total);
    if (fp32) S.v = ar.alloc<float>(total);
    else S.v = ar.alloc<double>(total);
    void *dg = nullptr, *di = nullptr;
    if (split) {
        if (fp32) { dg = ar.alloc<float>(n); di = ar.alloc<float>(n); }
        else { dg = ar.alloc<double>(n); di = ar.alloc<double>(n); }
        *diag = dg;
        *dinv = di;
    }
    if (S.nslices) {
        int64_t threads = (int64_t)S.nslices * 32;
        if (fp32)
            k_sell_fill<float><<<grid_for(threads, 256), 256, 0, s>>>(S.nslices, S.row0, S.nrow, S.off, S.width, s2n, n2s,
                                                                      A.rp, A.ci, A.v, split, S.col, (float *)S.v,
                                                                      (float *)dg, (float *)di);
        else
            k_sell_fill<double><<<grid_for(threads, 256), 256, 0, s>>>(S.nslices, S.row0, S.nrow, S.off, S.width, s2n,
                                                                       n2s, A.rp, A.ci, A.v, split, S.col,
                                                                       (double *)S.v, (double *)dg, (double *)di);
        VEMG_CHECK_LAUNCH();
    }
    // stored entries (rows of s2n)
    std::vector<int> hrp(A.n + 1);
    VEMG_CHECK_CUDA(cudaMemcpyAsync(hrp.data(), A.rp, sizeof(int) * (A.n + 1), cudaMemcpyDeviceToHost, s));
    VEMG_CHECK_CUDA(cudaStreamSynchronize(s));
    if (s2n) {
        std::vector<int> hs(n);
        VEMG_CHECK_CUDA(cudaMemcpy(hs.data(), s2n, sizeof(int) * n, cudaMemcpyDeviceToHost));
        for (int r = 0; r < n; ++r) S.nnz += hrp[hs[r] + 1] - hrp[hs[r]] - (split ? 1 : 0);
    } else {
        S.nnz = (int64_t)hrp[n] - (split ? n : 0);
    }
    return S;
}

__global__ void k_permute_dense(int n, const int *__restrict__ s2n, const double *__restrict__ G, double *Gs) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)n * n) return;
    int a = (int)(t / n), b = (int)(t % n);
    Gs[t] = G[(int64_t)s2n[a] * n + s2n[b]];
}

__global__ void k_to_float(int64_t n, const double *__restrict__ a, float *__restrict__ b) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) b[i] = (float)a[i];
}

// b = a rounded to BF16 (nearest, ties to even); a is overwritten by the same value in FP32
__global__ void k_f2bf(int64_t n, float *__restrict__ a, __nv_bfloat16 *__restrict__ b) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) {
        __nv_bfloat16 h = __float2bfloat16_rn(a[i]);
        b[i] = h;
        a[i] = __bfloat162float(h);
    }
}

// BF16 values of a sliced-ELL matrix, rounded from its FP32 values. The FP32 array keeps the
// rounded values, so that the kernels that read it (the batched solves, the coarse tails, the
// persistent cycle) apply the same operator as the per-phase kernels that read the BF16 array.
static void to_bf16(Arena &ar, Sell &S, cudaStream_t s) {
    __nv_bfloat16 *v = ar.alloc<__nv_bfloat16>(S.padded > 0 ? S.padded : 1);
    if (S.padded > 0) {
        k_f2bf<<<grid_for(S.padded, 256), 256, 0, s>>>(S.padded, (float *)S.v, v);
        VEMG_CHECK_LAUNCH();
    }
    S.vh = v;
}

// bf16: the chain's stored operators get BF16 copies, except on a chain with the near-nullspace
// {1, x, y}, whose coarse operators carry the fourth-order-like part of E~^T A E~ that BF16 values
// lose (measured on the 192x192x48 xy-jittered mesh: 1,593 iterations against 304 with FP32 values);
// it keeps FP32 values
static void layout_chain(Arena &ar, const Chain &C, SChain &S, bool fp32, cudaStream_t s, bool bf16 = false) {
    bf16 = bf16 && C.nsd == 1;
    S.nlev = C.nlev;
    S.direct = C.direct;
    S.singular = C.singular;
    S.fp32 = fp32;
    S.is_bar = C.is_bar;
    std::vector<int *> inv(C.nlev);
    for (int l = 0; l < C.nlev; ++l) {
        const Level &L = C.lv[l];
        inv[l] = ar.alloc<int>(L.A.n);
        k_inverse_perm<<<grid_for(L.A.n, 256), 256, 0, s>>>(L.A.n, L.crow, inv[l]);
        VEMG_CHECK_LAUNCH();
    }
    for (int l = 0; l < C.nlev; ++l) {
        const Level &L = C.lv[l];
        SLevel &T = S.lv[l];
        T.n = L.A.n;
        T.ncolours = L.ncolours;
        T.crow = L.cptr;
        T.cnnz.resize(L.ncolours);
        for (int c = 0; c < L.ncolours; ++c) T.cnnz[c] = L.cnnz[c] - (L.cptr[c + 1] - L.cptr[c]);
        T.A = build_sell(ar, L.A, L.A.n, L.crow, inv[l], L.A.n, L.cptr, true, fp32, &T.diag, &T.dinv, &T.cslice, s);
        if (l + 1 < C.nlev) {
            const Level &N = C.lv[l + 1];
            T.P = build_sell(ar, L.P, L.A.n, L.crow, inv[l + 1], N.A.n, {0, L.A.n}, false, fp32, nullptr, nullptr,
                             nullptr, s);
            T.PT = build_sell(ar, L.PT, N.A.n, N.crow, inv[l], L.A.n, {0, N.A.n}, false, fp32, nullptr, nullptr,
                              nullptr, s);
        }
        if (bf16) {
            to_bf16(ar, T.A, s);
            if (l + 1 < C.nlev) {
                to_bf16(ar, T.P, s);
                to_bf16(ar, T.PT, s);
            }
        }
        size_t es = fp32 ? sizeof(float) : sizeof(double);
        T.x = ar.alloc<char>((int64_t)es * T.n);
        T.b = ar.alloc<char>((int64_t)es * T.n);
        T.r = ar.alloc<char>((int64_t)es * T.n);
    }
    if (C.direct) {
        int n = C.nc;
        S.nc = n;
        S.G = ar.alloc<double>((int64_t)n * n);
        k_permute_dense<<<grid_for((int64_t)n * n, 256), 256, 0, s>>>(n, C.lv[C.nlev - 1].crow, C.G, S.G);
        VEMG_CHECK_LAUNCH();
        if (fp32) {   // FP32 cycles apply the dense inverse in FP32
            S.Gf = ar.alloc<float>((int64_t)n * n);
            k_to_float<<<grid_for((int64_t)n * n, 256), 256, 0, s>>>((int64_t)n * n, S.G, S.Gf);
            VEMG_CHECK_LAUNCH();
        }
    }
}

__global__ void k_outer_order(int n, int mtop, const int *__restrict__ surf_crow, const int *__restrict__ bar_crow,
                              int *s2n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    s2n[i] = i < mtop ? surf_crow[i] : mtop + bar_crow[i - mtop];
}

__global__ void k_compose(int n, const int *__restrict__ a, const int *__restrict__ b, int off, int *out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = a[off + b[i]];
}


__global__ void k_iota(int n, int *out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = i;
}

void build_solve_layout(vemg_hierarchy *h, cudaStream_t s) {
    Arena &ar = h->arena;
    bool fp32 = h->precision != VEMG_PREC_FP64;
    bool bf16 = h->precision == VEMG_PREC_BF16;
    int n = h->n, mt = h->mtop;
    if (!single_chain(h)) {
        layout_chain(ar, h->bar, h->sbar, fp32, s, bf16);
        layout_chain(ar, h->surf, h->ssurf, fp32, s, bf16);
        h->nu = n;
        Scratch<int> s2n(n), n2s(n);
        k_outer_order<<<grid_for(n, 256), 256, 0, s>>>(n, mt, h->surf.lv[0].crow, h->bar.lv[0].crow, s2n);
        VEMG_CHECK_LAUNCH();
        k_inverse_perm<<<grid_for(n, 256), 256, 0, s>>>(n, s2n, n2s);
        VEMG_CHECK_LAUNCH();
        Scratch<int> surf_inv(mt);
        k_inverse_perm<<<grid_for(mt, 256), 256, 0, s>>>(mt, h->surf.lv[0].crow, surf_inv);
        VEMG_CHECK_LAUNCH();
        h->Aop = build_sell(ar, h->A, n, s2n, n2s, n, {0, n}, false, false, nullptr, nullptr, nullptr, s);
        h->Enon = build_sell(ar, h->E, n - mt, s2n.p + mt, surf_inv, mt, {0, n - mt}, false, false, nullptr, nullptr,
                             nullptr, s);
        h->ETs = build_sell(ar, h->ET, mt, h->surf.lv[0].crow, n2s, n, {0, mt}, false, false, nullptr, nullptr, nullptr, s);
        if (fp32 && h->Enon.padded > 0) {
            // z = E~ y_s + x_bar is formed in FP32 when the V-cycles are FP32 (one conversion per row)
            h->Enon_vf = ar.alloc<float>(h->Enon.padded);
            k_to_float<<<grid_for(h->Enon.padded, 256), 256, 0, s>>>(h->Enon.padded, (const double *)h->Enon.v,
                                                                      h->Enon_vf);
            VEMG_CHECK_LAUNCH();
        }
        h->caller_of = ar.alloc<int>(n);
        k_compose<<<grid_for(n, 256), 256, 0, s>>>(n, h->new2old, s2n, 0, h->caller_of);
        VEMG_CHECK_LAUNCH();
    } else if (h->precond == VEMG_PRECOND_NONE && h->bc == VEMG_NEUMANN) {
        // plain CG: no cycle, the unknowns in their internal order
        h->nu = n;
        Scratch<int> iota(n);
        k_iota<<<grid_for(n, 256), 256, 0, s>>>(n, iota);
        VEMG_CHECK_LAUNCH();
        h->Aop = build_sell(ar, h->A, n, iota, iota, n, {0, n}, false, false, nullptr, nullptr, nullptr, s);
        h->caller_of = ar.alloc<int>(n);
        k_compose<<<grid_for(n, 256), 256, 0, s>>>(n, h->new2old, iota, 0, h->caller_of);
        VEMG_CHECK_LAUNCH();
    } else {
        // one chain whose level 0 is the operator of the unknowns (A_bar for Dirichlet-top, A for
        // the VL_SOR / SA preconditioners); the outer vectors use its level-0 colour order
        const Chain &C = the_chain(h);
        layout_chain(ar, C, h->sbar, fp32, s, bf16);
        int off = h->bc == VEMG_DIRICHLET_TOP ? mt : 0;
        int nb = n - off;
        h->nu = nb;
        const Level &L0 = C.lv[0];
        Scratch<int> inv(nb);
        k_inverse_perm<<<grid_for(nb, 256), 256, 0, s>>>(nb, L0.crow, inv);
        VEMG_CHECK_LAUNCH();
        h->Aop = build_sell(ar, L0.A, nb, L0.crow, inv, nb, {0, nb}, false, false, nullptr, nullptr, nullptr, s);
        h->caller_of = ar.alloc<int>(nb);
        k_compose<<<grid_for(nb, 256), 256, 0, s>>>(nb, h->new2old + off, L0.crow, 0, h->caller_of);
        VEMG_CHECK_LAUNCH();
    }
    VEMG_CHECK_CUDA(cudaStreamSynchronize(s));
}

}  // namespace vemg
