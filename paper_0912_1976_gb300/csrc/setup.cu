// setup.cu -- GPU setup of the vertical-extrapolation multigrid hierarchy.
//
// Compiled with -fmad=false: every floating-point operation here is rounded on its own, in the
// order written, so that the integer decisions taken from floating-point values (column
// location, strong couplings) and the setup values themselves are reproducible bit for bit.
//
// Steps (section numbers of Kramer, Cotter and Pain):
//   assembly of A and M f (section 3, Eq. Ax=b), top-first ordering (section 3,
//   Eqs. phi_decomposition / equation_decomposition), column location and vertical
//   extrapolation E~ (section 5.4, Fig. vertical_interpolation), Galerkin products
//   E~^T A E~ and P^T A P (section 5.1, Eq. reduced AMG), the Dirichlet-top block A_bar
//   (section 3), smoothed aggregation (section 5.1 and section 6), colouring for the SOR
//   sweeps, and the dense inverse of the coarsest level.
#include <math.h>

#include <algorithm>
#include <cstring>

#include "internal.cuh"

namespace vemg {

static constexpr int kMaxRowUnique = 256;  // neighbours of one node in the assembled pattern

// ------------------------------------------------------------------------------------------
// scans

__global__ void k_block_scan(const int *__restrict__ in, int64_t *__restrict__ out, int64_t *__restrict__ bsum,
                             int64_t n) {
    __shared__ int64_t ws[32];
    int64_t i = (int64_t)blockIdx.x * 1024 + threadIdx.x;
    int64_t v = i < n ? (int64_t)in[i] : 0;
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[w] = x;
    __syncthreads();
    if (w == 0) {
        int64_t s = ws[lane];
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        ws[lane] = s;
    }
    __syncthreads();
    int64_t incl = x + (w > 0 ? ws[w - 1] : 0);
    if (i < n) out[i] = incl - v;
    if (threadIdx.x == 1023) bsum[blockIdx.x] = incl;
}

__global__ void k_block_scan64(const int64_t *__restrict__ in, int64_t *__restrict__ out,
                               int64_t *__restrict__ bsum, int64_t n) {
    __shared__ int64_t ws[32];
    int64_t i = (int64_t)blockIdx.x * 1024 + threadIdx.x;
    int64_t v = i < n ? in[i] : 0;
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[w] = x;
    __syncthreads();
    if (w == 0) {
        int64_t s = ws[lane];
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        ws[lane] = s;
    }
    __syncthreads();
    int64_t incl = x + (w > 0 ? ws[w - 1] : 0);
    if (i < n) out[i] = incl - v;
    if (threadIdx.x == 1023) bsum[blockIdx.x] = incl;
}

__global__ void k_scan_add(int64_t *__restrict__ out, const int64_t *__restrict__ boff, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * 1024 + threadIdx.x;
    if (i < n) out[i] += boff[blockIdx.x];
}

static void scan64_inplace(int64_t *data, int64_t n, cudaStream_t s);

// exclusive scan of int64 values in place
static void scan64_inplace(int64_t *data, int64_t n, cudaStream_t s) {
    if (n <= 0) return;
    int64_t nb = (n + 1023) / 1024;
    Scratch<int64_t> bsum(nb);
    k_block_scan64<<<(unsigned)nb, 1024, 0, s>>>(data, data, bsum, n);
    VEMG_CHECK_LAUNCH();
    if (nb > 1) {
        scan64_inplace(bsum, nb, s);
        k_scan_add<<<(unsigned)nb, 1024, 0, s>>>(data, bsum, n);
        VEMG_CHECK_LAUNCH();
    }
}

// out64[0..n] = exclusive scan of in[0..n-1], out64[n] = total. Returns the total.
static int64_t scan_to64(const int *in, int64_t *out64, int64_t n, cudaStream_t s) {
    int64_t nb = (n + 1023) / 1024;
    if (n > 0) {
        Scratch<int64_t> bsum(nb);
        k_block_scan<<<(unsigned)nb, 1024, 0, s>>>(in, out64, bsum, n);
        VEMG_CHECK_LAUNCH();
        if (nb > 1) {
            scan64_inplace(bsum, nb, s);
            k_scan_add<<<(unsigned)nb, 1024, 0, s>>>(out64, bsum, n);
            VEMG_CHECK_LAUNCH();
        }
    }
    int64_t last_off = 0, total = 0;
    int last_in = 0;
    if (n > 0) {
        VEMG_CHECK_CUDA(cudaMemcpyAsync(&last_off, out64 + n - 1, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        VEMG_CHECK_CUDA(cudaMemcpyAsync(&last_in, in + n - 1, sizeof(int), cudaMemcpyDeviceToHost, s));
        VEMG_CHECK_CUDA(cudaStreamSynchronize(s));
        total = last_off + last_in;
    }
    VEMG_CHECK_CUDA(cudaMemcpyAsync(out64 + n, &total, sizeof(int64_t), cudaMemcpyHostToDevice, s));
    VEMG_CHECK_CUDA(cudaStreamSynchronize(s));
    return total;
}

__global__ void k_narrow(const int64_t *__restrict__ in, int *__restrict__ out, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (int)in[i];
}

// out[0..n] = exclusive scan of counts (int32 offsets); throws if the total needs 64 bits
static int scan_offsets(const int *counts, int *out, int64_t n, cudaStream_t s) {
    Scratch<int64_t> t(n + 1);
    int64_t total = scan_to64(counts, t, n, s);
    if (total > 0x7fffffffLL) throw Error{VEMG_EINTERNAL};
    k_narrow<<<grid_for(n + 1, 256), 256, 0, s>>>(t, out, n + 1);
    VEMG_CHECK_LAUNCH();
    return (int)total;
}

// ------------------------------------------------------------------------------------------
// small device helpers

__device__ __forceinline__ int bsearch_row(const int *__restrict__ ci, int lo, int hi, int j) {
    // position of j in ci[lo, hi), -1 if absent (sorted)
    hi -= 1;
    while (lo <= hi) {
        int mid = (lo + hi) >> 1;
        int c = ci[mid];
        if (c == j) return mid;
        if (c < j) lo = mid + 1;
        else hi = mid - 1;
    }
    return -1;
}

// insert v into the sorted unique array a[0..cnt) (capacity cap); returns the new count, or -1
// when full
template <class T>
__device__ __forceinline__ int insert_unique(T *a, int cnt, int cap, int v) {
    int lo = 0, hi = cnt - 1;
    while (lo <= hi) {
        int mid = (lo + hi) >> 1;
        int c = a[mid];
        if (c == v) return cnt;
        if (c < v) lo = mid + 1;
        else hi = mid - 1;
    }
    if (cnt >= cap) return -1;
    for (int k = cnt; k > lo; --k) a[k] = a[k - 1];
    a[lo] = v;
    return cnt + 1;
}

__device__ __forceinline__ void atomic_flag(int *err, int code) { atomicCAS(err, 0, code); }

static int read_flag(int *d_err, cudaStream_t s) {
    int e = 0;
    VEMG_CHECK_CUDA(cudaMemcpyAsync(&e, d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    VEMG_CHECK_CUDA(cudaStreamSynchronize(s));
    return e;
}

// MurmurHash3 32-bit finalizer (Austin Appleby, public domain), a bijection on 32-bit words:
// the fixed priority of the round-synchronous aggregation and colouring rules.
__device__ __forceinline__ uint32_t hash32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

// ------------------------------------------------------------------------------------------
// element matrices (section 3): K_ab = (c_a . c_b) / (6 det), c_1 = d2 x d3, c_2 = d3 x d1,
// c_3 = d1 x d2, c_0 = -((c_1 + c_2) + c_3), d_k = p_k - p_0, det = d1 . c_1 = 6 V.

struct Tet {
    double c[4][3];
    double det;
};

__device__ __forceinline__ void cross3(const double *u, const double *v, double *w) {
    w[0] = u[1] * v[2] - u[2] * v[1];
    w[1] = u[2] * v[0] - u[0] * v[2];
    w[2] = u[0] * v[1] - u[1] * v[0];
}

__device__ __forceinline__ double dot3(const double *u, const double *v) {
    return u[0] * v[0] + u[1] * v[1] + u[2] * v[2];
}

__device__ void tet_geometry(const double *__restrict__ xyz, const int *v, Tet &T) {
    double p0[3], d1[3], d2[3], d3[3];
    for (int k = 0; k < 3; ++k) p0[k] = xyz[3 * (int64_t)v[0] + k];
    for (int k = 0; k < 3; ++k) {
        d1[k] = xyz[3 * (int64_t)v[1] + k] - p0[k];
        d2[k] = xyz[3 * (int64_t)v[2] + k] - p0[k];
        d3[k] = xyz[3 * (int64_t)v[3] + k] - p0[k];
    }
    cross3(d2, d3, T.c[1]);
    cross3(d3, d1, T.c[2]);
    cross3(d1, d2, T.c[3]);
    T.det = dot3(d1, T.c[1]);
    for (int k = 0; k < 3; ++k) T.c[0][k] = -((T.c[1][k] + T.c[2][k]) + T.c[3][k]);
}

// ------------------------------------------------------------------------------------------
// node-to-element incidence

__global__ void k_inc_count(const int *__restrict__ tets, int64_t ne, int n, int *cnt, int *err) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ne) return;
    for (int a = 0; a < 4; ++a) {
        int v = tets[4 * e + a];
        if (v < 0 || v >= n) { atomic_flag(err, VEMG_EMESH); return; }
    }
    for (int a = 0; a < 4; ++a) atomicAdd(&cnt[tets[4 * e + a]], 1);
}

__global__ void k_inc_fill(const int *__restrict__ tets, int64_t ne, int *cur, int *inc) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ne) return;
    for (int a = 0; a < 4; ++a) {
        int p = atomicAdd(&cur[tets[4 * e + a]], 1);
        inc[p] = (int)e;
    }
}

// insertion sort of each segment data[ptr[i], ptr[i+1])
__global__ void k_sort_segments(const int *__restrict__ ptr, int *data, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int lo = ptr[i], hi = ptr[i + 1];
    for (int k = lo + 1; k < hi; ++k) {
        int x = data[k], j = k - 1;
        while (j >= lo && data[j] > x) { data[j + 1] = data[j]; --j; }
        data[j + 1] = x;
    }
}

// as above, carrying values along
__global__ void k_sort_rows_kv(const int *__restrict__ rp, int *ci, double *v, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int lo = rp[i], hi = rp[i + 1];
    for (int k = lo + 1; k < hi; ++k) {
        int x = ci[k];
        double y = v[k];
        int j = k - 1;
        while (j >= lo && ci[j] > x) { ci[j + 1] = ci[j]; v[j + 1] = v[j]; --j; }
        ci[j + 1] = x;
        v[j + 1] = y;
    }
}

struct Incidence {
    int *ptr = nullptr, *inc = nullptr;
    void release() {
        dev_free_raw(ptr);
        dev_free_raw(inc);
        ptr = inc = nullptr;
    }
};

static Incidence build_incidence(const int *d_tets, int64_t ne, int n, cudaStream_t s) {
    Incidence I;
    Scratch<int> cnt(n + 1), err(1);
    VEMG_CHECK_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * (n + 1), s));
    VEMG_CHECK_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
    k_inc_count<<<grid_for(ne, 256), 256, 0, s>>>(d_tets, ne, n, cnt, err);
    VEMG_CHECK_LAUNCH();
    if (read_flag(err, s)) throw Error{VEMG_EMESH};
    I.ptr = (int *)dev_alloc_raw(sizeof(int) * (n + 1));
    int total = scan_offsets(cnt, I.ptr, n, s);
    I.inc = (int *)dev_alloc_raw(sizeof(int) * (size_t)std::max(total, 1));
    Scratch<int> cur(n);
    VEMG_CHECK_CUDA(cudaMemcpyAsync(cur, I.ptr, sizeof(int) * n, cudaMemcpyDeviceToDevice, s));
    k_inc_fill<<<grid_for(ne, 256), 256, 0, s>>>(d_tets, ne, cur, I.inc);
    VEMG_CHECK_LAUNCH();
    k_sort_segments<<<grid_for(n, 128), 128, 0, s>>>(I.ptr, I.inc, n);
    VEMG_CHECK_LAUNCH();
    return I;
}

// ------------------------------------------------------------------------------------------
// assembly of A (caller order)

__global__ void k_asm_rowlen(int n, const int *__restrict__ iptr, const int *__restrict__ inc,
                             const int *__restrict__ tets, int *rowlen, int *err) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int nb[kMaxRowUnique];
    int cnt = 0;
    for (int k = iptr[i]; k < iptr[i + 1]; ++k) {
        const int *t = tets + 4 * (int64_t)inc[k];
        for (int a = 0; a < 4; ++a) {
            cnt = insert_unique(nb, cnt, kMaxRowUnique, t[a]);
            if (cnt < 0) { atomic_flag(err, VEMG_EINTERNAL); return; }
        }
    }
    rowlen[i] = cnt;
}

__global__ void k_asm_rowfill(int n, const int *__restrict__ iptr, const int *__restrict__ inc,
                              const int *__restrict__ tets, const int *__restrict__ rp, int *ci) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int nb[kMaxRowUnique];
    int cnt = 0;
    for (int k = iptr[i]; k < iptr[i + 1]; ++k) {
        const int *t = tets + 4 * (int64_t)inc[k];
        for (int a = 0; a < 4; ++a) cnt = insert_unique(nb, cnt, kMaxRowUnique, t[a]);
    }
    for (int k = 0; k < cnt; ++k) ci[rp[i] + k] = nb[k];
}

// A_ij = sum over the elements holding i and j, in ascending element index, of K_e[a][b]
__global__ void k_asm_values(int n, const int *__restrict__ iptr, const int *__restrict__ inc,
                             const int *__restrict__ tets, const double *__restrict__ xyz,
                             const int *__restrict__ rp, const int *__restrict__ ci, double *v, int *err) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int lo = rp[i], hi = rp[i + 1];
    for (int k = lo; k < hi; ++k) v[k] = 0.0;
    for (int k = iptr[i]; k < iptr[i + 1]; ++k) {
        const int *t = tets + 4 * (int64_t)inc[k];
        int vv[4] = {t[0], t[1], t[2], t[3]};
        Tet T;
        tet_geometry(xyz, vv, T);
        if (!(T.det > 0.0)) { atomic_flag(err, VEMG_EMESH); return; }
        int a = 0;
        while (vv[a] != i) ++a;
        double s = 6.0 * T.det;
        for (int b = 0; b < 4; ++b) {
            double kab = dot3(T.c[a], T.c[b]) / s;
            int pos = bsearch_row(ci, lo, hi, vv[b]);
            v[pos] = v[pos] + kab;
        }
    }
}

// b = M f: (M_e f)_a = V/20 (f_a + sum_b f_b), elements in ascending index
__global__ void k_load(int n, const int *__restrict__ iptr, const int *__restrict__ inc,
                       const int *__restrict__ tets, const double *__restrict__ xyz,
                       const double *__restrict__ f, double *b) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double acc = 0.0;
    for (int k = iptr[i]; k < iptr[i + 1]; ++k) {
        const int *t = tets + 4 * (int64_t)inc[k];
        int vv[4] = {t[0], t[1], t[2], t[3]};
        Tet T;
        tet_geometry(xyz, vv, T);
        double w = (T.det / 6.0) / 20.0;
        double s = ((f[vv[0]] + f[vv[1]]) + f[vv[2]]) + f[vv[3]];
        acc = acc + w * (f[i] + s);
    }
    b[i] = acc;
}

struct MeshDev {
    double *xyz = nullptr;
    int *tets = nullptr;
    int64_t ne = 0;
    int n = 0;
    void release() {
        dev_free_raw(xyz);
        dev_free_raw(tets);
        xyz = nullptr;
        tets = nullptr;
    }
};

static MeshDev upload_mesh(const vemg_mesh *m, cudaStream_t s) {
    if (!m || m->n_nodes <= 0 || m->n_tets <= 0 || !m->xyz || !m->tets) throw Error{VEMG_EINVAL};
    if (m->n_nodes > 0x7ffffff0LL || m->n_tets * 4 > 0x7ffffff0LL) throw Error{VEMG_EINVAL};
    MeshDev d;
    d.n = (int)m->n_nodes;
    d.ne = m->n_tets;
    d.xyz = (double *)dev_alloc_raw(sizeof(double) * 3 * (size_t)d.n);
    d.tets = (int *)dev_alloc_raw(sizeof(int) * 4 * (size_t)d.ne);
    VEMG_CHECK_CUDA(cudaMemcpyAsync(d.xyz, m->xyz, sizeof(double) * 3 * (size_t)d.n, cudaMemcpyHostToDevice, s));
    VEMG_CHECK_CUDA(cudaMemcpyAsync(d.tets, m->tets, sizeof(int) * 4 * (size_t)d.ne, cudaMemcpyHostToDevice, s));
    return d;
}

void assemble(const vemg_mesh *mesh, vemg_csr *out, cudaStream_t s) {
    if (!out) throw Error{VEMG_EINVAL};
    MeshDev md = upload_mesh(mesh, s);
    Incidence I;
    try {
        int n = md.n;
        I = build_incidence(md.tets, md.ne, n, s);
        Scratch<int> rowlen(n), err(1);
        VEMG_CHECK_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
        k_asm_rowlen<<<grid_for(n, 128), 128, 0, s>>>(n, I.ptr, I.inc, md.tets, rowlen, err);
        VEMG_CHECK_LAUNCH();
        if (int e = read_flag(err, s)) throw Error{e};
        int *rp = (int *)dev_alloc_raw(sizeof(int) * (n + 1));
        int nnz = scan_offsets(rowlen, rp, n, s);
        int *ci = (int *)dev_alloc_raw(sizeof(int) * (size_t)std::max(nnz, 1));
        double *v = (double *)dev_alloc_raw(sizeof(double) * (size_t)std::max(nnz, 1));
        k_asm_rowfill<<<grid_for(n, 128), 128, 0, s>>>(n, I.ptr, I.inc, md.tets, rp, ci);
        VEMG_CHECK_LAUNCH();
        k_asm_values<<<grid_for(n, 128), 128, 0, s>>>(n, I.ptr, I.inc, md.tets, md.xyz, rp, ci, v, err);
        VEMG_CHECK_LAUNCH();
        if (int e = read_flag(err, s)) {
            dev_free_raw(rp); dev_free_raw(ci); dev_free_raw(v);
            throw Error{e};
        }
        out->n = n;
        out->nnz = nnz;
        out->rowptr = rp;
        out->col = ci;
        out->val = v;
    } catch (...) {
        I.release();
        md.release();
        throw;
    }
    I.release();
    md.release();
}

void load_vector(const vemg_mesh *mesh, const double *f, double *b, cudaStream_t s) {
    if (!f || !b) throw Error{VEMG_EINVAL};
    MeshDev md = upload_mesh(mesh, s);
    Incidence I;
    try {
        I = build_incidence(md.tets, md.ne, md.n, s);
        k_load<<<grid_for(md.n, 128), 128, 0, s>>>(md.n, I.ptr, I.inc, md.tets, md.xyz, f, b);
        VEMG_CHECK_LAUNCH();
        VEMG_CHECK_CUDA(cudaStreamSynchronize(s));
    } catch (...) {
        I.release();
        md.release();
        throw;
    }
    I.release();
    md.release();
}

// ------------------------------------------------------------------------------------------
// generic CSR operations

static DCsr csr_alloc(Arena &ar, int n, int m, int nnz) {
    DCsr a;
    a.n = n;
    a.m = m;
    a.nnz = nnz;
    a.rp = ar.alloc<int>(n + 1);
    a.ci = ar.alloc<int>(nnz);
    a.v = ar.alloc<double>(nnz);
    return a;
}

__global__ void k_count_cols(const int *__restrict__ ci, int nnz, int *cnt) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < nnz) atomicAdd(&cnt[ci[k]], 1);
}

__global__ void k_fill_transpose(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                                 const double *__restrict__ v, int *cur, int *tci, double *tv) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int k = rp[i]; k < rp[i + 1]; ++k) {
        int p = atomicAdd(&cur[ci[k]], 1);
        tci[p] = i;
        tv[p] = v[k];
    }
}

// transpose; rows of the result hold source rows in ascending order
static DCsr csr_transpose(Arena &ar, const DCsr &a, cudaStream_t s) {
    Scratch<int> cnt(a.m + 1);
    VEMG_CHECK_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * (a.m + 1), s));
    k_count_cols<<<grid_for(a.nnz, 256), 256, 0, s>>>(a.ci, a.nnz, cnt);
    VEMG_CHECK_LAUNCH();
    DCsr t;
    t.n = a.m;
    t.m = a.n;
    t.nnz = a.nnz;
    t.rp = ar.alloc<int>(a.m + 1);
    scan_offsets(cnt, t.rp, a.m, s);
    t.ci = ar.alloc<int>(a.nnz);
    t.v = ar.alloc<double>(a.nnz);
    Scratch<int> cur(a.m + 1);
    VEMG_CHECK_CUDA(cudaMemcpyAsync(cur, t.rp, sizeof(int) * a.m, cudaMemcpyDeviceToDevice, s));
    k_fill_transpose<<<grid_for(a.n, 256), 256, 0, s>>>(a.n, a.rp, a.ci, a.v, cur, t.ci, t.v);
    VEMG_CHECK_LAUNCH();
    k_sort_rows_kv<<<grid_for(t.n, 128), 128, 0, s>>>(t.rp, t.ci, t.v, t.n);
    VEMG_CHECK_LAUNCH();
    return t;
}

// C = L R (Gustavson). Entry C_ij = sum over a ascending of L_ia R_aj, accumulated from 0.0 one
// product at a time; the pattern is structural.
__global__ void k_spgemm_ub(int n, const int *__restrict__ lrp, const int *__restrict__ lci,
                            const int *__restrict__ rrp, int *ub) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t c = 0;
    for (int k = lrp[i]; k < lrp[i + 1]; ++k) {
        int a = lci[k];
        c += rrp[a + 1] - rrp[a];
    }
    ub[i] = (int)(c > 0x7fffffff ? 0x7fffffff : c);
}

__global__ void k_spgemm_sym(int n, const int *__restrict__ lrp, const int *__restrict__ lci,
                             const int *__restrict__ rrp, const int *__restrict__ rci,
                             const int64_t *__restrict__ off, int *cand, int *ulen) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int *a_ = cand + off[i];
    int cap = (int)(off[i + 1] - off[i]);
    int cnt = 0;
    for (int k = lrp[i]; k < lrp[i + 1]; ++k) {
        int a = lci[k];
        for (int q = rrp[a]; q < rrp[a + 1]; ++q) cnt = insert_unique(a_, cnt, cap, rci[q]);
    }
    ulen[i] = cnt;
}

__global__ void k_spgemm_copy(int n, const int64_t *__restrict__ off, const int *__restrict__ cand,
                              const int *__restrict__ crp, int *cci) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int *a_ = cand + off[i];
    for (int k = crp[i]; k < crp[i + 1]; ++k) cci[k] = a_[k - crp[i]];
}

__global__ void k_spgemm_num(int n, const int *__restrict__ lrp, const int *__restrict__ lci,
                             const double *__restrict__ lv, const int *__restrict__ rrp,
                             const int *__restrict__ rci, const double *__restrict__ rv,
                             const int *__restrict__ crp, const int *__restrict__ cci, double *cv) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int lo = crp[i], hi = crp[i + 1];
    for (int k = lo; k < hi; ++k) cv[k] = 0.0;
    for (int k = lrp[i]; k < lrp[i + 1]; ++k) {
        int a = lci[k];
        double la = lv[k];
        for (int q = rrp[a]; q < rrp[a + 1]; ++q) {
            int pos = bsearch_row(cci, lo, hi, rci[q]);
            cv[pos] = cv[pos] + la * rv[q];
        }
    }
}

static DCsr csr_spgemm(Arena &ar, const DCsr &L, const DCsr &R, cudaStream_t s) {
    int n = L.n;
    Scratch<int> ub(n);
    k_spgemm_ub<<<grid_for(n, 256), 256, 0, s>>>(n, L.rp, L.ci, R.rp, ub);
    VEMG_CHECK_LAUNCH();
    Scratch<int64_t> off(n + 1);
    int64_t total = scan_to64(ub, off, n, s);
    Scratch<int> cand(total);
    Scratch<int> ulen(n);
    k_spgemm_sym<<<grid_for(n, 128), 128, 0, s>>>(n, L.rp, L.ci, R.rp, R.ci, off, cand, ulen);
    VEMG_CHECK_LAUNCH();
    DCsr C;
    C.n = n;
    C.m = R.m;
    C.rp = ar.alloc<int>(n + 1);
    C.nnz = scan_offsets(ulen, C.rp, n, s);
    C.ci = ar.alloc<int>(C.nnz);
    C.v = ar.alloc<double>(C.nnz);
    k_spgemm_copy<<<grid_for(n, 256), 256, 0, s>>>(n, off, cand, C.rp, C.ci);
    VEMG_CHECK_LAUNCH();
    k_spgemm_num<<<grid_for(n, 128), 128, 0, s>>>(n, L.rp, L.ci, L.v, R.rp, R.ci, R.v, C.rp, C.ci, C.v);
    VEMG_CHECK_LAUNCH();
    VEMG_CHECK_CUDA(cudaStreamSynchronize(s));
    return C;
}

// C_ij := C_ji for j < i (exact symmetry from the upper triangle)
__global__ void k_mirror_upper(int n, const int *__restrict__ rp, const int *__restrict__ ci, double *v) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int k = rp[i]; k < rp[i + 1]; ++k) {
        int j = ci[k];
        if (j >= i) break;
        int q = bsearch_row(ci, rp[j], rp[j + 1], i);
        if (q >= 0) v[k] = v[q];
    }
}

// Galerkin product P^T (A P), then exact symmetrisation (section 5.1, Eq. reduced AMG)
static DCsr galerkin(Arena &ar, const DCsr &A, const DCsr &P, const DCsr &PT, cudaStream_t s) {
    Arena tmp;
    DCsr AP = csr_spgemm(tmp, A, P, s);
    DCsr C = csr_spgemm(ar, PT, AP, s);
    k_mirror_upper<<<grid_for(C.n, 128), 128, 0, s>>>(C.n, C.rp, C.ci, C.v);
    VEMG_CHECK_LAUNCH();
    VEMG_CHECK_CUDA(cudaStreamSynchronize(s));
    tmp.release();
    return C;
}

// ------------------------------------------------------------------------------------------
// ordering: top nodes first, each group in caller order (section 3)

__global__ void k_top_flag(const uint8_t *__restrict__ tags, int n, int *flag) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) flag[i] = (tags[i] & VEMG_TAG_TOP) ? 1 : 0;
}

__global__ void k_perm(int n, int mtop, const int *__restrict__ flag, const int *__restrict__ topoff,
                       int *new2old, int *old2new) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int t = topoff[i];
    int r = flag[i] ? t : mtop + (i - t);
    new2old[r] = i;
    old2new[i] = r;
}

// symmetric permutation B = Q A Q^T: row r of B is row new2old[r] of A with mapped columns
__global__ void k_perm_rowlen(int n, const int *__restrict__ rp, const int *__restrict__ new2old, int *len) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) len[r] = rp[new2old[r] + 1] - rp[new2old[r]];
}

__global__ void k_perm_fill(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                            const double *__restrict__ v, const int *__restrict__ new2old,
                            const int *__restrict__ old2new, const int *__restrict__ brp, int *bci, double *bv) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    int i = new2old[r];
    int o = brp[r];
    for (int k = rp[i]; k < rp[i + 1]; ++k) {
        bci[o + k - rp[i]] = old2new[ci[k]];
        bv[o + k - rp[i]] = v[k];
    }
}

// trailing block: rows and columns >= mtop
__global__ void k_bar_rowlen(int nb, int mtop, const int *__restrict__ rp, const int *__restrict__ ci, int *len) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nb) return;
    int c = 0;
    for (int k = rp[mtop + i]; k < rp[mtop + i + 1]; ++k) c += ci[k] >= mtop;
    len[i] = c;
}

__global__ void k_bar_fill(int nb, int mtop, const int *__restrict__ rp, const int *__restrict__ ci,
                           const double *__restrict__ v, const int *__restrict__ brp, int *bci, double *bv) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nb) return;
    int o = brp[i];
    for (int k = rp[mtop + i]; k < rp[mtop + i + 1]; ++k)
        if (ci[k] >= mtop) {
            bci[o] = ci[k] - mtop;
            bv[o] = v[k];
            o++;
        }
}

// ------------------------------------------------------------------------------------------
// column location and vertical extrapolation (section 5.4)

__device__ __forceinline__ double orient2(double px, double py, double qx, double qy, double rx, double ry) {
    return (qx - px) * (ry - py) - (qy - py) * (rx - px);
}

__device__ __forceinline__ int bucket_of(double v, double v0, double sc, int nb) {
    double f = floor((v - v0) / sc * (double)nb);
    if (f < 0.0) return 0;
    if (f > (double)(nb - 1)) return nb - 1;
    return (int)f;
}

__global__ void k_tri_bbox(int nt, const int *__restrict__ tri, const double *__restrict__ xyz, double *bb,
                           const uint8_t *__restrict__ tags, int n, int *err) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    double a = INFINITY, b = -INFINITY, c = INFINITY, d = -INFINITY;
    for (int k = 0; k < 3; ++k) {
        int v = tri[3 * t + k];
        if (v < 0 || v >= n || !(tags[v] & VEMG_TAG_TOP)) { atomic_flag(err, VEMG_EMESH); return; }
        double x = xyz[3 * (int64_t)v], y = xyz[3 * (int64_t)v + 1];
        a = x < a ? x : a;
        b = x > b ? x : b;
        c = y < c ? y : c;
        d = y > d ? y : d;
    }
    bb[4 * t] = a;
    bb[4 * t + 1] = b;
    bb[4 * t + 2] = c;
    bb[4 * t + 3] = d;
}

struct Grid {
    double x0, y0, sx, sy;
    int nb;
};

__global__ void k_bucket_count(int nt, const double *__restrict__ bb, Grid g, int *cnt) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    int i0 = bucket_of(bb[4 * t], g.x0, g.sx, g.nb), i1 = bucket_of(bb[4 * t + 1], g.x0, g.sx, g.nb);
    int j0 = bucket_of(bb[4 * t + 2], g.y0, g.sy, g.nb), j1 = bucket_of(bb[4 * t + 3], g.y0, g.sy, g.nb);
    for (int j = j0; j <= j1; ++j)
        for (int i = i0; i <= i1; ++i) atomicAdd(&cnt[j * g.nb + i], 1);
}

__global__ void k_bucket_fill(int nt, const double *__restrict__ bb, Grid g, int *cur, int *idx) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    int i0 = bucket_of(bb[4 * t], g.x0, g.sx, g.nb), i1 = bucket_of(bb[4 * t + 1], g.x0, g.sx, g.nb);
    int j0 = bucket_of(bb[4 * t + 2], g.y0, g.sy, g.nb), j1 = bucket_of(bb[4 * t + 3], g.y0, g.sy, g.nb);
    for (int j = j0; j <= j1; ++j)
        for (int i = i0; i <= i1; ++i) idx[atomicAdd(&cur[j * g.nb + i], 1)] = t;
}

__device__ __forceinline__ void tri_bary(const int *__restrict__ tri, const double *__restrict__ xyz, int t,
                                         double px, double py, double w[3]) {
    const double *a = xyz + 3 * (int64_t)tri[3 * t], *b = xyz + 3 * (int64_t)tri[3 * t + 1],
                 *c = xyz + 3 * (int64_t)tri[3 * t + 2];
    double area = orient2(a[0], a[1], b[0], b[1], c[0], c[1]);
    w[0] = orient2(px, py, b[0], b[1], c[0], c[1]) / area;
    w[1] = orient2(a[0], a[1], px, py, c[0], c[1]) / area;
    w[2] = (1.0 - w[0]) - w[1];
}

// for each non-top internal node: among the top triangles whose bounding box holds (x, y), the
// one maximising the smallest barycentric coordinate (ties: lowest index)
__global__ void k_locate(int n, int mtop, const int *__restrict__ new2old, const double *__restrict__ xyz,
                         const int *__restrict__ tri, const double *__restrict__ bb, Grid g,
                         const int *__restrict__ bptr, const int *__restrict__ bidx, int *tri_of, double *bary,
                         int *err) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    if (r < mtop) {
        tri_of[r] = -1;
        bary[3 * (int64_t)r] = 1.0;
        bary[3 * (int64_t)r + 1] = 0.0;
        bary[3 * (int64_t)r + 2] = 0.0;
        return;
    }
    const double *p = xyz + 3 * (int64_t)new2old[r];
    double px = p[0], py = p[1];
    int bi = bucket_of(px, g.x0, g.sx, g.nb), bj = bucket_of(py, g.y0, g.sy, g.nb);
    int best = -1;
    double bm = 0.0;
    for (int k = bptr[bj * g.nb + bi]; k < bptr[bj * g.nb + bi + 1]; ++k) {
        int t = bidx[k];
        const double *q = bb + 4 * t;
        if (px < q[0] || px > q[1] || py < q[2] || py > q[3]) continue;
        double l[3];
        tri_bary(tri, xyz, t, px, py, l);
        double m = l[0] < l[1] ? l[0] : l[1];
        if (l[2] < m) m = l[2];
        if (best < 0 || m > bm || (m == bm && t < best)) {
            best = t;
            bm = m;
        }
    }
    tri_of[r] = best;
    if (best < 0) {
        atomic_flag(err, VEMG_EMESH);
        return;
    }
    double w[3];
    tri_bary(tri, xyz, best, px, py, w);
    bary[3 * (int64_t)r] = w[0];
    bary[3 * (int64_t)r + 1] = w[1];
    bary[3 * (int64_t)r + 2] = w[2];
}

__global__ void k_ext_rowlen(int n, int mtop, const double *__restrict__ bary, int *len) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    if (r < mtop) { len[r] = 1; return; }
    int c = 0;
    for (int k = 0; k < 3; ++k) c += bary[3 * (int64_t)r + k] != 0.0;
    len[r] = c;
}

// E~ = [I; F]: identity rows on top nodes, barycentric weights (exact zeros dropped) elsewhere
__global__ void k_ext_fill(int n, int mtop, const int *__restrict__ tri_of, const double *__restrict__ bary,
                           const int *__restrict__ tri, const int *__restrict__ old2new,
                           const int *__restrict__ rp, int *ci, double *v) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    int o = rp[r];
    if (r < mtop) { ci[o] = r; v[o] = 1.0; return; }
    int cols[3];
    double ws[3];
    int c = 0;
    for (int k = 0; k < 3; ++k) {
        double w = bary[3 * (int64_t)r + k];
        if (w != 0.0) {
            cols[c] = old2new[tri[3 * tri_of[r] + k]];
            ws[c] = w;
            c++;
        }
    }
    for (int a = 1; a < c; ++a) {
        int cc = cols[a];
        double ww = ws[a];
        int b = a - 1;
        while (b >= 0 && cols[b] > cc) { cols[b + 1] = cols[b]; ws[b + 1] = ws[b]; --b; }
        cols[b + 1] = cc;
        ws[b + 1] = ww;
    }
    for (int k = 0; k < c; ++k) { ci[o + k] = cols[k]; v[o + k] = ws[k]; }
}

// ------------------------------------------------------------------------------------------
// smoothed aggregation (section 5.1, section 6)

__global__ void k_diag(int n, const int *__restrict__ rp, const int *__restrict__ ci, const double *__restrict__ v,
                       double *d) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int q = bsearch_row(ci, rp[i], rp[i + 1], i);
    d[i] = q >= 0 ? v[q] : 0.0;
}

__device__ __forceinline__ bool strong(double aij, double di, double dj, double theta) {
    return fabs(aij) > theta * sqrt(di * dj);
}

__global__ void k_strong_len(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                             const double *__restrict__ v, const double *__restrict__ d, double theta, int *len) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int c = 0;
    for (int k = rp[i]; k < rp[i + 1]; ++k) {
        int j = ci[k];
        if (j != i && strong(v[k], d[i], d[j], theta)) c++;
    }
    len[i] = c;
}

__global__ void k_strong_fill(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                              const double *__restrict__ v, const double *__restrict__ d, double theta,
                              const int *__restrict__ srp, int *sci, double *sv) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int o = srp[i];
    for (int k = rp[i]; k < rp[i + 1]; ++k) {
        int j = ci[k];
        if (j != i && strong(v[k], d[i], d[j], theta)) {
            sci[o] = j;
            sv[o] = fabs(v[k]);
            o++;
        }
    }
}

__global__ void k_agg_keys(int n, const int *__restrict__ srp, uint64_t *key) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t deg = (uint64_t)(srp[i + 1] - srp[i]);
    key[i] = ((deg + 1u) << 32) | (uint64_t)hash32((uint32_t)i);
}

// phase 1 candidates: unaggregated with an unaggregated strong neighbourhood
// keep_isolated == 0: a node without strong couplings is never a candidate and stays
// unaggregated (zero prolongator row)
__global__ void k_phase1_cand(int n, const int *__restrict__ srp, const int *__restrict__ sci,
                              const int *__restrict__ agg, int keep_isolated, char *cand, char *thr, int *any) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    bool f = agg[i] < 0 && (keep_isolated || srp[i + 1] > srp[i]);
    for (int k = srp[i]; f && k < srp[i + 1]; ++k)
        if (agg[sci[k]] >= 0) f = false;
    cand[i] = f;
    thr[i] = 1;
    if (f) *any = 1;
}

__global__ void k_phase3_cand(int n, const int *__restrict__ srp, const int *__restrict__ agg, int keep_isolated,
                              char *cand, char *thr, int *any) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    bool f = agg[i] < 0 && (keep_isolated || srp[i + 1] > srp[i]);
    cand[i] = f;
    thr[i] = f;
    if (f) *any = 1;
}

__global__ void k_mis_m1(int n, const int *__restrict__ srp, const int *__restrict__ sci,
                         const uint64_t *__restrict__ key, const char *__restrict__ cand,
                         const char *__restrict__ thr, uint64_t *m1) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    uint64_t best = 0;
    if (thr[j]) {
        if (cand[j]) best = key[j];
        for (int k = srp[j]; k < srp[j + 1]; ++k) {
            int q = sci[k];
            if (cand[q] && key[q] > best) best = key[q];
        }
    }
    m1[j] = best;
}

__global__ void k_mis_root(int n, const int *__restrict__ srp, const int *__restrict__ sci,
                           const uint64_t *__restrict__ key, const char *__restrict__ cand,
                           const char *__restrict__ thr, const uint64_t *__restrict__ m1, int *isroot) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int r = 0;
    if (cand[i]) {
        uint64_t best = m1[i];
        for (int k = srp[i]; k < srp[i + 1]; ++k) {
            int q = sci[k];
            if (thr[q] && m1[q] > best) best = m1[q];
        }
        r = best == key[i];
    }
    isroot[i] = r;
}

// roots take new ids in ascending root index; each root's strong neighbours (restricted to
// candidates in phase 3) join it
__global__ void k_mis_assign(int n, const int *__restrict__ srp, const int *__restrict__ sci,
                             const int *__restrict__ isroot, const int *__restrict__ rootoff, int base,
                             const char *__restrict__ cand, int only_cand, int *agg) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !isroot[i]) return;
    int id = base + rootoff[i];
    agg[i] = id;
    for (int k = srp[i]; k < srp[i + 1]; ++k) {
        int j = sci[k];
        if (!only_cand || cand[j]) agg[j] = id;
    }
}

// phase 2: join the aggregate of the strongest neighbour in a phase-1 aggregate (ties: lowest id)
__global__ void k_phase2(int n, const int *__restrict__ srp, const int *__restrict__ sci,
                         const double *__restrict__ sv, const int *__restrict__ snap, int *agg) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || snap[i] >= 0) return;
    int best = -1;
    double bw = -1.0;
    for (int k = srp[i]; k < srp[i + 1]; ++k) {
        int j = sci[k];
        if (snap[j] < 0) continue;
        if (sv[k] > bw || (sv[k] == bw && snap[j] < best)) {
            bw = sv[k];
            best = snap[j];
        }
    }
    agg[i] = best;
}

static int read_int(const int *d, cudaStream_t s) {
    int v = 0;
    VEMG_CHECK_CUDA(cudaMemcpyAsync(&v, d, sizeof(int), cudaMemcpyDeviceToHost, s));
    VEMG_CHECK_CUDA(cudaStreamSynchronize(s));
    return v;
}

// Vanek's three aggregation phases made round-synchronous (see the oracle for the rule).
// Isolated nodes (no strong coupling) become singletons when keep_isolated is set (singular
// chains, where P 1 = 1 needs every node), else they stay unaggregated (agg = -1).
// Returns the number of aggregates; agg is allocated in the arena.
static int sa_aggregate(Arena &ar, const DCsr &A, const double *d, double theta, bool keep_isolated, int **agg_out,
                        cudaStream_t s) {
    int n = A.n;
    Scratch<int> slen(n);
    k_strong_len<<<grid_for(n, 256), 256, 0, s>>>(n, A.rp, A.ci, A.v, d, theta, slen);
    VEMG_CHECK_LAUNCH();
    Scratch<int> srp(n + 1);
    int snnz = scan_offsets(slen, srp, n, s);
    Scratch<int> sci(snnz);
    Scratch<double> sv(snnz);
    k_strong_fill<<<grid_for(n, 256), 256, 0, s>>>(n, A.rp, A.ci, A.v, d, theta, srp, sci, sv);
    VEMG_CHECK_LAUNCH();
    Scratch<uint64_t> key(n), m1(n);
    k_agg_keys<<<grid_for(n, 256), 256, 0, s>>>(n, srp, key);
    VEMG_CHECK_LAUNCH();
    int *agg = ar.alloc<int>(n);
    VEMG_CHECK_CUDA(cudaMemsetAsync(agg, 0xff, sizeof(int) * n, s));
    Scratch<char> cand(n), thr(n);
    Scratch<int> isroot(n), rootoff(n + 1), any(1);
    int nagg = 0;
    for (int phase : {1, 3}) {
        for (;;) {
            VEMG_CHECK_CUDA(cudaMemsetAsync(any, 0, sizeof(int), s));
            if (phase == 1)
                k_phase1_cand<<<grid_for(n, 256), 256, 0, s>>>(n, srp, sci, agg, keep_isolated, cand, thr, any);
            else
                k_phase3_cand<<<grid_for(n, 256), 256, 0, s>>>(n, srp, agg, keep_isolated, cand, thr, any);
            VEMG_CHECK_LAUNCH();
            if (!read_int(any, s)) break;
            k_mis_m1<<<grid_for(n, 256), 256, 0, s>>>(n, srp, sci, key, cand, thr, m1);
            VEMG_CHECK_LAUNCH();
            k_mis_root<<<grid_for(n, 256), 256, 0, s>>>(n, srp, sci, key, cand, thr, m1, isroot);
            VEMG_CHECK_LAUNCH();
            int nroots = scan_offsets(isroot, rootoff, n, s);
            k_mis_assign<<<grid_for(n, 256), 256, 0, s>>>(n, srp, sci, isroot, rootoff, nagg, cand, phase == 3, agg);
            VEMG_CHECK_LAUNCH();
            nagg += nroots;
        }
        if (phase == 1) {
            Scratch<int> snap(n);
            VEMG_CHECK_CUDA(cudaMemcpyAsync(snap, agg, sizeof(int) * n, cudaMemcpyDeviceToDevice, s));
            k_phase2<<<grid_for(n, 256), 256, 0, s>>>(n, srp, sci, sv, snap, agg);
            VEMG_CHECK_LAUNCH();
            VEMG_CHECK_CUDA(cudaStreamSynchronize(s));
        }
    }
    *agg_out = agg;
    return nagg;
}

// smoothed prolongator P = (I - omega (D^F)^-1 A^F) P_tent with Vanek's filtered matrix:
// weak off-diagonal entries dropped and lumped into the diagonal, so that each filtered row keeps
// the row sum of A and P keeps the constants (section 6: omega = 2/3). A row with no strong
// coupling, or a non-positive filtered diagonal, keeps its tentative row; an unaggregated row is
// empty.
__global__ void k_prolong_len(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                              const double *__restrict__ v, const double *__restrict__ d, double theta,
                              const int *__restrict__ agg, int *len, int *err) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (agg[i] < 0) {
        len[i] = 0;
        return;
    }
    int u[kMaxRowUnique];
    int c = 0;
    c = insert_unique(u, c, kMaxRowUnique, agg[i]);
    for (int k = rp[i]; k < rp[i + 1]; ++k) {
        int j = ci[k];
        if (j == i || !strong(v[k], d[i], d[j], theta)) continue;
        c = insert_unique(u, c, kMaxRowUnique, agg[j]);
        if (c < 0) { atomic_flag(err, VEMG_EINTERNAL); return; }
    }
    len[i] = c;
}

__global__ void k_prolong_fill(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                               const double *__restrict__ v, const double *__restrict__ d, double theta,
                               double omega, const int *__restrict__ agg, const int *__restrict__ prp, int *pci,
                               double *pv) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || agg[i] < 0) return;
    int lo = prp[i], hi = prp[i + 1];
    int c = 0;
    int *u = pci + lo;
    c = insert_unique(u, c, hi - lo, agg[i]);
    double dF = d[i];
    int nstrong = 0;
    for (int k = rp[i]; k < rp[i + 1]; ++k) {
        int j = ci[k];
        if (j == i) continue;
        if (strong(v[k], d[i], d[j], theta)) {
            c = insert_unique(u, c, hi - lo, agg[j]);
            nstrong++;
        } else {
            dF = dF + v[k];
        }
    }
    for (int k = lo; k < hi; ++k) pv[k] = 0.0;
    for (int k = rp[i]; k < rp[i + 1]; ++k) {
        int j = ci[k];
        double a;
        if (j == i) a = dF;
        else if (strong(v[k], d[i], d[j], theta)) a = v[k];
        else continue;
        int pos = bsearch_row(pci, lo, hi, agg[j]);
        pv[pos] = pv[pos] + a;
    }
    double w = (nstrong > 0 && dF > 0.0) ? omega / dF : 0.0;
    int ai = agg[i];
    for (int k = lo; k < hi; ++k) {
        double t = w * pv[k];
        pv[k] = (pci[k] == ai ? 1.0 : 0.0) - t;
    }
}

// ------------------------------------------------------------------------------------------
// smoothed aggregation with the near-nullspace {1, x, y} (the surface chain of vertically
// unstructured meshes; Vanek, Mandel and Brezina's recipe for fourth-order-like operators). Every
// step takes the oracle's operations in the oracle's order.

static constexpr int kNsd = 3;
static constexpr double kQrDrop = 1e-10;   // relative residual norm below which a column is dropped

// block strength matrix: entry (I, J) = Frobenius norm of the block A_IJ, squares summed over the
// block's rows in ascending order and each row's entries in ascending column order
__global__ void k_block_norm_len(int nblk, const int *__restrict__ bptr, const int *__restrict__ rp,
                                 const int *__restrict__ ci, const int *__restrict__ blk, int *len, int *err) {
    int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= nblk) return;
    int u[kMaxRowUnique];
    int c = 0;
    for (int i = bptr[I]; i < bptr[I + 1]; ++i)
        for (int k = rp[i]; k < rp[i + 1]; ++k) {
            c = insert_unique(u, c, kMaxRowUnique, blk[ci[k]]);
            if (c < 0) { atomic_flag(err, VEMG_EINTERNAL); return; }
        }
    len[I] = c;
}

__global__ void k_block_norm_fill(int nblk, const int *__restrict__ bptr, const int *__restrict__ rp,
                                  const int *__restrict__ ci, const double *__restrict__ v,
                                  const int *__restrict__ blk, const int *__restrict__ srp, int *sci, double *sv) {
    int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= nblk) return;
    const int lo = srp[I], hi = srp[I + 1];
    int c = 0;
    for (int i = bptr[I]; i < bptr[I + 1]; ++i)
        for (int k = rp[i]; k < rp[i + 1]; ++k) c = insert_unique(sci + lo, c, hi - lo, blk[ci[k]]);
    for (int q = lo; q < hi; ++q) sv[q] = 0.0;
    for (int i = bptr[I]; i < bptr[I + 1]; ++i)
        for (int k = rp[i]; k < rp[i + 1]; ++k) {
            int q = bsearch_row(sci, lo, hi, blk[ci[k]]);
            sv[q] = sv[q] + v[k] * v[k];
        }
    for (int q = lo; q < hi; ++q) sv[q] = sqrt(sv[q]);
}

__global__ void k_map_blocks(int n, const int *__restrict__ blk, const int *__restrict__ bagg, int *agg) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) agg[i] = bagg[blk ? blk[i] : i];
}

__global__ void k_member_fill(int n, const int *__restrict__ agg, const int *__restrict__ mptr, int *cur, int *mem) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) mem[mptr[agg[i]] + atomicAdd(cur + agg[i], 1)] = i;
}

// Local QR of each aggregate's near-nullspace rows (members ascending) by modified Gram-Schmidt in
// column order; one thread per aggregate. qv: rows of Q per unknown (n x 3), vt: a column being
// orthogonalised (n), R: Q^T B per aggregate (3 x 3), kept: columns kept per aggregate.
__global__ void k_tentative_qr(int nagg, const int *__restrict__ mptr, const int *__restrict__ mem,
                               const double *__restrict__ B, double *vt, double *qv, double *R, int *kept) {
    int J = blockIdx.x * blockDim.x + threadIdx.x;
    if (J >= nagg) return;
    const int lo = mptr[J], hi = mptr[J + 1];
    int kc = 0;
    for (int c = 0; c < kNsd; ++c) {
        double n0 = 0.0;
        for (int t = lo; t < hi; ++t) {
            int i = mem[t];
            double v = B[(int64_t)i * kNsd + c];
            vt[i] = v;
            n0 = n0 + v * v;
        }
        n0 = sqrt(n0);
        for (int a = 0; a < kc; ++a) {
            double s = 0.0;
            for (int t = lo; t < hi; ++t) {
                int i = mem[t];
                s = s + qv[(int64_t)i * kNsd + a] * vt[i];
            }
            for (int t = lo; t < hi; ++t) {
                int i = mem[t];
                vt[i] = vt[i] - s * qv[(int64_t)i * kNsd + a];
            }
        }
        double nr = 0.0;
        for (int t = lo; t < hi; ++t) nr = nr + vt[mem[t]] * vt[mem[t]];
        nr = sqrt(nr);
        if (!(nr > kQrDrop * n0)) continue;
        for (int t = lo; t < hi; ++t) {
            int i = mem[t];
            qv[(int64_t)i * kNsd + kc] = vt[i] / nr;
        }
        kc++;
    }
    for (int a = 0; a < kc; ++a)
        for (int c = 0; c < kNsd; ++c) {
            double s = 0.0;
            for (int t = lo; t < hi; ++t) {
                int i = mem[t];
                s = s + qv[(int64_t)i * kNsd + a] * B[(int64_t)i * kNsd + c];
            }
            R[(int64_t)J * kNsd * kNsd + a * kNsd + c] = s;
        }
    kept[J] = kc;
}

__global__ void k_pt_len(int n, const int *__restrict__ agg, const int *__restrict__ kept, int *len) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) len[i] = kept[agg[i]];
}

__global__ void k_pt_fill(int n, const int *__restrict__ agg, const int *__restrict__ kept,
                          const int64_t *__restrict__ col0, const int *__restrict__ prp,
                          const double *__restrict__ qv, int *pci, double *pv) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int J = agg[i];
    for (int a = 0; a < kept[J]; ++a) {
        pci[prp[i] + a] = (int)col0[J] + a;
        pv[prp[i] + a] = qv[(int64_t)i * kNsd + a];
    }
}

// coarse near-nullspace rows (the local R's) and node blocks of the coarse unknowns
__global__ void k_coarse_ns(int nagg, const int *__restrict__ kept, const int64_t *__restrict__ col0,
                            const double *__restrict__ R, double *Bc, int *blk, int *bptr) {
    int J = blockIdx.x * blockDim.x + threadIdx.x;
    if (J >= nagg) return;
    for (int a = 0; a < kept[J]; ++a) {
        const int64_t r = col0[J] + a;
        blk[r] = J;
        for (int c = 0; c < kNsd; ++c) Bc[r * kNsd + c] = R[(int64_t)J * kNsd * kNsd + a * kNsd + c];
    }
    bptr[J + 1] = (int)col0[J + 1];
    if (J == 0) bptr[0] = 0;
}

// P = P_t - (omega / A_ii) (A P_t) on the pattern of A P_t (AP holds A P_t and becomes P)
__global__ void k_smooth_unfiltered(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                                    const double *__restrict__ v, const int *__restrict__ trp,
                                    const int *__restrict__ tci, const double *__restrict__ tv,
                                    const int *__restrict__ arp, const int *__restrict__ aci, double *av,
                                    double omega) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int q = bsearch_row(ci, rp[i], rp[i + 1], i);
    double d = q >= 0 ? v[q] : 0.0;
    double w = d > 0.0 ? omega / d : 0.0;
    for (int k = arp[i]; k < arp[i + 1]; ++k) {
        int p = bsearch_row(tci, trp[i], trp[i + 1], aci[k]);
        double pt = p >= 0 ? tv[p] : 0.0;
        double t = w * av[k];
        av[k] = pt - t;
    }
}

__global__ void k_column0(int n, const double *__restrict__ B, double *nu) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) nu[i] = B[(int64_t)i * kNsd];
}

static DCsr csr_spgemm(Arena &ar, const DCsr &L, const DCsr &R, cudaStream_t s);

// One coarsening step of a {1, x, y} chain (singular: every unknown aggregated). Fills L.agg, L.P
// and the next level's B, blk, bptr, nblk; returns the number of coarse unknowns (0: the
// coarsening stops here).
static int coarsen_linear(Arena &ar, Level &L, Level &N, double theta, double omega, cudaStream_t s) {
    const int n = L.A.n;
    Arena tmp;
    int nagg = 0;
    int *bagg = nullptr;
    Scratch<int> err(1);
    VEMG_CHECK_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
    if (L.blk) {
        const int nb = L.nblk;
        Scratch<int> len(nb);
        k_block_norm_len<<<grid_for(nb, 128), 128, 0, s>>>(nb, L.bptr, L.A.rp, L.A.ci, L.blk, len, err);
        VEMG_CHECK_LAUNCH();
        if (int e = read_flag(err, s)) throw Error{e};
        DCsr S;
        S.n = S.m = nb;
        S.rp = tmp.alloc<int>(nb + 1);
        S.nnz = scan_offsets(len, S.rp, nb, s);
        S.ci = tmp.alloc<int>(S.nnz);
        S.v = tmp.alloc<double>(S.nnz);
        k_block_norm_fill<<<grid_for(nb, 128), 128, 0, s>>>(nb, L.bptr, L.A.rp, L.A.ci, L.A.v, L.blk, S.rp, S.ci, S.v);
        VEMG_CHECK_LAUNCH();
        Scratch<double> dS(nb);
        k_diag<<<grid_for(nb, 256), 256, 0, s>>>(nb, S.rp, S.ci, S.v, dS);
        VEMG_CHECK_LAUNCH();
        nagg = sa_aggregate(tmp, S, dS, theta, true, &bagg, s);
    } else {
        Scratch<double> d(n);
        k_diag<<<grid_for(n, 256), 256, 0, s>>>(n, L.A.rp, L.A.ci, L.A.v, d);
        VEMG_CHECK_LAUNCH();
        nagg = sa_aggregate(tmp, L.A, d, theta, true, &bagg, s);
    }
    if (nagg == 0) {
        tmp.release();
        return 0;
    }
    int *agg = ar.alloc<int>(n);
    k_map_blocks<<<grid_for(n, 256), 256, 0, s>>>(n, L.blk, bagg, agg);
    VEMG_CHECK_LAUNCH();
    // members of each aggregate, ascending
    Scratch<int> cnt(nagg + 1), mptr(nagg + 1), cur(nagg), mem(n);
    VEMG_CHECK_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * (nagg + 1), s));
    VEMG_CHECK_CUDA(cudaMemsetAsync(cur, 0, sizeof(int) * nagg, s));
    k_count_cols<<<grid_for(n, 256), 256, 0, s>>>(agg, n, cnt);
    VEMG_CHECK_LAUNCH();
    scan_offsets(cnt, mptr, nagg, s);
    k_member_fill<<<grid_for(n, 256), 256, 0, s>>>(n, agg, mptr, cur, mem);
    VEMG_CHECK_LAUNCH();
    k_sort_segments<<<grid_for(nagg, 128), 128, 0, s>>>(mptr, mem, nagg);
    VEMG_CHECK_LAUNCH();
    // local QR, tentative prolongator, coarse near-nullspace
    Scratch<double> vt(n), qv((int64_t)n * kNsd), R((int64_t)nagg * kNsd * kNsd);
    Scratch<int> kept(nagg);
    k_tentative_qr<<<grid_for(nagg, 64), 64, 0, s>>>(nagg, mptr, mem, L.B, vt, qv, R, kept);
    VEMG_CHECK_LAUNCH();
    Scratch<int64_t> col0(nagg + 1);
    const int64_t nc64 = scan_to64(kept, col0, nagg, s);
    if (nc64 == 0 || nc64 * 10 > (int64_t)n * 9) {
        tmp.release();
        return 0;
    }
    const int nc = (int)nc64;
    DCsr Pt;
    Pt.n = n;
    Pt.m = nc;
    {
        Scratch<int> plen(n);
        k_pt_len<<<grid_for(n, 256), 256, 0, s>>>(n, agg, kept, plen);
        VEMG_CHECK_LAUNCH();
        Pt.rp = tmp.alloc<int>(n + 1);
        Pt.nnz = scan_offsets(plen, Pt.rp, n, s);
        Pt.ci = tmp.alloc<int>(Pt.nnz);
        Pt.v = tmp.alloc<double>(Pt.nnz);
        k_pt_fill<<<grid_for(n, 256), 256, 0, s>>>(n, agg, kept, col0, Pt.rp, qv, Pt.ci, Pt.v);
        VEMG_CHECK_LAUNCH();
    }
    N.B = ar.alloc<double>((int64_t)nc * kNsd);
    N.blk = ar.alloc<int>(nc);
    N.bptr = ar.alloc<int>(nagg + 1);
    N.nblk = nagg;
    k_coarse_ns<<<grid_for(nagg, 128), 128, 0, s>>>(nagg, kept, col0, R, N.B, N.blk, N.bptr);
    VEMG_CHECK_LAUNCH();
    // P = (I - omega D^-1 A) P_t with the unfiltered A
    L.P = csr_spgemm(ar, L.A, Pt, s);
    k_smooth_unfiltered<<<grid_for(n, 128), 128, 0, s>>>(n, L.A.rp, L.A.ci, L.A.v, Pt.rp, Pt.ci, Pt.v, L.P.rp,
                                                         L.P.ci, L.P.v, omega);
    VEMG_CHECK_LAUNCH();
    L.agg = agg;
    VEMG_CHECK_CUDA(cudaStreamSynchronize(s));
    tmp.release();
    return nc;
}

// ------------------------------------------------------------------------------------------
// SOR colouring: greedy first-fit in round-synchronous smallest-last order
//
// Peeling: round t sets the threshold k_t = max(k_{t-1}, smallest remaining degree), k_{-1} = 0,
// and removes every remaining node with at most k_t remaining neighbours, giving it the rank t
// (a k-core peeling; every round removes at least one node). Colouring: a node takes
// the smallest colour absent from its coloured neighbours once every neighbour of larger key
// (rank, hash32(i)) is coloured (Jones-Plassmann rounds). With fixed distinct keys, Jones-
// Plassmann gives exactly the greedy colouring in decreasing key order: when a node is coloured,
// its coloured neighbours are precisely those of larger key.

static constexpr int kRoundBatch = 32;   // rounds launched between two host checks

__device__ __forceinline__ uint64_t colour_key(int rank, int i) {
    return ((uint64_t)(uint32_t)rank << 32) | hash32((uint32_t)i);
}

__global__ void k_offdiag_degree(int n, const int *__restrict__ rp, const int *__restrict__ ci, int *deg,
                                 int *rank) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int d = 0;
    for (int k = rp[i]; k < rp[i + 1]; ++k) d += ci[k] != i;
    deg[i] = d;
    rank[i] = -1;
}

// The rounds work on worklists: a round touches only the nodes it handles and their
// neighbours, so that a round costs about one small kernel launch (the peeling needs thousands
// of rounds on the finest levels).
static constexpr int kRoundBlocks = 152, kRoundThreads = 256;
static constexpr int kRing = 64;   // worklist sizes of the rounds, kept in a ring (> kRoundBatch + 2)

__device__ __forceinline__ void push(int *wl, int *count, int v) { wl[atomicAdd(count, 1)] = v; }

// Peeling round: every node of the worklist leaves with rank `round`; each remaining neighbour
// loses one degree, and one whose degree falls from k + 1 to k joins the next worklist. (A
// neighbour leaving in the same round has degree <= k already and never crosses.) One warp per
// node, its lanes over the node's row, so that the decrements of a row are one round trip.
// The worklist sizes live in a ring: round t reads slot t, fills slot t + 1 and clears slot
// t + 2 for the round after it.
__global__ void __launch_bounds__(kRoundThreads) k_peel_round(const int *__restrict__ wl_in, int *wl_out,
                                                             int *nring, const int *__restrict__ rp,
                                                             const int *__restrict__ ci, int *rank, int *deg, int k,
                                                             int round, int *removed) {
    const int cnt = nring[round % kRing];
    int *n_out = nring + (round + 1) % kRing;
    if (blockIdx.x == 0 && threadIdx.x == 0) nring[(round + 2) % kRing] = 0;
    const int lane = threadIdx.x & 31;
    const int w0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (int q = w0; q < cnt; q += nw) {
        int v = wl_in[q];
        if (lane == 0) rank[v] = round;
        for (int e = rp[v] + lane; e < rp[v + 1]; e += 32) {
            int j = ci[e];
            if (j != v && rank[j] < 0 && atomicSub(deg + j, 1) == k + 1) push(wl_out, n_out, j);
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(removed, cnt);
}

// threshold raise: the smallest degree of the remaining nodes, then every remaining node of at
// most that degree as the next worklist
__global__ void k_peel_min(int n, const int *__restrict__ deg, const int *__restrict__ rank, int *dmin) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    bool in = i < n && rank[i] < 0;
    unsigned d = in ? (unsigned)deg[i] : 0xffffffffu;
    unsigned m = __reduce_min_sync(0xffffffffu, d);
    if ((threadIdx.x & 31) == 0 && m != 0xffffffffu) atomicMin(dmin, (int)m);
}

__global__ void k_peel_fill(int n, const int *__restrict__ deg, const int *__restrict__ rank, int k, int *wl,
                            int *count) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && rank[i] < 0 && deg[i] <= k) push(wl, count, i);
}

// number of neighbours with a larger colouring key: a node is coloured once they all are
__global__ void k_jp_pred(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                          const int *__restrict__ rank, int *pc, int *wl, int *count) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t ki = colour_key(rank[i], i);
    int c = 0;
    for (int k = rp[i]; k < rp[i + 1]; ++k) {
        int j = ci[k];
        c += j != i && colour_key(rank[j], j) > ki;
    }
    pc[i] = c;
    if (c == 0) push(wl, count, i);
}

// Jones-Plassmann round: every node of the worklist (all its larger-key neighbours coloured; no
// two of them neighbours, since the smaller-key one would still wait for the other) takes the
// smallest colour none of its coloured neighbours has, then releases its smaller-key
// neighbours; one released by its last larger-key neighbour joins the next worklist. One warp
// per node: its lanes read the row's colours into a bit mask (colours below 64; a row that uses
// all 64 scans on), then decrement the counts.
__global__ void __launch_bounds__(kRoundThreads) k_jp_round(const int *__restrict__ wl_in, int *wl_out, int *nring,
                                                           int round, const int *__restrict__ rp,
                                                           const int *__restrict__ ci, const int *__restrict__ rank,
                                                           int *pc, int *colour, int *maxc) {
    const int cnt = nring[round % kRing];
    int *n_out = nring + (round + 1) % kRing;
    if (blockIdx.x == 0 && threadIdx.x == 0) nring[(round + 2) % kRing] = 0;
    const int lane = threadIdx.x & 31;
    const int w0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (int q = w0; q < cnt; q += nw) {
        const int v = wl_in[q];
        const int lo = rp[v], hi = rp[v + 1];
        int col = -1;
        for (int base = 0; col < 0; base += 64) {
            unsigned long long used = 0ull;
            for (int e = lo + lane; e < hi; e += 32) {
                int j = ci[e];
                int c = j != v ? colour[j] - base : -1;
                if (c >= 0 && c < 64) used |= 1ull << c;
            }
            unsigned lo32 = __reduce_or_sync(0xffffffffu, (unsigned)used);
            unsigned hi32 = __reduce_or_sync(0xffffffffu, (unsigned)(used >> 32));
            unsigned long long all = ((unsigned long long)hi32 << 32) | lo32;
            if (all != ~0ull) col = base + __ffsll((long long)~all) - 1;
        }
        if (lane == 0) {
            colour[v] = col;
            atomicMax(maxc, col);
        }
        const uint64_t kv = colour_key(rank[v], v);
        for (int e = lo + lane; e < hi; e += 32) {
            int j = ci[e];
            if (j != v && colour_key(rank[j], j) < kv && atomicSub(pc + j, 1) == 1) push(wl_out, n_out, j);
        }
    }
}

__global__ void k_eq_flag(int n, const int *__restrict__ key, int c, int *flag) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) flag[i] = key[i] == c;
}

__global__ void k_scatter_flagged(int n, const int *__restrict__ flag, const int *__restrict__ off, int base,
                                  int *out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && flag[i]) out[base + off[i]] = i;
}

static void colour_level(Arena &ar, Level &L, cudaStream_t s) {
    int n = L.A.n;
    L.colour = ar.alloc<int>(n);
    VEMG_CHECK_CUDA(cudaMemsetAsync(L.colour, 0xff, sizeof(int) * n, s));
    Scratch<int> deg(n), rank(n), pc(n), wl0(n), wl1(n), maxc(1), nring(kRing), removed(1), dmin(1);
    int *wl[2] = {wl0, wl1};
    VEMG_CHECK_CUDA(cudaMemsetAsync(maxc, 0, sizeof(int), s));
    if (n > 0) {
        k_offdiag_degree<<<grid_for(n, 256), 256, 0, s>>>(n, L.A.rp, L.A.ci, deg, rank);
        VEMG_CHECK_LAUNCH();
        VEMG_CHECK_CUDA(cudaMemsetAsync(nring, 0, sizeof(int) * kRing, s));
        VEMG_CHECK_CUDA(cudaMemsetAsync(removed, 0, sizeof(int), s));
    }
    // peeling: raise the threshold whenever the worklist runs empty, else kRoundBatch rounds per
    // host check (rounds after an empty worklist do nothing; their ranks stay unused, which
    // keeps the order of the ranks). Every batch removes a node (a raise guarantees one in its
    // first round): the bound on the batches turns a broken invariant into an error, not a hang.
    int t = 0, k = 0;
    for (int64_t batches = 0; n > 0 && read_int(removed, s) < n; ++batches) {
        if (batches > 2 * (int64_t)n + 64) throw Error{VEMG_EINTERNAL};
        if (read_int(nring + t % kRing, s) == 0) {
            VEMG_CHECK_CUDA(cudaMemsetAsync(dmin, 0x7f, sizeof(int), s));
            k_peel_min<<<grid_for(n, 256), 256, 0, s>>>(n, deg, rank, dmin);
            VEMG_CHECK_LAUNCH();
            k = std::max(k, read_int(dmin, s));
            k_peel_fill<<<grid_for(n, 256), 256, 0, s>>>(n, deg, rank, k, wl[t & 1], nring + t % kRing);
            VEMG_CHECK_LAUNCH();
        }
        for (int u = 0; u < kRoundBatch; ++u, ++t)
            k_peel_round<<<kRoundBlocks, kRoundThreads, 0, s>>>(wl[t & 1], wl[(t + 1) & 1], nring, L.A.rp, L.A.ci,
                                                                rank, deg, k, t, removed);
        VEMG_CHECK_LAUNCH();
    }
    // colouring in decreasing key order: Jones-Plassmann rounds on predecessor counts
    if (n > 0) {
        VEMG_CHECK_CUDA(cudaMemsetAsync(nring, 0, sizeof(int) * kRing, s));
        k_jp_pred<<<grid_for(n, 256), 256, 0, s>>>(n, L.A.rp, L.A.ci, rank, pc, wl[0], nring);
        VEMG_CHECK_LAUNCH();
    }
    t = 0;   // the colouring's first worklist sits in slot 0 of the ring
    for (int64_t batches = 0; n > 0; ++batches) {
        if (batches > (int64_t)n + 64) throw Error{VEMG_EINTERNAL};   // every batch colours a node
        for (int u = 0; u < kRoundBatch; ++u, ++t)
            k_jp_round<<<kRoundBlocks, kRoundThreads, 0, s>>>(wl[t & 1], wl[(t + 1) & 1], nring, t, L.A.rp, L.A.ci,
                                                              rank, pc, L.colour, maxc);
        VEMG_CHECK_LAUNCH();
        if (read_int(nring + t % kRing, s) == 0) break;   // every node coloured
    }
    L.ncolours = n > 0 ? read_int(maxc, s) + 1 : 0;
    L.crow = ar.alloc<int>(n);
    L.cptr.assign(L.ncolours + 1, 0);
    Scratch<int> flag(n), off(n + 1);
    int base = 0;
    for (int c = 0; c < L.ncolours; ++c) {
        k_eq_flag<<<grid_for(n, 256), 256, 0, s>>>(n, L.colour, c, flag);
        VEMG_CHECK_LAUNCH();
        int cnt = scan_offsets(flag, off, n, s);
        k_scatter_flagged<<<grid_for(n, 256), 256, 0, s>>>(n, flag, off, base, L.crow);
        VEMG_CHECK_LAUNCH();
        L.cptr[c] = base;
        base += cnt;
    }
    L.cptr[L.ncolours] = base;
    // entries per colour (for the algorithmic byte count of each sweep launch)
    std::vector<int> hrp(n + 1), hrow(n);
    VEMG_CHECK_CUDA(cudaMemcpyAsync(hrp.data(), L.A.rp, sizeof(int) * (n + 1), cudaMemcpyDeviceToHost, s));
    VEMG_CHECK_CUDA(cudaMemcpyAsync(hrow.data(), L.crow, sizeof(int) * n, cudaMemcpyDeviceToHost, s));
    VEMG_CHECK_CUDA(cudaStreamSynchronize(s));
    L.cnnz.assign(L.ncolours, 0);
    for (int c = 0; c < L.ncolours; ++c)
        for (int k = L.cptr[c]; k < L.cptr[c + 1]; ++k) L.cnnz[c] += hrp[hrow[k] + 1] - hrp[hrow[k]];
}

// ------------------------------------------------------------------------------------------
// coarsest level: dense inverse (projected onto the complement of constants if singular)

__global__ void k_dense_fill(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                             const double *__restrict__ v, double *D) {
    int i = blockIdx.x;
    for (int j = threadIdx.x; j < n; j += blockDim.x) D[(int64_t)i * n + j] = 0.0;
    __syncthreads();
    for (int k = rp[i] + threadIdx.x; k < rp[i + 1]; k += blockDim.x) D[(int64_t)i * n + ci[k]] = v[k];
}

// in-place right-looking Cholesky (lower) of D + sigma 1 1^T, one block
__global__ void k_dense_cholesky(int n, double *D, double sigma, int *err) {
    if (sigma != 0.0)
        for (int k = threadIdx.x; k < n * n; k += blockDim.x) D[k] = D[k] + sigma;
    __syncthreads();
    __shared__ double piv;
    for (int j = 0; j < n; ++j) {
        if (threadIdx.x == 0) {
            double djj = D[(int64_t)j * n + j];
            if (!(djj > 0.0)) {
                atomicCAS(err, 0, VEMG_EBREAKDOWN);
                djj = 1.0;
            }
            piv = sqrt(djj);
            D[(int64_t)j * n + j] = piv;
        }
        __syncthreads();
        for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) D[(int64_t)i * n + j] /= piv;
        __syncthreads();
        int m = n - j - 1;
        for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
            int i = j + 1 + t / m, k = j + 1 + t % m;
            if (k <= i) D[(int64_t)i * n + k] -= D[(int64_t)i * n + j] * D[(int64_t)k * n + j];
        }
        __syncthreads();
    }
}

// column c of the inverse: solve L L^T x = e_c; one thread per column
__global__ void k_dense_inverse_cols(int n, const double *__restrict__ L, double *G) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    // forward: L y = e_c (stored in column c of G)
    for (int i = 0; i < n; ++i) {
        double s = (i == c) ? 1.0 : 0.0;
        for (int k = 0; k < i; ++k) s -= L[(int64_t)i * n + k] * G[(int64_t)k * n + c];
        G[(int64_t)i * n + c] = s / L[(int64_t)i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = G[(int64_t)i * n + c];
        for (int k = i + 1; k < n; ++k) s -= L[(int64_t)k * n + i] * G[(int64_t)k * n + c];
        G[(int64_t)i * n + c] = s / L[(int64_t)i * n + i];
    }
}

// G := Q G Q, Q = I - 1 1^T / n (G symmetric)
__global__ void k_project_dense(int n, double *G) {
    __shared__ double rowmean[1024];
    __shared__ double total;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double s = 0.0;
        for (int j = 0; j < n; ++j) s += G[(int64_t)i * n + j];
        rowmean[i] = s / n;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += rowmean[i];
        total = s / n;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
        int i = t / n, j = t % n;
        G[t] = G[t] - rowmean[i] - rowmean[j] + total;
    }
}

__global__ void k_trace(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                        const double *__restrict__ v, double *out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double s = 0.0;
    for (int i = 0; i < n; ++i)
        for (int k = rp[i]; k < rp[i + 1]; ++k)
            if (ci[k] == i) s += v[k];
    *out = s;
}

// D += sigma nu nu^T (the rank-one regularisation of a singular chain with nullspace nu)
__global__ void k_dense_rank1(int n, double *D, double sigma, const double *__restrict__ nu) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n * n; t += gridDim.x * blockDim.x) {
        int i = t / n, j = t % n;
        D[t] += sigma * nu[i] * nu[j];
    }
}

// G := Q G Q, Q = I - nu nu^T / (nu^T nu) (G symmetric); one block
__global__ void k_project_dense_nu(int n, double *G, const double *__restrict__ nu) {
    __shared__ double gnu[1024];
    __shared__ double nn, nugnu;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double s = 0.0;
        for (int j = 0; j < n; ++j) s += G[(int64_t)i * n + j] * nu[j];
        gnu[i] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int i = 0; i < n; ++i) {
            a += nu[i] * nu[i];
            b += nu[i] * gnu[i];
        }
        nn = a;
        nugnu = b;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
        int i = t / n, j = t % n;
        G[t] = G[t] - (gnu[i] * nu[j] + nu[i] * gnu[j]) / nn + nu[i] * nu[j] * nugnu / (nn * nn);
    }
}

static void coarse_inverse(Arena &ar, Chain &C, cudaStream_t s) {
    Level &L = C.lv[C.nlev - 1];
    int n = L.A.n;
    C.nc = n;
    if (n > 1024) throw Error{VEMG_EINTERNAL};
    double sigma = 0.0;
    if (C.singular) {
        Scratch<double> tr(1);
        k_trace<<<1, 32, 0, s>>>(n, L.A.rp, L.A.ci, L.A.v, tr);
        VEMG_CHECK_LAUNCH();
        double t = 0.0;
        VEMG_CHECK_CUDA(cudaMemcpyAsync(&t, tr.p, sizeof(double), cudaMemcpyDeviceToHost, s));
        VEMG_CHECK_CUDA(cudaStreamSynchronize(s));
        if (C.nu) {
            // sigma nu^T nu = tr(A) / n
            std::vector<double> hnu(n);
            VEMG_CHECK_CUDA(cudaMemcpy(hnu.data(), C.nu, sizeof(double) * n, cudaMemcpyDeviceToHost));
            double nn = 0.0;
            for (int i = 0; i < n; ++i) nn = nn + hnu[i] * hnu[i];
            sigma = t / ((double)n * nn);
        } else {
            sigma = t / ((double)n * (double)n);
        }
    }
    Scratch<double> D((int64_t)n * n);
    Scratch<int> err(1);
    VEMG_CHECK_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
    k_dense_fill<<<n, 128, 0, s>>>(n, L.A.rp, L.A.ci, L.A.v, D);
    VEMG_CHECK_LAUNCH();
    if (C.nu) {
        k_dense_rank1<<<grid_for((int64_t)n * n, 256), 256, 0, s>>>(n, D, sigma, C.nu);
        VEMG_CHECK_LAUNCH();
    }
    k_dense_cholesky<<<1, 1024, 0, s>>>(n, D, C.nu ? 0.0 : sigma, err);
    VEMG_CHECK_LAUNCH();
    C.G = ar.alloc<double>((int64_t)n * n);
    k_dense_inverse_cols<<<grid_for(n, 64), 64, 0, s>>>(n, D, C.G);
    VEMG_CHECK_LAUNCH();
    if (C.singular && C.nu) {
        k_project_dense_nu<<<1, 1024, 0, s>>>(n, C.G, C.nu);
        VEMG_CHECK_LAUNCH();
    } else if (C.singular) {
        k_project_dense<<<1, 1024, 0, s>>>(n, C.G);
        VEMG_CHECK_LAUNCH();
    }
    if (int e = read_flag(err, s)) throw Error{e};
}

// ------------------------------------------------------------------------------------------
// chains

__global__ void k_top_nullspace(int mtop, const int *__restrict__ new2old, const double *__restrict__ xyz, double *B) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= mtop) return;
    const double *p = xyz + 3 * (int64_t)new2old[r];
    B[(int64_t)r * kNsd] = 1.0;
    B[(int64_t)r * kNsd + 1] = p[0];
    B[(int64_t)r * kNsd + 2] = p[1];
}

static DCsr copy_csr(Arena &ar, const DCsr &a, cudaStream_t s) {
    DCsr c = csr_alloc(ar, a.n, a.m, a.nnz);
    VEMG_CHECK_CUDA(cudaMemcpyAsync(c.rp, a.rp, sizeof(int) * (a.n + 1), cudaMemcpyDeviceToDevice, s));
    VEMG_CHECK_CUDA(cudaMemcpyAsync(c.ci, a.ci, sizeof(int) * a.nnz, cudaMemcpyDeviceToDevice, s));
    VEMG_CHECK_CUDA(cudaMemcpyAsync(c.v, a.v, sizeof(double) * a.nnz, cudaMemcpyDeviceToDevice, s));
    return c;
}

// B0: near-nullspace rows of level 0 (n x 3) for a {1, x, y} chain, else null
static void build_chain(Arena &ar, Chain &C, DCsr A0, bool singular, const vemg_options &o, cudaStream_t s,
                        double *B0 = nullptr) {
    C.singular = singular;
    C.nlev = 1;
    C.lv[0].A = A0;
    C.nsd = B0 ? kNsd : 1;
    C.lv[0].B = B0;
    C.lv[0].nblk = A0.n;
    int max_levels = std::min(std::max(o.max_levels, 1), kMaxLevels);
    while (C.nlev < max_levels && C.lv[C.nlev - 1].A.n > o.coarse_max) {
        Level &L = C.lv[C.nlev - 1];
        int n = L.A.n;
        if (C.nsd > 1) {
            Level &N = C.lv[C.nlev];
            if (coarsen_linear(ar, L, N, o.strength, o.omega_p, s) == 0) break;
            L.PT = csr_transpose(ar, L.P, s);
            N.A = galerkin(ar, L.A, L.P, L.PT, s);
            C.nlev++;
            continue;
        }
        Scratch<double> d(n);
        k_diag<<<grid_for(n, 256), 256, 0, s>>>(n, L.A.rp, L.A.ci, L.A.v, d);
        VEMG_CHECK_LAUNCH();
        int *agg = nullptr;
        Arena tmp;
        int nagg = sa_aggregate(tmp, L.A, d, o.strength, singular, &agg, s);
        if (nagg == 0 || (int64_t)nagg * 10 > (int64_t)n * 9) {
            tmp.release();
            break;
        }
        L.agg = ar.alloc<int>(n);
        VEMG_CHECK_CUDA(cudaMemcpyAsync(L.agg, agg, sizeof(int) * n, cudaMemcpyDeviceToDevice, s));
        tmp.release();
        Scratch<int> plen(n), err(1);
        VEMG_CHECK_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
        k_prolong_len<<<grid_for(n, 128), 128, 0, s>>>(n, L.A.rp, L.A.ci, L.A.v, d, o.strength, L.agg, plen, err);
        VEMG_CHECK_LAUNCH();
        if (int e = read_flag(err, s)) throw Error{e};
        L.P.n = n;
        L.P.m = nagg;
        L.P.rp = ar.alloc<int>(n + 1);
        L.P.nnz = scan_offsets(plen, L.P.rp, n, s);
        L.P.ci = ar.alloc<int>(L.P.nnz);
        L.P.v = ar.alloc<double>(L.P.nnz);
        k_prolong_fill<<<grid_for(n, 128), 128, 0, s>>>(n, L.A.rp, L.A.ci, L.A.v, d, o.strength, o.omega_p, L.agg,
                                                         L.P.rp, L.P.ci, L.P.v);
        VEMG_CHECK_LAUNCH();
        L.PT = csr_transpose(ar, L.P, s);
        C.lv[C.nlev].A = galerkin(ar, L.A, L.P, L.PT, s);
        C.nlev++;
    }
    for (int l = 0; l < C.nlev; ++l) {
        Level &L = C.lv[l];
        colour_level(ar, L, s);
        L.diag = ar.alloc<double>(L.A.n);
        k_diag<<<grid_for(L.A.n, 256), 256, 0, s>>>(L.A.n, L.A.rp, L.A.ci, L.A.v, L.diag);
        VEMG_CHECK_LAUNCH();
        L.x = ar.alloc<double>(L.A.n);
        L.b = ar.alloc<double>(L.A.n);
        L.r = ar.alloc<double>(L.A.n);
    }
    C.direct = C.lv[C.nlev - 1].A.n <= o.coarse_max;
    if (C.nsd > 1 && singular) {
        // the coarsest level's nullspace: its first near-nullspace column (the coarse constant)
        const Level &Lc = C.lv[C.nlev - 1];
        C.nu = ar.alloc<double>(Lc.A.n);
        k_column0<<<grid_for(Lc.A.n, 256), 256, 0, s>>>(Lc.A.n, Lc.B, C.nu);
        VEMG_CHECK_LAUNCH();
    }
    if (C.direct) coarse_inverse(ar, C, s);
    VEMG_CHECK_CUDA(cudaStreamSynchronize(s));
}

// ------------------------------------------------------------------------------------------
// the whole setup

void setup(vemg_hierarchy *h, const vemg_csr *Ain, const vemg_mesh *mesh, cudaStream_t s) {
    if (!Ain || !mesh || !mesh->tags || Ain->n != mesh->n_nodes || Ain->n <= 0) throw Error{VEMG_EINVAL};
    Arena &ar = h->arena;
    int n = (int)Ain->n;
    h->n = n;
    // upload the parts of the mesh the setup needs
    Scratch<uint8_t> tags(n);
    VEMG_CHECK_CUDA(cudaMemcpyAsync(tags, mesh->tags, n, cudaMemcpyHostToDevice, s));
    Scratch<int> flag(n), topoff(n + 1);
    k_top_flag<<<grid_for(n, 256), 256, 0, s>>>(tags, n, flag);
    VEMG_CHECK_LAUNCH();
    h->mtop = scan_offsets(flag, topoff, n, s);
    if (h->mtop == 0 || h->mtop == n) throw Error{VEMG_EMESH};
    h->new2old = ar.alloc<int>(n);
    h->old2new = ar.alloc<int>(n);
    k_perm<<<grid_for(n, 256), 256, 0, s>>>(n, h->mtop, flag, topoff, h->new2old, h->old2new);
    VEMG_CHECK_LAUNCH();

    // A in the internal order
    {
        Scratch<int> len(n);
        k_perm_rowlen<<<grid_for(n, 256), 256, 0, s>>>(n, Ain->rowptr, h->new2old, len);
        VEMG_CHECK_LAUNCH();
        DCsr &A = h->A;
        A.n = A.m = n;
        A.rp = ar.alloc<int>(n + 1);
        A.nnz = scan_offsets(len, A.rp, n, s);
        A.ci = ar.alloc<int>(A.nnz);
        A.v = ar.alloc<double>(A.nnz);
        k_perm_fill<<<grid_for(n, 256), 256, 0, s>>>(n, Ain->rowptr, Ain->col, Ain->val, h->new2old, h->old2new,
                                                     A.rp, A.ci, A.v);
        VEMG_CHECK_LAUNCH();
        k_sort_rows_kv<<<grid_for(n, 128), 128, 0, s>>>(A.rp, A.ci, A.v, n);
        VEMG_CHECK_LAUNCH();
    }
    // A_bar
    DCsr Abar;
    {
        int nb = n - h->mtop;
        Scratch<int> len(nb);
        k_bar_rowlen<<<grid_for(nb, 256), 256, 0, s>>>(nb, h->mtop, h->A.rp, h->A.ci, len);
        VEMG_CHECK_LAUNCH();
        Abar.n = Abar.m = nb;
        Abar.rp = ar.alloc<int>(nb + 1);
        Abar.nnz = scan_offsets(len, Abar.rp, nb, s);
        Abar.ci = ar.alloc<int>(Abar.nnz);
        Abar.v = ar.alloc<double>(Abar.nnz);
        k_bar_fill<<<grid_for(nb, 256), 256, 0, s>>>(nb, h->mtop, h->A.rp, h->A.ci, h->A.v, Abar.rp, Abar.ci, Abar.v);
        VEMG_CHECK_LAUNCH();
    }
    if (h->bc == VEMG_NEUMANN) {
        if (!mesh->xyz || !mesh->top_tris || mesh->n_top_tris <= 0) throw Error{VEMG_EINVAL};
        int nt = (int)mesh->n_top_tris;
        Scratch<double> xyz((int64_t)3 * n), bb((int64_t)4 * nt);
        Scratch<int> tri((int64_t)3 * nt), err(1);
        VEMG_CHECK_CUDA(cudaMemcpyAsync(xyz, mesh->xyz, sizeof(double) * 3 * (size_t)n, cudaMemcpyHostToDevice, s));
        VEMG_CHECK_CUDA(cudaMemcpyAsync(tri, mesh->top_tris, sizeof(int) * 3 * (size_t)nt, cudaMemcpyHostToDevice, s));
        VEMG_CHECK_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
        k_tri_bbox<<<grid_for(nt, 256), 256, 0, s>>>(nt, tri, xyz, bb, tags, n, err);
        VEMG_CHECK_LAUNCH();
        if (int e = read_flag(err, s)) throw Error{e};
        // bucket grid bounds (host reduction of the bounding boxes)
        std::vector<double> hb((size_t)4 * nt);
        VEMG_CHECK_CUDA(cudaMemcpyAsync(hb.data(), bb.p, sizeof(double) * 4 * (size_t)nt, cudaMemcpyDeviceToHost, s));
        VEMG_CHECK_CUDA(cudaStreamSynchronize(s));
        double xmin = INFINITY, xmax = -INFINITY, ymin = INFINITY, ymax = -INFINITY;
        for (int t = 0; t < nt; ++t) {
            xmin = std::min(xmin, hb[4 * t]);
            xmax = std::max(xmax, hb[4 * t + 1]);
            ymin = std::min(ymin, hb[4 * t + 2]);
            ymax = std::max(ymax, hb[4 * t + 3]);
        }
        Grid g;
        g.nb = std::max(1, (int)sqrt((double)nt));
        g.x0 = xmin;
        g.y0 = ymin;
        g.sx = xmax > xmin ? xmax - xmin : 1.0;
        g.sy = ymax > ymin ? ymax - ymin : 1.0;
        int nbk = g.nb * g.nb;
        Scratch<int> bcnt(nbk + 1), bptr(nbk + 1), bcur(nbk + 1);
        VEMG_CHECK_CUDA(cudaMemsetAsync(bcnt, 0, sizeof(int) * (nbk + 1), s));
        k_bucket_count<<<grid_for(nt, 256), 256, 0, s>>>(nt, bb, g, bcnt);
        VEMG_CHECK_LAUNCH();
        int tot = scan_offsets(bcnt, bptr, nbk, s);
        Scratch<int> bidx(tot);
        VEMG_CHECK_CUDA(cudaMemcpyAsync(bcur, bptr, sizeof(int) * nbk, cudaMemcpyDeviceToDevice, s));
        k_bucket_fill<<<grid_for(nt, 256), 256, 0, s>>>(nt, bb, g, bcur, bidx);
        VEMG_CHECK_LAUNCH();
        k_sort_segments<<<grid_for(nbk, 128), 128, 0, s>>>(bptr, bidx, nbk);
        VEMG_CHECK_LAUNCH();
        h->tri_of = ar.alloc<int>(n);
        h->bary = ar.alloc<double>((int64_t)3 * n);
        k_locate<<<grid_for(n, 128), 128, 0, s>>>(n, h->mtop, h->new2old, xyz, tri, bb, g, bptr, bidx, h->tri_of,
                                                  h->bary, err);
        VEMG_CHECK_LAUNCH();
        if (int e = read_flag(err, s)) throw Error{e};
        // E~ and its transpose
        Scratch<int> len(n);
        k_ext_rowlen<<<grid_for(n, 256), 256, 0, s>>>(n, h->mtop, h->bary, len);
        VEMG_CHECK_LAUNCH();
        DCsr &E = h->E;
        E.n = n;
        E.m = h->mtop;
        E.rp = ar.alloc<int>(n + 1);
        E.nnz = scan_offsets(len, E.rp, n, s);
        E.ci = ar.alloc<int>(E.nnz);
        E.v = ar.alloc<double>(E.nnz);
        k_ext_fill<<<grid_for(n, 256), 256, 0, s>>>(n, h->mtop, h->tri_of, h->bary, tri, h->old2new, E.rp, E.ci, E.v);
        VEMG_CHECK_LAUNCH();
        h->ET = csr_transpose(ar, E, s);
        h->Ac = galerkin(ar, h->A, h->E, h->ET, s);
        double *B0 = nullptr;
        if (h->opts.surf_nullspace == 3) {
            // {1, x, y} at the top nodes (internal rows 0 .. mtop - 1)
            B0 = ar.alloc<double>((int64_t)h->mtop * kNsd);
            k_top_nullspace<<<grid_for(h->mtop, 256), 256, 0, s>>>(h->mtop, h->new2old, xyz, B0);
            VEMG_CHECK_LAUNCH();
        }
        build_chain(ar, h->surf, copy_csr(ar, h->Ac, s), true, h->opts, s, B0);
    }
    h->bar.is_bar = true;
    build_chain(ar, h->bar, Abar, false, h->opts, s);
    if (h->bc == VEMG_NEUMANN && h->precond == VEMG_PRECOND_SA) {
        build_chain(ar, h->one, copy_csr(ar, h->A, s), true, h->opts, s);
    } else if (h->bc == VEMG_NEUMANN && h->precond == VEMG_PRECOND_VL_SOR) {
        // level 0: A with the vertical extrapolation E~ as its prolongator; below it the SA chain of
        // E~^T A E~ (section 6: the vertical lumping is the first coarsening of the cycle)
        Chain &V = h->one;
        const Chain &S = h->surf;
        if (S.nlev + 1 > kMaxLevels) throw Error{VEMG_EINVAL};
        V.singular = true;
        V.nlev = S.nlev + 1;
        V.lv[0].A = h->A;
        V.lv[0].P = h->E;
        V.lv[0].PT = h->ET;
        for (int l = 0; l < S.nlev; ++l) V.lv[l + 1] = S.lv[l];
        V.direct = S.direct;
        V.nc = S.nc;
        V.G = S.G;
        V.nsd = S.nsd;
        V.nu = S.nu;
        Level &L = V.lv[0];
        colour_level(ar, L, s);
        L.diag = ar.alloc<double>(L.A.n);
        k_diag<<<grid_for(L.A.n, 256), 256, 0, s>>>(L.A.n, L.A.rp, L.A.ci, L.A.v, L.diag);
        VEMG_CHECK_LAUNCH();
        L.x = ar.alloc<double>(L.A.n);
        L.b = ar.alloc<double>(L.A.n);
        L.r = ar.alloc<double>(L.A.n);
    }
    VEMG_CHECK_CUDA(cudaStreamSynchronize(s));
}

}  // namespace vemg
