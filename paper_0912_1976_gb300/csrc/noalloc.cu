// noalloc.cu -- y = A x without any device allocation, for callers that cannot allocate.
//
// vemg_spmv allocates per-call work buffers (the index map from solve order to internal order
// and solve-order copies of x and y). Some callers cannot allocate device memory at all: code
// running where cudaMalloc is forbidden or unsafe (inside a custom allocator's callback, in a
// process whose memory pool must not grow, under a memory budget that was fixed up front).
// vemg_spmv_static computes the same product with its work buffers in one file-scope device
// array of fixed size instead. The array belongs to the library: every device that loads
// libvemg holds it until the process exits.
#include <stdio.h>

#include <mutex>

#include "internal.cuh"

namespace vemg {

// Largest number of unknowns vemg_spmv_static accepts, and its static work array: one int
// (index map) and one double (x in solve order) per unknown, 12 MiB in total.
static constexpr int kStaticMaxUnknowns = 1 << 20;
static constexpr size_t kStaticBytes = (size_t)kStaticMaxUnknowns * (sizeof(int) + sizeof(double));

static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

// Host-side device addresses of g_static_scratch, one per device, resolved once. In host code
// the name g_static_scratch is only a host stand-in; kernels must be given this address.
static std::mutex g_static_mu;
static void *g_static_addr[64] = {nullptr};

static int static_scratch(void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return VEMG_ECUDA;
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p) {
            set_last_cuda_error(e, "cudaGetSymbolAddress", __FILE__, __LINE__);
            return VEMG_ECUDA;
        }
        g_static_addr[dev] = p;
    }
    *out = g_static_addr[dev];
    return VEMG_OK;
}

// index map (solve order -> internal order of the unknowns) and x in solve order
__global__ void k_static_gather(int nu, int off, const int *__restrict__ caller_of, const int *__restrict__ old2new,
                                const double *__restrict__ x, int *__restrict__ s2i, double *__restrict__ xs) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nu) return;
    int k = old2new[caller_of[i]] - off;
    s2i[i] = k;
    xs[i] = x[k];
}

// y[internal row] = sum over the row's sliced-ELL entries (in stored order) of A_ij xs_j
__global__ void k_static_spmv(int nsl, const int *__restrict__ row0, const int *__restrict__ nrow,
                              const int *__restrict__ off, const int *__restrict__ width, const int *__restrict__ col,
                              const double *__restrict__ v, const double *__restrict__ xs,
                              const int *__restrict__ s2i, double *__restrict__ y) {
    int s = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    int lane = threadIdx.x & 31;
    if (s >= nsl || lane >= nrow[s]) return;
    int o = off[s] + lane, w = width[s];
    double acc = 0.0;
    for (int k = 0; k < w; ++k) acc += v[o + 32 * k] * xs[col[o + 32 * k]];
    y[s2i[row0[s] + lane]] = acc;
}

static int spmv_static(vemg_hierarchy *h, const double *x_dev, double *y_dev, cudaStream_t s) {
    if (!h || !x_dev || !y_dev) return VEMG_EINVAL;
    if (!h->caller_of) {
        // vemg_setup builds the solve-order layout (index map and sliced-ELL operator); a
        // hierarchy without it did not come from a successful vemg_setup
        set_last_error_message("vemg_spmv_static: the hierarchy has no solve layout (not set up)");
        return VEMG_EINVAL;
    }
    if (h->nu > kStaticMaxUnknowns) {
        char msg[160];
        snprintf(msg, sizeof(msg), "vemg_spmv_static: %d unknowns, more than the %d its static work array holds",
                 h->nu, kStaticMaxUnknowns);
        set_last_error_message(msg);
        return VEMG_EINVAL;
    }
    void *base = nullptr;
    int rc = static_scratch(&base);
    if (rc != VEMG_OK) return rc;
    int *s2i = (int *)base;
    double *xs = (double *)((unsigned char *)base + (size_t)kStaticMaxUnknowns * sizeof(int));
    const int nu = h->nu, off = h->bc == VEMG_DIRICHLET_TOP ? h->mtop : 0;
    k_static_gather<<<grid_for(nu, 256), 256, 0, s>>>(nu, off, h->caller_of, h->old2new, x_dev, s2i, xs);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
        const Sell &A = h->Aop;
        int64_t threads = (int64_t)A.nslices * 32;
        k_static_spmv<<<grid_for(threads, 128), 128, 0, s>>>(A.nslices, A.row0, A.nrow, A.off, A.width, A.col,
                                                             (const double *)A.v, xs, s2i, y_dev);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        set_last_cuda_error(e, "vemg_spmv_static", __FILE__, __LINE__);
        return VEMG_ECUDA;
    }
    return VEMG_OK;
}

}  // namespace vemg

using namespace vemg;

extern "C" int vemg_spmv_static(vemg_hierarchy *h, const double *x_dev, double *y_dev, void *stream) {
    // no C++ exception crosses the ABI (the helpers above throw none; this is the backstop)
    try {
        return spmv_static(h, x_dev, y_dev, (cudaStream_t)stream);
    } catch (...) {
        return VEMG_EINTERNAL;
    }
}
