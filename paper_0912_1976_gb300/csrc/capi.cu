// capi.cu -- the extern "C" entry points of libvemg (declared in include/vemg.h): argument
// checks, the device allocator, status codes, and introspection of the hierarchy.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <unordered_map>

#include "internal.cuh"

namespace vemg {

// ------------------------------------------------------------------------------------------
// errors

static thread_local char g_cuda_err[256] = {0};

void set_last_cuda_error(cudaError_t e, const char *what, const char *file, int line) {
    snprintf(g_cuda_err, sizeof(g_cuda_err), "%s: %s (%s:%d)", cudaGetErrorString(e), what, file, line);
}

const char *last_cuda_error() { return g_cuda_err; }

void set_last_error_message(const char *msg) { snprintf(g_cuda_err, sizeof(g_cuda_err), "%s", msg); }

// ------------------------------------------------------------------------------------------
// allocator: every block remembers the allocator that made it

struct AllocFns {
    void *(*alloc)(size_t, void *) = nullptr;
    void (*free_fn)(void *, void *) = nullptr;
    void *ctx = nullptr;
};

static std::mutex g_alloc_mu;
static AllocFns g_alloc;
static std::unordered_map<void *, AllocFns> g_owner;

void *dev_alloc_raw(size_t bytes) {
    AllocFns fns;
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        fns = g_alloc;
    }
    void *p = nullptr;
    if (bytes == 0) bytes = 1;
    if (fns.alloc) {
        p = fns.alloc(bytes, fns.ctx);
        if (!p) throw Error{VEMG_ENOMEM};
    } else {
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e == cudaErrorMemoryAllocation) {
            cudaGetLastError();
            throw Error{VEMG_ENOMEM};
        }
        if (e != cudaSuccess) {
            set_last_cuda_error(e, "cudaMalloc", __FILE__, __LINE__);
            throw Error{VEMG_ECUDA};
        }
    }
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    g_owner[p] = fns;
    return p;
}

void dev_free_raw(void *p) {
    if (!p) return;
    AllocFns fns;
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        auto it = g_owner.find(p);
        if (it == g_owner.end()) return;
        fns = it->second;
        g_owner.erase(it);
    }
    if (fns.alloc) {
        if (fns.free_fn) fns.free_fn(p, fns.ctx);
    } else {
        cudaFree(p);
    }
}

static thread_local bool t_scratch_on = false;
static thread_local cudaStream_t t_scratch_s = nullptr;

ScratchStream::ScratchStream(cudaStream_t s) : prev_on(t_scratch_on), prev_s(t_scratch_s) {
    t_scratch_on = true;
    t_scratch_s = s;
}

ScratchStream::~ScratchStream() {
    t_scratch_on = prev_on;
    t_scratch_s = prev_s;
}

void *scratch_alloc(size_t bytes, bool *ordered, cudaStream_t *s) {
    bool custom;
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        custom = g_alloc.alloc != nullptr;
    }
    *ordered = false;
    if (!t_scratch_on || custom) return dev_alloc_raw(bytes);
    void *p = nullptr;
    cudaError_t e = cudaMallocAsync(&p, bytes > 0 ? bytes : 1, t_scratch_s);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        throw Error{VEMG_ENOMEM};
    }
    if (e != cudaSuccess) {
        set_last_cuda_error(e, "cudaMallocAsync", __FILE__, __LINE__);
        throw Error{VEMG_ECUDA};
    }
    *ordered = true;
    *s = t_scratch_s;
    return p;
}

void scratch_free(void *p, bool ordered, cudaStream_t s) {
    if (!p) return;
    if (ordered) cudaFreeAsync(p, s);
    else dev_free_raw(p);
}

template <class F>
static int guarded(F &&f) {
    try {
        return f();
    } catch (const Error &e) {
        return e.code;
    } catch (const std::bad_alloc &) {
        return VEMG_ENOMEM;
    } catch (...) {
        return VEMG_EINTERNAL;
    }
}

static const Chain *chain_of(const vemg_hierarchy *h, int c) {
    if (c == 0) return &h->surf;
    if (c == 1) return &h->bar;
    if (c == 2) return &h->one;
    return nullptr;
}

}  // namespace vemg

using namespace vemg;

extern "C" {

void vemg_default_options(vemg_options *o) {
    if (!o) return;
    o->bc = VEMG_NEUMANN;
    o->precision = VEMG_PREC_FP64;
    o->strength = 0.01;
    o->omega_p = 2.0 / 3.0;
    o->coarse_max = 1024;
    o->max_levels = 10;
    o->precond = VEMG_PRECOND_ADDITIVE;
    o->cycle = VEMG_CYCLE_AUTO;
    o->tail_rows = 0;
    o->surf_nullspace = 1;
    o->tail_cluster = 0;
}

const char *vemg_last_error(void) { return last_cuda_error(); }

int vemg_solve_coefficients(vemg_hierarchy *h, int capacity, double *alpha, double *beta, int *count) {
    return guarded([&] {
        if (!h || !count || capacity < 0) return VEMG_EINVAL;
        if (!h->coef) {
            *count = 0;
            return VEMG_OK;
        }
        if (h->precision != VEMG_PREC_FP64) return VEMG_EINVAL;
        double it = 0.0;
        std::vector<double> c(kCoefCap);
        VEMG_CHECK_CUDA(cudaDeviceSynchronize());
        VEMG_CHECK_CUDA(cudaMemcpy(&it, h->scal + solve_scalar_iters(), sizeof(double), cudaMemcpyDeviceToHost));
        VEMG_CHECK_CUDA(cudaMemcpy(c.data(), h->coef, sizeof(double) * kCoefCap, cudaMemcpyDeviceToHost));
        int k = std::min((int)it, kCoefCap / 2);
        *count = k;
        if (capacity < k || (k > 0 && (!alpha || !beta))) return VEMG_EINVAL;
        for (int j = 0; j < k; ++j) {
            alpha[j] = c[2 * j];
            beta[j] = j == 0 ? 0.0 : c[2 * j - 1];
        }
        return VEMG_OK;
    });
}

// number of eigenvalues of the symmetric tridiagonal (d, e) below x (Sturm sequence)
static int sturm_below(const std::vector<double> &d, const std::vector<double> &e, double x) {
    int cnt = 0;
    double q = 1.0;
    for (size_t j = 0; j < d.size(); ++j) {
        double off = j == 0 ? 0.0 : e[j - 1] * e[j - 1] / q;
        q = (d[j] - x) - off;
        if (q == 0.0) q = -1e-300;
        if (q < 0.0) ++cnt;
    }
    return cnt;
}

int vemg_lanczos_extremes(const double *alpha, const double *beta, int count, double *lmin, double *lmax) {
    if (!alpha || !beta || !lmin || !lmax || count < 1) return VEMG_EINVAL;
    for (int k = 0; k < count; ++k)
        if (!(alpha[k] > 0.0) || (k > 0 && !(beta[k] > 0.0))) return VEMG_EINVAL;
    std::vector<double> d(count), e(count > 1 ? count - 1 : 0);
    for (int k = 0; k < count; ++k) {
        d[k] = 1.0 / alpha[k] + (k > 0 ? beta[k] / alpha[k - 1] : 0.0);
        if (k + 1 < count) e[k] = std::sqrt(beta[k + 1]) / alpha[k];
    }
    // Gershgorin interval
    double lo = d[0], hi = d[0];
    for (int k = 0; k < count; ++k) {
        double rad = (k > 0 ? std::fabs(e[k - 1]) : 0.0) + (k + 1 < count ? std::fabs(e[k]) : 0.0);
        lo = std::min(lo, d[k] - rad);
        hi = std::max(hi, d[k] + rad);
    }
    auto kth = [&](int which) {   // the eigenvalue with index `which` (0 = smallest)
        double a = lo, b = hi;
        for (int it = 0; it < 200 && b - a > 1e-15 * std::max(std::fabs(a), std::fabs(b)); ++it) {
            double m = 0.5 * (a + b);
            if (sturm_below(d, e, m) > which) b = m;
            else a = m;
        }
        return 0.5 * (a + b);
    };
    *lmin = kth(0);
    *lmax = kth(count - 1);
    return VEMG_OK;
}

int vemg_selftest_barrier(int claimed_blocks, int launched_blocks, void *stream) {
    return guarded([&] { return barrier_selftest(claimed_blocks, launched_blocks, (cudaStream_t)stream); });
}

const char *vemg_strerror(int s) {
    switch (s) {
        case VEMG_OK: return "VEMG_OK";
        case VEMG_EINVAL: return "VEMG_EINVAL: invalid argument";
        case VEMG_EMESH: return "VEMG_EMESH: invalid mesh";
        case VEMG_ENOMEM: return "VEMG_ENOMEM: device allocation failed";
        case VEMG_ENOTCONV: return "VEMG_ENOTCONV: not converged within max_it";
        case VEMG_EBREAKDOWN: return "VEMG_EBREAKDOWN: Krylov breakdown (p^T A p <= 0 or NaN)";
        case VEMG_ETIMEOUT: return "VEMG_ETIMEOUT: bounded device wait expired";
        case VEMG_ECUDA: return "VEMG_ECUDA: CUDA runtime error";
        case VEMG_EINTERNAL: return "VEMG_EINTERNAL: internal capacity exceeded";
        default: return "unknown vemg status";
    }
}

int vemg_set_allocator(void *(*alloc)(size_t, void *), void (*free_fn)(void *, void *), void *ctx) {
    if (alloc && !free_fn) return VEMG_EINVAL;
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    g_alloc.alloc = alloc;
    g_alloc.free_fn = alloc ? free_fn : nullptr;
    g_alloc.ctx = alloc ? ctx : nullptr;
    return VEMG_OK;
}

int vemg_assemble(const vemg_mesh *mesh, vemg_csr *A_out, void *stream) {
    return guarded([&] {
        if (!mesh || !A_out) return VEMG_EINVAL;
        ScratchStream scratch((cudaStream_t)stream);
        assemble(mesh, A_out, (cudaStream_t)stream);
        return VEMG_OK;
    });
}

int vemg_load(const vemg_mesh *mesh, const double *f_dev, double *b_dev, void *stream) {
    return guarded([&] {
        if (!mesh || !f_dev || !b_dev) return VEMG_EINVAL;
        load_vector(mesh, f_dev, b_dev, (cudaStream_t)stream);
        return VEMG_OK;
    });
}

void vemg_csr_free(vemg_csr *A) {
    if (!A) return;
    dev_free_raw(A->rowptr);
    dev_free_raw(A->col);
    dev_free_raw(A->val);
    A->rowptr = nullptr;
    A->col = nullptr;
    A->val = nullptr;
    A->n = A->nnz = 0;
}

int vemg_setup(const vemg_csr *A, const vemg_mesh *mesh, const vemg_options *opts, void *stream,
               vemg_hierarchy **out) {
    if (!out) return VEMG_EINVAL;
    *out = nullptr;
    vemg_hierarchy *h = nullptr;
    int rc = guarded([&] {
        if (!A || !mesh || !A->rowptr || !A->col || !A->val) return VEMG_EINVAL;
        vemg_options o;
        vemg_default_options(&o);
        if (opts) o = *opts;
        if ((o.bc != VEMG_NEUMANN && o.bc != VEMG_DIRICHLET_TOP) ||
            (o.precision != VEMG_PREC_FP64 && o.precision != VEMG_PREC_FP32 && o.precision != VEMG_PREC_BF16) ||
            !(o.strength >= 0.0) ||
            !(o.omega_p > 0.0) || o.coarse_max < 1 || o.coarse_max > 1024 || o.max_levels < 1 ||
            o.tail_rows < 0 || o.tail_rows > (o.tail_cluster > 0 ? 262144 : 65536) || o.tail_cluster < 0 ||
            o.tail_cluster == 1 || o.tail_cluster > 16 || (o.surf_nullspace != 1 && o.surf_nullspace != 3) ||
            o.max_levels > kMaxLevels || o.precond < VEMG_PRECOND_ADDITIVE || o.precond > VEMG_PRECOND_NONE ||
            (o.precond == VEMG_PRECOND_VL_SOR && o.bc != VEMG_NEUMANN) ||
            (o.cycle != VEMG_CYCLE_PERSISTENT && o.cycle != VEMG_CYCLE_LAUNCHES && o.cycle != VEMG_CYCLE_AUTO &&
             o.cycle != VEMG_CYCLE_HYBRID))
            return VEMG_EINVAL;
        h = new vemg_hierarchy();
        if (o.precond == VEMG_PRECOND_NONE) {   // plain CG: nothing to run in FP32 or persistently
            o.precision = VEMG_PREC_FP64;
            o.cycle = VEMG_CYCLE_LAUNCHES;
        }
        if (o.precision == VEMG_PREC_BF16) o.cycle = VEMG_CYCLE_LAUNCHES;   // BF16 values: per-phase kernels
        // one kernel per phase, each loading its operator rows before it waits on its
        // predecessor, measured fastest for every precision on the 256x256x32 workload
        if (o.cycle == VEMG_CYCLE_AUTO) o.cycle = VEMG_CYCLE_LAUNCHES;
        h->opts = o;
        h->bc = o.bc;
        h->precision = o.precision;
        h->precond = (o.bc == VEMG_DIRICHLET_TOP && o.precond != VEMG_PRECOND_NONE) ? VEMG_PRECOND_ADDITIVE
                                                                                   : o.precond;
        ScratchStream scratch((cudaStream_t)stream);
        setup(h, A, mesh, (cudaStream_t)stream);
        prepare_solve(h, (cudaStream_t)stream);
        return VEMG_OK;
    });
    if (rc != VEMG_OK) {
        if (h) {
            cudaStreamSynchronize((cudaStream_t)stream);
            release_graphs(h);
            release_batch(h);
            h->arena.release();
            delete h;
        }
        return rc;
    }
    *out = h;
    return VEMG_OK;
}

void vemg_destroy(vemg_hierarchy *h) {
    if (!h) return;
    cudaDeviceSynchronize();
    release_graphs(h);
    release_batch(h);
    release_persist(h);
    release_ctail(h->ssurf);
    release_ctail(h->sbar);
    for (auto &e : h->probe.ev) cudaEventDestroy(e);
    h->arena.release();
    delete h;
}

int vemg_solve(vemg_hierarchy *h, const double *b_dev, double *x_dev, double rtol, int max_it, vemg_info *info,
               void *stream) {
    vemg_info local{};
    if (!info) info = &local;
    return guarded([&] {
        if (!h || !b_dev || !x_dev || !(rtol >= 0.0) || max_it < 0) return VEMG_EINVAL;
        return solve(h, b_dev, x_dev, rtol, max_it, info, (cudaStream_t)stream);
    });
}

int vemg_solve_host(vemg_hierarchy *h, const double *b_host, double *x_host, double rtol, int max_it,
                    vemg_info *info, void *stream) {
    vemg_info local{};
    if (!info) info = &local;
    return guarded([&] {
        if (!h || !b_host || !x_host || !(rtol >= 0.0) || max_it < 0) return VEMG_EINVAL;
        cudaStream_t s = (cudaStream_t)stream;
        if (!h->host_b || !h->host_x) {   // kept with the hierarchy: no allocation (nor its free) per call
            double *hb = h->host_b ? h->host_b : h->arena.alloc<double>(h->n);
            h->host_b = hb;
            h->host_x = h->arena.alloc<double>(h->n);
        }
        VEMG_CHECK_CUDA(cudaMemcpyAsync(h->host_b, b_host, sizeof(double) * h->n, cudaMemcpyHostToDevice, s));
        int rc = solve(h, h->host_b, h->host_x, rtol, max_it, info, s);
        VEMG_CHECK_CUDA(cudaMemcpyAsync(x_host, h->host_x, sizeof(double) * h->n, cudaMemcpyDeviceToHost, s));
        VEMG_CHECK_CUDA(cudaStreamSynchronize(s));
        return rc;
    });
}

int vemg_solve_batch(vemg_hierarchy *h, int k, const double *B_dev, int64_t ldb, double *X_dev, int64_t ldx,
                     double rtol, int max_it, vemg_info *infos, void *stream) {
    return guarded([&] {
        if (!h || k < 0 || (k > 0 && (!B_dev || !X_dev || !infos)) || ldb < h->n || ldx < h->n ||
            !(rtol >= 0.0) || max_it < 0)
            return VEMG_EINVAL;
        return solve_batch(h, k, B_dev, ldb, X_dev, ldx, rtol, max_it, infos, (cudaStream_t)stream);
    });
}

int vemg_hierarchy_bytes(const vemg_hierarchy *h, size_t *bytes) {
    if (!h || !bytes) return VEMG_EINVAL;
    *bytes = h->arena.bytes;
    return VEMG_OK;
}

int vemg_get_size(const vemg_hierarchy *h, const char *key, int chain, int level, int64_t *out) {
    if (!h || !key || !out) return VEMG_EINVAL;
    const Chain *C = chain_of(h, chain);
    *out = -1;
    if (!strcmp(key, "n")) *out = h->n;
    else if (!strcmp(key, "mtop")) *out = h->mtop;
    else if (!strcmp(key, "nnzA")) *out = h->A.nnz;
    else if (!strcmp(key, "nnzE")) *out = h->E.nnz;
    else if (!strcmp(key, "nnzAc")) *out = h->Ac.nnz;
    else if (C && !strcmp(key, "nlev")) *out = C->nlev;
    else if (C && !strcmp(key, "direct")) *out = C->direct;
    else if (C && !strcmp(key, "nsd")) *out = C->nsd;
    else if (C && level >= 0 && level < C->nlev) {
        const Level &L = C->lv[level];
        if (!strcmp(key, "lev.n")) *out = L.A.n;
        else if (!strcmp(key, "lev.nnz")) *out = L.A.nnz;
        else if (!strcmp(key, "lev.nnzP")) *out = L.P.nnz;
        else if (!strcmp(key, "lev.ncolours")) *out = L.ncolours;
    }
    return VEMG_OK;
}

int vemg_get_nullspace(const vemg_hierarchy *h, int chain, int level, double *out) {
    return guarded([&] {
        const Chain *C = h ? chain_of(h, chain) : nullptr;
        if (!C || !out || level < 0 || level >= C->nlev || !C->lv[level].B) return VEMG_EINVAL;
        VEMG_CHECK_CUDA(cudaDeviceSynchronize());
        VEMG_CHECK_CUDA(cudaMemcpy(out, C->lv[level].B, sizeof(double) * 3 * (size_t)C->lv[level].A.n,
                                   cudaMemcpyDeviceToHost));
        return VEMG_OK;
    });
}

int vemg_get_csr(const vemg_hierarchy *h, const char *name, int chain, int level, int32_t *rp, int32_t *ci,
                 double *v) {
    return guarded([&] {
        if (!h || !name || !rp || !ci || !v) return VEMG_EINVAL;
        const DCsr *a = nullptr;
        const Chain *C = chain_of(h, chain);
        if (!strcmp(name, "A")) a = &h->A;
        else if (!strcmp(name, "E")) a = &h->E;
        else if (!strcmp(name, "Ac")) a = &h->Ac;
        else if (C && level >= 0 && level < C->nlev) {
            if (!strcmp(name, "lev.A")) a = &C->lv[level].A;
            else if (!strcmp(name, "lev.P")) a = &C->lv[level].P;
        }
        if (!a || !a->rp) return VEMG_EINVAL;
        VEMG_CHECK_CUDA(cudaDeviceSynchronize());
        VEMG_CHECK_CUDA(cudaMemcpy(rp, a->rp, sizeof(int) * (a->n + 1), cudaMemcpyDeviceToHost));
        VEMG_CHECK_CUDA(cudaMemcpy(ci, a->ci, sizeof(int) * a->nnz, cudaMemcpyDeviceToHost));
        VEMG_CHECK_CUDA(cudaMemcpy(v, a->v, sizeof(double) * a->nnz, cudaMemcpyDeviceToHost));
        return VEMG_OK;
    });
}

int vemg_get_int(const vemg_hierarchy *h, const char *name, int chain, int level, int32_t *out) {
    return guarded([&] {
        if (!h || !name || !out) return VEMG_EINVAL;
        const int *src = nullptr;
        int cnt = 0;
        const Chain *C = chain_of(h, chain);
        if (!strcmp(name, "new2old")) { src = h->new2old; cnt = h->n; }
        else if (!strcmp(name, "tri_of")) { src = h->tri_of; cnt = h->n; }
        else if (C && level >= 0 && level < C->nlev) {
            if (!strcmp(name, "lev.agg")) { src = C->lv[level].agg; cnt = C->lv[level].A.n; }
            else if (!strcmp(name, "lev.colour")) { src = C->lv[level].colour; cnt = C->lv[level].A.n; }
        }
        if (!src) return VEMG_EINVAL;
        VEMG_CHECK_CUDA(cudaDeviceSynchronize());
        VEMG_CHECK_CUDA(cudaMemcpy(out, src, sizeof(int) * cnt, cudaMemcpyDeviceToHost));
        return VEMG_OK;
    });
}

int vemg_spmv(vemg_hierarchy *h, const double *x, double *y, void *stream) {
    return guarded([&] {
        if (!h || !x || !y) return VEMG_EINVAL;
        spmv_op(h, x, y, (cudaStream_t)stream);
        VEMG_CHECK_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
        return VEMG_OK;
    });
}

int vemg_precond(vemg_hierarchy *h, const double *r, double *z, void *stream) {
    return guarded([&] {
        if (!h || !r || !z) return VEMG_EINVAL;
        precond(h, r, z, (cudaStream_t)stream);
        VEMG_CHECK_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
        return VEMG_OK;
    });
}

int vemg_vcycle(vemg_hierarchy *h, int chain, const double *b, double *x, void *stream) {
    return guarded([&] {
        if (!h || !b || !x || chain < 0 || chain > 2) return VEMG_EINVAL;
        vcycle(h, chain, b, x, (cudaStream_t)stream);
        VEMG_CHECK_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
        return VEMG_OK;
    });
}

int vemg_kernel_launches(const vemg_hierarchy *h, int64_t *count) {
    if (!h || !count) return VEMG_EINVAL;
    *count = h->launches;
    return VEMG_OK;
}

int vemg_probe(vemg_hierarchy *h, int kind) {
    return guarded([&] {
        if (!h || kind < VEMG_PROBE_NONE || kind > VEMG_PROBE_TAIL) return VEMG_EINVAL;
        probe_start(h, kind);
        if (kind == VEMG_PROBE_VCYCLE) persist_profile_reset(h);
        if (kind == VEMG_PROBE_TAIL) {
            ctail_profile_reset(h->ssurf);
            ctail_profile_reset(h->sbar);
        }
        return VEMG_OK;
    });
}

int vemg_probe_phases(vemg_hierarchy *h, int capacity, int *count, int *op, int *level, int *group,
                      double *cycles) {
    return guarded([&] {
        if (!h || !count || capacity < 0 || (capacity > 0 && (!op || !level || !group || !cycles)))
            return VEMG_EINVAL;
        if (h->persist || !(h->ssurf.ctail || h->sbar.ctail))
            return persist_profile(h, capacity, count, op, level, group, cycles);
        // the cluster tails: the surface chain's as group 0, the A_bar chain's as group 1
        std::vector<int> o, l, g;
        std::vector<double> c;
        ctail_profile(h->ssurf, 0, o, l, g, c);
        ctail_profile(h->sbar, 1, o, l, g, c);
        *count = (int)o.size();
        if (capacity < *count) return VEMG_EINVAL;
        for (int k = 0; k < *count; ++k) {
            op[k] = o[k];
            level[k] = l[k];
            group[k] = g[k];
            cycles[k] = c[k];
        }
        return VEMG_OK;
    });
}

int vemg_probe_read(vemg_hierarchy *h, double *total_ms, int64_t *launches, double *bytes) {
    return guarded([&] {
        if (!h || !total_ms || !launches || !bytes) return VEMG_EINVAL;
        probe_read(h, total_ms, launches, bytes);
        return VEMG_OK;
    });
}

}  // extern "C"
