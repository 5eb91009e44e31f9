/*
 * vemg_oracle.c -- plain, slow, FP64 CPU oracle of the vertical-extrapolation multigrid PCG
 * of Kramer, Cotter and Pain, "Solving the Poisson equation on small aspect ratio domains
 * using unstructured meshes".
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the benchmark's CPU-baseline
 * leg may load this library. The product path (libvemg) shares no code with it.
 *
 * Build: gcc -O2 -ffp-contract=off -shared -fPIC (no fused multiply-add, so that every
 * floating-point decision in the setup is reproducible bit for bit). A timing build adds -fopenmp:
 * the solve's row loops (SpMV, the rows of one SOR colour, residuals, transfers, vector updates)
 * then run on all host cores, and every sum over a vector is taken in fixed blocks of OR_BLOCK
 * entries added in block order, so that both builds give the same bits whatever the thread count.
 *
 * What it computes, in the paper's order and notation:
 *   - P1 stiffness matrix A of -Laplace(phi) with all-Neumann boundaries (section 3, Eq. Ax=b)
 *     and the load vector M f;
 *   - the block ordering phi = (phi', phi_bar): top-surface nodes first (section 3,
 *     Eqs. phi_decomposition / equation_decomposition), so that A_bar, the Dirichlet-top
 *     matrix, is the trailing principal block;
 *   - the vertical extrapolation operator E~ (section 5.4, Fig. vertical_interpolation):
 *     each node is projected straight up onto the top triangulation and interpolated
 *     barycentrically from the three vertices of the triangle it lands in;
 *   - the Galerkin surface operator E~^T A E~ (section 5.1, Eq. reduced AMG);
 *   - smoothed-aggregation AMG (section 5.1 and section 6: strength |A_ij| > 0.01
 *     sqrt(A_ii A_jj), prolongator smoothing with omega = 2/3, one forward SOR sweep
 *     (omega = 1) before and one backward sweep after the coarse correction);
 *   - the additive preconditioner of Eq. ourpreconditioner (section 5.5):
 *       z = E~ MG(E~^T A E~) E~^T r + [0; I] MG_SA(A_bar) [0; I]^T r;
 *   - preconditioned CG with the constant nullspace projected out of each preconditioned
 *     residual (section 3, the BoLe05 remark), or flexible CG (Notay's FCG(1)).
 *
 * Readings where the paper is silent (all shared with the GPU path by definition, not by code):
 *   aggregation is made round-synchronous (distance-2 maximal independent sets with a fixed
 *   integer hash), the SOR ordering is multicolour with the colours of a greedy colouring in
 *   round-synchronous smallest-last order (ties broken by the same hash), the Galerkin product is
 *   P^T (A P) with entries summed in ascending index order and the lower triangle copied from
 *   the upper, the coarsest level is a dense Cholesky solve (regularised by a rank-one term
 *   on the singular surface chain).
 */
#include <math.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#define OR_PARALLEL_FOR _Pragma("omp parallel for schedule(static)")
#else
#define OR_PARALLEL_FOR
#endif
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_EINVAL 1
#define OR_EMESH 2
#define OR_ENOMEM 3
#define OR_ENOTCONV 4
#define OR_EBREAKDOWN 5

#define TAG_TOP 1

#define BC_NEUMANN 0
#define BC_DIRICHLET_TOP 1

/* the three preconditioners compared in section 6 */
#define PC_ADDITIVE 0   /* vertical lumping + additive smoother, Eq. ourpreconditioner (section 5.5) */
#define PC_VL_SOR 1     /* vertical lumping as the first coarsening of a V-cycle with SOR smoothing on A */
#define PC_SA 2         /* smoothed-aggregation AMG on A */
#define PC_NONE 3       /* no preconditioner: plain CG (the spectrum of A itself, section 4) */

#define MAX_LEVELS_CAP 16

/* ------------------------------------------------------------------------------------------ */
/* small helpers                                                                              */

typedef struct {
    int n, m; /* rows, cols */
    int *rp;  /* n + 1 */
    int *ci;  /* nnz */
    double *v;/* nnz */
} csr;

static void *xcalloc(size_t n, size_t s) {
    void *p = calloc(n ? n : 1, s);
    if (!p) { fprintf(stderr, "oracle: out of memory\n"); abort(); }
    return p;
}

static csr csr_new(int n, int m, int nnz) {
    csr a;
    a.n = n; a.m = m;
    a.rp = (int *)xcalloc((size_t)n + 1, sizeof(int));
    a.ci = (int *)xcalloc((size_t)nnz, sizeof(int));
    a.v = (double *)xcalloc((size_t)nnz, sizeof(double));
    return a;
}

static void csr_del(csr *a) {
    free(a->rp); free(a->ci); free(a->v);
    a->rp = NULL; a->ci = NULL; a->v = NULL; a->n = a->m = 0;
}

static int csr_nnz(const csr *a) { return a->rp[a->n]; }

/* position of column j in row i, -1 if absent (rows are sorted) */
static int csr_find(const csr *a, int i, int j) {
    int lo = a->rp[i], hi = a->rp[i + 1] - 1;
    while (lo <= hi) {
        int mid = (lo + hi) >> 1;
        if (a->ci[mid] == j) return mid;
        if (a->ci[mid] < j) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

static void isort(int *a, int n) {
    for (int i = 1; i < n; ++i) {
        int x = a[i], j = i - 1;
        while (j >= 0 && a[j] > x) { a[j + 1] = a[j]; --j; }
        a[j + 1] = x;
    }
}

static int cmp_int(const void *a, const void *b) {
    int x = *(const int *)a, y = *(const int *)b;
    return (x > y) - (x < y);
}

/* MurmurHash3 32-bit finalizer (Austin Appleby, public domain): a bijection on 32-bit words,
   used as the fixed priority of the round-synchronous aggregation and colouring rules. */
static uint32_t hash32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

/* transpose with rows of the result in ascending column order of the source */
static csr csr_transpose(const csr *a) {
    int nnz = csr_nnz(a);
    csr t = csr_new(a->m, a->n, nnz);
    for (int k = 0; k < nnz; ++k) t.rp[a->ci[k] + 1]++;
    for (int i = 0; i < a->m; ++i) t.rp[i + 1] += t.rp[i];
    int *cur = (int *)xcalloc((size_t)a->m, sizeof(int));
    memcpy(cur, t.rp, sizeof(int) * (size_t)a->m);
    for (int i = 0; i < a->n; ++i)
        for (int k = a->rp[i]; k < a->rp[i + 1]; ++k) {
            int p = cur[a->ci[k]]++;
            t.ci[p] = i;
            t.v[p] = a->v[k];
        }
    free(cur);
    return t;
}

/* C = L R, Gustavson's row-by-row product. Entry C_ij = sum over a ascending of L_ia R_aj,
   accumulated from 0.0 one product at a time. The pattern is structural (every (i, j) that
   receives a product is stored, even if its value is zero). */
static csr csr_spgemm(const csr *L, const csr *R) {
    int n = L->n, m = R->m;
    int *mark = (int *)xcalloc((size_t)m, sizeof(int));
    for (int j = 0; j < m; ++j) mark[j] = -1;
    int *rp = (int *)xcalloc((size_t)n + 1, sizeof(int));
    for (int i = 0; i < n; ++i) {
        int cnt = 0;
        for (int ka = L->rp[i]; ka < L->rp[i + 1]; ++ka) {
            int a = L->ci[ka];
            for (int kb = R->rp[a]; kb < R->rp[a + 1]; ++kb) {
                int j = R->ci[kb];
                if (mark[j] != i) { mark[j] = i; cnt++; }
            }
        }
        rp[i + 1] = rp[i] + cnt;
    }
    csr c = csr_new(n, m, rp[n]);
    memcpy(c.rp, rp, sizeof(int) * ((size_t)n + 1));
    free(rp);
    double *acc = (double *)xcalloc((size_t)m, sizeof(double));
    for (int j = 0; j < m; ++j) mark[j] = -1;
    for (int i = 0; i < n; ++i) {
        int cnt = 0, base = c.rp[i];
        for (int ka = L->rp[i]; ka < L->rp[i + 1]; ++ka) {
            int a = L->ci[ka];
            double la = L->v[ka];
            for (int kb = R->rp[a]; kb < R->rp[a + 1]; ++kb) {
                int j = R->ci[kb];
                if (mark[j] != i) { mark[j] = i; acc[j] = 0.0; c.ci[base + cnt++] = j; }
                acc[j] = acc[j] + la * R->v[kb];
            }
        }
        qsort(c.ci + base, (size_t)cnt, sizeof(int), cmp_int);
        for (int k = 0; k < cnt; ++k) c.v[base + k] = acc[c.ci[base + k]];
    }
    free(acc); free(mark);
    return c;
}

/* copy the upper triangle onto the lower one: C_ij := C_ji for j < i (exact symmetry) */
static void csr_mirror_upper(csr *c) {
    for (int i = 0; i < c->n; ++i)
        for (int k = c->rp[i]; k < c->rp[i + 1]; ++k) {
            int j = c->ci[k];
            if (j < i) {
                int q = csr_find(c, j, i);
                if (q >= 0) c->v[k] = c->v[q];
            }
        }
}

/* Galerkin product P^T (A P), then exact symmetrisation from the upper triangle */
static csr galerkin(const csr *A, const csr *P, const csr *PT) {
    csr AP = csr_spgemm(A, P);
    csr C = csr_spgemm(PT, &AP);
    csr_del(&AP);
    csr_mirror_upper(&C);
    return C;
}

static void csr_spmv(const csr *a, const double *x, double *y) {
    OR_PARALLEL_FOR
    for (int i = 0; i < a->n; ++i) {
        double s = 0.0;
        for (int k = a->rp[i]; k < a->rp[i + 1]; ++k) s += a->v[k] * x[a->ci[k]];
        y[i] = s;
    }
}

/* Sums over vectors: the partial sums of fixed blocks of OR_BLOCK entries (each in index order),
   added in block order. The blocks do not depend on the number of threads. */
#define OR_BLOCK 4096

static double dot(int n, const double *a, const double *b) {
    int nb = (n + OR_BLOCK - 1) / OR_BLOCK;
    double *part = (double *)xcalloc((size_t)(nb > 0 ? nb : 1), sizeof(double));
    OR_PARALLEL_FOR
    for (int k = 0; k < nb; ++k) {
        double s = 0.0;
        int hi = (k + 1) * OR_BLOCK < n ? (k + 1) * OR_BLOCK : n;
        for (int i = k * OR_BLOCK; i < hi; ++i) s += a[i] * b[i];
        part[k] = s;
    }
    double s = 0.0;
    for (int k = 0; k < nb; ++k) s += part[k];
    free(part);
    return s;
}

static double vsum(int n, const double *a) {
    int nb = (n + OR_BLOCK - 1) / OR_BLOCK;
    double *part = (double *)xcalloc((size_t)(nb > 0 ? nb : 1), sizeof(double));
    OR_PARALLEL_FOR
    for (int k = 0; k < nb; ++k) {
        double s = 0.0;
        int hi = (k + 1) * OR_BLOCK < n ? (k + 1) * OR_BLOCK : n;
        for (int i = k * OR_BLOCK; i < hi; ++i) s += a[i];
        part[k] = s;
    }
    double s = 0.0;
    for (int k = 0; k < nb; ++k) s += part[k];
    free(part);
    return s;
}

/* the number of threads the solve's loops use (1 without OpenMP) */
int or_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void or_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------------------------------ */
/* P1 element matrices (section 3: A_ij = integral of grad N_i . grad N_j, M_ij = integral N_i N_j) */

static void cross3(const double *u, const double *v, double *w) {
    w[0] = u[1] * v[2] - u[2] * v[1];
    w[1] = u[2] * v[0] - u[0] * v[2];
    w[2] = u[0] * v[1] - u[1] * v[0];
}

static double dot3(const double *u, const double *v) { return u[0] * v[0] + u[1] * v[1] + u[2] * v[2]; }

/* Element stiffness K_ab = V grad(lambda_a) . grad(lambda_b) of the linear tetrahedron p0..p3.
   With d_k = p_k - p0 and det = d1 . (d2 x d3) = 6 V, the barycentric gradients are
   grad lambda_1 = (d2 x d3)/det, grad lambda_2 = (d3 x d1)/det, grad lambda_3 = (d1 x d2)/det,
   grad lambda_0 = -(sum of the others); hence K_ab = (c_a . c_b) / (6 det). Returns det. */
static double elem_stiffness(const double *p0, const double *p1, const double *p2, const double *p3,
                             double K[16]) {
    double d1[3], d2[3], d3[3], c[4][3];
    for (int k = 0; k < 3; ++k) { d1[k] = p1[k] - p0[k]; d2[k] = p2[k] - p0[k]; d3[k] = p3[k] - p0[k]; }
    cross3(d2, d3, c[1]);
    cross3(d3, d1, c[2]);
    cross3(d1, d2, c[3]);
    double det = dot3(d1, c[1]);
    for (int k = 0; k < 3; ++k) c[0][k] = -((c[1][k] + c[2][k]) + c[3][k]);
    double s = 6.0 * det;
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) K[a * 4 + b] = dot3(c[a], c[b]) / s;
    return det;
}

static double elem_det(const double *p0, const double *p1, const double *p2, const double *p3) {
    double d1[3], d2[3], d3[3], c1[3];
    for (int k = 0; k < 3; ++k) { d1[k] = p1[k] - p0[k]; d2[k] = p2[k] - p0[k]; d3[k] = p3[k] - p0[k]; }
    cross3(d2, d3, c1);
    return dot3(d1, c1);
}

/* ------------------------------------------------------------------------------------------ */
/* smoothed aggregation (section 5.1 and section 6)                                           */

typedef struct {
    csr A;        /* level operator */
    csr P, PT;    /* transfer to the next coarser level (absent on the coarsest) */
    int *agg;     /* aggregate of each node (absent on the coarsest) */
    int ncolours;
    int *colour;  /* SOR colour of each node (smallest-last greedy) */
    int *cptr;    /* ncolours + 1 offsets into crow */
    int *crow;    /* rows grouped by colour, ascending within a colour */
    double *x, *b, *r; /* work vectors */
    double *B;    /* near-nullspace rows (n x nsd, row-major) of a chain with nsd > 1, else NULL */
    int *blk;     /* node block of each unknown (the aggregate it came from), NULL on level 0 */
    int nblk;     /* number of node blocks */
} level;

typedef struct {
    int nlev;
    level lv[MAX_LEVELS_CAP];
    int singular;      /* constants are the nullspace (Neumann surface chain) */
    int direct;        /* coarsest level solved by dense Cholesky */
    int nc;            /* coarsest size */
    double *Lc;        /* dense Cholesky factor, nc x nc row-major lower */
    double sigma;      /* rank-one regularisation added on singular chains */
    int natural;       /* use natural-order (sequential) Gauss-Seidel instead of multicolour */
    int nsd;           /* near-nullspace vectors: 1 (constants) or 3 ({1, x, y}) */
    double *nu;        /* nsd > 1: the coarsest level's nullspace vector (the coarse constant) */
} chain;

/* strength of connection: |A_ij| > theta sqrt(A_ii A_jj), i != j (section 6) */
static csr strength_graph(const csr *A, double theta) {
    int n = A->n;
    double *d = (double *)xcalloc((size_t)n, sizeof(double));
    for (int i = 0; i < n; ++i) {
        int q = csr_find(A, i, i);
        d[i] = q >= 0 ? A->v[q] : 0.0;
    }
    int *rp = (int *)xcalloc((size_t)n + 1, sizeof(int));
    for (int i = 0; i < n; ++i) {
        int c = 0;
        for (int k = A->rp[i]; k < A->rp[i + 1]; ++k) {
            int j = A->ci[k];
            if (j != i && fabs(A->v[k]) > theta * sqrt(d[i] * d[j])) c++;
        }
        rp[i + 1] = rp[i] + c;
    }
    csr S = csr_new(n, n, rp[n]);
    memcpy(S.rp, rp, sizeof(int) * ((size_t)n + 1));
    for (int i = 0; i < n; ++i) {
        int c = S.rp[i];
        for (int k = A->rp[i]; k < A->rp[i + 1]; ++k) {
            int j = A->ci[k];
            if (j != i && fabs(A->v[k]) > theta * sqrt(d[i] * d[j])) { S.ci[c] = j; S.v[c] = fabs(A->v[k]); c++; }
        }
    }
    free(rp); free(d);
    return S;
}

/* One round of root selection: node i is a root if it is a candidate and its key is the
   largest among the candidates within strong-graph distance 2 (paths restricted to
   'through' nodes). Returns the number of roots; roots are flagged in isroot. */
static int mis2_round(const csr *S, const uint64_t *key, const char *cand, const char *through,
                      uint64_t *m1, char *isroot) {
    int n = S->n, nroots = 0;
    for (int j = 0; j < n; ++j) {
        uint64_t best = 0;
        if (through[j]) {
            if (cand[j]) best = key[j];
            for (int k = S->rp[j]; k < S->rp[j + 1]; ++k) {
                int q = S->ci[k];
                if (cand[q] && key[q] > best) best = key[q];
            }
        }
        m1[j] = best;
    }
    for (int i = 0; i < n; ++i) {
        isroot[i] = 0;
        if (!cand[i]) continue;
        uint64_t best = m1[i];
        for (int k = S->rp[i]; k < S->rp[i + 1]; ++k) {
            int q = S->ci[k];
            if (through[q] && m1[q] > best) best = m1[q];
        }
        if (best == key[i]) { isroot[i] = 1; nroots++; }
    }
    return nroots;
}

/* Vanek's three aggregation phases, made round-synchronous:
   1. roots whose whole strong neighbourhood is unaggregated, chosen as distance-2 maxima of
      the key (strong degree, hash); each root takes its strong neighbourhood;
   2. every remaining node with a strong neighbour in a phase-1 aggregate joins the aggregate
      of its strongest such neighbour (ties: lowest aggregate id);
   3. the rest are aggregated among themselves by the rule of phase 1 restricted to
      unaggregated nodes.
   Isolated nodes (no strong coupling) become singleton aggregates when keep_isolated is set
   (singular chains: every node must keep a coarse representative for P 1 = 1); otherwise they
   stay unaggregated (agg = -1), as in Vanek, Mandel and Brezina: their prolongator rows are
   zero and the smoother alone treats them.
   Returns the number of aggregates. */
int or_sa_aggregate(int n, const int *rp, const int *ci, const double *v, double theta, int keep_isolated,
                    int *agg) {
    csr A;
    A.n = n; A.m = n; A.rp = (int *)rp; A.ci = (int *)ci; A.v = (double *)v;
    csr S = strength_graph(&A, theta);
    uint64_t *key = (uint64_t *)xcalloc((size_t)n, sizeof(uint64_t));
    for (int i = 0; i < n; ++i) {
        uint64_t deg = (uint64_t)(S.rp[i + 1] - S.rp[i]);
        key[i] = ((deg + 1u) << 32) | (uint64_t)hash32((uint32_t)i);
    }
    uint64_t *m1 = (uint64_t *)xcalloc((size_t)n, sizeof(uint64_t));
    char *cand = (char *)xcalloc((size_t)n, 1), *thr = (char *)xcalloc((size_t)n, 1),
         *isroot = (char *)xcalloc((size_t)n, 1);
    for (int i = 0; i < n; ++i) agg[i] = -1;
    int nagg = 0;

    /* phase 1 */
    for (;;) {
        int any = 0;
        for (int i = 0; i < n; ++i) {
            int f = agg[i] < 0 && (keep_isolated || S.rp[i + 1] > S.rp[i]);
            for (int k = S.rp[i]; f && k < S.rp[i + 1]; ++k)
                if (agg[S.ci[k]] >= 0) f = 0;
            cand[i] = (char)f;
            thr[i] = 1;
            any |= f;
        }
        if (!any) break;
        mis2_round(&S, key, cand, thr, m1, isroot);
        for (int i = 0; i < n; ++i)
            if (isroot[i]) {
                agg[i] = nagg;
                for (int k = S.rp[i]; k < S.rp[i + 1]; ++k) agg[S.ci[k]] = nagg;
                nagg++;
            }
    }
    /* phase 2 (decisions taken on the phase-1 snapshot) */
    int *snap = (int *)xcalloc((size_t)n, sizeof(int));
    memcpy(snap, agg, sizeof(int) * (size_t)n);
    for (int i = 0; i < n; ++i) {
        if (snap[i] >= 0) continue;
        int best = -1;
        double bw = -1.0;
        for (int k = S.rp[i]; k < S.rp[i + 1]; ++k) {
            int j = S.ci[k];
            if (snap[j] < 0) continue;
            if (S.v[k] > bw || (S.v[k] == bw && snap[j] < best)) { bw = S.v[k]; best = snap[j]; }
        }
        agg[i] = best;
    }
    free(snap);
    /* phase 3 */
    for (;;) {
        int any = 0;
        for (int i = 0; i < n; ++i) {
            cand[i] = (char)(agg[i] < 0 && (keep_isolated || S.rp[i + 1] > S.rp[i]));
            thr[i] = cand[i];
            any |= cand[i];
        }
        if (!any) break;
        mis2_round(&S, key, cand, thr, m1, isroot);
        for (int i = 0; i < n; ++i)
            if (isroot[i]) {
                agg[i] = nagg;
                for (int k = S.rp[i]; k < S.rp[i + 1]; ++k)
                    if (cand[S.ci[k]]) agg[S.ci[k]] = nagg;
                nagg++;
            }
    }
    free(key); free(m1); free(cand); free(thr); free(isroot);
    csr_del(&S);
    return nagg;
}

/* Round-synchronous smallest-last ranks (a k-core peeling): round t first sets the threshold
   k_t = max(k_{t-1}, the smallest remaining degree), k_{-1} = 0, then removes every remaining
   node with at most k_t remaining neighbours and gives it the rank t. Every round removes at
   least one node. The nodes that qualify in the next round at the same threshold are
   neighbours of the removed ones, so a round costs the work of the nodes it removes; only
   a raise of the threshold scans all remaining nodes. */
void or_sl_ranks(int n, const int *rp, const int *ci, int *rank) {
    int *deg = (int *)xcalloc((size_t)n, sizeof(int));
    int *cur = (int *)xcalloc((size_t)n, sizeof(int));
    int *nxt = (int *)xcalloc((size_t)n, sizeof(int));
    char *queued = (char *)xcalloc((size_t)n, 1);
    for (int i = 0; i < n; ++i) {
        for (int k = rp[i]; k < rp[i + 1]; ++k) if (ci[k] != i) deg[i]++;
        rank[i] = -1;
    }
    int left = n, k = 0, ncur = 0;
    for (int round = 0; left > 0; ++round) {
        if (ncur == 0) {
            /* nothing at or below the threshold: raise it to the smallest remaining degree */
            int dmin = -1;
            for (int i = 0; i < n; ++i)
                if (rank[i] < 0 && (dmin < 0 || deg[i] < dmin)) dmin = deg[i];
            if (dmin > k) k = dmin;
            for (int i = 0; i < n; ++i)
                if (rank[i] < 0 && deg[i] <= k) { cur[ncur++] = i; queued[i] = 1; }
        }
        for (int t = 0; t < ncur; ++t) rank[cur[t]] = round;
        left -= ncur;
        int nn = 0;
        for (int t = 0; t < ncur; ++t) {
            int i = cur[t];
            for (int q = rp[i]; q < rp[i + 1]; ++q) {
                int j = ci[q];
                if (j == i || rank[j] >= 0) continue;
                deg[j]--;
                if (deg[j] <= k && !queued[j]) { queued[j] = 1; nxt[nn++] = j; }
            }
        }
        int *sw = cur; cur = nxt; nxt = sw;
        ncur = nn;
    }
    free(deg); free(cur); free(nxt); free(queued);
}

static const int *g_key_rank;   /* comparator context of the colouring order */
static int cmp_key_desc(const void *a, const void *b) {
    int i = *(const int *)a, j = *(const int *)b;
    uint64_t ki = ((uint64_t)(uint32_t)g_key_rank[i] << 32) | hash32((uint32_t)i);
    uint64_t kj = ((uint64_t)(uint32_t)g_key_rank[j] << 32) | hash32((uint32_t)j);
    return ki < kj ? 1 : (ki > kj ? -1 : 0);
}

/* Colouring of the matrix graph for the multicolour SOR sweeps: greedy first-fit in
   smallest-last order. Nodes are coloured by decreasing key (rank, hash32(i)) -- removed last,
   coloured first, ties in a round broken by the fixed hash -- each taking the smallest colour
   that no already coloured neighbour has. A node's already coloured neighbours were all still
   present when its round began, so it meets at most that round's threshold of them; the
   threshold never exceeds the graph's degeneracy (it only rises to a minimum degree of a
   subgraph), so the colours number at most the degeneracy + 1. Returns the number of colours. */
int or_colour(int n, const int *rp, const int *ci, int *colour) {
    int *rank = (int *)xcalloc((size_t)n, sizeof(int));
    int *order = (int *)xcalloc((size_t)n, sizeof(int));
    or_sl_ranks(n, rp, ci, rank);
    for (int i = 0; i < n; ++i) { order[i] = i; colour[i] = -1; }
    g_key_rank = rank;
    qsort(order, (size_t)n, sizeof(int), cmp_key_desc);
    int maxdeg = 0;
    for (int i = 0; i < n; ++i) if (rp[i + 1] - rp[i] > maxdeg) maxdeg = rp[i + 1] - rp[i];
    char *used = (char *)xcalloc((size_t)maxdeg + 2, 1);
    int ncol = 0;
    for (int t = 0; t < n; ++t) {
        int i = order[t];
        memset(used, 0, (size_t)maxdeg + 2);
        for (int k = rp[i]; k < rp[i + 1]; ++k) {
            int j = ci[k];
            if (j != i && colour[j] >= 0 && colour[j] <= maxdeg) used[colour[j]] = 1;
        }
        int c = 0;
        while (used[c]) c++;
        colour[i] = c;
        if (c + 1 > ncol) ncol = c + 1;
    }
    free(rank); free(order); free(used);
    return ncol;
}

/* smoothed prolongator P = (I - omega (D^F)^-1 A^F) P_tent (section 6: omega = 2/3), with the
   filtered matrix of Vanek, Mandel and Brezina (1996): weak off-diagonal entries are dropped and
   lumped into the diagonal, A^F_ii = A_ii + sum_{j weak} A_ij, so that A^F 1 = A 1. A row with no
   strong coupling (or a non-positive filtered diagonal) keeps its tentative row. Sums run over
   the row in ascending column order. */
static csr smoothed_prolongator(const csr *A, const int *agg, int nagg, double omega, double theta) {
    int n = A->n;
    double *d = (double *)xcalloc((size_t)n, sizeof(double));
    for (int i = 0; i < n; ++i) {
        int q = csr_find(A, i, i);
        d[i] = q >= 0 ? A->v[q] : 0.0;
    }
    int *mark = (int *)xcalloc((size_t)nagg, sizeof(int));
    for (int j = 0; j < nagg; ++j) mark[j] = -1;
    int *rp = (int *)xcalloc((size_t)n + 1, sizeof(int));
    for (int i = 0; i < n; ++i) {
        int c = 0;
        if (agg[i] < 0) { rp[i + 1] = rp[i]; continue; }   /* unaggregated: zero row */
        mark[agg[i]] = i; c++;
        for (int k = A->rp[i]; k < A->rp[i + 1]; ++k) {
            int j = A->ci[k];
            if (j == i || !(fabs(A->v[k]) > theta * sqrt(d[i] * d[j]))) continue;
            int J = agg[j];
            if (mark[J] != i) { mark[J] = i; c++; }
        }
        rp[i + 1] = rp[i] + c;
    }
    csr P = csr_new(n, nagg, rp[n]);
    memcpy(P.rp, rp, sizeof(int) * ((size_t)n + 1));
    free(rp);
    double *acc = (double *)xcalloc((size_t)nagg, sizeof(double));
    for (int j = 0; j < nagg; ++j) mark[j] = -1;
    for (int i = 0; i < n; ++i) {
        int base = P.rp[i], c = 0, nstrong = 0;
        if (agg[i] < 0) continue;
        /* filtered diagonal: the dropped (weak) couplings are lumped into it, so that the
           filtered row has the row sum of A's row and P keeps the constants A annihilates */
        double dF = d[i];
        for (int k = A->rp[i]; k < A->rp[i + 1]; ++k) {
            int j = A->ci[k];
            if (j == i) continue;
            if (fabs(A->v[k]) > theta * sqrt(d[i] * d[j])) nstrong++;
            else dF = dF + A->v[k];
        }
        mark[agg[i]] = i; acc[agg[i]] = 0.0; P.ci[base + c++] = agg[i];
        for (int k = A->rp[i]; k < A->rp[i + 1]; ++k) {
            int j = A->ci[k];
            double a;
            if (j == i) a = dF;
            else if (fabs(A->v[k]) > theta * sqrt(d[i] * d[j])) a = A->v[k];
            else continue;
            int J = agg[j];
            if (mark[J] != i) { mark[J] = i; acc[J] = 0.0; P.ci[base + c++] = J; }
            acc[J] = acc[J] + a;
        }
        qsort(P.ci + base, (size_t)c, sizeof(int), cmp_int);
        /* a row without strong couplings (or a non-positive filtered diagonal) keeps its
           tentative row: nothing to smooth against */
        double w = (nstrong > 0 && dF > 0.0) ? omega / dF : 0.0;
        for (int k = 0; k < c; ++k) {
            int J = P.ci[base + k];
            double t = w * acc[J];
            P.v[base + k] = (J == agg[i] ? 1.0 : 0.0) - t;
        }
    }
    free(acc); free(mark); free(d);
    return P;
}

/* exported for the closed-form tests of the prolongator weights: P of the given aggregates
   (agg[i] = -1: unaggregated) written to prp (n + 1), pci and pv (cap entries at most).
   Returns the number of entries, or -1 when cap is too small. */
int or_smoothed_prolongator(int n, const int *rp, const int *ci, const double *v, const int *agg, int nagg,
                            double omega, double theta, int *prp, int *pci, double *pv, int cap) {
    csr A;
    A.n = n; A.m = n; A.rp = (int *)rp; A.ci = (int *)ci; A.v = (double *)v;
    csr P = smoothed_prolongator(&A, agg, nagg, omega, theta);
    int nnz = csr_nnz(&P);
    if (nnz > cap) { csr_del(&P); return -1; }
    memcpy(prp, P.rp, sizeof(int) * ((size_t)n + 1));
    memcpy(pci, P.ci, sizeof(int) * (size_t)nnz);
    memcpy(pv, P.v, sizeof(double) * (size_t)nnz);
    csr_del(&P);
    return nnz;
}

/* ------------------------------------------------------------------------------------------ */
/* smoothed aggregation with the near-nullspace {1, x, y} (Vanek, Mandel and Brezina 1996, the    */
/* fourth-order recipe), for the surface operator E~^T A E~ of vertically unstructured meshes    */

/* Block strength matrix of a level whose unknowns come in node blocks (the coarse unknowns of
   one aggregate): entry (I, J) is the Frobenius norm of the block A_IJ, its squares summed over
   the rows of block I in ascending order and each row's entries in ascending column order. The
   rows of a block are consecutive. */
static csr block_norm_matrix(const csr *A, const int *blk, int nblk) {
    int n = A->n;
    int *bptr = (int *)xcalloc((size_t)nblk + 1, sizeof(int));
    for (int i = 0; i < n; ++i) bptr[blk[i] + 1]++;
    for (int I = 0; I < nblk; ++I) bptr[I + 1] += bptr[I];
    int *mark = (int *)xcalloc((size_t)nblk, sizeof(int));
    for (int J = 0; J < nblk; ++J) mark[J] = -1;
    int *rp = (int *)xcalloc((size_t)nblk + 1, sizeof(int));
    for (int I = 0; I < nblk; ++I) {
        int c = 0;
        for (int i = bptr[I]; i < bptr[I + 1]; ++i)
            for (int k = A->rp[i]; k < A->rp[i + 1]; ++k) {
                int J = blk[A->ci[k]];
                if (mark[J] != I) { mark[J] = I; c++; }
            }
        rp[I + 1] = rp[I] + c;
    }
    csr S = csr_new(nblk, nblk, rp[nblk]);
    memcpy(S.rp, rp, sizeof(int) * ((size_t)nblk + 1));
    double *acc = (double *)xcalloc((size_t)nblk, sizeof(double));
    for (int J = 0; J < nblk; ++J) mark[J] = -1;
    for (int I = 0; I < nblk; ++I) {
        int base = S.rp[I], c = 0;
        for (int i = bptr[I]; i < bptr[I + 1]; ++i)
            for (int k = A->rp[i]; k < A->rp[i + 1]; ++k) {
                int J = blk[A->ci[k]];
                if (mark[J] != I) { mark[J] = I; acc[J] = 0.0; S.ci[base + c++] = J; }
                acc[J] = acc[J] + A->v[k] * A->v[k];
            }
        qsort(S.ci + base, (size_t)c, sizeof(int), cmp_int);
        for (int q = 0; q < c; ++q) S.v[base + q] = sqrt(acc[S.ci[base + q]]);
    }
    free(acc); free(mark); free(rp); free(bptr);
    return S;
}

/* exported for tests: the block strength matrix (returns its entries, -1 if cap is too small) */
int or_block_norms(int n, const int *rp, const int *ci, const double *v, const int *blk, int nblk, int *srp,
                   int *sci, double *sv, int cap) {
    csr A;
    A.n = n; A.m = n; A.rp = (int *)rp; A.ci = (int *)ci; A.v = (double *)v;
    csr S = block_norm_matrix(&A, blk, nblk);
    int nnz = csr_nnz(&S);
    if (nnz <= cap) {
        memcpy(srp, S.rp, sizeof(int) * ((size_t)nblk + 1));
        memcpy(sci, S.ci, sizeof(int) * (size_t)nnz);
        memcpy(sv, S.v, sizeof(double) * (size_t)nnz);
    }
    csr_del(&S);
    return nnz <= cap ? nnz : -1;
}

#define QR_DROP 1e-10   /* a near-nullspace column whose part outside the kept ones is below this
                           fraction of its norm adds no coarse unknown (e.g. 1 or 2 nodes) */

/* Local QR of one aggregate's near-nullspace rows Bj (k x d, row-major) by modified Gram-Schmidt
   in column order, every sum in ascending row order: Q (k x d, row-major, kept columns first)
   with orthonormal columns spanning Bj's columns, and R = Q^T Bj (kept x d, row-major). A column
   whose residual after the kept ones has norm <= QR_DROP times its own norm is dropped. Returns
   the number of kept columns. */
int or_tentative_qr(int k, int d, const double *Bj, double *Q, double *R) {
    int kept = 0;
    double *v = (double *)xcalloc((size_t)k, sizeof(double));
    for (int c = 0; c < d; ++c) {
        double n0 = 0.0;
        for (int i = 0; i < k; ++i) { v[i] = Bj[i * d + c]; n0 = n0 + v[i] * v[i]; }
        n0 = sqrt(n0);
        for (int a = 0; a < kept; ++a) {
            double t = 0.0;
            for (int i = 0; i < k; ++i) t = t + Q[i * d + a] * v[i];
            for (int i = 0; i < k; ++i) v[i] = v[i] - t * Q[i * d + a];
        }
        double nr = 0.0;
        for (int i = 0; i < k; ++i) nr = nr + v[i] * v[i];
        nr = sqrt(nr);
        if (!(nr > QR_DROP * n0)) continue;
        for (int i = 0; i < k; ++i) Q[i * d + kept] = v[i] / nr;
        kept++;
    }
    for (int a = 0; a < kept; ++a)
        for (int c = 0; c < d; ++c) {
            double t = 0.0;
            for (int i = 0; i < k; ++i) t = t + Q[i * d + a] * Bj[i * d + c];
            R[a * d + c] = t;
        }
    free(v);
    return kept;
}

/* Tentative prolongator of aggregates agg (every unknown aggregated) with near-nullspace rows B
   (n x d): aggregate J's unknowns, ascending, get the rows of its local Q; its kept columns are
   the coarse unknowns of J, numbered aggregate by aggregate. The coarse near-nullspace rows are
   the local R's (nc x d), and the coarse unknowns' blocks their aggregates. */
static csr tentative_linear(int n, const int *agg, int nagg, const double *B, int d, double **Bc_out,
                            int **blk_out) {
    int *cnt = (int *)xcalloc((size_t)nagg + 1, sizeof(int));
    for (int i = 0; i < n; ++i) cnt[agg[i] + 1]++;
    for (int J = 0; J < nagg; ++J) cnt[J + 1] += cnt[J];
    int *mem = (int *)xcalloc((size_t)n, sizeof(int)), *cur = (int *)xcalloc((size_t)nagg, sizeof(int));
    memcpy(cur, cnt, sizeof(int) * (size_t)nagg);
    for (int i = 0; i < n; ++i) mem[cur[agg[i]]++] = i;   /* ascending within each aggregate */
    int kmax = 1;
    for (int J = 0; J < nagg; ++J) if (cnt[J + 1] - cnt[J] > kmax) kmax = cnt[J + 1] - cnt[J];
    double *Bj = (double *)xcalloc((size_t)kmax * d, sizeof(double)), *Q = (double *)xcalloc((size_t)kmax * d, sizeof(double));
    double *R = (double *)xcalloc((size_t)nagg * d * d, sizeof(double));
    int *kept = (int *)xcalloc((size_t)nagg, sizeof(int)), *col0 = (int *)xcalloc((size_t)nagg + 1, sizeof(int));
    double *qv = (double *)xcalloc((size_t)n * d, sizeof(double));
    for (int J = 0; J < nagg; ++J) {
        int k = cnt[J + 1] - cnt[J];
        for (int t = 0; t < k; ++t)
            for (int c = 0; c < d; ++c) Bj[t * d + c] = B[(size_t)mem[cnt[J] + t] * d + c];
        kept[J] = or_tentative_qr(k, d, Bj, Q, R + (size_t)J * d * d);
        col0[J + 1] = col0[J] + kept[J];
        for (int t = 0; t < k; ++t)
            for (int a = 0; a < kept[J]; ++a) qv[(size_t)mem[cnt[J] + t] * d + a] = Q[t * d + a];
    }
    int nc = col0[nagg];
    csr Pt = csr_new(n, nc, 0);
    free(Pt.ci); free(Pt.v);
    for (int i = 0; i < n; ++i) Pt.rp[i + 1] = Pt.rp[i] + kept[agg[i]];
    Pt.ci = (int *)xcalloc((size_t)Pt.rp[n], sizeof(int));
    Pt.v = (double *)xcalloc((size_t)Pt.rp[n], sizeof(double));
    for (int i = 0; i < n; ++i)
        for (int a = 0; a < kept[agg[i]]; ++a) {
            Pt.ci[Pt.rp[i] + a] = col0[agg[i]] + a;
            Pt.v[Pt.rp[i] + a] = qv[(size_t)i * d + a];
        }
    double *Bc = (double *)xcalloc((size_t)nc * d, sizeof(double));
    int *blk = (int *)xcalloc((size_t)nc, sizeof(int));
    for (int J = 0; J < nagg; ++J)
        for (int a = 0; a < kept[J]; ++a) {
            blk[col0[J] + a] = J;
            for (int c = 0; c < d; ++c) Bc[(size_t)(col0[J] + a) * d + c] = R[(size_t)J * d * d + a * d + c];
        }
    free(cnt); free(mem); free(cur); free(Bj); free(Q); free(R); free(kept); free(col0); free(qv);
    *Bc_out = Bc;
    *blk_out = blk;
    return Pt;
}

/* P = (I - omega D^-1 A) P_t with the unfiltered A and its diagonal D (section 6: omega = 2/3):
   A P_t by Gustavson's rule, then P_ij = (P_t)_ij - (omega / A_ii) (A P_t)_ij on the pattern of
   A P_t. (The filtered matrix of the constant chains keeps the constants only; with {1, x, y} the
   unfiltered matrix keeps the linear functions as well.) */
static csr smooth_unfiltered(const csr *A, const csr *Pt, double omega) {
    csr AP = csr_spgemm(A, Pt);
    for (int i = 0; i < A->n; ++i) {
        int q = csr_find(A, i, i);
        double d = q >= 0 ? A->v[q] : 0.0;
        double w = d > 0.0 ? omega / d : 0.0;
        for (int k = AP.rp[i]; k < AP.rp[i + 1]; ++k) {
            int p = csr_find(Pt, i, AP.ci[k]);
            double pt = p >= 0 ? Pt->v[p] : 0.0;
            double t = w * AP.v[k];
            AP.v[k] = pt - t;
        }
    }
    return AP;
}

/* exported for tests: the tentative and smoothed prolongators of the {1, x, y} chain for given
   aggregates (every unknown aggregated); Bc receives the coarse near-nullspace rows (nc x d) */
int or_linear_prolongator(int n, const int *rp, const int *ci, const double *v, const int *agg, int nagg,
                          const double *B, int d, double omega, int smoothed, int *prp, int *pci, double *pv,
                          double *Bc, int cap) {
    csr A;
    A.n = n; A.m = n; A.rp = (int *)rp; A.ci = (int *)ci; A.v = (double *)v;
    double *bc = NULL;
    int *blk = NULL;
    csr Pt = tentative_linear(n, agg, nagg, B, d, &bc, &blk);
    csr P = smoothed ? smooth_unfiltered(&A, &Pt, omega) : Pt;
    int nnz = csr_nnz(&P), nc = P.m;
    if (nnz <= cap) {
        memcpy(prp, P.rp, sizeof(int) * ((size_t)n + 1));
        memcpy(pci, P.ci, sizeof(int) * (size_t)nnz);
        memcpy(pv, P.v, sizeof(double) * (size_t)nnz);
        memcpy(Bc, bc, sizeof(double) * (size_t)nc * d);
    }
    if (smoothed) csr_del(&P);
    csr_del(&Pt);
    free(bc); free(blk);
    return nnz <= cap ? nc : -1;
}

static void level_colour(level *L) {
    int n = L->A.n;
    L->colour = (int *)xcalloc((size_t)n, sizeof(int));
    L->ncolours = or_colour(n, L->A.rp, L->A.ci, L->colour);
    L->cptr = (int *)xcalloc((size_t)L->ncolours + 1, sizeof(int));
    L->crow = (int *)xcalloc((size_t)n, sizeof(int));
    for (int i = 0; i < n; ++i) L->cptr[L->colour[i] + 1]++;
    for (int c = 0; c < L->ncolours; ++c) L->cptr[c + 1] += L->cptr[c];
    int *cur = (int *)xcalloc((size_t)L->ncolours + 1, sizeof(int));
    memcpy(cur, L->cptr, sizeof(int) * (size_t)L->ncolours);
    for (int i = 0; i < n; ++i) L->crow[cur[L->colour[i]]++] = i;
    free(cur);
    L->x = (double *)xcalloc((size_t)n, sizeof(double));
    L->b = (double *)xcalloc((size_t)n, sizeof(double));
    L->r = (double *)xcalloc((size_t)n, sizeof(double));
}

/* dense Cholesky of the coarsest operator (plus sigma 1 1^T on singular chains) */
static int chain_factor_coarsest(chain *C) {
    level *L = &C->lv[C->nlev - 1];
    int n = L->A.n;
    C->nc = n;
    double *a = (double *)xcalloc((size_t)n * n, sizeof(double));
    double tr = 0.0;
    for (int i = 0; i < n; ++i)
        for (int k = L->A.rp[i]; k < L->A.rp[i + 1]; ++k) {
            a[(size_t)i * n + L->A.ci[k]] = L->A.v[k];
            if (L->A.ci[k] == i) tr += L->A.v[k];
        }
    C->sigma = 0.0;
    if (C->singular && C->nu) {
        /* nullspace nu (the coarse constant of a {1, x, y} chain): A + sigma nu nu^T with
           sigma nu^T nu = tr(A) / n */
        double nn = 0.0;
        for (int i = 0; i < n; ++i) nn = nn + C->nu[i] * C->nu[i];
        C->sigma = tr / ((double)n * nn);
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) a[(size_t)i * n + j] += C->sigma * C->nu[i] * C->nu[j];
    } else if (C->singular) {
        C->sigma = tr / ((double)n * (double)n);
        for (size_t k = 0; k < (size_t)n * n; ++k) a[k] += C->sigma;
    }
    for (int j = 0; j < n; ++j) {
        double s = a[(size_t)j * n + j];
        for (int k = 0; k < j; ++k) s -= a[(size_t)j * n + k] * a[(size_t)j * n + k];
        if (!(s > 0.0)) { free(a); return OR_EBREAKDOWN; }
        double d = sqrt(s);
        a[(size_t)j * n + j] = d;
        for (int i = j + 1; i < n; ++i) {
            double t = a[(size_t)i * n + j];
            for (int k = 0; k < j; ++k) t -= a[(size_t)i * n + k] * a[(size_t)j * n + k];
            a[(size_t)i * n + j] = t / d;
        }
    }
    C->Lc = a;
    return OR_OK;
}

/* B0: near-nullspace rows of level 0 (n x nsd) for nsd > 1 (owned by the chain afterwards) */
static int chain_build(chain *C, csr A0, int singular, double theta, double omega_p, int coarse_max,
                       int max_levels, int natural, int nsd, double *B0) {
    memset(C, 0, sizeof(*C));
    C->singular = singular;
    C->natural = natural;
    C->nsd = nsd;
    if (max_levels > MAX_LEVELS_CAP) max_levels = MAX_LEVELS_CAP;
    if (max_levels < 1) max_levels = 1;
    C->lv[0].A = A0;
    C->lv[0].B = B0;
    C->lv[0].nblk = A0.n;
    C->nlev = 1;
    while (C->nlev < max_levels && C->lv[C->nlev - 1].A.n > coarse_max) {
        level *L = &C->lv[C->nlev - 1];
        int n = L->A.n;
        if (nsd > 1) {
            /* aggregates of node blocks, by the block strength (level 0: the unknowns themselves) */
            int nb = L->nblk;
            int *bagg = (int *)xcalloc((size_t)nb, sizeof(int));
            int nagg;
            if (L->blk) {
                csr S = block_norm_matrix(&L->A, L->blk, nb);
                nagg = or_sa_aggregate(nb, S.rp, S.ci, S.v, theta, singular, bagg);
                csr_del(&S);
            } else {
                nagg = or_sa_aggregate(n, L->A.rp, L->A.ci, L->A.v, theta, singular, bagg);
            }
            int *agg = (int *)xcalloc((size_t)n, sizeof(int));
            for (int i = 0; i < n; ++i) agg[i] = bagg[L->blk ? L->blk[i] : i];
            free(bagg);
            double *Bc = NULL;
            int *blk = NULL;
            csr Pt = tentative_linear(n, agg, nagg, L->B, nsd, &Bc, &blk);
            if (nagg == 0 || (long)Pt.m * 10 > (long)n * 9) { csr_del(&Pt); free(Bc); free(blk); free(agg); break; }
            L->agg = agg;
            L->P = smooth_unfiltered(&L->A, &Pt, omega_p);
            csr_del(&Pt);
            L->PT = csr_transpose(&L->P);
            level *Nx = &C->lv[C->nlev];
            Nx->A = galerkin(&L->A, &L->P, &L->PT);
            Nx->B = Bc;
            Nx->blk = blk;
            Nx->nblk = nagg;
            C->nlev++;
            continue;
        }
        int *agg = (int *)xcalloc((size_t)n, sizeof(int));
        int nagg = or_sa_aggregate(n, L->A.rp, L->A.ci, L->A.v, theta, singular, agg);
        if (nagg == 0 || (long)nagg * 10 > (long)n * 9) { free(agg); break; }
        L->agg = agg;
        L->P = smoothed_prolongator(&L->A, agg, nagg, omega_p, theta);
        L->PT = csr_transpose(&L->P);
        level *Nx = &C->lv[C->nlev];
        Nx->A = galerkin(&L->A, &L->P, &L->PT);
        C->nlev++;
    }
    if (nsd > 1 && singular) {
        /* the coarsest level's nullspace: the first near-nullspace column (the coarse constant) */
        level *Lc = &C->lv[C->nlev - 1];
        C->nu = (double *)xcalloc((size_t)Lc->A.n, sizeof(double));
        for (int i = 0; i < Lc->A.n; ++i) C->nu[i] = Lc->B[(size_t)i * nsd];
    }
    for (int l = 0; l < C->nlev; ++l) level_colour(&C->lv[l]);
    C->direct = C->lv[C->nlev - 1].A.n <= coarse_max;
    if (C->direct) return chain_factor_coarsest(C);
    return OR_OK;
}

static void chain_free(chain *C) {
    for (int l = 0; l < C->nlev; ++l) {
        level *L = &C->lv[l];
        csr_del(&L->A); csr_del(&L->P); csr_del(&L->PT);
        free(L->agg); free(L->colour); free(L->cptr); free(L->crow);
        free(L->x); free(L->b); free(L->r);
        free(L->B); free(L->blk);
    }
    free(C->Lc); free(C->nu);
    memset(C, 0, sizeof(*C));
}

/* one SOR (omega = 1) update of row i: x_i = (b_i - sum_{j != i} A_ij x_j) / A_ii */
static void sor_row(const csr *A, const double *b, double *x, int i) {
    double s = b[i], d = 0.0;
    for (int k = A->rp[i]; k < A->rp[i + 1]; ++k) {
        int j = A->ci[k];
        if (j == i) d = A->v[k]; else s -= A->v[k] * x[j];
    }
    x[i] = s / d;
}

static void sor_sweep(const chain *C, const level *L, const double *b, double *x, int forward) {
    if (C->natural) {
        if (forward) for (int i = 0; i < L->A.n; ++i) sor_row(&L->A, b, x, i);
        else for (int i = L->A.n - 1; i >= 0; --i) sor_row(&L->A, b, x, i);
        return;
    }
    for (int cc = 0; cc < L->ncolours; ++cc) {
        int c = forward ? cc : L->ncolours - 1 - cc;
        /* the rows of one colour are not coupled: any order gives the same values */
        OR_PARALLEL_FOR
        for (int k = L->cptr[c]; k < L->cptr[c + 1]; ++k) sor_row(&L->A, b, x, L->crow[k]);
    }
}

static void coarse_solve(const chain *C, const level *L, const double *b, double *x) {
    int n = L->A.n;
    if (!C->direct) {
        /* coarsening stalled above the direct-solve size: one symmetric SOR pass */
        memset(x, 0, sizeof(double) * (size_t)n);
        sor_sweep(C, L, b, x, 1);
        sor_sweep(C, L, b, x, 0);
        return;
    }
    const double *a = C->Lc;
    const double *nu = C->nu;
    double mu = 0.0, nn = 0.0;
    if (C->singular && nu) {
        /* project the right-hand side on the complement of the nullspace nu */
        double t = 0.0;
        for (int i = 0; i < n; ++i) { t = t + nu[i] * b[i]; nn = nn + nu[i] * nu[i]; }
        mu = t / nn;
    } else if (C->singular) {
        mu = vsum(n, b) / (double)n;
    }
    for (int i = 0; i < n; ++i) {
        double s = b[i] - (nu ? mu * nu[i] : mu);
        for (int k = 0; k < i; ++k) s -= a[(size_t)i * n + k] * x[k];
        x[i] = s / a[(size_t)i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = x[i];
        for (int k = i + 1; k < n; ++k) s -= a[(size_t)k * n + i] * x[k];
        x[i] = s / a[(size_t)i * n + i];
    }
    if (C->singular && nu) {
        double t = 0.0;
        for (int i = 0; i < n; ++i) t = t + nu[i] * x[i];
        double m2 = t / nn;
        for (int i = 0; i < n; ++i) x[i] -= m2 * nu[i];
    } else if (C->singular) {
        double m2 = vsum(n, x) / (double)n;
        for (int i = 0; i < n; ++i) x[i] -= m2;
    }
}

/* V-cycle with zero initial guess (section 5.1): forward SOR, restrict the residual,
   recurse, prolong and add, backward SOR. */
static void vcycle(const chain *C, int l, const double *b, double *x) {
    const level *L = &C->lv[l];
    int n = L->A.n;
    if (l == C->nlev - 1) { coarse_solve(C, L, b, x); return; }
    memset(x, 0, sizeof(double) * (size_t)n);
    sor_sweep(C, L, b, x, 1);
    csr_spmv(&L->A, x, L->r);
    OR_PARALLEL_FOR
    for (int i = 0; i < n; ++i) L->r[i] = b[i] - L->r[i];
    const level *Nx = &C->lv[l + 1];
    csr_spmv(&L->PT, L->r, Nx->b);
    vcycle(C, l + 1, Nx->b, Nx->x);
    OR_PARALLEL_FOR
    for (int i = 0; i < n; ++i) {
        double s = 0.0;
        for (int k = L->P.rp[i]; k < L->P.rp[i + 1]; ++k) s += L->P.v[k] * Nx->x[L->P.ci[k]];
        x[i] += s;
    }
    sor_sweep(C, L, b, x, 0);
}

/* ------------------------------------------------------------------------------------------ */
/* the problem: ordering, assembly, vertical extrapolation, Galerkin surface operator          */

typedef struct {
    int n, mtop, bc;
    int *new2old, *old2new;
    csr A;               /* internal (top-first) ordering; Neumann operator */
    int ntri;
    int *tri_of;         /* located top triangle of each internal node (-1 for top nodes) */
    double *bary;        /* 3 barycentric weights per internal node */
    csr E, ET;           /* vertical extrapolation E~ (n x mtop) and its transpose */
    csr Ac;              /* E~^T A E~ */
    chain surf;          /* SA chain on Ac (Neumann only) */
    chain bar;           /* SA chain on A_bar */
    int precond;         /* PC_ADDITIVE, PC_VL_SOR or PC_SA */
    chain one;           /* the single chain of PC_VL_SOR / PC_SA */
    /* copy of the mesh needed for the load vector */
    int ntet;
    int *tets;
    double *xyz;
    double *wr, *wz, *wq, *wp, *wx, *wb; /* solver work vectors */
} problem;

static int build_order(problem *h, const unsigned char *tags) {
    int n = h->n, t = 0;
    for (int i = 0; i < n; ++i) if (tags[i] & TAG_TOP) t++;
    h->mtop = t;
    h->new2old = (int *)xcalloc((size_t)n, sizeof(int));
    h->old2new = (int *)xcalloc((size_t)n, sizeof(int));
    int a = 0, b = t;
    for (int i = 0; i < n; ++i) {
        int r = (tags[i] & TAG_TOP) ? a++ : b++;
        h->new2old[r] = i;
        h->old2new[i] = r;
    }
    return OR_OK;
}

/* A in the internal ordering; entries summed over elements in ascending element index */
static int assemble(problem *h) {
    int n = h->n, ne = h->ntet;
    const int *T = h->tets;
    int *cnt = (int *)xcalloc((size_t)n + 1, sizeof(int));
    for (int e = 0; e < ne; ++e) for (int a = 0; a < 4; ++a) cnt[T[4 * e + a] + 1]++;
    for (int i = 0; i < n; ++i) cnt[i + 1] += cnt[i];
    int *inc = (int *)xcalloc((size_t)cnt[n], sizeof(int));
    int *cur = (int *)xcalloc((size_t)n, sizeof(int));
    memcpy(cur, cnt, sizeof(int) * (size_t)n);
    for (int e = 0; e < ne; ++e) for (int a = 0; a < 4; ++a) inc[cur[T[4 * e + a]]++] = e;
    free(cur);
    /* row patterns in the internal ordering */
    int *rp = (int *)xcalloc((size_t)n + 1, sizeof(int));
    int maxc = 0;
    for (int i = 0; i < n; ++i) if (cnt[i + 1] - cnt[i] > maxc) maxc = cnt[i + 1] - cnt[i];
    int *buf = (int *)xcalloc((size_t)maxc * 4 + 1, sizeof(int));
    for (int r = 0; r < n; ++r) {
        int i = h->new2old[r], m = 0;
        for (int k = cnt[i]; k < cnt[i + 1]; ++k)
            for (int a = 0; a < 4; ++a) buf[m++] = h->old2new[T[4 * inc[k] + a]];
        isort(buf, m);
        int u = 0;
        for (int k = 0; k < m; ++k) if (k == 0 || buf[k] != buf[k - 1]) u++;
        rp[r + 1] = rp[r] + u;
    }
    csr A = csr_new(n, n, rp[n]);
    memcpy(A.rp, rp, sizeof(int) * ((size_t)n + 1));
    free(rp);
    for (int r = 0; r < n; ++r) {
        int i = h->new2old[r], m = 0;
        for (int k = cnt[i]; k < cnt[i + 1]; ++k)
            for (int a = 0; a < 4; ++a) buf[m++] = h->old2new[T[4 * inc[k] + a]];
        isort(buf, m);
        int u = A.rp[r];
        for (int k = 0; k < m; ++k) if (k == 0 || buf[k] != buf[k - 1]) A.ci[u++] = buf[k];
    }
    free(buf); free(inc); free(cnt);
    for (int e = 0; e < ne; ++e) {
        double K[16];
        const int *v = T + 4 * e;
        double det = elem_stiffness(h->xyz + 3 * v[0], h->xyz + 3 * v[1], h->xyz + 3 * v[2],
                                    h->xyz + 3 * v[3], K);
        if (!(det > 0.0)) { csr_del(&A); return OR_EMESH; }
        for (int a = 0; a < 4; ++a) {
            int r = h->old2new[v[a]];
            for (int b = 0; b < 4; ++b) {
                int q = csr_find(&A, r, h->old2new[v[b]]);
                A.v[q] = A.v[q] + K[a * 4 + b];
            }
        }
    }
    h->A = A;
    return OR_OK;
}

static double orient2(double px, double py, double qx, double qy, double rx, double ry) {
    return (qx - px) * (ry - py) - (qy - py) * (rx - px);
}

/* Column location (section 5.4): for a point p, among the top triangles whose bounding box
   holds p, the one maximising the smallest barycentric coordinate (ties: lowest index).
   lambda_a = orient(p,b,c)/orient(a,b,c), lambda_b = orient(a,p,c)/orient(a,b,c),
   lambda_c = (1 - lambda_a) - lambda_b. Returns -1 if no bounding box holds p. */
typedef struct {
    int ntri, nb;
    const int *tri;        /* ntri x 3 node ids */
    const double *xyz;
    double x0, y0, sx, sy; /* bucket grid origin and extent */
    int *bptr, *bidx;
    double *bb;            /* ntri x 4: xmin xmax ymin ymax */
} locator;

static int bucket_of(double v, double v0, double s, int nb) {
    double f = floor((v - v0) / s * (double)nb);
    if (f < 0.0) return 0;
    if (f > (double)(nb - 1)) return nb - 1;
    return (int)f;
}

static void locator_build(locator *L, int ntri, const int *tri, const double *xyz) {
    L->ntri = ntri; L->tri = tri; L->xyz = xyz;
    L->bb = (double *)xcalloc((size_t)ntri * 4, sizeof(double));
    double xmin = INFINITY, xmax = -INFINITY, ymin = INFINITY, ymax = -INFINITY;
    for (int t = 0; t < ntri; ++t) {
        double a = INFINITY, b = -INFINITY, c = INFINITY, d = -INFINITY;
        for (int k = 0; k < 3; ++k) {
            const double *p = xyz + 3 * tri[3 * t + k];
            if (p[0] < a) a = p[0];
            if (p[0] > b) b = p[0];
            if (p[1] < c) c = p[1];
            if (p[1] > d) d = p[1];
        }
        L->bb[4 * t] = a; L->bb[4 * t + 1] = b; L->bb[4 * t + 2] = c; L->bb[4 * t + 3] = d;
        if (a < xmin) xmin = a;
        if (b > xmax) xmax = b;
        if (c < ymin) ymin = c;
        if (d > ymax) ymax = d;
    }
    int nb = (int)sqrt((double)ntri);
    if (nb < 1) nb = 1;
    L->nb = nb;
    L->x0 = xmin; L->y0 = ymin;
    L->sx = xmax > xmin ? xmax - xmin : 1.0;
    L->sy = ymax > ymin ? ymax - ymin : 1.0;
    L->bptr = (int *)xcalloc((size_t)nb * nb + 1, sizeof(int));
    for (int pass = 0; pass < 2; ++pass) {
        int *cur = NULL;
        if (pass == 1) {
            for (int k = 0; k < nb * nb; ++k) L->bptr[k + 1] += L->bptr[k];
            L->bidx = (int *)xcalloc((size_t)L->bptr[nb * nb], sizeof(int));
            cur = (int *)xcalloc((size_t)nb * nb, sizeof(int));
            memcpy(cur, L->bptr, sizeof(int) * (size_t)nb * nb);
        }
        for (int t = 0; t < ntri; ++t) {
            int i0 = bucket_of(L->bb[4 * t], L->x0, L->sx, nb), i1 = bucket_of(L->bb[4 * t + 1], L->x0, L->sx, nb);
            int j0 = bucket_of(L->bb[4 * t + 2], L->y0, L->sy, nb), j1 = bucket_of(L->bb[4 * t + 3], L->y0, L->sy, nb);
            for (int j = j0; j <= j1; ++j)
                for (int i = i0; i <= i1; ++i) {
                    if (pass == 0) L->bptr[j * nb + i + 1]++;
                    else L->bidx[cur[j * nb + i]++] = t;
                }
        }
        free(cur);
    }
}

static void locator_free(locator *L) { free(L->bb); free(L->bptr); free(L->bidx); }

static void tri_bary(const locator *L, int t, double px, double py, double w[3]) {
    const double *a = L->xyz + 3 * L->tri[3 * t], *b = L->xyz + 3 * L->tri[3 * t + 1],
                 *c = L->xyz + 3 * L->tri[3 * t + 2];
    double area = orient2(a[0], a[1], b[0], b[1], c[0], c[1]);
    w[0] = orient2(px, py, b[0], b[1], c[0], c[1]) / area;
    w[1] = orient2(a[0], a[1], px, py, c[0], c[1]) / area;
    w[2] = (1.0 - w[0]) - w[1];
}

static int locate(const locator *L, double px, double py, double w[3]) {
    int bi = bucket_of(px, L->x0, L->sx, L->nb), bj = bucket_of(py, L->y0, L->sy, L->nb);
    int k0 = L->bptr[bj * L->nb + bi], k1 = L->bptr[bj * L->nb + bi + 1];
    int best = -1;
    double bm = 0.0;
    for (int k = k0; k < k1; ++k) {
        int t = L->bidx[k];
        const double *bb = L->bb + 4 * t;
        if (px < bb[0] || px > bb[1] || py < bb[2] || py > bb[3]) continue;
        double l[3];
        tri_bary(L, t, px, py, l);
        double m = l[0] < l[1] ? l[0] : l[1];
        if (l[2] < m) m = l[2];
        if (best < 0 || m > bm || (m == bm && t < best)) { best = t; bm = m; }
    }
    if (best >= 0) tri_bary(L, best, px, py, w);
    return best;
}

/* standalone location of arbitrary points (for brute-force comparisons in tests) */
int or_locate_points(int ntri, const int *tri, const double *xyz, int npts, const double *pts_xy,
                     int *tri_out, double *w_out) {
    locator L;
    locator_build(&L, ntri, tri, xyz);
    for (int p = 0; p < npts; ++p) tri_out[p] = locate(&L, pts_xy[2 * p], pts_xy[2 * p + 1], w_out + 3 * p);
    locator_free(&L);
    return OR_OK;
}

/* E~ = [I; F]: identity rows for top nodes, barycentric rows elsewhere (exact zeros dropped) */
static int build_extrapolation(problem *h, int ntri, const int *tris, const unsigned char *tags) {
    int n = h->n, mt = h->mtop;
    for (int t = 0; t < 3 * ntri; ++t) {
        if (tris[t] < 0 || tris[t] >= n || !(tags[tris[t]] & TAG_TOP)) return OR_EMESH;
    }
    h->ntri = ntri;
    h->tri_of = (int *)xcalloc((size_t)n, sizeof(int));
    h->bary = (double *)xcalloc((size_t)n * 3, sizeof(double));
    locator L;
    locator_build(&L, ntri, tris, h->xyz);
    int rc = OR_OK;
    for (int r = 0; r < n; ++r) {
        if (r < mt) { h->tri_of[r] = -1; h->bary[3 * r] = 1.0; continue; }
        const double *p = h->xyz + 3 * h->new2old[r];
        int t = locate(&L, p[0], p[1], h->bary + 3 * r);
        h->tri_of[r] = t;
        if (t < 0) rc = OR_EMESH;
    }
    locator_free(&L);
    if (rc) return rc;
    int *rp = (int *)xcalloc((size_t)n + 1, sizeof(int));
    for (int r = 0; r < n; ++r) {
        int c = 0;
        if (r < mt) c = 1;
        else for (int k = 0; k < 3; ++k) if (h->bary[3 * r + k] != 0.0) c++;
        rp[r + 1] = rp[r] + c;
    }
    csr E = csr_new(n, mt, rp[n]);
    memcpy(E.rp, rp, sizeof(int) * ((size_t)n + 1));
    free(rp);
    for (int r = 0; r < n; ++r) {
        int base = E.rp[r];
        if (r < mt) { E.ci[base] = r; E.v[base] = 1.0; continue; }
        int c = 0, cols[3];
        double ws[3];
        for (int k = 0; k < 3; ++k)
            if (h->bary[3 * r + k] != 0.0) {
                cols[c] = h->old2new[tris[3 * h->tri_of[r] + k]];
                ws[c] = h->bary[3 * r + k];
                c++;
            }
        /* sort by column */
        for (int a = 1; a < c; ++a) {
            int cc = cols[a]; double ww = ws[a]; int b = a - 1;
            while (b >= 0 && cols[b] > cc) { cols[b + 1] = cols[b]; ws[b + 1] = ws[b]; --b; }
            cols[b + 1] = cc; ws[b + 1] = ww;
        }
        for (int k = 0; k < c; ++k) { E.ci[base + k] = cols[k]; E.v[base + k] = ws[k]; }
    }
    h->E = E;
    h->ET = csr_transpose(&E);
    return OR_OK;
}

/* A_bar: the trailing block of A on non-top rows and columns (section 3) */
static csr extract_bar(const csr *A, int mt) {
    int n = A->n, nb = n - mt;
    int *rp = (int *)xcalloc((size_t)nb + 1, sizeof(int));
    for (int i = 0; i < nb; ++i) {
        int c = 0;
        for (int k = A->rp[mt + i]; k < A->rp[mt + i + 1]; ++k) if (A->ci[k] >= mt) c++;
        rp[i + 1] = rp[i] + c;
    }
    csr B = csr_new(nb, nb, rp[nb]);
    memcpy(B.rp, rp, sizeof(int) * ((size_t)nb + 1));
    free(rp);
    for (int i = 0; i < nb; ++i) {
        int c = B.rp[i];
        for (int k = A->rp[mt + i]; k < A->rp[mt + i + 1]; ++k)
            if (A->ci[k] >= mt) { B.ci[c] = A->ci[k] - mt; B.v[c] = A->v[k]; c++; }
    }
    return B;
}

static csr csr_copy(const csr *a) {
    csr c = csr_new(a->n, a->m, csr_nnz(a));
    memcpy(c.rp, a->rp, sizeof(int) * ((size_t)a->n + 1));
    memcpy(c.ci, a->ci, sizeof(int) * (size_t)csr_nnz(a));
    memcpy(c.v, a->v, sizeof(double) * (size_t)csr_nnz(a));
    return c;
}

void or_free(void *hp);

/* surf_ns: near-nullspace of the surface chain's smoothed aggregation, 1 (constants) or 3
   ({1, x, y} with the top nodes' horizontal coordinates) */
void *or_setup(int n, const double *xyz, int ntet, const int *tets, const unsigned char *tags, int ntri,
               const int *tris, int bc, double theta, double omega_p, int coarse_max, int max_levels,
               int natural_order, int precond, int surf_ns, int *status) {
    *status = OR_OK;
    if (n <= 0 || ntet <= 0 || (bc != BC_NEUMANN && bc != BC_DIRICHLET_TOP) || precond < PC_ADDITIVE ||
        precond > PC_NONE || (precond == PC_VL_SOR && bc != BC_NEUMANN) || (surf_ns != 1 && surf_ns != 3)) {
        *status = OR_EINVAL;
        return NULL;
    }
    for (int e = 0; e < 4 * ntet; ++e) if (tets[e] < 0 || tets[e] >= n) { *status = OR_EMESH; return NULL; }
    problem *h = (problem *)xcalloc(1, sizeof(problem));
    h->n = n; h->bc = bc; h->ntet = ntet;
    /* with Dirichlet on top, smoothed aggregation on A_bar is the additive preconditioner itself */
    h->precond = (bc == BC_DIRICHLET_TOP && precond != PC_NONE) ? PC_ADDITIVE : precond;
    h->tets = (int *)xcalloc((size_t)ntet * 4, sizeof(int));
    memcpy(h->tets, tets, sizeof(int) * (size_t)ntet * 4);
    h->xyz = (double *)xcalloc((size_t)n * 3, sizeof(double));
    memcpy(h->xyz, xyz, sizeof(double) * (size_t)n * 3);
    build_order(h, tags);
    if (h->mtop == 0 || h->mtop == n) { or_free(h); *status = OR_EMESH; return NULL; }
    int rc = assemble(h);
    if (rc) { or_free(h); *status = rc; return NULL; }
    csr Abar = extract_bar(&h->A, h->mtop);
    if (bc == BC_NEUMANN) {
        rc = build_extrapolation(h, ntri, tris, tags);
        if (rc) { csr_del(&Abar); or_free(h); *status = rc; return NULL; }
        h->Ac = galerkin(&h->A, &h->E, &h->ET);
        double *B0 = NULL;
        if (surf_ns == 3) {
            /* {1, x, y} at the top nodes (internal rows 0 .. mtop-1) */
            B0 = (double *)xcalloc((size_t)h->mtop * 3, sizeof(double));
            for (int r = 0; r < h->mtop; ++r) {
                const double *p = h->xyz + 3 * h->new2old[r];
                B0[3 * r] = 1.0;
                B0[3 * r + 1] = p[0];
                B0[3 * r + 2] = p[1];
            }
        }
        rc = chain_build(&h->surf, csr_copy(&h->Ac), 1, theta, omega_p, coarse_max, max_levels, natural_order,
                         surf_ns, B0);
        if (rc) { csr_del(&Abar); or_free(h); *status = rc; return NULL; }
    }
    rc = chain_build(&h->bar, Abar, 0, theta, omega_p, coarse_max, max_levels, natural_order, 1, NULL);
    if (rc) { or_free(h); *status = rc; return NULL; }
    if (h->precond == PC_SA) {
        rc = chain_build(&h->one, csr_copy(&h->A), 1, theta, omega_p, coarse_max, max_levels, natural_order, 1, NULL);
        if (rc) { or_free(h); *status = rc; return NULL; }
    } else if (h->precond == PC_VL_SOR) {
        /* level 0: A with the vertical extrapolation E~ as its prolongator; below it, the SA chain
           of E~^T A E~ (section 6 treats the vertical lumping as the top coarsening step of one
           multigrid cycle) */
        chain *V = &h->one, *S = &h->surf;
        memset(V, 0, sizeof(*V));
        if (S->nlev + 1 > MAX_LEVELS_CAP) { or_free(h); *status = OR_EINVAL; return NULL; }
        V->singular = 1;
        V->natural = natural_order;
        V->nlev = S->nlev + 1;
        V->lv[0].A = csr_copy(&h->A);
        V->lv[0].P = csr_copy(&h->E);
        V->lv[0].PT = csr_copy(&h->ET);
        for (int l = 0; l < S->nlev; ++l) V->lv[l + 1] = S->lv[l];
        V->direct = S->direct; V->nc = S->nc; V->Lc = S->Lc; V->sigma = S->sigma;
        V->nsd = S->nsd; V->nu = S->nu;
        memset(S, 0, sizeof(*S));
        level_colour(&V->lv[0]);
    }
    h->wr = (double *)xcalloc((size_t)n, sizeof(double));
    h->wz = (double *)xcalloc((size_t)n, sizeof(double));
    h->wq = (double *)xcalloc((size_t)n, sizeof(double));
    h->wp = (double *)xcalloc((size_t)n, sizeof(double));
    h->wx = (double *)xcalloc((size_t)n, sizeof(double));
    h->wb = (double *)xcalloc((size_t)n, sizeof(double));
    return h;
}

void or_free(void *hp) {
    problem *h = (problem *)hp;
    if (!h) return;
    free(h->new2old); free(h->old2new);
    csr_del(&h->A); csr_del(&h->E); csr_del(&h->ET); csr_del(&h->Ac);
    free(h->tri_of); free(h->bary);
    chain_free(&h->surf); chain_free(&h->bar); chain_free(&h->one);
    free(h->tets); free(h->xyz);
    free(h->wr); free(h->wz); free(h->wq); free(h->wp); free(h->wx); free(h->wb);
    free(h);
}

/* ------------------------------------------------------------------------------------------ */
/* preconditioner and Krylov solver                                                            */

/* Eq. ourpreconditioner: z = E~ V(Ac)(E~^T r) + [0; I] V(A_bar)([0; I]^T r), each inverse
   replaced by one V-cycle; Dirichlet-top keeps only the second term. r and z are in the
   internal ordering over the unknowns of the chosen boundary condition. */
void or_precond(void *hp, const double *r, double *z) {
    problem *h = (problem *)hp;
    int mt = h->mtop, n = h->n;
    if (h->precond == PC_NONE) { memcpy(z, r, sizeof(double) * (size_t)(h->n - (h->bc == BC_NEUMANN ? 0 : mt))); return; }
    if (h->bc == BC_DIRICHLET_TOP) { vcycle(&h->bar, 0, r, z); return; }
    if (h->precond != PC_ADDITIVE) { vcycle(&h->one, 0, r, z); return; }
    level *s0 = &h->surf.lv[0];
    csr_spmv(&h->ET, r, s0->b);
    vcycle(&h->surf, 0, s0->b, s0->x);
    csr_spmv(&h->E, s0->x, z);
    level *b0 = &h->bar.lv[0];
    vcycle(&h->bar, 0, r + mt, b0->x);
    OR_PARALLEL_FOR
    for (int i = 0; i < n - mt; ++i) z[mt + i] += b0->x[i];
}

/* y = A x on the unknowns of the chosen boundary condition (internal ordering) */
void or_spmv(void *hp, const double *x, double *y) {
    problem *h = (problem *)hp;
    if (h->bc == BC_DIRICHLET_TOP) csr_spmv(&h->bar.lv[0].A, x, y);
    else csr_spmv(&h->A, x, y);
}

/* Preconditioned CG (flexible = 0) or flexible CG, Notay's FCG(1) (flexible = 1), x0 = 0.
   Neumann: b is projected to mean zero, each preconditioned residual z is projected to mean
   zero before use, and x is returned with zero mean. Stops when ||r_k||_2 <= tol ||b||_2 on the
   recursively updated residual. b and x are in the caller's node ordering. */
/* Preconditioned CG (section 6) on the unknowns of the boundary condition. coef (optional):
   coef[2k] = alpha_k, coef[2k + 1] = beta_{k+1}, the coefficients from which the Lanczos
   tridiagonal of the preconditioned operator follows (plain CG only, flexible = 0). */
int or_solve(void *hp, const double *b_orig, double *x_orig, double tol, int maxit, int flexible,
             int *iters, double *relres, double *true_relres, double *hist, int hist_len, double *coef,
             int coef_len) {
    problem *h = (problem *)hp;
    int neu = h->bc == BC_NEUMANN;
    int off = neu ? 0 : h->mtop;
    int m = h->n - off;
    double *r = h->wr, *z = h->wz, *q = h->wq, *p = h->wp, *x = h->wx, *b = h->wb;
    for (int i = 0; i < m; ++i) b[i] = b_orig[h->new2old[off + i]];
    if (neu) {
        double mu = vsum(m, b) / (double)m;
        for (int i = 0; i < m; ++i) b[i] -= mu;
    }
    double bn = sqrt(dot(m, b, b));
    memset(x, 0, sizeof(double) * (size_t)m);
    *iters = 0; *relres = 0.0; *true_relres = 0.0;
    int status = OR_OK;
    if (bn == 0.0) goto out;
    memcpy(r, b, sizeof(double) * (size_t)m);
    or_precond(h, r, z);
    if (neu) {
        double mu = vsum(m, z) / (double)m;
        OR_PARALLEL_FOR
        for (int i = 0; i < m; ++i) z[i] -= mu;
    }
    memcpy(p, z, sizeof(double) * (size_t)m);
    double rz = dot(m, r, z);
    status = OR_ENOTCONV;
    for (int k = 0; k < maxit; ++k) {
        or_spmv(h, p, q);
        double pq = dot(m, p, q);
        if (!(pq > 0.0)) { status = OR_EBREAKDOWN; break; }
        double alpha = rz / pq;
        if (coef && 2 * k < coef_len) coef[2 * k] = alpha;
        OR_PARALLEL_FOR
        for (int i = 0; i < m; ++i) { x[i] += alpha * p[i]; r[i] -= alpha * q[i]; }
        double rn = sqrt(dot(m, r, r));
        *iters = k + 1;
        *relres = rn / bn;
        if (hist && k < hist_len) hist[k] = *relres;
        if (!(rn == rn)) { status = OR_EBREAKDOWN; break; }
        if (rn <= tol * bn) { status = OR_OK; break; }
        or_precond(h, r, z);
        if (neu) {
            double mu = vsum(m, z) / (double)m;
            OR_PARALLEL_FOR
            for (int i = 0; i < m; ++i) z[i] -= mu;
        }
        double beta;
        if (flexible) {
            beta = -dot(m, z, q) / pq;
        } else {
            double rzn = dot(m, r, z);
            beta = rzn / rz;
            rz = rzn;
        }
        if (coef && 2 * k + 1 < coef_len) coef[2 * k + 1] = beta;
        OR_PARALLEL_FOR
        for (int i = 0; i < m; ++i) p[i] = z[i] + beta * p[i];
        if (flexible) rz = dot(m, r, z);
    }
    if (neu) { double mu = vsum(m, x) / (double)m; for (int i = 0; i < m; ++i) x[i] -= mu; }
    or_spmv(h, x, q);
    for (int i = 0; i < m; ++i) q[i] = b[i] - q[i];
    *true_relres = sqrt(dot(m, q, q)) / bn;
out:
    for (int i = 0; i < h->n; ++i) x_orig[i] = 0.0;
    for (int i = 0; i < m; ++i) x_orig[h->new2old[off + i]] = x[i];
    return status;
}

/* b = M f (section 3, Eq. Ax=b) in the caller's ordering: per element, M_e = V/20 (1 + delta_ab),
   so (M_e f)_a = V/20 (f_a + sum_b f_b); elements are added in ascending index. */
int or_load(void *hp, const double *f, double *b) {
    problem *h = (problem *)hp;
    for (int i = 0; i < h->n; ++i) b[i] = 0.0;
    for (int e = 0; e < h->ntet; ++e) {
        const int *v = h->tets + 4 * e;
        double det = elem_det(h->xyz + 3 * v[0], h->xyz + 3 * v[1], h->xyz + 3 * v[2], h->xyz + 3 * v[3]);
        double w = (det / 6.0) / 20.0;
        double s = ((f[v[0]] + f[v[1]]) + f[v[2]]) + f[v[3]];
        for (int a = 0; a < 4; ++a) b[v[a]] = b[v[a]] + w * (f[v[a]] + s);
    }
    return OR_OK;
}

/* ------------------------------------------------------------------------------------------ */
/* introspection for tests                                                                     */

static const chain *pick_chain(const problem *h, int which) {
    return which == 0 ? &h->surf : which == 2 ? &h->one : &h->bar;
}

/* sizes: key in {"n","mtop","nnzA","nnzE","nnzAc","nlev","lev.n","lev.nnz","lev.nnzP",
   "lev.ncolours","direct"} */
long or_size(void *hp, const char *key, int which, int l) {
    problem *h = (problem *)hp;
    const chain *C = pick_chain(h, which);
    if (!strcmp(key, "n")) return h->n;
    if (!strcmp(key, "mtop")) return h->mtop;
    if (!strcmp(key, "nnzA")) return csr_nnz(&h->A);
    if (!strcmp(key, "nnzE")) return h->E.rp ? csr_nnz(&h->E) : 0;
    if (!strcmp(key, "nnzAc")) return h->Ac.rp ? csr_nnz(&h->Ac) : 0;
    if (!strcmp(key, "nlev")) return C->nlev;
    if (!strcmp(key, "direct")) return C->direct;
    if (!strcmp(key, "nsd")) return C->nsd;
    if (l < 0 || l >= C->nlev) return -1;
    if (!strcmp(key, "lev.n")) return C->lv[l].A.n;
    if (!strcmp(key, "lev.nnz")) return csr_nnz(&C->lv[l].A);
    if (!strcmp(key, "lev.nnzP")) return C->lv[l].P.rp ? csr_nnz(&C->lv[l].P) : 0;
    if (!strcmp(key, "lev.ncolours")) return C->lv[l].ncolours;
    return -1;
}

static const csr *pick_csr(const problem *h, const char *name, int which, int l) {
    const chain *C = pick_chain(h, which);
    if (!strcmp(name, "A")) return &h->A;
    if (!strcmp(name, "E")) return &h->E;
    if (!strcmp(name, "ET")) return &h->ET;
    if (!strcmp(name, "Ac")) return &h->Ac;
    if (l < 0 || l >= C->nlev) return NULL;
    if (!strcmp(name, "lev.A")) return &C->lv[l].A;
    if (!strcmp(name, "lev.P")) return &C->lv[l].P;
    return NULL;
}

/* copy a CSR matrix out (rp: rows+1, ci/v: nnz) */
int or_get_csr(void *hp, const char *name, int which, int l, int *rp, int *ci, double *v) {
    problem *h = (problem *)hp;
    const csr *a = pick_csr(h, name, which, l);
    if (!a || !a->rp) return OR_EINVAL;
    memcpy(rp, a->rp, sizeof(int) * ((size_t)a->n + 1));
    memcpy(ci, a->ci, sizeof(int) * (size_t)csr_nnz(a));
    memcpy(v, a->v, sizeof(double) * (size_t)csr_nnz(a));
    return OR_OK;
}

/* integer arrays: "new2old" (n), "tri_of" (n), "lev.agg" (lev.n), "lev.colour" (lev.n) */
int or_get_int(void *hp, const char *name, int which, int l, int *out) {
    problem *h = (problem *)hp;
    const chain *C = pick_chain(h, which);
    if (!strcmp(name, "new2old")) { memcpy(out, h->new2old, sizeof(int) * (size_t)h->n); return OR_OK; }
    if (!strcmp(name, "tri_of")) {
        if (!h->tri_of) return OR_EINVAL;
        memcpy(out, h->tri_of, sizeof(int) * (size_t)h->n); return OR_OK;
    }
    if (l < 0 || l >= C->nlev) return OR_EINVAL;
    if (!strcmp(name, "lev.agg")) {
        if (!C->lv[l].agg) return OR_EINVAL;
        memcpy(out, C->lv[l].agg, sizeof(int) * (size_t)C->lv[l].A.n); return OR_OK;
    }
    if (!strcmp(name, "lev.colour")) { memcpy(out, C->lv[l].colour, sizeof(int) * (size_t)C->lv[l].A.n); return OR_OK; }
    return OR_EINVAL;
}

/* the near-nullspace rows of a level of a {1, x, y} chain (lev.n x nsd, row-major) */
int or_get_nullspace(void *hp, int which, int l, double *out) {
    problem *h = (problem *)hp;
    const chain *C = pick_chain(h, which);
    if (l < 0 || l >= C->nlev || !C->lv[l].B) return OR_EINVAL;
    memcpy(out, C->lv[l].B, sizeof(double) * (size_t)C->lv[l].A.n * C->nsd);
    return OR_OK;
}

/* one V-cycle of a chain on its finest level (for tests of the cycle alone) */
int or_vcycle(void *hp, int which, const double *b, double *x) {
    problem *h = (problem *)hp;
    const chain *C = pick_chain(h, which);
    if (C->nlev == 0) return OR_EINVAL;
    vcycle(C, 0, b, x);
    return OR_OK;
}

/* element stiffness of one tetrahedron (for the closed-form test); returns det = 6 V */
/* ------------------------------------------------------------------------------------------ */
/* BF16 operator values                                                                        */

/* a rounded to binary32 (the C conversion, nearest even), then to bfloat16, the format with
   binary32's sign and 8-bit exponent and 7 stored significand bits: keep the upper 16 bits of
   the binary32 pattern and round the dropped 16 bits to nearest, ties to the even result.
   Adding one unit of the kept part to the magnitude carries into the exponent where it must
   (up to infinity). Infinities and NaNs pass through. */
double or_round_bf16(double a) {
    float f = (float)a;
    uint32_t u;
    memcpy(&u, &f, sizeof u);
    if ((u & 0x7f800000u) == 0x7f800000u) return (double)f;
    uint32_t kept = u & 0xffff0000u, dropped = u & 0x0000ffffu;
    if (dropped > 0x8000u || (dropped == 0x8000u && (kept & 0x00010000u))) kept += 0x00010000u;
    memcpy(&f, &kept, sizeof f);
    return (double)f;
}

static void round_offdiag_bf16(csr *a, int keep_diagonal) {
    for (int i = 0; i < a->n; ++i)
        for (int k = a->rp[i]; k < a->rp[i + 1]; ++k)
            if (!(keep_diagonal && a->ci[k] == i)) a->v[k] = or_round_bf16(a->v[k]);
}

/* the operators of every level of every chain, as the BF16 variant of the cycle stores them:
   off-diagonal entries of each level matrix and every entry of P and P^T rounded to BF16; the
   diagonal and the dense coarsest factor keep their FP64 values (the setup is unchanged, only
   the stored operators of the cycle are rounded). A chain with the near-nullspace {1, x, y} keeps
   its values (the BF16 variant stores that chain in FP32: BF16 loses the fourth-order-like part
   of its coarse operators). */
void or_round_operators_bf16(void *hp) {
    problem *h = (problem *)hp;
    chain *cs[3] = {&h->surf, &h->bar, &h->one};
    for (int c = 0; c < 3; ++c)
        for (int l = 0; l < cs[c]->nlev && cs[c]->nsd <= 1; ++l) {
            level *L = &cs[c]->lv[l];
            round_offdiag_bf16(&L->A, 1);
            if (l + 1 < cs[c]->nlev) {
                round_offdiag_bf16(&L->P, 0);
                round_offdiag_bf16(&L->PT, 0);
            }
        }
}

double or_elem_stiffness(const double *p, double *K) {
    return elem_stiffness(p, p + 3, p + 6, p + 9, K);
}
