/*
 * ORACLE -- test infrastructure only.  A plain, slow, single-threaded FP64 CPU implementation
 * of the SpHcurlAMG method (Tuminaro & Glusa, "A structure preserving H-curl algebraic
 * multigrid method for the eddy current equations").  Only the tests, the package's smoke
 * check and the benchmark's CPU-baseline leg may load it.  It shares no code, header or table
 * with the GPU library.
 *
 * Every step follows the paper's definitions literally, with library-free sparse algebra:
 *   - sparse products use a dense accumulator (SPA) and keep every structurally reached entry;
 *     numerically zero entries are never dropped, so all patterns are structural;
 *   - nodal operator  A_n = D_h^T A_e D_h          (nodal problem, Sec. 2 eq. (5); Hiptmair Sec. 6.1)
 *   - smoothed-aggregation nodal prolongator, drop tolerance 0 (Sec. 4.1; Sec. 6.1)
 *       P_n = rowscale((I - w D^-1 A_n) Pbar),  w = 4 / (3 rho(D^-1 A_n))   (Sec. 3, eq. (9) text;
 *       rows scaled to sum one, Sec. 4.2)
 *   - coarse gradient from Z = Pbar^T D_h^T D_h Pbar, one coarse edge per strictly upper
 *     nonzero (Sec. 2 eq. (4), Sec. 4.1 eq. (11)), plus one single-node coarse edge per
 *     coarse node reached by the interior node of a single-node fine edge (Sec. 2);
 *   - Alg. 2 (Emin_Setup): T = |D_h||P_n|, W = Diag(3 - |D_H| 1), B = |T||D_H|^T W,
 *     N_ij = 1 iff B_ij = 2, irreducibility of each local graph (Sec. 4.2, Fig. 3),
 *     make_irreducible by the largest |(P_n^T D_h^T D_h P_n)_uv| candidate, QR of the local
 *     sub-matrix [D_H]_{I,J}, Reduce_Dimension when no Dirichlet coarse edge is present;
 *   - initial guess: ones on the pattern, then the least-norm local correction (Sec. 6.1);
 *   - projected Jacobi energy minimisation (Sec. 3 eq. (9)), D = diag(A_e), omega = 0.5;
 *   - Galerkin A_H = P_e^T A_e P_e (Sec. 2); nodal hierarchy A_n,H = P_n^T A_n P_n;
 *   - V-cycle with one pre and one post symmetric Hiptmair sweep, direct coarsest solve
 *     (Sec. 6.1), inside CG with x0 = 0 and ||r|| <= tol ||b|| (Sec. 6.1).
 *
 * Built plain (single-threaded) for the tests, or with -fopenmp as the timed CPU baseline: the
 * pragmas split only loops whose rows are independent (product rows, mat-vec rows, the rows of
 * one Gauss-Seidel colour, the per-row local solves), each row computed exactly as in the plain
 * build, so both builds give bit-identical results.
 *
 * Readings where the paper is open (stated once here, used throughout):
 *   - random priorities: splitmix64(seed, id); higher hash = higher priority, ties -> lower id;
 *   - Gauss-Seidel order: multicolour, colours from greedy colouring in priority order
 *     (identical to Jones-Plassmann); forward sweep colours 0..C-1, backward C-1..0;
 *   - aggregation: maximal distance-2 independent set chosen greedily in priority order,
 *     aggregate = root + its neighbours, each remaining node joins the aggregate it has the most
 *     edges to (ties -> lowest aggregate id) in synchronous rounds; aggregate ids follow root ids;
 *   - rho(D^-1 A_n): power iteration, 15 steps, start vector uniform(0,1) from splitmix64;
 *   - coarse edges: two-node edges in (tail, head) order with tail < head (tail -1, head +1),
 *     then single-node edges (+1) in node order;
 *   - Reduce_Dimension drops the column of the largest coarse node in J;
 *   - make_irreducible: per disconnected row, repeatedly join two components by the pair (u,v)
 *     with the largest |Z_uv| (values within a relative 1e-9 of the maximum tie; ties -> lowest
 *     (u,v)); all rows are checked against the same D_H, new edges are merged and N rebuilt.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#include <stdio.h>
#ifdef _OPENMP
#include <omp.h>
#define ORC_THREADS() omp_get_max_threads()
#define ORC_TID() omp_get_thread_num()
#else
#define ORC_THREADS() 1
#define ORC_TID() 0
#endif

/* a failure flag shared by the rows of a parallel loop (set once, read to skip the rest) */
#ifdef _OPENMP
#define ORC_FAIL(flag, code) do { _Pragma("omp atomic write") flag = (code); } while (0)
#define ORC_FAILED(flag) orc_read_flag(&(flag))
static int orc_read_flag(int *f) { int v; _Pragma("omp atomic read") v = *f; return v != 0; }
#else
#define ORC_FAIL(flag, code) do { flag = (code); } while (0)
#define ORC_FAILED(flag) ((flag) != 0)
#endif

#define ORC_MAXLEV 16
/* smallest row sum of the smoothed nodal prolongator that is rescaled to one */
#define SA_MIN_ROWSUM 0.125

/* ------------------------------------------------------------------ CSR basics */
typedef struct {
    int64_t nr, nc;
    int64_t *rp;
    int32_t *ci;
    double *v;
} ocsr;

static ocsr csr_alloc(int64_t nr, int64_t nc, int64_t nnz) {
    ocsr a;
    a.nr = nr; a.nc = nc;
    a.rp = (int64_t *)calloc((size_t)(nr + 1), sizeof(int64_t));
    a.ci = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
    a.v = (double *)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
    return a;
}
static void csr_free(ocsr *a) {
    free(a->rp); free(a->ci); free(a->v);
    a->rp = NULL; a->ci = NULL; a->v = NULL; a->nr = a->nc = 0;
}
static int64_t nnz_of(const ocsr *a) { return a->rp ? a->rp[a->nr] : 0; }

static ocsr csr_copy(const ocsr *a) {
    ocsr b = csr_alloc(a->nr, a->nc, nnz_of(a));
    memcpy(b.rp, a->rp, sizeof(int64_t) * (size_t)(a->nr + 1));
    memcpy(b.ci, a->ci, sizeof(int32_t) * (size_t)nnz_of(a));
    memcpy(b.v, a->v, sizeof(double) * (size_t)nnz_of(a));
    return b;
}

/* transpose; rows of the result list their columns in increasing order */
static ocsr csr_transpose(const ocsr *a) {
    int64_t nnz = nnz_of(a);
    ocsr t = csr_alloc(a->nc, a->nr, nnz);
    for (int64_t k = 0; k < nnz; ++k) t.rp[a->ci[k] + 1]++;
    for (int64_t i = 0; i < a->nc; ++i) t.rp[i + 1] += t.rp[i];
    int64_t *pos = (int64_t *)malloc(sizeof(int64_t) * (size_t)(a->nc + 1));
    memcpy(pos, t.rp, sizeof(int64_t) * (size_t)(a->nc + 1));
    for (int64_t i = 0; i < a->nr; ++i)
        for (int64_t k = a->rp[i]; k < a->rp[i + 1]; ++k) {
            int64_t q = pos[a->ci[k]]++;
            t.ci[q] = (int32_t)i;
            t.v[q] = a->v[k];
        }
    free(pos);
    return t;
}

static int cmp_i32(const void *x, const void *y) {
    int32_t a = *(const int32_t *)x, b = *(const int32_t *)y;
    return (a > b) - (a < b);
}

/* C = A * B keeping every structurally reached entry (dense accumulator per row) */
static ocsr csr_spgemm(const ocsr *A, const ocsr *B) {
    int64_t n = A->nr, m = B->nc;
    int nth = ORC_THREADS();
    size_t mm = (size_t)(m > 0 ? m : 1);
    /* one dense accumulator (SPA) per thread; rows are independent */
    int64_t *mark = (int64_t *)malloc(sizeof(int64_t) * mm * (size_t)nth);
    double *acc = (double *)calloc(mm * (size_t)nth, sizeof(double));
    int32_t *cols = (int32_t *)malloc(sizeof(int32_t) * mm * (size_t)nth);
    for (size_t j = 0; j < mm * (size_t)nth; ++j) mark[j] = -1;
    /* pass 1: row sizes */
    int64_t *rp = (int64_t *)calloc((size_t)(n + 1), sizeof(int64_t));
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < n; ++i) {
        int64_t *mk = mark + mm * (size_t)ORC_TID();
        int64_t cnt = 0;
        for (int64_t ka = A->rp[i]; ka < A->rp[i + 1]; ++ka) {
            int32_t k = A->ci[ka];
            for (int64_t kb = B->rp[k]; kb < B->rp[k + 1]; ++kb) {
                int32_t j = B->ci[kb];
                if (mk[j] != i) { mk[j] = i; ++cnt; }
            }
        }
        rp[i + 1] = cnt;
    }
    for (int64_t i = 0; i < n; ++i) rp[i + 1] += rp[i];
    ocsr C = csr_alloc(n, m, rp[n]);
    memcpy(C.rp, rp, sizeof(int64_t) * (size_t)(n + 1));
    free(rp);
    for (size_t j = 0; j < mm * (size_t)nth; ++j) mark[j] = -1;
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < n; ++i) {
        int64_t *mk = mark + mm * (size_t)ORC_TID();
        double *ac = acc + mm * (size_t)ORC_TID();
        int32_t *cl = cols + mm * (size_t)ORC_TID();
        int64_t cnt = 0;
        for (int64_t ka = A->rp[i]; ka < A->rp[i + 1]; ++ka) {
            int32_t k = A->ci[ka];
            double a = A->v[ka];
            for (int64_t kb = B->rp[k]; kb < B->rp[k + 1]; ++kb) {
                int32_t j = B->ci[kb];
                if (mk[j] != i) { mk[j] = i; ac[j] = 0.0; cl[cnt++] = j; }
                ac[j] += a * B->v[kb];
            }
        }
        qsort(cl, (size_t)cnt, sizeof(int32_t), cmp_i32);
        for (int64_t q = 0; q < cnt; ++q) {
            C.ci[C.rp[i] + q] = cl[q];
            C.v[C.rp[i] + q] = ac[cl[q]];
        }
    }
    free(mark); free(acc); free(cols);
    return C;
}

static ocsr csr_add(const ocsr *A, double alpha, const ocsr *B, double beta) {
    int64_t n = A->nr;
    int64_t *rp = (int64_t *)calloc((size_t)(n + 1), sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) {
        int64_t ka = A->rp[i], kb = B->rp[i], cnt = 0;
        while (ka < A->rp[i + 1] || kb < B->rp[i + 1]) {
            if (kb >= B->rp[i + 1] || (ka < A->rp[i + 1] && A->ci[ka] < B->ci[kb])) ++ka;
            else if (ka >= A->rp[i + 1] || B->ci[kb] < A->ci[ka]) ++kb;
            else { ++ka; ++kb; }
            ++cnt;
        }
        rp[i + 1] = rp[i] + cnt;
    }
    ocsr C = csr_alloc(n, A->nc, rp[n]);
    memcpy(C.rp, rp, sizeof(int64_t) * (size_t)(n + 1));
    free(rp);
    for (int64_t i = 0; i < n; ++i) {
        int64_t ka = A->rp[i], kb = B->rp[i], q = C.rp[i];
        while (ka < A->rp[i + 1] || kb < B->rp[i + 1]) {
            if (kb >= B->rp[i + 1] || (ka < A->rp[i + 1] && A->ci[ka] < B->ci[kb])) {
                C.ci[q] = A->ci[ka]; C.v[q] = alpha * A->v[ka]; ++ka;
            } else if (ka >= A->rp[i + 1] || B->ci[kb] < A->ci[ka]) {
                C.ci[q] = B->ci[kb]; C.v[q] = beta * B->v[kb]; ++kb;
            } else {
                C.ci[q] = A->ci[ka]; C.v[q] = alpha * A->v[ka] + beta * B->v[kb]; ++ka; ++kb;
            }
            ++q;
        }
    }
    return C;
}

static double csr_diag(const ocsr *A, int64_t i) {
    for (int64_t k = A->rp[i]; k < A->rp[i + 1]; ++k)
        if (A->ci[k] == i) return A->v[k];
    return 0.0;
}

static void csr_matvec(const ocsr *A, const double *x, double *y) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < A->nr; ++i) {
        double s = 0.0;
        for (int64_t k = A->rp[i]; k < A->rp[i + 1]; ++k) s += A->v[k] * x[A->ci[k]];
        y[i] = s;
    }
}

/* ------------------------------------------------------------------ random priorities */
static uint64_t splitmix64(uint64_t seed, uint64_t counter) {
    uint64_t z = seed + (counter + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
static double uniform01(uint64_t seed, uint64_t counter) {
    return (double)(splitmix64(seed, counter) >> 11) * (1.0 / 9007199254740992.0);
}

typedef struct { uint64_t h; int32_t id; } prio_t;
/* sort descending by priority: larger hash first, ties -> smaller id first */
static int cmp_prio(const void *x, const void *y) {
    const prio_t *a = (const prio_t *)x, *b = (const prio_t *)y;
    if (a->h != b->h) return a->h > b->h ? -1 : 1;
    return (a->id > b->id) - (a->id < b->id);
}
static prio_t *priority_order(int64_t n, uint64_t seed) {
    prio_t *p = (prio_t *)malloc(sizeof(prio_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) { p[i].h = splitmix64(seed, (uint64_t)i); p[i].id = (int32_t)i; }
    qsort(p, (size_t)n, sizeof(prio_t), cmp_prio);
    return p;
}

/* ------------------------------------------------------------------ colouring (greedy in priority order) */
static int32_t color_graph(const ocsr *G, uint64_t seed, int32_t *color) {
    int64_t n = G->nr;
    prio_t *ord = priority_order(n, seed);
    for (int64_t i = 0; i < n; ++i) color[i] = -1;
    int32_t ncol = 0;
    int32_t *used = (int32_t *)malloc(sizeof(int32_t) * 4096);
    for (int32_t c = 0; c < 4096; ++c) used[c] = -1;
    for (int64_t t = 0; t < n; ++t) {
        int32_t v = ord[t].id;
        for (int64_t k = G->rp[v]; k < G->rp[v + 1]; ++k) {
            int32_t w = G->ci[k];
            if (w != v && color[w] >= 0 && color[w] < 4096) used[color[w]] = v;
        }
        int32_t c = 0;
        while (c < 4096 && used[c] == v) ++c;
        color[v] = c;
        if (c + 1 > ncol) ncol = c + 1;
    }
    free(used); free(ord);
    return ncol;
}

/* ------------------------------------------------------------------ aggregation */
/* returns the number of aggregates, agg[n] filled; -1 on failure */
static int64_t aggregate_mis2(const ocsr *G, uint64_t seed, int32_t *agg) {
    int64_t n = G->nr;
    prio_t *ord = priority_order(n, seed);
    char *blocked = (char *)calloc((size_t)(n > 0 ? n : 1), 1);
    char *root = (char *)calloc((size_t)(n > 0 ? n : 1), 1);
    /* maximal distance-2 independent set, greedy in priority order */
    for (int64_t t = 0; t < n; ++t) {
        int32_t v = ord[t].id;
        if (blocked[v]) continue;
        root[v] = 1;
        blocked[v] = 1;
        for (int64_t k = G->rp[v]; k < G->rp[v + 1]; ++k) {
            int32_t w = G->ci[k];
            blocked[w] = 1;
            for (int64_t k2 = G->rp[w]; k2 < G->rp[w + 1]; ++k2) blocked[G->ci[k2]] = 1;
        }
    }
    free(ord); free(blocked);
    /* aggregate ids in root-id order */
    int64_t nagg = 0;
    for (int64_t i = 0; i < n; ++i) agg[i] = -1;
    for (int64_t i = 0; i < n; ++i) if (root[i]) agg[i] = (int32_t)(nagg++);
    /* root + its neighbours */
    for (int64_t i = 0; i < n; ++i) {
        if (!root[i]) continue;
        for (int64_t k = G->rp[i]; k < G->rp[i + 1]; ++k) {
            int32_t w = G->ci[k];
            if (w == i) continue;
            if (agg[w] >= 0 && agg[w] != agg[i]) { free(root); return -1; }  /* roots >= 3 apart */
            agg[w] = agg[i];
        }
    }
    free(root);
    /* remaining nodes: synchronous rounds, join the aggregate with the most edges */
    int32_t *next = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t *cnt_agg = (int32_t *)malloc(sizeof(int32_t) * 256);
    int32_t *cnt_val = (int32_t *)malloc(sizeof(int32_t) * 256);
    for (int round = 0; round < 64; ++round) {
        int64_t left = 0, changed = 0;
        for (int64_t i = 0; i < n; ++i) {
            next[i] = agg[i];
            if (agg[i] >= 0) continue;
            ++left;
            int nc = 0;
            for (int64_t k = G->rp[i]; k < G->rp[i + 1]; ++k) {
                int32_t w = G->ci[k];
                if (w == i || agg[w] < 0) continue;
                int q = 0;
                while (q < nc && cnt_agg[q] != agg[w]) ++q;
                if (q == nc) { if (nc == 256) continue; cnt_agg[nc] = agg[w]; cnt_val[nc] = 0; ++nc; }
                cnt_val[q]++;
            }
            int32_t best = -1, bestc = 0;
            for (int q = 0; q < nc; ++q)
                if (cnt_val[q] > bestc || (cnt_val[q] == bestc && cnt_agg[q] < best)) {
                    best = cnt_agg[q]; bestc = cnt_val[q];
                }
            if (best >= 0) { next[i] = best; ++changed; }
        }
        memcpy(agg, next, sizeof(int32_t) * (size_t)n);
        if (left == 0) break;
        if (changed == 0) { free(next); free(cnt_agg); free(cnt_val); return -1; }
    }
    free(next); free(cnt_agg); free(cnt_val);
    for (int64_t i = 0; i < n; ++i) if (agg[i] < 0) return -1;
    return nagg;
}

/* ------------------------------------------------------------------ nodal prolongator */
static double power_rho(const ocsr *A, uint64_t seed, int iters) {
    int64_t n = A->nr;
    if (n == 0) return 1.0;
    double *v = (double *)malloc(sizeof(double) * (size_t)n);
    double *w = (double *)malloc(sizeof(double) * (size_t)n);
    double *dinv = (double *)malloc(sizeof(double) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) { v[i] = uniform01(seed, (uint64_t)i); dinv[i] = 1.0 / csr_diag(A, i); }
    double rho = 1.0;
    for (int it = 0; it < iters; ++it) {
        csr_matvec(A, v, w);
        double nv = 0.0, nw = 0.0;
        for (int64_t i = 0; i < n; ++i) { w[i] *= dinv[i]; nw += w[i] * w[i]; nv += v[i] * v[i]; }
        nv = sqrt(nv); nw = sqrt(nw);
        rho = nw / nv;
        for (int64_t i = 0; i < n; ++i) v[i] = w[i] / nw;
    }
    free(v); free(w); free(dinv);
    return rho;
}

/* Drop tolerance theta > 0 (the symmetric smoothed-aggregation criterion the paper uses with
 * MueLu in Sec. 7): off-diagonal a_ij is strong when |a_ij| >= theta sqrt(a_ii a_jj).  The filtered
 * matrix keeps the diagonal and the strong entries; each dropped entry is added to the diagonal,
 * in column order, so that its row sums equal A's. */
static ocsr strength_filter(const ocsr *A, double theta) {
    int64_t n = A->nr;
    double *d = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) d[i] = csr_diag(A, i);
    int64_t nnz = 0;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t k = A->rp[i]; k < A->rp[i + 1]; ++k) {
            int32_t j = A->ci[k];
            if (j == i || fabs(A->v[k]) >= theta * sqrt(d[i] * d[j])) ++nnz;
        }
    ocsr F = csr_alloc(n, A->nc, nnz);
    int64_t q = 0;
    for (int64_t i = 0; i < n; ++i) {
        double diag = d[i];
        int64_t qd = -1;
        for (int64_t k = A->rp[i]; k < A->rp[i + 1]; ++k) {
            int32_t j = A->ci[k];
            if (j == i) { qd = q; F.ci[q] = j; F.v[q++] = 0.0; }
            else if (fabs(A->v[k]) >= theta * sqrt(d[i] * d[j])) { F.ci[q] = j; F.v[q++] = A->v[k]; }
            else diag += A->v[k];
        }
        if (qd >= 0) F.v[qd] = diag;
        F.rp[i + 1] = q;
    }
    free(d);
    return F;
}

/* Alg. 1 (Gen_Piecewise_Const, Sec. 4.1): assign every row of the smoothed P (m_h x m_H) to one
 * column, largest entries first, for the construction of D_H.  Readings (the paper leaves them
 * open or states a sequential sweep):
 *   - target_j = ceil(nnz(P_:j) m_h / nnz(P)) (proportional to the column's entries, summing to
 *     about m_h); a pass assigns up to ceil(target_j / nPasses) rows to column j;
 *   - within a pass the columns choose simultaneously: column j proposes its assignable rows
 *     (unassigned when the pass starts) of largest |P_rj| (ties: lower row), and a row proposed by
 *     several columns goes to the largest |P_rj| (ties: lower column);
 *   - Greedy_Assign: each row still unassigned goes to its column of largest |P_rj| (ties: lower
 *     column);
 *   - safeguard: in column order, a column without rows takes its row of largest |P_rj| if that
 *     row's column keeps another row.
 * Returns the number of columns (m_H). */
typedef struct { double a; int32_t r; } aent;
static int cmp_aent(const void *x, const void *y) {
    const aent *p = (const aent *)x, *q = (const aent *)y;
    if (p->a != q->a) return p->a > q->a ? -1 : 1;
    return p->r < q->r ? -1 : (p->r > q->r);
}
static int64_t gen_piecewise_const(const ocsr *P, int passes, int32_t *assign) {
    int64_t m = P->nr, nc = P->nc, nnz = nnz_of(P);
    ocsr Pt = csr_transpose(P);
    for (int64_t r = 0; r < m; ++r) assign[r] = -1;
    int64_t *nass = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nc > 0 ? nc : 1));
    for (int64_t j = 0; j < nc; ++j) {
        int64_t cnt = Pt.rp[j + 1] - Pt.rp[j];
        int64_t target = nnz > 0 ? (cnt * m + nnz - 1) / nnz : 0;
        nass[j] = (target + passes - 1) / passes;
    }
    double *best = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    int32_t *bcol = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
    char *prop = (char *)calloc((size_t)(nnz > 0 ? nnz : 1), 1);
    aent *buf = (aent *)malloc(sizeof(aent) * (size_t)(m > 0 ? m : 1));
    for (int pass = 0; pass < passes; ++pass) {
        memset(prop, 0, (size_t)(nnz > 0 ? nnz : 1));
        for (int64_t r = 0; r < m; ++r) { best[r] = -1.0; bcol[r] = -1; }
        for (int64_t j = 0; j < nc; ++j) {              /* proposals against the state at the pass start */
            int64_t nb = 0;
            for (int64_t k = Pt.rp[j]; k < Pt.rp[j + 1]; ++k)
                if (assign[Pt.ci[k]] < 0) { buf[nb].a = fabs(Pt.v[k]); buf[nb].r = Pt.ci[k]; ++nb; }
            qsort(buf, (size_t)nb, sizeof(aent), cmp_aent);
            for (int64_t t = 0; t < nb && t < nass[j]; ++t)
                for (int64_t k = Pt.rp[j]; k < Pt.rp[j + 1]; ++k)
                    if (Pt.ci[k] == buf[t].r) prop[k] = 1;
        }
        for (int64_t j = 0; j < nc; ++j)               /* a contested row: largest |P_rj|, then lower j */
            for (int64_t k = Pt.rp[j]; k < Pt.rp[j + 1]; ++k) {
                if (!prop[k]) continue;
                int32_t r = Pt.ci[k];
                double a = fabs(Pt.v[k]);
                if (a > best[r] || (a == best[r] && (bcol[r] < 0 || j < bcol[r]))) { best[r] = a; bcol[r] = (int32_t)j; }
            }
        for (int64_t r = 0; r < m; ++r) if (bcol[r] >= 0) assign[r] = bcol[r];
    }
    for (int64_t r = 0; r < m; ++r) {                   /* Greedy_Assign */
        if (assign[r] >= 0) continue;
        double ba = -1.0;
        int32_t bj = -1;
        for (int64_t k = P->rp[r]; k < P->rp[r + 1]; ++k) {
            double a = fabs(P->v[k]);
            if (a > ba || (a == ba && P->ci[k] < bj)) { ba = a; bj = P->ci[k]; }
        }
        assign[r] = bj;
    }
    int64_t *cnt = (int64_t *)calloc((size_t)(nc > 0 ? nc : 1), sizeof(int64_t));
    for (int64_t r = 0; r < m; ++r) if (assign[r] >= 0) cnt[assign[r]]++;
    for (int64_t j = 0; j < nc; ++j) {                  /* safeguard, in column order */
        if (cnt[j] > 0 || Pt.rp[j + 1] == Pt.rp[j]) continue;
        double ba = -1.0;
        int32_t br = -1;
        for (int64_t k = Pt.rp[j]; k < Pt.rp[j + 1]; ++k) {
            double a = fabs(Pt.v[k]);
            if (a > ba || (a == ba && Pt.ci[k] < br)) { ba = a; br = Pt.ci[k]; }
        }
        if (br >= 0 && assign[br] >= 0 && cnt[assign[br]] >= 2) { cnt[assign[br]]--; assign[br] = (int32_t)j; cnt[j]++; }
    }
    free(cnt); free(nass); free(best); free(bcol); free(prop); free(buf);
    csr_free(&Pt);
    return nc;
}

/* entry point of the tests */
int64_t orc_gen_piecewise_const(int64_t nr, int64_t nc, const int64_t *rp, const int32_t *ci, const double *v,
                                int passes, int32_t *assign) {
    ocsr P = csr_alloc(nr, nc, rp[nr]);
    memcpy(P.rp, rp, sizeof(int64_t) * (size_t)(nr + 1));
    memcpy(P.ci, ci, sizeof(int32_t) * (size_t)rp[nr]);
    memcpy(P.v, v, sizeof(double) * (size_t)rp[nr]);
    int64_t r = gen_piecewise_const(&P, passes, assign);
    csr_free(&P);
    return r;
}

/* Pbar: one 1 per row in column agg(i) */
static ocsr pbar_matrix(int64_t n, int64_t nagg, const int32_t *agg) {
    ocsr P = csr_alloc(n, nagg, n);
    for (int64_t i = 0; i < n; ++i) { P.rp[i + 1] = i + 1; P.ci[i] = agg[i]; P.v[i] = 1.0; }
    return P;
}

/* ------------------------------------------------------------------ small dense linear algebra */
/* Householder QR of G (np x k, column-major in a[np*k]); R stored in the upper triangle of a,
 * Householder vectors below it; tau[k].  Returns 0, or -1 if a diagonal of R vanishes. */
static int house_qr(int np, int k, double *a, double *tau) {
    for (int j = 0; j < k; ++j) {
        double *col = a + (size_t)j * np;
        double norm = 0.0;
        for (int i = j; i < np; ++i) norm += col[i] * col[i];
        norm = sqrt(norm);
        if (norm == 0.0) { tau[j] = 0.0; return -1; }
        double alpha = col[j] > 0 ? -norm : norm;
        double v0 = col[j] - alpha;
        /* v = (col[j]-alpha, col[j+1..]) normalised so v[0] = 1 */
        for (int i = j + 1; i < np; ++i) col[i] /= v0;
        double vnorm2 = 1.0;
        for (int i = j + 1; i < np; ++i) vnorm2 += col[i] * col[i];
        tau[j] = 2.0 / vnorm2;
        col[j] = alpha;
        for (int c = j + 1; c < k; ++c) {
            double *cc = a + (size_t)c * np;
            double s = cc[j];
            for (int i = j + 1; i < np; ++i) s += col[i] * cc[i];
            s *= tau[j];
            cc[j] -= s;
            for (int i = j + 1; i < np; ++i) cc[i] -= s * col[i];
        }
        if (fabs(alpha) < 1e-12) return -1;
    }
    return 0;
}
/* y := Q x  (Q = H_0 H_1 ... H_{k-1}); x has length np */
static void house_apply_q(int np, int k, const double *a, const double *tau, double *x) {
    for (int j = k - 1; j >= 0; --j) {
        const double *col = a + (size_t)j * np;
        double s = x[j];
        for (int i = j + 1; i < np; ++i) s += col[i] * x[i];
        s *= tau[j];
        x[j] -= s;
        for (int i = j + 1; i < np; ++i) x[i] -= s * col[i];
    }
}
/* y := Q^T x */
static void house_apply_qt(int np, int k, const double *a, const double *tau, double *x) {
    for (int j = 0; j < k; ++j) {
        const double *col = a + (size_t)j * np;
        double s = x[j];
        for (int i = j + 1; i < np; ++i) s += col[i] * x[i];
        s *= tau[j];
        x[j] -= s;
        for (int i = j + 1; i < np; ++i) x[i] -= s * col[i];
    }
}

/* Least-norm solution of Gt^T p = rt (Gt = QR, np x k): p = Q [R^-T rt; 0]. */
static void qr_minnorm(int np, int k, const double *a, const double *tau, const double *rt, double *p) {
    for (int i = 0; i < np; ++i) p[i] = 0.0;
    for (int i = 0; i < k; ++i) {        /* solve R^T y = rt (R upper => R^T lower) */
        double s = rt[i];
        for (int j = 0; j < i; ++j) s -= a[(size_t)i * np + j] * p[j];
        p[i] = s / a[(size_t)i * np + i];
    }
    house_apply_q(np, k, a, tau, p);
}
/* Remove from x its component in range(Gt): x -= Q_k Q_k^T x */
static void qr_project_null(int np, int k, const double *a, const double *tau, double *x, double *tmp) {
    memcpy(tmp, x, sizeof(double) * (size_t)np);
    house_apply_qt(np, k, a, tau, tmp);
    for (int i = k; i < np; ++i) tmp[i] = 0.0;
    house_apply_q(np, k, a, tau, tmp);
    for (int i = 0; i < np; ++i) x[i] -= tmp[i];
}

/* ------------------------------------------------------------------ hierarchy */
typedef struct {
    int32_t max_levels;
    int32_t emin_iters;
    int64_t max_coarse;
    double emin_omega;
    uint64_t seed;
    int32_t power_iters;
    int32_t unsmoothed_pn;      /* 1: P_n := Pbar (the Reitzinger-Schoeberl special case) */
    const int32_t *agg0;        /* injected level-0 aggregates (or NULL) */
    int64_t nagg0;
    double p0_value;            /* initial pattern value before the least-norm correction */
    int32_t emin_method;        /* 0: projected Jacobi, eq. (9); 1: projected CG on the KKT system, eq. (8) */
    double sa_theta;            /* SA drop tolerance (0: every structural entry strong, Sec. 6.1) */
    int32_t pn_alg1;            /* 1: D_H from Alg. 1 on the smoothed P_n (Sec. 4.1) */
    int32_t alg1_passes;        /* passes of Alg. 1 */
} orc_opts;

typedef struct {
    ocsr A, D, An;
    int32_t *col_e, *col_n;
    int32_t ncol_e, ncol_n;
    /* transfer data (absent on the coarsest level) */
    int32_t *agg; int64_t nagg;
    ocsr Pn, DH, T, Pe, P0, PeT;
    double rho, omega_sa;
    int64_t n_added;            /* coarse edges added by make_irreducible */
    int64_t n_infeasible0;      /* rows found reducible before the fix */
    int64_t n_rows_unsmoothed;  /* P_n rows whose smoothed sum fell below SA_MIN_ROWSUM */
    int64_t hist[33][33];       /* least-squares sub-problem sizes |I| x |J| (clipped at 32) */
    double energy0, energy1;    /* trace(P^T A P) of P0 and of the final P_e */
} olevel;

typedef struct {
    int nlev;
    olevel L[ORC_MAXLEV];
    double *chol; int64_t nc;   /* dense Cholesky factor of the coarsest operator (row-major lower) */
    int status;
    double setup_seconds;
} ohier;

static double energy_trace(const ocsr *A, const ocsr *P) {
    /* sum_j P_:j^T A P_:j = sum_ij P_ij (A P)_ij */
    ocsr AP = csr_spgemm(A, P);
    double e = 0.0;
    for (int64_t i = 0; i < P->nr; ++i) {
        int64_t ka = AP.rp[i];
        for (int64_t k = P->rp[i]; k < P->rp[i + 1]; ++k) {
            while (ka < AP.rp[i + 1] && AP.ci[ka] < P->ci[k]) ++ka;
            if (ka < AP.rp[i + 1] && AP.ci[ka] == P->ci[k]) e += P->v[k] * AP.v[ka];
        }
    }
    csr_free(&AP);
    return e;
}

/* coarse gradient from the piecewise-constant prolongator (eqs. (4), (11)) */
static ocsr coarse_gradient(const ocsr *D, const int32_t *agg, int64_t nagg) {
    ocsr Pb = pbar_matrix(D->nc, nagg, agg);
    ocsr DP = csr_spgemm(D, &Pb);
    ocsr DPt = csr_transpose(&DP);
    ocsr Z = csr_spgemm(&DPt, &DP);
    /* single-node coarse edges: coarse nodes of the interior node of single-node fine edges */
    char *single = (char *)calloc((size_t)(nagg > 0 ? nagg : 1), 1);
    for (int64_t e = 0; e < D->nr; ++e)
        if (D->rp[e + 1] - D->rp[e] == 1) single[agg[D->ci[D->rp[e]]]] = 1;
    int64_t n2 = 0, n1 = 0;
    for (int64_t u = 0; u < nagg; ++u) {
        for (int64_t k = Z.rp[u]; k < Z.rp[u + 1]; ++k) if (Z.ci[k] > u) ++n2;
        n1 += single[u];
    }
    ocsr H = csr_alloc(n2 + n1, nagg, 2 * n2 + n1);
    int64_t e = 0, q = 0;
    for (int64_t u = 0; u < nagg; ++u)
        for (int64_t k = Z.rp[u]; k < Z.rp[u + 1]; ++k)
            if (Z.ci[k] > u) {
                H.ci[q] = (int32_t)u; H.v[q] = -1.0; ++q;
                H.ci[q] = Z.ci[k]; H.v[q] = 1.0; ++q;
                H.rp[++e] = q;
            }
    for (int64_t u = 0; u < nagg; ++u)
        if (single[u]) { H.ci[q] = (int32_t)u; H.v[q] = 1.0; ++q; H.rp[++e] = q; }
    free(single);
    csr_free(&Pb); csr_free(&DP); csr_free(&DPt); csr_free(&Z);
    return H;
}

/* Alg. 2 Initial_Pattern: N_ij = 1 iff B_ij = 2, B = |T| |D_H|^T W, W = Diag(3 - |D_H| 1) */
static ocsr initial_pattern(const ocsr *T, const ocsr *DH) {
    ocsr absT = csr_copy(T);
    for (int64_t k = 0; k < nnz_of(&absT); ++k) absT.v[k] = 1.0;
    ocsr absDHt = csr_transpose(DH);       /* m_H x n_H */
    for (int64_t u = 0; u < absDHt.nr; ++u)
        for (int64_t k = absDHt.rp[u]; k < absDHt.rp[u + 1]; ++k) {
            int32_t j = absDHt.ci[k];
            double w = 3.0 - (double)(DH->rp[j + 1] - DH->rp[j]);
            absDHt.v[k] = 1.0 * w;
        }
    ocsr B = csr_spgemm(&absT, &absDHt);
    int64_t cnt = 0;
    for (int64_t k = 0; k < nnz_of(&B); ++k) if (B.v[k] == 2.0) ++cnt;
    ocsr N = csr_alloc(B.nr, B.nc, cnt);
    int64_t q = 0;
    for (int64_t i = 0; i < B.nr; ++i) {
        for (int64_t k = B.rp[i]; k < B.rp[i + 1]; ++k)
            if (B.v[k] == 2.0) { N.ci[q] = B.ci[k]; N.v[q] = 0.0; ++q; }
        N.rp[i + 1] = q;
    }
    csr_free(&absT); csr_free(&absDHt); csr_free(&B);
    return N;
}

static int32_t uf_find(int32_t *par, int32_t x) {
    while (par[x] != x) { par[x] = par[par[x]]; x = par[x]; }
    return x;
}

/* component labels of the local graph of row i (nodes T_i, two-node edges of N_i);
 * returns the number of components; comp[] indexed by position in T_i */
static int local_components(const ocsr *T, const ocsr *N, const ocsr *DH, int64_t i, int32_t *comp) {
    int m = (int)(T->rp[i + 1] - T->rp[i]);
    const int32_t *J = T->ci + T->rp[i];
    for (int a = 0; a < m; ++a) comp[a] = a;
    for (int64_t k = N->rp[i]; k < N->rp[i + 1]; ++k) {
        int32_t j = N->ci[k];
        if (DH->rp[j + 1] - DH->rp[j] != 2) continue;
        int32_t u = DH->ci[DH->rp[j]], v = DH->ci[DH->rp[j] + 1];
        int a = -1, b = -1;
        for (int q = 0; q < m; ++q) { if (J[q] == u) a = q; if (J[q] == v) b = q; }
        if (a < 0 || b < 0) continue;
        int32_t ra = uf_find(comp, a), rb = uf_find(comp, b);
        if (ra != rb) comp[ra < rb ? rb : ra] = ra < rb ? ra : rb;
    }
    int nc = 0;
    for (int a = 0; a < m; ++a) { comp[a] = uf_find(comp, a); if (comp[a] == a) ++nc; }
    return nc;
}

typedef struct { int32_t u, v; } opair;
static int cmp_pair(const void *x, const void *y) {
    const opair *a = (const opair *)x, *b = (const opair *)y;
    if (a->u != b->u) return (a->u > b->u) - (a->u < b->u);
    return (a->v > b->v) - (a->v < b->v);
}

/* sparse dot product of rows u and v of a CSR with sorted columns */
static double row_dot(const ocsr *M, int32_t u, int32_t v) {
    int64_t a = M->rp[u], b = M->rp[v];
    double s = 0.0;
    while (a < M->rp[u + 1] && b < M->rp[v + 1]) {
        if (M->ci[a] < M->ci[b]) ++a;
        else if (M->ci[b] < M->ci[a]) ++b;
        else { s += M->v[a] * M->v[b]; ++a; ++b; }
    }
    return s;
}

/* make_irreducible (Alg. 2): returns the number of coarse edges added, modifies DH */
static int64_t make_irreducible(ocsr *DH, const ocsr *T, const ocsr *N, int64_t *n_bad) {
    /* columns of M = D_h P_n are the rows of T^T (T holds D_h P_n) */
    ocsr Mt = csr_transpose(T);
    int64_t cap = 1024, np = 0;
    opair *add = (opair *)malloc(sizeof(opair) * (size_t)cap);
    int32_t comp[1024];
    *n_bad = 0;
    for (int64_t i = 0; i < T->nr; ++i) {
        int m = (int)(T->rp[i + 1] - T->rp[i]);
        if (m <= 1 || m > 1024) continue;
        int nc = local_components(T, N, DH, i, comp);
        if (nc <= 1) continue;
        (*n_bad)++;
        const int32_t *J = T->ci + T->rp[i];
        while (nc > 1) {
            double best = -1.0;
            for (int a = 0; a < m; ++a) for (int b = a + 1; b < m; ++b)
                if (comp[a] != comp[b]) { double z = fabs(row_dot(&Mt, J[a], J[b])); if (z > best) best = z; }
            int ba = -1, bb = -1;
            for (int a = 0; a < m && ba < 0; ++a) for (int b = a + 1; b < m; ++b)
                if (comp[a] != comp[b] && fabs(row_dot(&Mt, J[a], J[b])) >= best * (1.0 - 1e-9)) {
                    ba = a; bb = b; break;
                }
            if (np == cap) { cap *= 2; add = (opair *)realloc(add, sizeof(opair) * (size_t)cap); }
            add[np].u = J[ba]; add[np].v = J[bb]; ++np;
            int32_t ca = comp[ba], cb = comp[bb], lo = ca < cb ? ca : cb, hi = ca < cb ? cb : ca;
            for (int a = 0; a < m; ++a) if (comp[a] == hi) comp[a] = lo;
            --nc;
        }
    }
    csr_free(&Mt);
    if (np == 0) { free(add); return 0; }
    /* merge: existing two-node edges + new ones, sorted and unique; single-node edges after */
    int64_t n2 = 0, n1 = 0;
    for (int64_t j = 0; j < DH->nr; ++j) { if (DH->rp[j + 1] - DH->rp[j] == 2) ++n2; else ++n1; }
    opair *all = (opair *)malloc(sizeof(opair) * (size_t)(n2 + np));
    int32_t *singles = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n1 > 0 ? n1 : 1));
    int64_t q2 = 0, q1 = 0;
    for (int64_t j = 0; j < DH->nr; ++j) {
        if (DH->rp[j + 1] - DH->rp[j] == 2) { all[q2].u = DH->ci[DH->rp[j]]; all[q2].v = DH->ci[DH->rp[j] + 1]; ++q2; }
        else singles[q1++] = DH->ci[DH->rp[j]];
    }
    for (int64_t t = 0; t < np; ++t) all[q2++] = add[t];
    qsort(all, (size_t)q2, sizeof(opair), cmp_pair);
    int64_t nu = 0;
    for (int64_t t = 0; t < q2; ++t)
        if (nu == 0 || all[t].u != all[nu - 1].u || all[t].v != all[nu - 1].v) all[nu++] = all[t];
    int64_t added = nu - n2;
    ocsr H = csr_alloc(nu + n1, DH->nc, 2 * nu + n1);
    int64_t q = 0, e = 0;
    for (int64_t t = 0; t < nu; ++t) {
        H.ci[q] = all[t].u; H.v[q] = -1.0; ++q;
        H.ci[q] = all[t].v; H.v[q] = 1.0; ++q;
        H.rp[++e] = q;
    }
    for (int64_t t = 0; t < n1; ++t) { H.ci[q] = singles[t]; H.v[q] = 1.0; ++q; H.rp[++e] = q; }
    csr_free(DH);
    *DH = H;
    free(all); free(singles); free(add);
    return added;
}

/* Local sub-problem of row i: G = [D_H]_{I,J} as a dense np x k column-major block (k = rank
 * columns kept), rt = the kept entries of r_i.  Returns k, or -1 when infeasible. */
static int local_system(const ocsr *T, const ocsr *N, const ocsr *DH, int64_t i, double *G, double *rt,
                        int *np_out) {
    int m = (int)(T->rp[i + 1] - T->rp[i]);
    int np = (int)(N->rp[i + 1] - N->rp[i]);
    const int32_t *J = T->ci + T->rp[i];
    int singular = 1;
    for (int64_t kk = N->rp[i]; kk < N->rp[i + 1]; ++kk) {
        int32_t j = N->ci[kk];
        if (DH->rp[j + 1] - DH->rp[j] == 1) singular = 0;
    }
    int k = singular ? m - 1 : m;    /* Reduce_Dimension: drop the largest coarse node */
    if (k < 0) k = 0;
    *np_out = np;
    if (k > np) return -1;
    for (int c = 0; c < k; ++c) {
        for (int r = 0; r < np; ++r) G[(size_t)c * np + r] = 0.0;
        rt[c] = T->v[T->rp[i] + c];
    }
    for (int r = 0; r < np; ++r) {
        int32_t j = N->ci[N->rp[i] + r];
        for (int64_t q = DH->rp[j]; q < DH->rp[j + 1]; ++q) {
            int32_t u = DH->ci[q];
            for (int c = 0; c < k; ++c) if (J[c] == u) G[(size_t)c * np + r] = DH->v[q];
        }
    }
    return k;
}

static void hier_free_level(olevel *L) {
    csr_free(&L->A); csr_free(&L->D); csr_free(&L->An);
    free(L->col_e); free(L->col_n); free(L->agg);
    csr_free(&L->Pn); csr_free(&L->DH); csr_free(&L->T); csr_free(&L->Pe); csr_free(&L->P0);
    csr_free(&L->PeT);
}

void orc_free(ohier *h) {
    if (!h) return;
    for (int l = 0; l < h->nlev; ++l) hier_free_level(&h->L[l]);
    free(h->chol);
    free(h);
}

#define ORC_OK 0
#define ORC_EINVAL_REUSE -7     /* the related system did not reproduce the previous hierarchy's levels */
#define ORC_EINVAL -1
#define ORC_EINFEASIBLE -6
#define ORC_ENUMERIC -9

/* The projected, D^-1-scaled gradient of the energy sum_j P_:j^T A P_:j at P (values on the
 * pattern N): g_i = Pi_i (D^-1 A P)_{i, N_i} row by row, Pi_i the orthogonal projection onto the
 * null space of row i's constraint matrix G~^T (Sec. 3: masking to N, then the row constraints). */
static int projected_gradient(const olevel *L, const ocsr *N, const double *Pv, double *g, int cap) {
    ocsr P = csr_copy(N);
    memcpy(P.v, Pv, sizeof(double) * (size_t)N->rp[N->nr]);
    ocsr AP = csr_spgemm(&L->A, &P);
    int nth = ORC_THREADS();
    double *G = (double *)malloc(sizeof(double) * (size_t)cap * cap * (size_t)nth);
    double *rt = (double *)malloc(sizeof(double) * (size_t)cap * (size_t)nth);
    double *tau = (double *)malloc(sizeof(double) * (size_t)cap * (size_t)nth);
    double *tmp = (double *)malloc(sizeof(double) * (size_t)cap * (size_t)nth);
    int status = ORC_OK;
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < L->A.nr; ++i) {
        if (ORC_FAILED(status)) continue;
        const size_t t = (size_t)ORC_TID();
        double *Gt = G + t * (size_t)cap * cap, *rtt = rt + t * (size_t)cap, *taut = tau + t * (size_t)cap;
        double *tmpt = tmp + t * (size_t)cap;
        double d = csr_diag(&L->A, i);
        int np;
        int k = local_system(&L->T, N, &L->DH, i, Gt, rtt, &np);
        if (np == 0) continue;
        double *gi = g + N->rp[i];
        int64_t ka = AP.rp[i];
        for (int r = 0; r < np; ++r) {
            int32_t j = N->ci[N->rp[i] + r];
            while (ka < AP.rp[i + 1] && AP.ci[ka] < j) ++ka;
            gi[r] = (ka < AP.rp[i + 1] && AP.ci[ka] == j) ? AP.v[ka] / d : 0.0;
        }
        if (k > 0) {
            if (house_qr(np, k, Gt, taut)) { ORC_FAIL(status, ORC_EINFEASIBLE); continue; }
            qr_project_null(np, k, Gt, taut, gi, tmpt);
        }
    }
    free(G); free(rt); free(tau); free(tmp);
    csr_free(&AP);
    csr_free(&P);
    return status;
}
/* sum_i a_ii x_i . y_i over the pattern rows: the inner product of the projected CG below in
 * which D^-1 is the preconditioner (it scales whole rows, so it commutes with each Pi_i) */
static double row_weighted_dot(const olevel *L, const ocsr *N, const double *x, const double *y) {
    double s = 0.0;
    for (int64_t i = 0; i < L->A.nr; ++i) {
        double d = csr_diag(&L->A, i), si = 0.0;
        for (int64_t k = N->rp[i]; k < N->rp[i + 1]; ++k) si += x[k] * y[k];
        s += d * si;
    }
    return s;
}
/* Projected CG for the saddle-point system of eq. (8) (Sec. 3): CG on the energy restricted to
 * corrections that keep the pattern and the row constraints, preconditioned by D^-1, started
 * from the feasible P (so that only one projection per iteration is needed), iters steps. */
static int emin_projected_cg(const olevel *L, const ocsr *N, double *Pv, int iters, int cap) {
    int64_t nz = N->rp[N->nr];
    double *z = (double *)calloc((size_t)(nz > 0 ? nz : 1), sizeof(double));
    double *pd = (double *)calloc((size_t)(nz > 0 ? nz : 1), sizeof(double));
    double *w = (double *)calloc((size_t)(nz > 0 ? nz : 1), sizeof(double));
    int status = projected_gradient(L, N, Pv, w, cap);
    for (int64_t q = 0; q < nz; ++q) { z[q] = -w[q]; pd[q] = z[q]; }
    double rz = row_weighted_dot(L, N, z, z);
    for (int it = 0; it < iters && status == ORC_OK && rz > 0.0; ++it) {
        status = projected_gradient(L, N, pd, w, cap);
        if (status != ORC_OK) break;
        double pq = row_weighted_dot(L, N, pd, w);
        if (!(pq > 0.0)) break;
        double alpha = rz / pq;
        for (int64_t q = 0; q < nz; ++q) { Pv[q] += alpha * pd[q]; z[q] -= alpha * w[q]; }
        double rz_new = row_weighted_dot(L, N, z, z);
        double beta = rz_new / rz;
        rz = rz_new;
        for (int64_t q = 0; q < nz; ++q) pd[q] = z[q] + beta * pd[q];
    }
    free(z); free(pd); free(w);
    return status;
}

/* one level of Alg. 3 plus the emin iteration; fills L's transfer data and returns the
 * next-level operators through Anext/Dnext/Annext. */
/* prev != NULL: a related system (new values of A on the same patterns, Sec. 3 warm-start
 * remark).  The structural parts of prev's level are reused (aggregates, D_H, the pattern N),
 * the initial guess starts from prev's P_e instead of the pattern value, the rest is recomputed. */
static int build_level(olevel *L, int lev, const orc_opts *o, ocsr *Anext, ocsr *Dnext, ocsr *Annext,
                       const olevel *prev) {
    uint64_t s = o->seed + 1000ULL * (uint64_t)lev;
    int64_t nv = L->An.nr, ne = L->A.nr;
    /* drop tolerance: aggregation and prolongator smoothing on the filtered nodal matrix */
    ocsr Af = {0, 0, NULL, NULL, NULL};
    if (o->sa_theta > 0.0) Af = strength_filter(&L->An, o->sa_theta);
    const ocsr *Ag = o->sa_theta > 0.0 ? &Af : &L->An;
    /* aggregation on the nodal graph (drop tolerance 0: every structural entry is strong) */
    L->agg = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nv > 0 ? nv : 1));
    if (prev) {
        memcpy(L->agg, prev->agg, sizeof(int32_t) * (size_t)nv);
        L->nagg = prev->nagg;
    } else if (lev == 0 && o->agg0) {
        memcpy(L->agg, o->agg0, sizeof(int32_t) * (size_t)nv);
        L->nagg = o->nagg0;
    } else {
        L->nagg = aggregate_mis2(Ag, s + 1, L->agg);
        if (L->nagg < 0) { if (Af.rp) csr_free(&Af); return ORC_ENUMERIC; }
    }
    /* nodal prolongator */
    ocsr Pb = pbar_matrix(nv, L->nagg, L->agg);
    if (o->unsmoothed_pn) {
        L->Pn = csr_copy(&Pb);
        L->rho = 0.0; L->omega_sa = 0.0;
    } else {
        L->rho = power_rho(Ag, s + 4, o->power_iters);
        L->omega_sa = 4.0 / (3.0 * L->rho);
        ocsr APb = csr_spgemm(Ag, &Pb);
        for (int64_t i = 0; i < nv; ++i) {
            double d = csr_diag(Ag, i);
            for (int64_t k = APb.rp[i]; k < APb.rp[i + 1]; ++k) APb.v[k] /= d;
        }
        ocsr Pn = csr_add(&Pb, 1.0, &APb, -L->omega_sa);
        for (int64_t i = 0; i < nv; ++i) {
            double rs = 0.0;
            for (int64_t k = Pn.rp[i]; k < Pn.rp[i + 1]; ++k) rs += Pn.v[k];
            if (!isfinite(rs)) {
                csr_free(&APb); csr_free(&Pn); csr_free(&Pb);
                if (Af.rp) csr_free(&Af);
                return ORC_ENUMERIC;
            }
            if (rs <= SA_MIN_ROWSUM) {
                /* smoothing left no usable row: keep the tentative row (same pattern) */
                for (int64_t k = Pn.rp[i]; k < Pn.rp[i + 1]; ++k) Pn.v[k] = Pn.ci[k] == L->agg[i] ? 1.0 : 0.0;
                L->n_rows_unsmoothed++;
                continue;
            }
            for (int64_t k = Pn.rp[i]; k < Pn.rp[i + 1]; ++k) Pn.v[k] /= rs;
        }
        csr_free(&APb);
        L->Pn = Pn;
    }
    if (Af.rp) csr_free(&Af);
    /* coarse gradient from the piecewise-constant aggregates, or from Alg. 1 applied to P_n */
    if (prev) {
        L->DH = csr_copy(&prev->DH);
    } else if (o->pn_alg1) {
        int32_t *pc = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nv > 0 ? nv : 1));
        gen_piecewise_const(&L->Pn, o->alg1_passes, pc);
        L->DH = coarse_gradient(&L->D, pc, L->nagg);
        free(pc);
    } else {
        L->DH = coarse_gradient(&L->D, L->agg, L->nagg);
    }
    /* Alg. 2: T (with the values r = D_h P_n), N, irreducibility */
    L->T = csr_spgemm(&L->D, &L->Pn);
    ocsr N = prev ? csr_copy(&prev->Pe) : initial_pattern(&L->T, &L->DH);
    L->n_added = prev ? prev->n_added : 0;
    for (int pass = 0; pass < 8 && !prev; ++pass) {
        int64_t bad = 0;
        int64_t added = make_irreducible(&L->DH, &L->T, &N, &bad);
        if (pass == 0) L->n_infeasible0 = bad;
        if (added == 0) break;
        L->n_added += added;
        csr_free(&N);
        N = initial_pattern(&L->T, &L->DH);
    }
    int64_t nH = L->DH.nr;
    /* initial guess: ones on the pattern + least-norm correction, then emin iterations */
    memset(L->hist, 0, sizeof(L->hist));
    L->P0 = csr_copy(&N);
    int maxnp = 0, maxm = 0;
    for (int64_t i = 0; i < ne; ++i) {
        int np = (int)(N.rp[i + 1] - N.rp[i]), m = (int)(L->T.rp[i + 1] - L->T.rp[i]);
        if (np > maxnp) maxnp = np;
        if (m > maxm) maxm = m;
    }
    int cap = (maxnp > maxm ? maxnp : maxm) + 1;
    int nth = ORC_THREADS();
    /* per-thread scratch of the row-local solves (rows are independent) */
    double *G = (double *)malloc(sizeof(double) * (size_t)cap * cap * (size_t)nth);
    double *rt = (double *)malloc(sizeof(double) * (size_t)cap * (size_t)nth);
    double *tau = (double *)malloc(sizeof(double) * (size_t)cap * (size_t)nth);
    double *p = (double *)malloc(sizeof(double) * (size_t)cap * (size_t)nth);
    double *tmp = (double *)malloc(sizeof(double) * (size_t)cap * (size_t)nth);
    int status = ORC_OK;
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < ne; ++i) {
        if (ORC_FAILED(status)) continue;
        const size_t t = (size_t)ORC_TID();
        double *Gt = G + t * (size_t)cap * cap, *rtt = rt + t * (size_t)cap, *taut = tau + t * (size_t)cap;
        double *pt = p + t * (size_t)cap, *tmpt = tmp + t * (size_t)cap;
        int np;
        int m = (int)(L->T.rp[i + 1] - L->T.rp[i]);
        int k = local_system(&L->T, &N, &L->DH, i, Gt, rtt, &np);
        if (k < 0) { ORC_FAIL(status, ORC_EINFEASIBLE); continue; }
#pragma omp atomic
        L->hist[np < 32 ? np : 32][m < 32 ? m : 32]++;
        if (np == 0) continue;
        if (k > 0 && house_qr(np, k, Gt, taut)) { ORC_FAIL(status, ORC_EINFEASIBLE); continue; }
        double *pi = L->P0.v + N.rp[i];
        for (int r = 0; r < np; ++r) pi[r] = prev ? prev->Pe.v[N.rp[i] + r] : o->p0_value;
        if (k > 0) {
            /* p += Q R^-T (rt - Gt^T p): Gt^T p = R^T Q^T p (first k entries) */
            memcpy(tmpt, pi, sizeof(double) * (size_t)np);
            house_apply_qt(np, k, Gt, taut, tmpt);
            double *res = (double *)malloc(sizeof(double) * (size_t)k);
            for (int c = 0; c < k; ++c) {
                double sv = 0.0;
                for (int q = 0; q <= c; ++q) sv += Gt[(size_t)c * np + q] * tmpt[q];
                res[c] = rtt[c] - sv;
            }
            qr_minnorm(np, k, Gt, taut, res, pt);
            for (int r = 0; r < np; ++r) pi[r] += pt[r];
            free(res);
        }
    }
    L->Pe = csr_copy(&L->P0);
    if (o->emin_method == 1 && status == ORC_OK)
        status = emin_projected_cg(L, &N, L->Pe.v, o->emin_iters, cap);
    for (int it = 0; it < o->emin_iters && status == ORC_OK && o->emin_method == 0; ++it) {
        /* dP = D^-1 A P (full product), then the projection: mask to N, row constraint */
        ocsr AP = csr_spgemm(&L->A, &L->Pe);
#pragma omp parallel for schedule(dynamic, 256)
        for (int64_t i = 0; i < ne; ++i) {
            if (ORC_FAILED(status)) continue;
            const size_t t = (size_t)ORC_TID();
            double *Gt = G + t * (size_t)cap * cap, *rtt = rt + t * (size_t)cap, *taut = tau + t * (size_t)cap;
            double *tmpt = tmp + t * (size_t)cap;
            double d = csr_diag(&L->A, i);
            int np;
            int k = local_system(&L->T, &N, &L->DH, i, Gt, rtt, &np);
            if (np == 0) continue;
            double *dp = p + t * (size_t)cap;
            int64_t ka = AP.rp[i];
            for (int r = 0; r < np; ++r) {
                int32_t j = N.ci[N.rp[i] + r];
                while (ka < AP.rp[i + 1] && AP.ci[ka] < j) ++ka;
                dp[r] = (ka < AP.rp[i + 1] && AP.ci[ka] == j) ? AP.v[ka] / d : 0.0;
            }
            if (k > 0) {
                if (house_qr(np, k, Gt, taut)) { ORC_FAIL(status, ORC_EINFEASIBLE); continue; }
                qr_project_null(np, k, Gt, taut, dp, tmpt);
            }
            double *pi = L->Pe.v + N.rp[i];
            for (int r = 0; r < np; ++r) pi[r] -= o->emin_omega * dp[r];
        }
        csr_free(&AP);
    }
    free(G); free(rt); free(tau); free(p); free(tmp);
    csr_free(&N); csr_free(&Pb);
    if (status != ORC_OK) return status;
    (void)nH;
    L->energy0 = energy_trace(&L->A, &L->P0);
    L->energy1 = energy_trace(&L->A, &L->Pe);
    /* Galerkin coarse operators */
    L->PeT = csr_transpose(&L->Pe);
    ocsr AP = csr_spgemm(&L->A, &L->Pe);
    *Anext = csr_spgemm(&L->PeT, &AP);
    csr_free(&AP);
    ocsr PnT = csr_transpose(&L->Pn);
    ocsr AnP = csr_spgemm(&L->An, &L->Pn);
    *Annext = csr_spgemm(&PnT, &AnP);
    csr_free(&PnT); csr_free(&AnP);
    *Dnext = csr_copy(&L->DH);
    return ORC_OK;
}

static int dense_cholesky(int64_t n, double *a) {
    for (int64_t j = 0; j < n; ++j) {
        double d = a[j * n + j];
        for (int64_t k = 0; k < j; ++k) d -= a[j * n + k] * a[j * n + k];
        if (!(d > 0.0)) return -1;
        d = sqrt(d);
        a[j * n + j] = d;
        for (int64_t i = j + 1; i < n; ++i) {
            double s = a[i * n + j];
            for (int64_t k = 0; k < j; ++k) s -= a[i * n + k] * a[j * n + k];
            a[i * n + j] = s / d;
        }
        for (int64_t i = 0; i < j; ++i) a[i * n + j] = 0.0;
    }
    return 0;
}

static ocsr csr_from(int64_t nr, int64_t nc, const int64_t *rp, const int32_t *ci, const double *v) {
    ocsr a = csr_alloc(nr, nc, rp[nr]);
    memcpy(a.rp, rp, sizeof(int64_t) * (size_t)(nr + 1));
    memcpy(a.ci, ci, sizeof(int32_t) * (size_t)rp[nr]);
    memcpy(a.v, v, sizeof(double) * (size_t)rp[nr]);
    return a;
}

/* Setup of the whole hierarchy from A_e (ne x ne) and D_h (ne x nv). */
static ohier *setup_hier(int64_t ne, int64_t nv, const int64_t *A_rp, const int32_t *A_ci, const double *A_v,
                         const int64_t *D_rp, const int32_t *D_ci, const double *D_v, const orc_opts *o,
                         const ohier *prev, int *status) {
    ohier *h = (ohier *)calloc(1, sizeof(ohier));
    olevel *L0 = &h->L[0];
    L0->A = csr_from(ne, ne, A_rp, A_ci, A_v);
    L0->D = csr_from(ne, nv, D_rp, D_ci, D_v);
    /* nodal operator D_h^T A_e D_h */
    ocsr Dt = csr_transpose(&L0->D);
    ocsr AD = csr_spgemm(&L0->A, &L0->D);
    L0->An = csr_spgemm(&Dt, &AD);
    csr_free(&Dt); csr_free(&AD);
    int st = ORC_OK;
    int lev = 0;
    for (;;) {
        olevel *L = &h->L[lev];
        uint64_t s = o->seed + 1000ULL * (uint64_t)lev;
        L->col_e = (int32_t *)malloc(sizeof(int32_t) * (size_t)(L->A.nr > 0 ? L->A.nr : 1));
        L->col_n = (int32_t *)malloc(sizeof(int32_t) * (size_t)(L->An.nr > 0 ? L->An.nr : 1));
        L->ncol_e = color_graph(&L->A, s + 2, L->col_e);
        L->ncol_n = color_graph(&L->An, s + 3, L->col_n);
        int coarsest = (L->A.nr <= o->max_coarse) || (lev + 1 >= o->max_levels) || (L->An.nr <= 1);
        if (coarsest) break;
        ocsr An1, D1, A1;
        const olevel *pl = prev && lev + 1 < prev->nlev ? &prev->L[lev] : NULL;
        if (prev && !pl) { st = ORC_EINVAL_REUSE; break; }
        st = build_level(L, lev, o, &A1, &D1, &An1, pl);
        if (st != ORC_OK) break;
        if (L->nagg >= L->An.nr) {          /* no coarsening: stop here */
            csr_free(&A1); csr_free(&D1); csr_free(&An1);
            free(L->agg); L->agg = NULL;
            csr_free(&L->Pn); csr_free(&L->DH); csr_free(&L->T); csr_free(&L->Pe);
            csr_free(&L->P0); csr_free(&L->PeT);
            break;
        }
        h->L[lev + 1].A = A1; h->L[lev + 1].D = D1; h->L[lev + 1].An = An1;
        ++lev;
    }
    h->nlev = lev + 1;
    if (st == ORC_OK) {
        olevel *C = &h->L[lev];
        int64_t n = C->A.nr;
        h->nc = n;
        h->chol = (double *)calloc((size_t)(n * n > 0 ? n * n : 1), sizeof(double));
        for (int64_t i = 0; i < n; ++i)
            for (int64_t k = C->A.rp[i]; k < C->A.rp[i + 1]; ++k) h->chol[i * n + C->A.ci[k]] = C->A.v[k];
        if (dense_cholesky(n, h->chol)) st = ORC_ENUMERIC;
    }
    if (st == ORC_OK && prev && h->nlev != prev->nlev) st = ORC_EINVAL_REUSE;
    h->status = st;
    if (status) *status = st;
    return h;
}

ohier *orc_setup(int64_t ne, int64_t nv, const int64_t *A_rp, const int32_t *A_ci, const double *A_v,
                 const int64_t *D_rp, const int32_t *D_ci, const double *D_v, const orc_opts *o,
                 int *status) {
    return setup_hier(ne, nv, A_rp, A_ci, A_v, D_rp, D_ci, D_v, o, NULL, status);
}

/* The hierarchy of a related system: new values A_v on prev's level-0 pattern (see build_level). */
ohier *orc_update(const ohier *prev, const double *A_v, const orc_opts *o, int *status) {
    const olevel *P0 = &prev->L[0];
    return setup_hier(P0->A.nr, P0->D.nc, P0->A.rp, P0->A.ci, A_v, P0->D.rp, P0->D.ci, P0->D.v, o, prev, status);
}

/* ------------------------------------------------------------------ solve */
static void sgs_sweep(const ocsr *A, const int32_t *color, int32_t ncol, const double *b, double *x) {
    for (int dir = 0; dir < 2; ++dir)
        for (int32_t cc = 0; cc < ncol; ++cc) {
            int32_t c = dir == 0 ? cc : ncol - 1 - cc;
            /* the rows of one colour do not couple: each reads x only at other colours */
#pragma omp parallel for schedule(static)
            for (int64_t i = 0; i < A->nr; ++i) {
                if (color[i] != c) continue;
                double s = b[i], d = 0.0;
                for (int64_t k = A->rp[i]; k < A->rp[i + 1]; ++k) {
                    if (A->ci[k] == i) d = A->v[k];
                    else s -= A->v[k] * x[A->ci[k]];
                }
                x[i] = s / d;
            }
        }
}

/* one symmetric Hiptmair sweep (Sec. 6.1) */
static void hiptmair(const olevel *L, const double *b, double *x) {
    int64_t ne = L->A.nr, nv = L->An.nr;
    sgs_sweep(&L->A, L->col_e, L->ncol_e, b, x);
    double *r = (double *)malloc(sizeof(double) * (size_t)(ne > 0 ? ne : 1));
    csr_matvec(&L->A, x, r);
    for (int64_t i = 0; i < ne; ++i) r[i] = b[i] - r[i];
    double *g = (double *)calloc((size_t)(nv > 0 ? nv : 1), sizeof(double));
    double *c = (double *)calloc((size_t)(nv > 0 ? nv : 1), sizeof(double));
    for (int64_t e = 0; e < ne; ++e)
        for (int64_t k = L->D.rp[e]; k < L->D.rp[e + 1]; ++k) g[L->D.ci[k]] += L->D.v[k] * r[e];
    sgs_sweep(&L->An, L->col_n, L->ncol_n, g, c);
    for (int64_t e = 0; e < ne; ++e)
        for (int64_t k = L->D.rp[e]; k < L->D.rp[e + 1]; ++k) x[e] += L->D.v[k] * c[L->D.ci[k]];
    sgs_sweep(&L->A, L->col_e, L->ncol_e, b, x);
    free(r); free(g); free(c);
}

static void vcycle(const ohier *h, int lev, const double *b, double *x) {
    const olevel *L = &h->L[lev];
    int64_t n = L->A.nr;
    if (lev == h->nlev - 1) {
        /* x = (L L^T)^-1 b */
        for (int64_t i = 0; i < n; ++i) {
            double s = b[i];
            for (int64_t k = 0; k < i; ++k) s -= h->chol[i * n + k] * x[k];
            x[i] = s / h->chol[i * n + i];
        }
        for (int64_t i = n - 1; i >= 0; --i) {
            double s = x[i];
            for (int64_t k = i + 1; k < n; ++k) s -= h->chol[k * n + i] * x[k];
            x[i] = s / h->chol[i * n + i];
        }
        return;
    }
    for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
    hiptmair(L, b, x);
    double *r = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    csr_matvec(&L->A, x, r);
    for (int64_t i = 0; i < n; ++i) r[i] = b[i] - r[i];
    int64_t nH = L->PeT.nr;
    double *bH = (double *)malloc(sizeof(double) * (size_t)(nH > 0 ? nH : 1));
    double *xH = (double *)malloc(sizeof(double) * (size_t)(nH > 0 ? nH : 1));
    csr_matvec(&L->PeT, r, bH);
    vcycle(h, lev + 1, bH, xH);
    csr_matvec(&L->Pe, xH, r);
    for (int64_t i = 0; i < n; ++i) x[i] += r[i];
    hiptmair(L, b, x);
    free(r); free(bH); free(xH);
}

void orc_vcycle(const ohier *h, const double *r, double *z) { vcycle(h, 0, r, z); }

static double dot(int64_t n, const double *a, const double *b) {
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

/* PCG with x0 = 0, stop when ||r_k|| <= tol ||b|| (recursive residual).  Returns 0 on
 * convergence, -4 not converged, -5 breakdown.  relres_true = ||b - A x|| / ||b||. */
int orc_solve(const ohier *h, const double *b, double *x, double tol, int max_iter, int precond,
              int *iters, double *relres_true, double *history) {
    const ocsr *A = &h->L[0].A;
    int64_t n = A->nr;
    double *r = (double *)malloc(sizeof(double) * (size_t)n);
    double *z = (double *)malloc(sizeof(double) * (size_t)n);
    double *p = (double *)malloc(sizeof(double) * (size_t)n);
    double *q = (double *)malloc(sizeof(double) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) { x[i] = 0.0; r[i] = b[i]; }
    double bnorm = sqrt(dot(n, b, b));
    int status = -4, it = 0;
    if (bnorm == 0.0) { status = 0; goto done; }
    if (precond) vcycle(h, 0, r, z); else memcpy(z, r, sizeof(double) * (size_t)n);
    memcpy(p, z, sizeof(double) * (size_t)n);
    double rz = dot(n, r, z);
    for (it = 0; it < max_iter;) {
        csr_matvec(A, p, q);
        double pq = dot(n, p, q);
        if (!(pq > 0.0)) { status = -5; break; }
        double alpha = rz / pq;
        for (int64_t i = 0; i < n; ++i) { x[i] += alpha * p[i]; r[i] -= alpha * q[i]; }
        ++it;
        double rn = sqrt(dot(n, r, r));
        if (history) history[it - 1] = rn / bnorm;
        if (rn <= tol * bnorm) { status = 0; break; }
        if (precond) vcycle(h, 0, r, z); else memcpy(z, r, sizeof(double) * (size_t)n);
        double rz1 = dot(n, r, z);
        double beta = rz1 / rz;
        rz = rz1;
        for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
    }
done:
    csr_matvec(A, x, q);
    for (int64_t i = 0; i < n; ++i) q[i] = b[i] - q[i];
    if (relres_true) *relres_true = bnorm > 0 ? sqrt(dot(n, q, q)) / bnorm : 0.0;
    if (iters) *iters = it;
    free(r); free(z); free(p); free(q);
    return status;
}

/* ------------------------------------------------------------------ accessors for the tests */
int orc_num_levels(const ohier *h) { return h->nlev; }
int orc_status(const ohier *h) { return h->status; }

/* sizes of level l:  [ne, nv, nnzA, nnzD, nnzAn, nagg, nnzPn, nH, nnzDH, nnzPe, ncol_e, ncol_n,
 *                     n_added, nnzT, n_infeasible0, has_transfer, n_rows_unsmoothed] */
int orc_level_sizes(const ohier *h, int l, int64_t *out) {
    if (l < 0 || l >= h->nlev) return -1;
    const olevel *L = &h->L[l];
    int tr = L->agg != NULL;
    out[0] = L->A.nr; out[1] = L->An.nr; out[2] = nnz_of(&L->A); out[3] = nnz_of(&L->D);
    out[4] = nnz_of(&L->An); out[5] = tr ? L->nagg : 0; out[6] = tr ? nnz_of(&L->Pn) : 0;
    out[7] = tr ? L->DH.nr : 0; out[8] = tr ? nnz_of(&L->DH) : 0; out[9] = tr ? nnz_of(&L->Pe) : 0;
    out[10] = L->ncol_e; out[11] = L->ncol_n; out[12] = tr ? L->n_added : 0;
    out[13] = tr ? nnz_of(&L->T) : 0; out[14] = tr ? L->n_infeasible0 : 0; out[15] = tr;
    out[16] = tr ? L->n_rows_unsmoothed : 0;
    return 0;
}

/* scalars of level l: [rho, omega_sa, energy(P0), energy(Pe)] */
int orc_level_scalars(const ohier *h, int l, double *out) {
    if (l < 0 || l >= h->nlev) return -1;
    const olevel *L = &h->L[l];
    out[0] = L->rho; out[1] = L->omega_sa; out[2] = L->energy0; out[3] = L->energy1;
    return 0;
}

int orc_level_hist(const ohier *h, int l, int64_t *out /*33*33*/) {
    if (l < 0 || l >= h->nlev) return -1;
    memcpy(out, h->L[l].hist, sizeof(h->L[l].hist));
    return 0;
}

/* matrix ids: 0 A, 1 D, 2 An, 3 Pn, 4 DH, 5 T (values r), 6 Pe, 7 P0 */
static const ocsr *level_matrix(const ohier *h, int l, int which) {
    const olevel *L = &h->L[l];
    switch (which) {
        case 0: return &L->A; case 1: return &L->D; case 2: return &L->An; case 3: return &L->Pn;
        case 4: return &L->DH; case 5: return &L->T; case 6: return &L->Pe; case 7: return &L->P0;
    }
    return NULL;
}
int orc_matrix_nnz(const ohier *h, int l, int which, int64_t *nr, int64_t *nc, int64_t *nnz) {
    if (l < 0 || l >= h->nlev) return -1;
    const ocsr *m = level_matrix(h, l, which);
    if (!m || !m->rp) return -1;
    *nr = m->nr; *nc = m->nc; *nnz = nnz_of(m);
    return 0;
}
int orc_matrix_get(const ohier *h, int l, int which, int64_t *rp, int32_t *ci, double *v) {
    const ocsr *m = level_matrix(h, l, which);
    if (!m || !m->rp) return -1;
    memcpy(rp, m->rp, sizeof(int64_t) * (size_t)(m->nr + 1));
    memcpy(ci, m->ci, sizeof(int32_t) * (size_t)nnz_of(m));
    memcpy(v, m->v, sizeof(double) * (size_t)nnz_of(m));
    return 0;
}
/* int vectors: 0 agg, 1 col_e, 2 col_n */
int orc_level_ivec(const ohier *h, int l, int which, int32_t *out) {
    if (l < 0 || l >= h->nlev) return -1;
    const olevel *L = &h->L[l];
    if (which == 0) { if (!L->agg) return -1; memcpy(out, L->agg, sizeof(int32_t) * (size_t)L->An.nr); }
    else if (which == 1) memcpy(out, L->col_e, sizeof(int32_t) * (size_t)L->A.nr);
    else if (which == 2) memcpy(out, L->col_n, sizeof(int32_t) * (size_t)L->An.nr);
    else return -1;
    return 0;
}

/* ------------------------------------------------------------------ unit entry points */
/* colour a graph given in CSR (self loops ignored) */
int orc_color(int64_t n, const int64_t *rp, const int32_t *ci, uint64_t seed, int32_t *color) {
    ocsr G; G.nr = n; G.nc = n; G.rp = (int64_t *)rp; G.ci = (int32_t *)ci; G.v = NULL;
    return color_graph(&G, seed, color);
}
int64_t orc_aggregate(int64_t n, const int64_t *rp, const int32_t *ci, uint64_t seed, int32_t *agg) {
    ocsr G; G.nr = n; G.nc = n; G.rp = (int64_t *)rp; G.ci = (int32_t *)ci; G.v = NULL;
    return aggregate_mis2(&G, seed, agg);
}
/* coarse gradient of D (ne x nv) under aggregates; returns nH, fills up to cap rows */
int64_t orc_coarse_gradient(int64_t ne, int64_t nv, const int64_t *rp, const int32_t *ci, const double *v,
                            const int32_t *agg, int64_t nagg, int64_t cap, int64_t *H_rp, int32_t *H_ci,
                            double *H_v) {
    ocsr D; D.nr = ne; D.nc = nv; D.rp = (int64_t *)rp; D.ci = (int32_t *)ci; D.v = (double *)v;
    ocsr H = coarse_gradient(&D, agg, nagg);
    int64_t nH = H.nr;
    if (nH <= cap && H_rp) {
        memcpy(H_rp, H.rp, sizeof(int64_t) * (size_t)(nH + 1));
        memcpy(H_ci, H.ci, sizeof(int32_t) * (size_t)nnz_of(&H));
        memcpy(H_v, H.v, sizeof(double) * (size_t)nnz_of(&H));
    }
    csr_free(&H);
    return nH;
}
/* least-norm solution of G^T p = r for a dense G (np x m, row-major) with the given
 * singularity flag; p[np].  Returns k (columns kept) or -1. */
int orc_minnorm(int np, int m, const double *Grow, const double *r, int singular, double *p) {
    int k = singular ? m - 1 : m;
    if (k < 0) k = 0;
    if (k > np) return -1;
    double *a = (double *)malloc(sizeof(double) * (size_t)(np * (k > 0 ? k : 1)));
    double *tau = (double *)malloc(sizeof(double) * (size_t)(k > 0 ? k : 1));
    for (int c = 0; c < k; ++c) for (int i = 0; i < np; ++i) a[(size_t)c * np + i] = Grow[(size_t)i * m + c];
    int rc = k;
    if (k > 0 && house_qr(np, k, a, tau)) rc = -1;
    else if (k > 0) qr_minnorm(np, k, a, tau, r, p);
    else for (int i = 0; i < np; ++i) p[i] = 0.0;
    free(a); free(tau);
    return rc;
}
/* orthogonal projection of x onto null(G^T) (same G convention) */
int orc_project(int np, int m, const double *Grow, int singular, double *x) {
    int k = singular ? m - 1 : m;
    if (k <= 0) return 0;
    if (k > np) return -1;
    double *a = (double *)malloc(sizeof(double) * (size_t)(np * k));
    double *tau = (double *)malloc(sizeof(double) * (size_t)k);
    double *tmp = (double *)malloc(sizeof(double) * (size_t)np);
    for (int c = 0; c < k; ++c) for (int i = 0; i < np; ++i) a[(size_t)c * np + i] = Grow[(size_t)i * m + c];
    int rc = 0;
    if (house_qr(np, k, a, tau)) rc = -1;
    else qr_project_null(np, k, a, tau, x, tmp);
    free(a); free(tau); free(tmp);
    return rc;
}
