/*
 * Seeded synthetic inputs for the eddy-current edge-element system (Sec. 1, eqs. (1)-(2)):
 * the unit cube cut into n^3 hexahedra, each split into six tetrahedra (the Kuhn split
 * named in Sec. 6.1), lowest-order Whitney/Nedelec edge elements, A_e = S_e + M_e, and the
 * discrete gradient D_h (Sec. 1, the +-1 edge/node matrix).
 *
 * This file only manufactures inputs.  It holds none of the AMG method: no aggregation,
 * prolongators, smoothers or Krylov iterations.  Both the GPU library and the CPU oracle
 * receive the matrices written here as plain arrays.
 *
 * Conventions (the paper leaves them open):
 *   - nodes (i,j,k), 0 <= i,j,k <= n, global id g = i + N*(j + N*k) with N = n+1;
 *   - every edge joins a node to node + d for one of the seven non-negative directions
 *     d in {x, y, z, x+y, x+z, y+z, x+y+z}; it is oriented from the lower global id (tail,
 *     -1 in D_h) to the higher one (head, +1);
 *   - Dirichlet mode: every edge lying in a face of the cube and every boundary node is
 *     eliminated; D_h rows of edges with one boundary end keep one entry, rows with two
 *     boundary ends (interior edges between two faces) are empty;
 *   - natural mode: every edge and node is kept;
 *   - edge ids follow (tail global id, direction) order; interior node ids follow global
 *     order;
 *   - random numbers: splitmix64 (Steele, Lea, Flood 2014) on a counter, uniform on [0,1) from
 *     the top 53 bits, normal by Box-Muller.
 *
 * Element matrices on a tetrahedron T with barycentric coordinates l_a:
 *   w_ab = l_a grad l_b - l_b grad l_a,  curl w_ab = 2 grad l_a x grad l_b,
 *   S_T(e,f) = |T| curl w_e . curl w_f,
 *   M_T(e,f) = sigma_T * int_T w_e . w_f, with int_T l_a l_b = |T| (1 + delta_ab) / 20.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

typedef struct {
    int32_t n;            /* cells per axis */
    int32_t natural;      /* 1: keep boundary (natural BC); 0: eliminate (tangential Dirichlet) */
    double jitter;        /* interior node jitter amplitude as a fraction of h */
    uint64_t seed_jitter;
    int32_t sigma_kind;   /* 0: constant; 1: box [0.25,0.75]^3 -> sigma_in else sigma_out; 2: log-normal */
    double sigma_in, sigma_out;  /* kind 0 uses sigma_in; kind 2: log10 sigma ~ N(0, sigma_in^2) clipped */
    double log_lo, log_hi;       /* clip range for kind 2 */
    uint64_t seed_sigma;
    int32_t which;        /* 0: A = S + M, 1: S only, 2: M only */
    int32_t nthreads;     /* OpenMP threads (0 = default) */
} kg_params;

static inline uint64_t kg_splitmix64(uint64_t seed, uint64_t counter) {
    uint64_t z = seed + (counter + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
static inline double kg_uniform(uint64_t seed, uint64_t counter) {
    return (double)(kg_splitmix64(seed, counter) >> 11) * (1.0 / 9007199254740992.0);
}

static const int DIRS[7][3] = {{1,0,0},{0,1,0},{0,0,1},{1,1,0},{1,0,1},{0,1,1},{1,1,1}};
static const int PERMS[6][3] = {{0,1,2},{0,2,1},{1,0,2},{1,2,0},{2,0,1},{2,1,0}};
/* local edges of a tet (v0,v1,v2,v3) */
static const int TET_EDGES[6][2] = {{0,1},{0,2},{0,3},{1,2},{1,3},{2,3}};

typedef struct {
    int n, N, natural;
    int64_t nnode_all;
    int32_t *edge_id;     /* [nnode_all*7] -> interior-edge id or -1 */
    int32_t *node_id;     /* [nnode_all] -> interior-node id or -1 */
    int64_t n_edges, n_nodes;
    double *X;            /* [nnode_all*3] coordinates */
    double *sig;          /* [6 n^3] per-tet sigma */
} kg_mesh;

static int dir_index(int dx, int dy, int dz) {
    for (int d = 0; d < 7; ++d)
        if (DIRS[d][0] == dx && DIRS[d][1] == dy && DIRS[d][2] == dz) return d;
    return -1;
}

static int kg_mesh_init(const kg_params *p, kg_mesh *m, int need_geom) {
    int n = p->n, N = n + 1;
    m->n = n; m->N = N; m->natural = p->natural;
    m->nnode_all = (int64_t)N * N * N;
    m->edge_id = (int32_t *)malloc(sizeof(int32_t) * m->nnode_all * 7);
    m->node_id = (int32_t *)malloc(sizeof(int32_t) * m->nnode_all);
    m->X = NULL; m->sig = NULL;
    if (!m->edge_id || !m->node_id) return -1;
    int64_t ne = 0, nv = 0;
    for (int k = 0; k <= n; ++k) for (int j = 0; j <= n; ++j) for (int i = 0; i <= n; ++i) {
        int64_t g = i + (int64_t)N * (j + (int64_t)N * k);
        int bnd = (i == 0 || j == 0 || k == 0 || i == n || j == n || k == n);
        m->node_id[g] = (p->natural || !bnd) ? (int32_t)(nv++) : -1;
        for (int d = 0; d < 7; ++d) {
            int hi = i + DIRS[d][0], hj = j + DIRS[d][1], hk = k + DIRS[d][2];
            int32_t id = -1;
            if (hi <= n && hj <= n && hk <= n) {
                int in_face = 0;
                if (!p->natural) {
                    /* the edge lies in a boundary face iff both ends share a boundary coordinate */
                    if ((i == 0 && hi == 0) || (i == n && hi == n)) in_face = 1;
                    if ((j == 0 && hj == 0) || (j == n && hj == n)) in_face = 1;
                    if ((k == 0 && hk == 0) || (k == n && hk == n)) in_face = 1;
                }
                if (!in_face) id = (int32_t)(ne++);
            }
            m->edge_id[g * 7 + d] = id;
        }
    }
    m->n_edges = ne; m->n_nodes = nv;
    if (!need_geom) return 0;
    m->X = (double *)malloc(sizeof(double) * m->nnode_all * 3);
    int64_t ntet = 6LL * n * n * n;
    m->sig = (double *)malloc(sizeof(double) * ntet);
    if (!m->X || !m->sig) return -1;
    double h = 1.0 / n;
    for (int k = 0; k <= n; ++k) for (int j = 0; j <= n; ++j) for (int i = 0; i <= n; ++i) {
        int64_t g = i + (int64_t)N * (j + (int64_t)N * k);
        int bnd = (i == 0 || j == 0 || k == 0 || i == n || j == n || k == n);
        int c[3] = {i, j, k};
        for (int a = 0; a < 3; ++a) {
            double x = c[a] * h;
            if (!bnd && p->jitter != 0.0)
                x += p->jitter * h * (2.0 * kg_uniform(p->seed_jitter, (uint64_t)(3 * g + a)) - 1.0);
            m->X[3 * g + a] = x;
        }
    }
    for (int64_t t = 0; t < ntet; ++t) {
        double s = p->sigma_in;
        if (p->sigma_kind == 1) {
            int64_t cell = t / 6; int pm = (int)(t % 6);
            int ci = (int)(cell % n), cj = (int)((cell / n) % n), ck = (int)(cell / ((int64_t)n * n));
            int v[4][3]; v[0][0] = ci; v[0][1] = cj; v[0][2] = ck;
            for (int q = 0; q < 3; ++q) { for (int a = 0; a < 3; ++a) v[q + 1][a] = v[q][a]; v[q + 1][PERMS[pm][q]] += 1; }
            double cen[3] = {0, 0, 0};
            for (int q = 0; q < 4; ++q) {
                int64_t g = v[q][0] + (int64_t)N * (v[q][1] + (int64_t)N * v[q][2]);
                for (int a = 0; a < 3; ++a) cen[a] += 0.25 * m->X[3 * g + a];
            }
            int inside = 1;
            for (int a = 0; a < 3; ++a) if (cen[a] < 0.25 || cen[a] > 0.75) inside = 0;
            s = inside ? p->sigma_in : p->sigma_out;
        } else if (p->sigma_kind == 2) {
            double u1 = 1.0 - kg_uniform(p->seed_sigma, (uint64_t)(2 * t));
            double u2 = kg_uniform(p->seed_sigma, (uint64_t)(2 * t + 1));
            double z = sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2);
            double l = p->sigma_in * z;
            if (l < p->log_lo) l = p->log_lo;
            if (l > p->log_hi) l = p->log_hi;
            s = pow(10.0, l);
        }
        m->sig[t] = s;
    }
    return 0;
}

static void kg_mesh_free(kg_mesh *m) {
    free(m->edge_id); free(m->node_id); free(m->X); free(m->sig);
}

/* global ids of the 4 vertices of tet pm of cell (ci,cj,ck), in increasing order */
static inline void tet_vertices(const kg_mesh *m, int ci, int cj, int ck, int pm, int64_t g[4], int v[4][3]) {
    v[0][0] = ci; v[0][1] = cj; v[0][2] = ck;
    for (int q = 0; q < 3; ++q) {
        for (int a = 0; a < 3; ++a) v[q + 1][a] = v[q][a];
        v[q + 1][PERMS[pm][q]] += 1;
    }
    for (int q = 0; q < 4; ++q) g[q] = v[q][0] + (int64_t)m->N * (v[q][1] + (int64_t)m->N * v[q][2]);
}

/* interior-edge id of the tet's local edge q (or -1) */
static inline int32_t tet_edge_id(const kg_mesh *m, int v[4][3], const int64_t g[4], int q) {
    int a = TET_EDGES[q][0], b = TET_EDGES[q][1];
    int d = dir_index(v[b][0] - v[a][0], v[b][1] - v[a][1], v[b][2] - v[a][2]);
    return m->edge_id[g[a] * 7 + d];
}

/* element matrix row: local edge q against the 6 local edges, for A/S/M */
static void tet_row(const kg_mesh *m, const int64_t g[4], double sigma, int which, int q, double out[6]) {
    double P[4][3];
    for (int a = 0; a < 4; ++a) for (int c = 0; c < 3; ++c) P[a][c] = m->X[3 * g[a] + c];
    double J[3][3];
    for (int r = 0; r < 3; ++r) for (int c = 0; c < 3; ++c) J[r][c] = P[r + 1][c] - P[0][c];
    double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1])
               - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0])
               + J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
    double vol = fabs(det) / 6.0;
    /* inverse of J: grad l_{r+1} = column r of J^{-1} */
    double Ji[3][3];
    Ji[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
    Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
    Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
    Ji[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
    Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
    Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
    Ji[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
    Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
    Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
    double G[4][3];
    for (int r = 0; r < 3; ++r) for (int c = 0; c < 3; ++c) G[r + 1][c] = Ji[c][r];
    for (int c = 0; c < 3; ++c) G[0][c] = -(G[1][c] + G[2][c] + G[3][c]);
    double GG[4][4];
    for (int a = 0; a < 4; ++a) for (int b = 0; b < 4; ++b)
        GG[a][b] = G[a][0] * G[b][0] + G[a][1] * G[b][1] + G[a][2] * G[b][2];
    int ea = TET_EDGES[q][0], eb = TET_EDGES[q][1];
    double ce[3] = {2.0 * (G[ea][1] * G[eb][2] - G[ea][2] * G[eb][1]),
                    2.0 * (G[ea][2] * G[eb][0] - G[ea][0] * G[eb][2]),
                    2.0 * (G[ea][0] * G[eb][1] - G[ea][1] * G[eb][0])};
    for (int f = 0; f < 6; ++f) {
        int fa = TET_EDGES[f][0], fb = TET_EDGES[f][1];
        double v = 0.0;
        if (which != 2) {
            double cf[3] = {2.0 * (G[fa][1] * G[fb][2] - G[fa][2] * G[fb][1]),
                            2.0 * (G[fa][2] * G[fb][0] - G[fa][0] * G[fb][2]),
                            2.0 * (G[fa][0] * G[fb][1] - G[fa][1] * G[fb][0])};
            v += vol * (ce[0] * cf[0] + ce[1] * cf[1] + ce[2] * cf[2]);
        }
        if (which != 1) {
            /* int (l_a grad l_b - l_b grad l_a).(l_c grad l_d - l_d grad l_c) */
#define LL(x, y) (vol * ((x) == (y) ? 2.0 : 1.0) / 20.0)
            double mm = GG[eb][fb] * LL(ea, fa) - GG[eb][fa] * LL(ea, fb)
                      - GG[ea][fb] * LL(eb, fa) + GG[ea][fa] * LL(eb, fb);
#undef LL
            v += sigma * mm;
        }
        out[f] = v;
    }
}

#define KG_MAXROW 64

/* Row e of the operator: columns (sorted) and values.  Returns the row length. */
static int kg_row(const kg_mesh *m, int64_t tail_g, int dir, int which, int32_t *cols, double *vals,
                  double *sigma_mean) {
    int n = m->n, N = m->N;
    int ti = (int)(tail_g % N), tj = (int)((tail_g / N) % N), tk = (int)(tail_g / ((int64_t)N * N));
    int hi = ti + DIRS[dir][0], hj = tj + DIRS[dir][1], hk = tk + DIRS[dir][2];
    int len = 0; double ssum = 0.0; int scnt = 0;
    for (int ck = tk - 1; ck <= tk; ++ck) for (int cj = tj - 1; cj <= tj; ++cj) for (int ci = ti - 1; ci <= ti; ++ci) {
        if (ci < 0 || cj < 0 || ck < 0 || ci >= n || cj >= n || ck >= n) continue;
        if (hi - ci > 1 || hj - cj > 1 || hk - ck > 1) continue;
        for (int pm = 0; pm < 6; ++pm) {
            int64_t g[4]; int v[4][3];
            tet_vertices(m, ci, cj, ck, pm, g, v);
            int q = -1;
            for (int l = 0; l < 6; ++l) {
                int a = TET_EDGES[l][0], b = TET_EDGES[l][1];
                if (g[a] == tail_g && v[b][0] == hi && v[b][1] == hj && v[b][2] == hk) q = l;
            }
            if (q < 0) continue;
            int64_t tet = 6 * (ci + (int64_t)n * (cj + (int64_t)n * ck)) + pm;
            double sg = m->sig ? m->sig[tet] : 1.0;
            ssum += sg; scnt++;
            double rowv[6] = {0, 0, 0, 0, 0, 0};
            if (vals) tet_row(m, g, sg, which, q, rowv);
            for (int f = 0; f < 6; ++f) {
                int32_t c = tet_edge_id(m, v, g, f);
                if (c < 0) continue;
                int pos = 0;
                while (pos < len && cols[pos] < c) ++pos;
                if (pos < len && cols[pos] == c) {
                    if (vals) vals[pos] += rowv[f];
                } else {
                    if (len >= KG_MAXROW) return -1;
                    memmove(cols + pos + 1, cols + pos, sizeof(int32_t) * (len - pos));
                    if (vals) memmove(vals + pos + 1, vals + pos, sizeof(double) * (len - pos));
                    cols[pos] = c;
                    if (vals) vals[pos] = rowv[f];
                    ++len;
                }
            }
        }
    }
    if (sigma_mean) *sigma_mean = scnt ? ssum / scnt : 0.0;
    return len;
}

/* sizes: out[0] = #edges (rows), out[1] = #nodes (D_h columns), out[2] = nnz(A), out[3] = nnz(D_h),
 * out[4] = #tets, out[5] = #all grid nodes */
int kg_count(const kg_params *p, int64_t *out) {
    kg_mesh m;
    if (kg_mesh_init(p, &m, 0)) { kg_mesh_free(&m); return -1; }
    int64_t nnzA = 0, nnzD = 0;
    int bad = 0;
#pragma omp parallel for reduction(+:nnzA,nnzD) reduction(|:bad) schedule(dynamic, 4096) num_threads(p->nthreads > 0 ? p->nthreads : 1)
    for (int64_t g = 0; g < m.nnode_all; ++g) {
        int32_t cols[KG_MAXROW];
        for (int d = 0; d < 7; ++d) {
            if (m.edge_id[g * 7 + d] < 0) continue;
            int len = kg_row(&m, g, d, 0, cols, NULL, NULL);
            if (len < 0) bad = 1; else nnzA += len;
            int N = m.N;
            int i = (int)(g % N), j = (int)((g / N) % N), k = (int)(g / ((int64_t)N * N));
            int64_t hg = (i + DIRS[d][0]) + (int64_t)N * ((j + DIRS[d][1]) + (int64_t)N * (k + DIRS[d][2]));
            nnzD += (m.node_id[g] >= 0) + (m.node_id[hg] >= 0);
        }
    }
    out[0] = m.n_edges; out[1] = m.n_nodes; out[2] = nnzA; out[3] = nnzD;
    out[4] = 6LL * p->n * p->n * p->n; out[5] = m.nnode_all;
    kg_mesh_free(&m);
    return bad ? -2 : 0;
}

/*
 * Fill the arrays (any output pointer may be NULL to skip it).
 *   A: CSR (rowptr[n_edges+1], col[nnzA], val[nnzA]) of the operator chosen by p->which;
 *   D: CSR of D_h (rowptr[n_edges+1], col[nnzD], val[nnzD] = -1 tail / +1 head);
 *   coords_nodes[n_nodes*3]: coordinates of the kept nodes (D_h column order);
 *   sigma_edge[n_edges]: mean sigma over the tets containing the edge;
 *   edge_ends[n_edges*2]: global (tail, head) node ids of each kept edge;
 *   coords_all[N^3*3], tets[6n^3*4] (global ids), tet_sigma[6n^3]: raw mesh for test assembly.
 */
int kg_fill(const kg_params *p,
            int64_t *A_rp, int32_t *A_ci, double *A_v,
            int64_t *D_rp, int32_t *D_ci, double *D_v,
            double *coords_nodes, double *sigma_edge, int64_t *edge_ends,
            double *coords_all, int64_t *tets, double *tet_sigma) {
    kg_mesh m;
    int need_geom = (A_v || coords_nodes || sigma_edge || coords_all || tet_sigma);
    if (kg_mesh_init(p, &m, need_geom)) { kg_mesh_free(&m); return -1; }
    int N = m.N, n = m.n;
    int nth = p->nthreads > 0 ? p->nthreads : 1;
    /* per-row lengths in edge order */
    int64_t ne = m.n_edges;
    int64_t *etail = (int64_t *)malloc(sizeof(int64_t) * ne);
    int8_t *edir = (int8_t *)malloc(ne);
    if (!etail || !edir) { kg_mesh_free(&m); return -1; }
    for (int64_t g = 0; g < m.nnode_all; ++g)
        for (int d = 0; d < 7; ++d) {
            int32_t id = m.edge_id[g * 7 + d];
            if (id >= 0) { etail[id] = g; edir[id] = (int8_t)d; }
        }
    int bad = 0;
    if (A_rp) {
        A_rp[0] = 0;
#pragma omp parallel for schedule(dynamic, 4096) num_threads(nth) reduction(|:bad)
        for (int64_t e = 0; e < ne; ++e) {
            int32_t cols[KG_MAXROW];
            int len = kg_row(&m, etail[e], edir[e], p->which, cols, NULL, NULL);
            if (len < 0) bad = 1;
            A_rp[e + 1] = len;
        }
        for (int64_t e = 0; e < ne; ++e) A_rp[e + 1] += A_rp[e];
    }
#pragma omp parallel for schedule(dynamic, 4096) num_threads(nth) reduction(|:bad)
    for (int64_t e = 0; e < ne; ++e) {
        int32_t cols[KG_MAXROW]; double vals[KG_MAXROW]; double smean = 0.0;
        if (A_ci || A_v || sigma_edge) {
            int len = kg_row(&m, etail[e], edir[e], p->which, cols, (A_v || sigma_edge) ? vals : NULL,
                             sigma_edge ? &smean : NULL);
            if (len < 0) { bad = 1; continue; }
            if (A_ci) memcpy(A_ci + A_rp[e], cols, sizeof(int32_t) * len);
            if (A_v) memcpy(A_v + A_rp[e], vals, sizeof(double) * len);
            if (sigma_edge) sigma_edge[e] = smean;
        }
        int64_t g = etail[e]; int d = edir[e];
        int i = (int)(g % N), j = (int)((g / N) % N), k = (int)(g / ((int64_t)N * N));
        int64_t hg = (i + DIRS[d][0]) + (int64_t)N * ((j + DIRS[d][1]) + (int64_t)N * (k + DIRS[d][2]));
        if (edge_ends) { edge_ends[2 * e] = g; edge_ends[2 * e + 1] = hg; }
    }
    if (D_rp) {
        D_rp[0] = 0;
        for (int64_t e = 0; e < ne; ++e) {
            int64_t g = etail[e]; int d = edir[e];
            int i = (int)(g % N), j = (int)((g / N) % N), k = (int)(g / ((int64_t)N * N));
            int64_t hg = (i + DIRS[d][0]) + (int64_t)N * ((j + DIRS[d][1]) + (int64_t)N * (k + DIRS[d][2]));
            int64_t pos = D_rp[e];
            if (m.node_id[g] >= 0) { if (D_ci) D_ci[pos] = m.node_id[g]; if (D_v) D_v[pos] = -1.0; ++pos; }
            if (m.node_id[hg] >= 0) { if (D_ci) D_ci[pos] = m.node_id[hg]; if (D_v) D_v[pos] = 1.0; ++pos; }
            D_rp[e + 1] = pos;
        }
    }
    if (coords_nodes)
        for (int64_t g = 0; g < m.nnode_all; ++g)
            if (m.node_id[g] >= 0)
                for (int a = 0; a < 3; ++a) coords_nodes[3 * (int64_t)m.node_id[g] + a] = m.X[3 * g + a];
    if (coords_all) memcpy(coords_all, m.X, sizeof(double) * 3 * m.nnode_all);
    int64_t ntet = 6LL * n * n * n;
    if (tets)
        for (int64_t t = 0; t < ntet; ++t) {
            int64_t cell = t / 6; int pm = (int)(t % 6);
            int ci = (int)(cell % n), cj = (int)((cell / n) % n), ck = (int)(cell / ((int64_t)n * n));
            int64_t g[4]; int v[4][3];
            tet_vertices(&m, ci, cj, ck, pm, g, v);
            for (int q = 0; q < 4; ++q) tets[4 * t + q] = g[q];
        }
    if (tet_sigma) memcpy(tet_sigma, m.sig, sizeof(double) * ntet);
    free(etail); free(edir);
    kg_mesh_free(&m);
    return bad ? -2 : 0;
}

/* Uniform[-1,1] right-hand side entries from a seed (counter = entry index). */
void kg_rhs(uint64_t seed, int64_t len, double *out) {
    for (int64_t i = 0; i < len; ++i) out[i] = 2.0 * kg_uniform(seed, (uint64_t)i) - 1.0;
}
