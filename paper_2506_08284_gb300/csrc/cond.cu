// 1-norm condition estimate of D^-1 A_e (D = diag(A_e)), which the paper (Sec. 6.1) uses to cap
// the CG tolerance at kappa(D^-1 A) / 1e16 where rounding limits the reachable accuracy.
//
// ||D^-1 A||_1 is computed exactly: A is symmetric, so column j's sum is sum_i |a_ji| / a_ii.
// ||(D^-1 A)^-1||_1 is estimated by Hager's method (W. W. Hager, "Condition estimates", SIAM J.
// Sci. Stat. Comput. 5 (1984)), the iteration behind Matlab's condest: with B = D^-1 A,
//   x = (1/n, ..., 1/n);  repeat: y = B^-1 x, est = ||y||_1, xi = sign(y), z = B^-T xi;
//   stop when max_j |z_j| <= z^T x, else x = e_j for the j of the largest |z_j|.
// B^-1 x = A^-1 (D x) and B^-T xi = D (A^-1 xi) (A symmetric) are solves with the handle's own
// preconditioned CG to a relative residual of 1e-10.
#include <cmath>

#include "sphc_level.cuh"

using namespace sphc;

namespace {

constexpr int CN_BLOCKS = 512;

// per row j of A: sum_i |a_ji| / a_ii (a column sum of |D^-1 A|, by symmetry)
__global__ void k_col_abs_sum(const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                              const double* __restrict__ v, const double* __restrict__ d, int64_t n,
                              double* __restrict__ out) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double s = 0.0;
    for (int64_t k = rp[j]; k < rp[j + 1]; ++k) s += fabs(v[k]) / d[ci[k]];
    out[j] = s;
}
// block partials of (max |a_i|, its first index) and of sum |a_i|
__global__ void __launch_bounds__(256) k_abs_stats(const double* __restrict__ a, int64_t n, double* __restrict__ pmax,
                                                   int64_t* __restrict__ parg, double* __restrict__ psum) {
    __shared__ double smax[256], ssum[256];
    __shared__ int64_t sarg[256];
    double m = -1.0, sm = 0.0;
    int64_t arg = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double x = fabs(a[i]);
        sm += x;
        if (x > m) { m = x; arg = i; }
    }
    smax[threadIdx.x] = m;
    sarg[threadIdx.x] = arg;
    ssum[threadIdx.x] = sm;
    __syncthreads();
    if (threadIdx.x == 0) {
        double bm = -1.0, bs = 0.0;
        int64_t ba = 0;
        for (int t = 0; t < (int)blockDim.x; ++t) {
            bs += ssum[t];
            if (smax[t] > bm || (smax[t] == bm && sarg[t] < ba)) { bm = smax[t]; ba = sarg[t]; }
        }
        pmax[blockIdx.x] = bm;
        parg[blockIdx.x] = ba;
        psum[blockIdx.x] = bs;
    }
}
__global__ void k_scale_vec(const double* __restrict__ d, const double* __restrict__ x, int64_t n, double* __restrict__ y) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = d[i] * x[i];
}
__global__ void k_sign_vec(const double* __restrict__ y, int64_t n, double* __restrict__ s) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) s[i] = y[i] >= 0.0 ? 1.0 : -1.0;
}
__global__ void k_fill(double* a, int64_t n, double v) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = v;
}

// max |a_i| with its index, and sum |a_i| (host reduction of CN_BLOCKS partials in a fixed order)
int abs_stats(const double* a, int64_t n, DBuf<double>& pmax, DBuf<int64_t>& parg, DBuf<double>& psum, double* mx,
              int64_t* arg, double* sum, cudaStream_t s) {
    SPHC_LAUNCH(k_abs_stats<<<CN_BLOCKS, 256, 0, s>>>(a, n, pmax.p, parg.p, psum.p));
    std::vector<double> hm(CN_BLOCKS), hs(CN_BLOCKS);
    std::vector<int64_t> ha(CN_BLOCKS);
    SPHC_CK(cudaMemcpyAsync(hm.data(), pmax.p, sizeof(double) * CN_BLOCKS, cudaMemcpyDeviceToHost, s));
    SPHC_CK(cudaMemcpyAsync(ha.data(), parg.p, sizeof(int64_t) * CN_BLOCKS, cudaMemcpyDeviceToHost, s));
    SPHC_CK(cudaMemcpyAsync(hs.data(), psum.p, sizeof(double) * CN_BLOCKS, cudaMemcpyDeviceToHost, s));
    SPHC_CK(cudaStreamSynchronize(s));
    double bm = -1.0, bs = 0.0;
    int64_t ba = 0;
    for (int b = 0; b < CN_BLOCKS; ++b) {
        bs += hs[b];
        if (hm[b] > bm || (hm[b] == bm && ha[b] < ba)) { bm = hm[b]; ba = ha[b]; }
    }
    *mx = bm;
    *arg = ba;
    *sum = bs;
    return SPHC_OK;
}

}  // namespace

namespace {
__global__ void k_uniform_pm1(double* x, int64_t n, uint64_t seed) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] = 2.0 * ((double)(splitmix64(seed, (uint64_t)i) >> 11) * (1.0 / 9007199254740992.0)) - 1.0;
}
__global__ void k_add_to(const double* __restrict__ z, double* __restrict__ x, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] += z[i];
}
__global__ void k_negate(double* a, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = -a[i];
}
}  // namespace

// V-cycle convergence factor: the stationary iteration x <- x + M^-1 (b - A x) with b = 0 from a
// seeded random x; ratios of successive A-norms ||x_k||_A / ||x_{k-1}||_A, geometric mean of the
// last `tail` of `iters` iterations.
extern "C" int sphc_vcycle_factor(sphc_handle* h, int iters, int tail, uint64_t seed, double* factor, void* stream) {
    if (!h || !factor || iters < 2 || tail < 1 || tail > iters) {
        set_error("sphc_vcycle_factor: invalid argument");
        return SPHC_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    Hierarchy& H = h->H;
    const DCSR& A = H.L[0].A;
    const int64_t n = A.nr;
    DBuf<double> x, r, z, sc;
    for (DBuf<double>* b : {&x, &r, &z}) SPHC_TRY(b->alloc(n, s));
    SPHC_TRY(sc.alloc(1, s));
    SPHC_LAUNCH(k_uniform_pm1<<<grid_for(n, 256), 256, 0, s>>>(x.p, n, seed));
    auto anorm = [&](double* out) -> int {
        SPHC_TRY(spmv64(A, x.p, r.p, s));
        SPHC_TRY(dot64(x.p, r.p, n, sc.p, s));
        double v = 0.0;
        SPHC_CK(cudaMemcpyAsync(&v, sc.p, sizeof(double), cudaMemcpyDeviceToHost, s));
        SPHC_CK(cudaStreamSynchronize(s));
        *out = sqrt(v > 0.0 ? v : 0.0);
        return SPHC_OK;
    };
    double e_prev = 0.0, logsum = 0.0;
    SPHC_TRY(anorm(&e_prev));
    for (int k = 1; k <= iters; ++k) {
        // r = -A x (anorm left A x in r), z = M^-1 r, x += z
        SPHC_LAUNCH(k_negate<<<grid_for(n, 256), 256, 0, s>>>(r.p, n));
        SPHC_TRY(apply_vcycle_user(H, r.p, z.p, s));
        SPHC_LAUNCH(k_add_to<<<grid_for(n, 256), 256, 0, s>>>(z.p, x.p, n));
        double e = 0.0;
        SPHC_TRY(anorm(&e));
        if (k > iters - tail) logsum += log(e_prev > 0.0 ? e / e_prev : 1.0);
        e_prev = e;
    }
    *factor = exp(logsum / tail);
    SPHC_CK(cudaGetLastError());
    return SPHC_OK;
}

namespace {
// per row i: e_i = sum_t P_it (A P)_{i, N_i(t)} (warp per row; lanes own pattern entries; a
// binary search of column N_i(t) in every P row f of A's row i)
__global__ void k_row_energy(int64_t ne, const int64_t* __restrict__ arp, const int32_t* __restrict__ aci,
                             const double* __restrict__ av, const int64_t* __restrict__ prp,
                             const int32_t* __restrict__ pci, const double* __restrict__ pv, double* __restrict__ e) {
    const int lane = threadIdx.x & 31;
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= ne) return;
    const int64_t n0 = prp[i], n1 = prp[i + 1];
    double sum = 0.0;
    for (int64_t q = n0 + lane; q < n1; q += 32) {
        const int32_t key = pci[q];
        double ap = 0.0;
        for (int64_t ka = arp[i]; ka < arp[i + 1]; ++ka) {
            const int32_t f = aci[ka];
            int64_t lo = prp[f], hi = prp[f + 1];
            while (lo < hi) {
                const int64_t mid = (lo + hi) >> 1;
                if (pci[mid] < key) lo = mid + 1; else hi = mid;
            }
            if (lo < prp[f + 1] && pci[lo] == key) ap += av[ka] * pv[lo];
        }
        sum += pv[q] * ap;
    }
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (lane == 0) e[i] = sum;
}
}  // namespace

// trace(P_e^T A P_e) of level `level` (the A-energy the energy minimisation of Sec. 3 reduces)
extern "C" int sphc_prolongator_energy(const sphc_handle* h, int level, double* energy, void* stream) {
    if (!h || !energy || level < 0 || level + 1 >= h->H.nlev || !h->H.L[level].has_transfer) {
        set_error("sphc_prolongator_energy: level %d has no prolongator", level);
        return SPHC_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const Level& L = h->H.L[level];
    const int64_t n = L.A.nr;
    DBuf<double> e, sc, ones;
    SPHC_TRY(e.alloc(n, s));
    SPHC_TRY(ones.alloc(n, s));
    SPHC_TRY(sc.alloc(1, s));
    SPHC_LAUNCH(k_row_energy<<<grid_for(n * 32, 256), 256, 0, s>>>(n, L.A.rp.p, L.A.ci.p, L.A.v.p, L.Pe.rp.p, L.Pe.ci.p,
                                                                   L.Pe.v.p, e.p));
    SPHC_LAUNCH(k_fill<<<grid_for(n, 256), 256, 0, s>>>(ones.p, n, 1.0));
    SPHC_TRY(dot64(e.p, ones.p, n, sc.p, s));
    SPHC_CK(cudaMemcpyAsync(energy, sc.p, sizeof(double), cudaMemcpyDeviceToHost, s));
    SPHC_CK(cudaStreamSynchronize(s));
    return SPHC_OK;
}

extern "C" int sphc_cond_estimate(sphc_handle* h, int max_steps, double* kappa, double* norm_b, double* norm_binv,
                                  void* stream) {
    if (!h || max_steps < 1) {
        set_error("sphc_cond_estimate: invalid argument");
        return SPHC_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    Hierarchy& H = h->H;
    const DCSR& A = H.L[0].A;
    const int64_t n = A.nr;
    if (n == 0) {
        set_error("sphc_cond_estimate: empty operator");
        return SPHC_EINVAL;
    }
    DBuf<double> d, col, x, y, z, t, pmax, psum;
    DBuf<int64_t> parg;
    for (DBuf<double>* b : {&d, &col, &x, &y, &z, &t}) SPHC_TRY(b->alloc(n, s));
    SPHC_TRY(pmax.alloc(CN_BLOCKS, s));
    SPHC_TRY(psum.alloc(CN_BLOCKS, s));
    SPHC_TRY(parg.alloc(CN_BLOCKS, s));
    SPHC_TRY(csr_diag(A, d.p, s));
    // ||D^-1 A||_1
    SPHC_LAUNCH(k_col_abs_sum<<<grid_for(n, 256), 256, 0, s>>>(A.rp.p, A.ci.p, A.v.p, d.p, n, col.p));
    double nb = 0.0, unused = 0.0;
    int64_t unused_i = 0;
    SPHC_TRY(abs_stats(col.p, n, pmax, parg, psum, &nb, &unused_i, &unused, s));
    // Hager's iteration for ||B^-1||_1
    SPHC_LAUNCH(k_fill<<<grid_for(n, 256), 256, 0, s>>>(x.p, n, 1.0 / (double)n));
    double est = 0.0;
    const double tol = 1e-10;
    for (int step = 0; step < max_steps; ++step) {
        int it = 0;
        double rr = 0.0;
        SPHC_LAUNCH(k_scale_vec<<<grid_for(n, 256), 256, 0, s>>>(d.p, x.p, n, t.p));       // D x
        int rc = pcg_solve(H, t.p, y.p, tol, s, &it, &rr);                                  // y = A^-1 D x
        if (rc != SPHC_OK && rc != SPHC_ENOTCONV && rc != SPHC_ESTAGNATION) return rc;
        double ymax = 0.0, ysum = 0.0;
        int64_t yarg = 0;
        SPHC_TRY(abs_stats(y.p, n, pmax, parg, psum, &ymax, &yarg, &ysum, s));
        est = ysum;
        SPHC_LAUNCH(k_sign_vec<<<grid_for(n, 256), 256, 0, s>>>(y.p, n, t.p));             // xi
        rc = pcg_solve(H, t.p, z.p, tol, s, &it, &rr);                                      // A^-1 xi
        if (rc != SPHC_OK && rc != SPHC_ENOTCONV && rc != SPHC_ESTAGNATION) return rc;
        SPHC_LAUNCH(k_scale_vec<<<grid_for(n, 256), 256, 0, s>>>(d.p, z.p, n, z.p));       // z = D A^-1 xi
        double zmax = 0.0, zsum = 0.0;
        int64_t zarg = 0;
        SPHC_TRY(abs_stats(z.p, n, pmax, parg, psum, &zmax, &zarg, &zsum, s));
        SPHC_TRY(dot64(z.p, x.p, n, pmax.p, s));                                           // z^T x
        double ztx = 0.0;
        SPHC_CK(cudaMemcpyAsync(&ztx, pmax.p, sizeof(double), cudaMemcpyDeviceToHost, s));
        SPHC_CK(cudaStreamSynchronize(s));
        if (step > 0 && zmax <= ztx) break;
        SPHC_CK(cudaMemsetAsync(x.p, 0, sizeof(double) * n, s));                            // x = e_j
        const double one = 1.0;
        SPHC_CK(cudaMemcpyAsync(x.p + zarg, &one, sizeof(double), cudaMemcpyHostToDevice, s));
        SPHC_CK(cudaStreamSynchronize(s));
    }
    SPHC_CK(cudaGetLastError());
    if (norm_b) *norm_b = nb;
    if (norm_binv) *norm_binv = est;
    if (kappa) *kappa = nb * est;
    return SPHC_OK;
}
