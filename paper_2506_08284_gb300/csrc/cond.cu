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
