// extern "C" entry points of libsphc.so (declared and documented in include/sphc.h).
#include <chrono>
#include <cmath>
#include <cstring>
#include <algorithm>
#include <atomic>
#include <new>
#include <thread>
#include <string>
#include <vector>

#include "sphc_level.cuh"

using namespace sphc;

namespace {

// bytes allocated from the library pool of the current device (0 without a pool)
int64_t pool_used() {
    cudaMemPool_t pool = device_pool();
    uint64_t v = 0;
    if (!pool || cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &v) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return (int64_t)v;
}

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// copy a caller CSR (host or device) into a device CSR
int ingest_csr(const sphc_csr* M, DCSR& D, cudaStream_t s) {
    if (!M || M->nrows < 0 || M->ncols < 0 || !M->rowptr) {
        set_error("malformed CSR descriptor");
        return SPHC_EINVAL;
    }
    int64_t nnz = 0;
    SPHC_CK(cudaMemcpyAsync(&nnz, M->rowptr + M->nrows, sizeof(int64_t), cudaMemcpyDefault, s));
    SPHC_CK(cudaStreamSynchronize(s));
    if (nnz < 0 || (nnz > 0 && (!M->col || !M->val))) {
        set_error("malformed CSR arrays");
        return SPHC_EINVAL;
    }
    SPHC_TRY(D.alloc(M->nrows, M->ncols, nnz, s));
    SPHC_CK(cudaMemcpyAsync(D.rp.p, M->rowptr, sizeof(int64_t) * (M->nrows + 1), cudaMemcpyDefault, s));
    if (nnz > 0) {
        SPHC_CK(cudaMemcpyAsync(D.ci.p, M->col, sizeof(int32_t) * nnz, cudaMemcpyDefault, s));
        SPHC_CK(cudaMemcpyAsync(D.v.p, M->val, sizeof(double) * nnz, cudaMemcpyDefault, s));
    }
    return SPHC_OK;
}

// flags: 0 rowptr not monotone / wrong ends, 1 column out of range or unsorted, 2 non-finite
// value, 3 gradient row with >2 entries or entries not +-1 or two entries of equal sign,
// 4 missing/non-positive diagonal
__global__ void k_validate(const int64_t* rp, const int32_t* ci, const double* v, int64_t nr, int64_t nc, int64_t nnz,
                           int gradient, int* flags) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nr) return;
    int64_t b = rp[i], e = rp[i + 1];
    if (b < 0 || e < b || e > nnz || (i == 0 && b != 0) || (i == nr - 1 && e != nnz)) { atomicExch(&flags[0], 1); return; }
    bool diag = false;
    for (int64_t k = b; k < e; ++k) {
        int32_t c = ci[k];
        if (c < 0 || c >= nc || (k > b && ci[k - 1] >= c)) atomicExch(&flags[1], 1);
        if (!isfinite(v[k])) atomicExch(&flags[2], 1);
        if (c == i && v[k] > 0) diag = true;
    }
    if (gradient) {
        if (e - b > 2) atomicExch(&flags[3], 1);
        for (int64_t k = b; k < e; ++k) if (v[k] != 1.0 && v[k] != -1.0) atomicExch(&flags[3], 1);
        if (e - b == 2 && v[b] == v[b + 1]) atomicExch(&flags[3], 1);
    } else if (!diag) {
        atomicExch(&flags[4], 1);
    }
}

int validate(const DCSR& M, int gradient, const char* name, cudaStream_t s) {
    DBuf<int> f;
    SPHC_TRY(f.alloc(5, s));
    SPHC_TRY(f.zero(s));
    if (M.nr > 0) SPHC_LAUNCH(k_validate<<<grid_for(M.nr, 256), 256, 0, s>>>(M.rp.p, M.ci.p, M.v.p, M.nr, M.nc, M.nnz, gradient, f.p));
    int h[5];
    SPHC_CK(cudaMemcpyAsync(h, f.p, sizeof(h), cudaMemcpyDeviceToHost, s));
    SPHC_CK(cudaStreamSynchronize(s));
    const char* what[5] = {"row pointers are not monotone", "a column index is out of range or unsorted",
                           "a value is not finite", "a row is not a gradient row (<=2 entries of +-1, opposite signs)",
                           "a diagonal entry is missing or not positive"};
    for (int q = 0; q < 5; ++q)
        if (h[q]) {
            set_error("%s: %s", name, what[q]);
            return SPHC_EINVAL;
        }
    return SPHC_OK;
}

int setup_impl(sphc_handle* h, const sphc_csr* A_e, const sphc_csr* D_h, const double* coords,
               const double* sigma_edge, cudaStream_t s) {
    Hierarchy& H = h->H;
    const sphc_opts& o = H.opts;
    if (o.sweep_form < 0 || o.sweep_form > 3) {
        set_error("opts.sweep_form must be 0, 1, 2 or 3 (got %d)", (int)o.sweep_form);
        return SPHC_EINVAL;
    }
    {
        const int l = o.sell_lpr0, c = o.sell_ch0;
        if (!(l == 0 || l == 1 || l == 2 || l == 4 || l == 8 || l == 16 || l == 32) || !(c == 0 || c == 1 || c == 2 || c == 4)) {
            set_error("opts.sell_lpr0 must be 0 or a power of two up to 32 and opts.sell_ch0 0, 1, 2 or 4 (got %d, %d)",
                      l, c);
            return SPHC_EINVAL;
        }
        if (o.emin_method < 0 || o.emin_method > 1) {
            set_error("opts.emin_method must be 0 (projected Jacobi) or 1 (projected CG) (got %d)", (int)o.emin_method);
            return SPHC_EINVAL;
        }
        if (!(o.sa_theta >= 0.0 && o.sa_theta < 1.0) || o.pn_alg1 < 0 || o.pn_alg1 > 1 || o.alg1_passes < 1 ||
            o.grid_wait_polls < 0) {
            set_error("opts: sa_theta must lie in [0, 1), pn_alg1 be 0 or 1, alg1_passes >= 1 and grid_wait_polls >= 0");
            return SPHC_EINVAL;
        }
        if (o.mlp_wait_polls < 0) {
            set_error("opts.mlp_wait_polls must be >= 0 (got %d)", (int)o.mlp_wait_polls);
            return SPHC_EINVAL;
        }
    }
    H.L.clear();
    H.L.reserve(o.max_levels > 0 ? o.max_levels : 1);
    H.L.emplace_back();
    Level& L0 = H.L[0];
    Profiler* prof = H.prof.on ? &H.prof : nullptr;
    Section total(prof, "setup_total", s);
    Section* sec_in = new Section(prof, "setup_ingest", s);
    SPHC_TRY(ingest_csr(A_e, L0.A, s));
    SPHC_TRY(ingest_csr(D_h, L0.D, s));
    if (L0.A.nr != L0.A.nc || L0.D.nr != L0.A.nr) {
        set_error("A_e must be n_e x n_e and D_h n_e x n_v (got %lldx%lld and %lldx%lld)", (long long)L0.A.nr,
                  (long long)L0.A.nc, (long long)L0.D.nr, (long long)L0.D.nc);
        return SPHC_EINVAL;
    }
    SPHC_TRY(validate(L0.A, 0, "A_e", s));
    SPHC_TRY(validate(L0.D, 1, "D_h", s));
    if (coords) {
        SPHC_TRY(L0.X.alloc(L0.D.nc * 3, s));
        SPHC_CK(cudaMemcpyAsync(L0.X.p, coords, sizeof(double) * L0.D.nc * 3, cudaMemcpyDefault, s));
    }
    if (sigma_edge) {
        SPHC_TRY(L0.sig.alloc(L0.D.nr, s));
        SPHC_CK(cudaMemcpyAsync(L0.sig.p, sigma_edge, sizeof(double) * L0.D.nr, cudaMemcpyDefault, s));
    }
    if (o.learned) {
        if (!o.mlp_params || !coords) {
            set_error("learned warm start needs opts.mlp_params and coords");
            return SPHC_EINVAL;
        }
        SPHC_TRY(H.mlp.alloc(SPHC_MLP_NPARAM, s));
        SPHC_CK(cudaMemcpyAsync(H.mlp.p, o.mlp_params, sizeof(float) * SPHC_MLP_NPARAM, cudaMemcpyDefault, s));
    }
    delete sec_in;
    // nodal operator D_h^T A_e D_h
    {
        Section sec(prof, "setup_Dt_l0", s);
        SPHC_TRY(transpose(L0.D, L0.Dt, s));
    }
    {
        Section sec(prof, "setup_nodal_op", s);
        {
            Section sub(prof, "setup_nodal_AD", s);
            SPHC_TRY(amul_d(L0.A, L0.D, L0.AD, s));
        }
        if (prof) {
            auto csr_bytes = [](const DCSR& M) { return 12.0 * (double)M.nnz + 8.0 * (double)(M.nr + 1); };
            prof->timers[prof->find("setup_nodal_AD", 0.0)].bytes = csr_bytes(L0.A) + csr_bytes(L0.D) + csr_bytes(L0.AD);
        }
        SPHC_TRY(spgemm_sym(L0.Dt, L0.AD, L0.An, s));
    }
    int lev = 0;
    for (;;) {
        Level& L = H.L[lev];
        uint64_t seed = o.seed + 1000ULL * (uint64_t)lev;
        {
            Section sec(prof, lev == 0 ? "setup_colour_l0" : "setup_colour_ge1", s);
            SPHC_TRY(color_graph(L.A, seed + 2, L.col_e, &L.ncol_e, s, &L.rounds_e, prof, lev == 0 ? "e_l0" : "e_ge1"));
            SPHC_TRY(color_graph(L.An, seed + 3, L.col_n, &L.ncol_n, s, &L.rounds_n, prof, lev == 0 ? "n_l0" : "n_ge1"));
        }
        bool coarsest = L.A.nr <= o.max_coarse || lev + 1 >= o.max_levels || L.An.nr <= 1;
        if (coarsest) break;
        DCSR A1, D1, An1;
        DBuf<double> X1;
        Section sec(lev >= 1 ? prof : nullptr, "setup_levels_ge1", s);
        SPHC_TRY(build_level(L, lev, o, A1, D1, An1, X1, H.mlp.p, prof, s));
        if (L.nagg >= L.An.nr) break;      // no coarsening: this level is solved directly
        L.has_transfer = true;
        H.L.emplace_back();
        Level& N = H.L[lev + 1];
        N.A = std::move(A1);
        N.D = std::move(D1);
        N.An = std::move(An1);
        N.X = std::move(X1);
        Section sec_t(prof, "setup_Dt_ge1", s);
        SPHC_TRY(transpose(N.D, N.Dt, s));
        ++lev;
    }
    H.nlev = lev + 1;
    H.n_coarse = H.L[lev].A.nr;
    {
        Section sec(prof, "setup_coarse_inverse", s);
        SPHC_TRY(coarse_inverse(H.L[lev].A, H.coarse_inv, false, s));
        if (o.vcycle_fp32) {
            H.n_coarse_nodes = H.L[lev].An.nr;
            SPHC_TRY(coarse_inverse(H.L[lev].An, H.coarse_inv_n, true, s));
        }
    }
    {
        Section sec(prof, "setup_vcycle_ops", s);
        SPHC_TRY(build_vcycle_ops(H, s));
        if (o.autotune) SPHC_TRY(autotune_vcycle(H, s));
    }
    SPHC_CK(cudaStreamSynchronize(s));
    return SPHC_OK;
}

}  // namespace

extern "C" {

int sphc_default_opts(sphc_opts* o) {
    if (!o) return SPHC_EINVAL;
    memset(o, 0, sizeof(*o));
    o->max_levels = 8;
    o->emin_iters = 1;
    o->max_coarse = 1000;
    o->emin_omega = 0.5;
    o->seed = 0;
    o->power_iters = 15;
    o->vcycle_fp32 = 1;
    o->max_iter = 500;
    o->flexible = -1;
    o->profile = 0;
    o->cg_graph = 1;
    o->learned = 0;
    o->learned_emin_iters = 0;
    o->mlp_params = nullptr;
    o->autotune = 0;
    o->block_rhs = 1;
    o->alg1_passes = 2;
    return SPHC_OK;
}

int sphc_setup(const sphc_csr* A_e, const sphc_csr* D_h, const double* coords, const double* sigma_edge,
               const sphc_opts* opts, void* stream, sphc_handle** out) {
    if (!out || !A_e || !D_h) {
        set_error("sphc_setup: NULL argument");
        return SPHC_EINVAL;
    }
    *out = nullptr;
    sphc_handle* h = new (std::nothrow) sphc_handle();
    if (!h) {
        set_error("host allocation failed");
        return SPHC_ENOMEM;
    }
    if (opts) h->H.opts = *opts;
    else sphc_default_opts(&h->H.opts);
    sphc_opts& o = h->H.opts;
    if (o.flexible < 0) o.flexible = o.vcycle_fp32 ? 1 : 0;
    if (o.max_levels < 1 || o.max_levels > 32 || o.emin_iters < 0 || o.power_iters < 1 || o.max_iter < 1 ||
        !(o.emin_omega >= 0.0)) {
        set_error("sphc_setup: invalid options");
        delete h;
        return SPHC_EINVAL;
    }
    cudaGetDevice(&h->device);
    h->H.prof.on = o.profile != 0;
    cudaStream_t s = (cudaStream_t)stream;
    auto t0 = std::chrono::steady_clock::now();
    int64_t used0 = pool_used();
    int rc = setup_impl(h, A_e, D_h, coords, sigma_edge, s);
    if (rc != SPHC_OK) {
        cudaStreamSynchronize(s);
        sphc_destroy(h);
        return rc;
    }
    h->H.setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    cudaStreamSynchronize(s);                 // frees of setup temporaries have completed
    h->device_bytes = pool_used() - used0;
    *out = h;
    return SPHC_OK;
}

int sphc_setup_update(sphc_handle* h, const double* A_values, void* stream) {
    if (!h || !A_values) {
        set_error("sphc_setup_update: NULL argument");
        return SPHC_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    Hierarchy& H = h->H;
    const sphc_opts& o = H.opts;
    if (o.sa_theta > 0.0) {
        set_error("sphc_setup_update: the strength graph of a drop tolerance theta > 0 depends on the values, so the "
                  "aggregates cannot be kept; set up the new system instead");
        return SPHC_EINVAL;
    }
    auto t0 = std::chrono::steady_clock::now();
    Level& L0 = H.L[0];
    if (L0.A.nnz > 0) SPHC_CK(cudaMemcpyAsync(L0.A.v.p, A_values, sizeof(double) * L0.A.nnz, cudaMemcpyDefault, s));
    SPHC_TRY(validate(L0.A, 0, "A_e", s));
    Profiler* prof = H.prof.on ? &H.prof : nullptr;
    {
        Section sec(prof, "update_nodal_op", s);
        SPHC_TRY(amul_d(L0.A, L0.D, L0.AD, s));
        SPHC_TRY(spgemm_sym(L0.Dt, L0.AD, L0.An, s));
    }
    for (int lev = 0; lev + 1 < H.nlev; ++lev) {
        Level& L = H.L[lev];
        DCSR A1, D1, An1;
        DBuf<double> X1;
        Section sec(prof, "update_levels", s);
        SPHC_TRY(build_level(L, lev, o, A1, D1, An1, X1, H.mlp.p, prof, s, true));
        H.L[lev + 1].A = std::move(A1);
        H.L[lev + 1].An = std::move(An1);
    }
    {
        Section sec(prof, "update_coarse_inverse", s);
        const int lev = H.nlev - 1;
        SPHC_TRY(coarse_inverse(H.L[lev].A, H.coarse_inv, false, s));
        if (o.vcycle_fp32) SPHC_TRY(coarse_inverse(H.L[lev].An, H.coarse_inv_n, true, s));
    }
    // the V-cycle copies are rebuilt; the captured CG graphs refer to the old buffers
    SPHC_CK(cudaStreamSynchronize(s));
    if (H.cg_exec) cudaGraphExecDestroy(H.cg_exec);
    if (H.cg_graph) cudaGraphDestroy(H.cg_graph);
    H.cg_exec = nullptr;
    H.cg_graph = nullptr;
    H.blk.reset();
    {
        Section sec(prof, "update_vcycle_ops", s);
        SPHC_TRY(build_vcycle_ops(H, s));
        if (o.autotune) SPHC_TRY(autotune_vcycle(H, s));
    }
    SPHC_CK(cudaStreamSynchronize(s));
    H.setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return SPHC_OK;
}

int sphc_solve(sphc_handle* h, const double* b, double* x, int nrhs, double tol, void* stream, int* iters,
               double* relres) {
    if (!h || !b || !x || nrhs < 1 || !(tol > 0.0)) {
        set_error("sphc_solve: invalid argument");
        return SPHC_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    Hierarchy& H = h->H;
    int64_t n = H.L[0].A.nr;
    bool bdev = is_device_ptr(b), xdev = is_device_ptr(x);
    DBuf<double> bb, xb;
    auto t0 = std::chrono::steady_clock::now();
    if (nrhs >= 2 && H.opts.block_rhs) {
        // blocks of up to 16 right-hand sides, each one CG per column sharing the operator reads
        constexpr int BMAX = 16;
        const int64_t cap = (int64_t)(nrhs < BMAX ? nrhs : BMAX) * n;
        if (!bdev) SPHC_TRY(bb.alloc(cap, s));
        if (!xdev) SPHC_TRY(xb.alloc(cap, s));
        std::vector<int> it(nrhs, 0);
        std::vector<double> rr(nrhs, 0.0);
        int status = SPHC_OK;
        for (int k0 = 0; k0 < nrhs; k0 += BMAX) {
            const int m = nrhs - k0 < BMAX ? nrhs - k0 : BMAX;
            const double* bd = b + (int64_t)k0 * n;
            double* xd = x + (int64_t)k0 * n;
            if (!bdev) {
                SPHC_CK(cudaMemcpyAsync(bb.p, bd, sizeof(double) * n * m, cudaMemcpyDefault, s));
                bd = bb.p;
            }
            int rc = pcg_block(H, bd, xdev ? xd : xb.p, m, tol, s, it.data() + k0, rr.data() + k0);
            if (!xdev) SPHC_CK(cudaMemcpyAsync(xd, xb.p, sizeof(double) * n * m, cudaMemcpyDefault, s));
            if (rc != SPHC_OK && status == SPHC_OK) status = rc;
            if (rc == SPHC_ECUDA || rc == SPHC_ENOMEM) break;
        }
        SPHC_CK(cudaStreamSynchronize(s));
        for (int k = 0; k < nrhs; ++k) {
            if (iters) iters[k] = it[k];
            if (relres) relres[k] = rr[k];
        }
        H.last_iters = it[0];
        H.last_relres = rr[0];
        H.solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        return status;
    }
    if (!bdev) SPHC_TRY(bb.alloc(n, s));
    if (!xdev) SPHC_TRY(xb.alloc(n, s));
    int status = SPHC_OK;
    for (int k = 0; k < nrhs; ++k) {
        const double* bk = b + (int64_t)k * n;
        double* xk = x + (int64_t)k * n;
        const double* bd = bk;
        double* xd = xk;
        if (!bdev) {
            SPHC_CK(cudaMemcpyAsync(bb.p, bk, sizeof(double) * n, cudaMemcpyDefault, s));
            bd = bb.p;
        }
        if (!xdev) xd = xb.p;
        int it = 0;
        double rr = 0.0;
        int rc = pcg_solve(H, bd, xd, tol, s, &it, &rr);
        if (!xdev) {
            SPHC_CK(cudaMemcpyAsync(xk, xb.p, sizeof(double) * n, cudaMemcpyDefault, s));
        }
        if (iters) iters[k] = it;
        if (relres) relres[k] = rr;
        if (k == 0) { H.last_iters = it; H.last_relres = rr; }
        if (rc != SPHC_OK && status == SPHC_OK) status = rc;
        if (rc == SPHC_ECUDA || rc == SPHC_ENOMEM) break;
    }
    SPHC_CK(cudaStreamSynchronize(s));
    H.solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return status;
}

int sphc_vcycle(sphc_handle* h, const double* r, double* z, void* stream) {
    if (!h || !r || !z) {
        set_error("sphc_vcycle: NULL argument");
        return SPHC_EINVAL;
    }
    if (!is_device_ptr(r) || !is_device_ptr(z)) {
        set_error("sphc_vcycle: r and z must be device pointers");
        return SPHC_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    SPHC_TRY(apply_vcycle_user(h->H, r, z, s));
    SPHC_CK(cudaStreamSynchronize(s));
    return SPHC_OK;
}

int sphc_grid_barrier_check(int extra_arrivals, int polls, int* timed_out, void* stream) {
    if (extra_arrivals < 0 || polls < 0 || !timed_out) {
        set_error("sphc_grid_barrier_check: invalid argument");
        return SPHC_EINVAL;
    }
    *timed_out = 0;
    return grid_barrier_check(extra_arrivals, polls > 0 ? (unsigned)polls : GRID_BAR_POLLS, timed_out,
                              (cudaStream_t)stream);
}

int sphc_get_stats(const sphc_handle* h, sphc_stats* st) {
    if (!h || !st) return SPHC_EINVAL;
    const Hierarchy& H = h->H;
    memset(st, 0, sizeof(*st));
    st->n_levels = H.nlev;
    double tot = 0.0;
    for (int l = 0; l < H.nlev; ++l) tot += (double)H.L[l].A.nnz;
    st->operator_complexity = H.L[0].A.nnz > 0 ? tot / (double)H.L[0].A.nnz : 0.0;
    st->setup_ms = H.setup_ms;
    st->solve_ms = H.solve_ms;
    st->last_iters = H.last_iters;
    st->last_relres = H.last_relres;
    st->device_bytes = h->device_bytes;
    return SPHC_OK;
}

int sphc_get_level_info(const sphc_handle* h, int level, sphc_level_info* info) {
    if (!h || !info || level < 0 || level >= h->H.nlev) {
        set_error("sphc_get_level_info: invalid level");
        return SPHC_EINVAL;
    }
    const Level& L = h->H.L[level];
    memset(info, 0, sizeof(*info));
    info->n_edges = L.A.nr;
    info->n_nodes = L.An.nr;
    info->nnz_A = L.A.nnz;
    info->nnz_An = L.An.nnz;
    info->n_colors_edge = L.ncol_e;
    info->n_colors_node = L.ncol_n;
    info->colour_rounds_edge = L.rounds_e;
    info->colour_rounds_node = L.rounds_n;
    if (L.has_transfer) {
        info->n_aggregates = L.nagg;
        info->n_coarse_edges = L.DH.nr;
        info->nnz_Pn = L.Pn.nnz;
        info->nnz_Pe = L.Pe.nnz;
        info->nnz_T = L.T.nnz;
        info->n_added_edges = L.n_added;
        info->n_rows_unsmoothed = L.n_rows_unsmoothed;
        info->rho = L.rho;
        info->omega_sa = L.omega_sa;
        info->max_pattern_row = L.max_np;
        info->max_T_row = L.max_m;
    }
    const Hierarchy& H = h->H;
    auto shape = [&](const auto& V) {
        if (level >= (int)V.size()) return;
        info->sell_lpr_edge = V[level].A.m.lpr * (V[level].A.m.nslice > 0);
        info->sell_ch_edge = V[level].A.m.ch * (V[level].A.m.nslice > 0);
        info->sell_stored_edge = V[level].A.m.stored;
        info->sell_lpr_node = V[level].An.m.lpr * (V[level].An.m.nslice > 0);
        info->sell_ch_node = V[level].An.m.ch * (V[level].An.m.nslice > 0);
        info->sell_stored_node = V[level].An.m.stored;
        info->sweep_kind_edge = sweep_kind(V[level].A);
        info->sweep_kind_node = sweep_kind(V[level].An);
    };
    if (H.opts.vcycle_fp32) shape(H.V32); else shape(H.V64);
    return SPHC_OK;
}

static const DCSR* export_csr(const Level& L, int what) {
    switch (what) {
        case SPHC_X_A: return &L.A;
        case SPHC_X_D: return &L.D;
        case SPHC_X_AN: return &L.An;
        case SPHC_X_PN: return L.has_transfer ? &L.Pn : nullptr;
        case SPHC_X_DH: return L.has_transfer ? &L.DH : nullptr;
        case SPHC_X_T: return L.has_transfer ? &L.T : nullptr;
        case SPHC_X_PE: return L.has_transfer ? &L.Pe : nullptr;
        case SPHC_X_P0: return L.has_transfer ? &L.P0 : nullptr;
    }
    return nullptr;
}
static const DBuf<int32_t>* export_vec(const Level& L, int what, int64_t* len) {
    switch (what) {
        case SPHC_X_AGG: *len = L.An.nr; return L.has_transfer ? &L.agg : nullptr;
        case SPHC_X_COLE: *len = L.A.nr; return &L.col_e;
        case SPHC_X_COLN: *len = L.An.nr; return &L.col_n;
    }
    return nullptr;
}

int sphc_export_size(const sphc_handle* h, int level, int what, int64_t* nrows, int64_t* ncols, int64_t* nnz) {
    if (!h || level < 0 || level >= h->H.nlev) {
        set_error("sphc_export_size: invalid level");
        return SPHC_EINVAL;
    }
    const Level& L = h->H.L[level];
    if (const DCSR* M = export_csr(L, what)) {
        if (nrows) *nrows = M->nr;
        if (ncols) *ncols = M->nc;
        if (nnz) *nnz = M->nnz;
        return SPHC_OK;
    }
    int64_t len = 0;
    if (export_vec(L, what, &len)) {
        if (nrows) *nrows = len;
        if (ncols) *ncols = 1;
        if (nnz) *nnz = len;
        return SPHC_OK;
    }
    set_error("sphc_export_size: array %d not present on level %d", what, level);
    return SPHC_EINVAL;
}

int sphc_export(const sphc_handle* h, int level, int what, int64_t* rowptr, int32_t* col, double* val, int32_t* ivec,
                void* stream) {
    if (!h || level < 0 || level >= h->H.nlev) {
        set_error("sphc_export: invalid level");
        return SPHC_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const Level& L = h->H.L[level];
    if (const DCSR* M = export_csr(L, what)) {
        if (rowptr) SPHC_CK(cudaMemcpyAsync(rowptr, M->rp.p, sizeof(int64_t) * (M->nr + 1), cudaMemcpyDefault, s));
        if (col && M->nnz) SPHC_CK(cudaMemcpyAsync(col, M->ci.p, sizeof(int32_t) * M->nnz, cudaMemcpyDefault, s));
        if (val && M->nnz) SPHC_CK(cudaMemcpyAsync(val, M->v.p, sizeof(double) * M->nnz, cudaMemcpyDefault, s));
        SPHC_CK(cudaStreamSynchronize(s));
        return SPHC_OK;
    }
    int64_t len = 0;
    if (const DBuf<int32_t>* v = export_vec(L, what, &len)) {
        if (ivec && len) SPHC_CK(cudaMemcpyAsync(ivec, v->p, sizeof(int32_t) * len, cudaMemcpyDefault, s));
        SPHC_CK(cudaStreamSynchronize(s));
        return SPHC_OK;
    }
    set_error("sphc_export: array %d not present on level %d", what, level);
    return SPHC_EINVAL;
}

void sphc_destroy(sphc_handle* h) {
    if (!h) return;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaSetDevice(h->device);
    cudaDeviceSynchronize();
    g_sync_free = true;
    delete h;
    g_sync_free = false;
    cudaSetDevice(dev);
}

int sphc_trim_memory(int device, uint64_t keep_bytes) {
    int dev = 0;
    SPHC_CK(cudaGetDevice(&dev));
    if (device != dev) SPHC_CK(cudaSetDevice(device));
    cudaMemPool_t pool = device_pool();
    cudaError_t e = pool ? cudaMemPoolTrimTo(pool, (size_t)keep_bytes) : cudaErrorInvalidValue;
    if (device != dev) cudaSetDevice(dev);
    if (!pool) {
        set_error("sphc_trim_memory: no memory pool on device %d", device);
        return SPHC_EINVAL;
    }
    if (e != cudaSuccess) {
        set_error("sphc_trim_memory: %s", cudaGetErrorString(e));
        return SPHC_ECUDA;
    }
    return SPHC_OK;
}

int sphc_get_profile(sphc_handle* h, sphc_timer* out, int max, int* n) {
    if (!h || (max > 0 && !out) || !n) {
        set_error("sphc_get_profile: invalid argument");
        return SPHC_EINVAL;
    }
    Profiler& P = h->H.prof;
    P.resolve();
    *n = (int)P.timers.size();
    for (int i = 0; i < max && i < (int)P.timers.size(); ++i) {
        memset(&out[i], 0, sizeof(sphc_timer));
        strncpy(out[i].name, P.timers[i].name.c_str(), sizeof(out[i].name) - 1);
        out[i].ms = P.timers[i].ms;
        out[i].calls = P.timers[i].calls;
        out[i].bytes_per_call = P.timers[i].bytes;
    }
    return SPHC_OK;
}

int64_t sphc_launch_count(void) { return (int64_t)g_launches.load(); }

int sphc_memory_usage(int device, int64_t* used, int64_t* reserved) {
    int dev = 0;
    SPHC_CK(cudaGetDevice(&dev));
    if (device != dev) SPHC_CK(cudaSetDevice(device));
    cudaMemPool_t pool = device_pool();
    uint64_t u = 0, r = 0;
    cudaError_t e = cudaSuccess;
    if (pool) {
        e = cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &u);
        if (e == cudaSuccess) e = cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &r);
    }
    if (device != dev) cudaSetDevice(dev);
    if (!pool) {
        set_error("sphc_memory_usage: no memory pool on device %d", device);
        return SPHC_EINVAL;
    }
    if (e != cudaSuccess) {
        set_error("sphc_memory_usage: %s", cudaGetErrorString(e));
        return SPHC_ECUDA;
    }
    if (used) *used = (int64_t)u;
    if (reserved) *reserved = (int64_t)r;
    return SPHC_OK;
}

}  // extern "C"

struct sphc_batch {
    std::vector<sphc_handle*> hs;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    cudaStream_t cs = nullptr;
    std::vector<cudaStream_t> bs;
    std::vector<cudaEvent_t> ev;
    // streams the systems were set up on (their buffers were allocated stream-ordered there, so
    // the streams live as long as the handles)
    std::vector<cudaStream_t> ws;
};

static void batch_free(sphc_batch* B) {
    if (!B) return;
    if (B->ge) cudaGraphExecDestroy(B->ge);
    if (B->g) cudaGraphDestroy(B->g);
    for (auto e : B->ev) cudaEventDestroy(e);
    for (auto st : B->bs) cudaStreamDestroy(st);
    if (B->cs) cudaStreamDestroy(B->cs);
    for (auto h : B->hs) sphc_destroy(h);
    for (auto st : B->ws) cudaStreamDestroy(st);
    delete B;
}

static int batch_capture(sphc_batch* B) {
    int n = (int)B->hs.size();
    SPHC_CK(cudaStreamCreateWithFlags(&B->cs, cudaStreamNonBlocking));
    B->bs.resize(n);
    B->ev.resize(n + 1);
    for (int k = 0; k < n; ++k) SPHC_CK(cudaStreamCreateWithFlags(&B->bs[k], cudaStreamNonBlocking));
    for (int k = 0; k <= n; ++k) SPHC_CK(cudaEventCreateWithFlags(&B->ev[k], cudaEventDisableTiming));
    SPHC_CK(cudaStreamBeginCapture(B->cs, cudaStreamCaptureModeThreadLocal));
    cudaEventRecord(B->ev[n], B->cs);
    int rc = SPHC_OK;
    for (int k = 0; k < n && rc == SPHC_OK; ++k) {
        cudaStreamWaitEvent(B->bs[k], B->ev[n], 0);
        rc = capture_cg(B->hs[k]->H, B->bs[k]);
        cudaEventRecord(B->ev[k], B->bs[k]);
        cudaStreamWaitEvent(B->cs, B->ev[k], 0);
    }
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(B->cs, &g);
    if (rc != SPHC_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) {
        set_error("batched CG capture failed: %s", cudaGetErrorString(e));
        return SPHC_ECUDA;
    }
    B->g = g;
    SPHC_CK(cudaGraphInstantiate(&B->ge, B->g, 0));
    return SPHC_OK;
}

extern "C" {

int sphc_setup_batched(int nsys, const sphc_csr* A_e, const sphc_csr* D_h, const double* const* coords,
                       const double* const* sigma_edge, const sphc_opts* opts, void* stream, sphc_batch** out) {
    if (nsys < 1 || !A_e || !D_h || !out) {
        set_error("sphc_setup_batched: invalid argument");
        return SPHC_EINVAL;
    }
    *out = nullptr;
    sphc_batch* B = new (std::nothrow) sphc_batch();
    if (!B) return SPHC_ENOMEM;
    // The systems are set up concurrently by up to BATCH_WORKERS host threads, each on its own
    // stream, largest systems first: a small system's setup is a chain of short kernels and host
    // synchronisations that leaves most of the GPU idle.  Inputs the caller produced on `stream`
    // are complete before any worker reads them.
    constexpr int BATCH_WORKERS = 8;
    SPHC_CK(cudaStreamSynchronize((cudaStream_t)stream));
    int dev = 0;
    SPHC_CK(cudaGetDevice(&dev));
    const int nw = nsys < BATCH_WORKERS ? nsys : BATCH_WORKERS;
    B->hs.assign(nsys, nullptr);
    B->ws.assign(nw, nullptr);
    for (int w = 0; w < nw; ++w) {
        cudaError_t e = cudaStreamCreateWithFlags(&B->ws[w], cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            batch_free(B);
            set_error("sphc_setup_batched: cudaStreamCreate: %s", cudaGetErrorString(e));
            return SPHC_ECUDA;
        }
    }
    std::vector<int> order(nsys);
    for (int k = 0; k < nsys; ++k) order[k] = k;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return A_e[a].nrows > A_e[b].nrows; });
    std::vector<int> rcs(nsys, SPHC_OK);
    std::vector<std::string> msgs(nsys);
    std::atomic<int> next{0};
    auto work = [&](int w) {
        cudaSetDevice(dev);
        for (;;) {
            const int q = next.fetch_add(1);
            if (q >= nsys) break;
            const int k = order[q];
            rcs[k] = sphc_setup(&A_e[k], &D_h[k], coords ? coords[k] : nullptr, sigma_edge ? sigma_edge[k] : nullptr,
                                opts, B->ws[w], &B->hs[k]);
            if (rcs[k] != SPHC_OK) msgs[k] = last_error();
        }
    };
    std::vector<std::thread> threads;
    for (int w = 1; w < nw; ++w) threads.emplace_back(work, w);
    work(0);
    for (auto& t : threads) t.join();
    for (int k = 0; k < nsys; ++k)
        if (rcs[k] != SPHC_OK) {
            const int rc = rcs[k];
            batch_free(B);
            set_error("system %d: %s", k, msgs[k].c_str());
            return rc;
        }
    int rc = batch_capture(B);
    if (rc != SPHC_OK) {
        batch_free(B);
        return rc;
    }
    *out = B;
    return SPHC_OK;
}

int sphc_solve_batched(sphc_batch* B, const double* const* b, double* const* x, int nrhs, double tol, void* stream,
                       int* iters, double* relres) {
    if (!B || !b || !x || nrhs < 1 || !(tol > 0.0)) {
        set_error("sphc_solve_batched: invalid argument");
        return SPHC_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    int n = (int)B->hs.size();
    double tol2 = tol * tol;
    std::vector<int> hit(2 * n);
    std::vector<double> hsc(2 * n);
    int status = SPHC_OK;
    for (int r = 0; r < nrhs; ++r) {
        for (int k = 0; k < n; ++k) {
            Hierarchy& H = B->hs[k]->H;
            int64_t m = H.L[0].A.nr;
            SPHC_CK(cudaMemcpyAsync(H.bin.p, b[k] + (int64_t)r * m, sizeof(double) * m, cudaMemcpyDefault, s));
            SPHC_CK(cudaMemcpyAsync(H.scal.p + 8, &tol2, sizeof(double), cudaMemcpyHostToDevice, s));
        }
        SPHC_CK(cudaGraphLaunch(B->ge, s));
        for (int k = 0; k < n; ++k) {
            Hierarchy& H = B->hs[k]->H;
            int64_t m = H.L[0].A.nr;
            SPHC_CK(cudaMemcpyAsync(x[k] + (int64_t)r * m, H.xo.p, sizeof(double) * m, cudaMemcpyDefault, s));
            SPHC_CK(cudaMemcpyAsync(&hit[2 * k], H.itc.p, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
            SPHC_CK(cudaMemcpyAsync(&hsc[2 * k], H.scal.p + 5, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
        }
        SPHC_CK(cudaStreamSynchronize(s));
        for (int k = 0; k < n; ++k) {
            Hierarchy& H = B->hs[k]->H;
            int it = hit[2 * k], st = hit[2 * k + 1];
            g_launches.fetch_add(H.branch_launches + H.body_launches * (long long)it);
            double rel = hsc[2 * k] == 0.0 ? 0.0 : sqrt(hsc[2 * k + 1]) / sqrt(hsc[2 * k]);
            if (iters) iters[(int64_t)k * nrhs + r] = it;
            if (relres) relres[(int64_t)k * nrhs + r] = rel;
            int rc = st == 0 ? SPHC_OK
                             : (st == 1 ? SPHC_EBREAKDOWN : (st == 4 ? SPHC_ESTAGNATION : SPHC_ENOTCONV));
            if (rc != SPHC_OK && status == SPHC_OK) {
                status = rc;
                set_error("system %d, right side %d: %s after %d iterations", k, r,
                          rc == SPHC_EBREAKDOWN ? "CG breakdown"
                                                : (rc == SPHC_ESTAGNATION ? "CG stagnation" : "no convergence"),
                          it);
            }
        }
    }
    return status;
}

void sphc_batch_destroy(sphc_batch* B) {
    if (!B) return;
    cudaDeviceSynchronize();
    batch_free(B);
}

__global__ void k_target(const double* pe, const double* p0, int64_t n, float* y) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < n) y[q] = (float)(pe[q] - p0[q]);
}

int sphc_export_features(const sphc_handle* h, int level, float* X, float* y, void* stream) {
    if (!h || level < 0 || level + 1 >= h->H.nlev || !h->H.L[level].has_transfer) {
        set_error("sphc_export_features: level %d has no prolongator", level);
        return SPHC_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const Level& L = h->H.L[level];
    int64_t nnz = L.P0.nnz;
    DBuf<float> F, Y;
    if (X) {
        SPHC_TRY(F.alloc(nnz * SPHC_MLP_NFEAT, s));
        SPHC_TRY(level_features(L, h->H.L[level + 1].X, level, F.p, s));
        SPHC_CK(cudaMemcpyAsync(X, F.p, sizeof(float) * nnz * SPHC_MLP_NFEAT, cudaMemcpyDefault, s));
    }
    if (y) {
        SPHC_TRY(Y.alloc(nnz, s));
        if (nnz > 0) SPHC_LAUNCH(k_target<<<grid_for(nnz, 256), 256, 0, s>>>(L.Pe.v.p, L.P0.v.p, nnz, Y.p));
        SPHC_CK(cudaMemcpyAsync(y, Y.p, sizeof(float) * nnz, cudaMemcpyDefault, s));
    }
    SPHC_CK(cudaStreamSynchronize(s));
    return SPHC_OK;
}

int sphc_mlp_predict_level(const sphc_handle* h, int level, const float* params, float* out, void* stream) {
    if (!h || !params || !out || level < 0 || level + 1 >= h->H.nlev || !h->H.L[level].has_transfer) {
        set_error("sphc_mlp_predict_level: invalid argument or level %d has no prolongator", level);
        return SPHC_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const Level& L = h->H.L[level];
    int64_t nnz = L.P0.nnz;
    DBuf<float> P, Y;
    SPHC_TRY(P.alloc(SPHC_MLP_NPARAM, s));
    SPHC_CK(cudaMemcpyAsync(P.p, params, sizeof(float) * SPHC_MLP_NPARAM, cudaMemcpyDefault, s));
    SPHC_TRY(Y.alloc(nnz, s));
    SPHC_TRY(level_prediction(L, h->H.L[level + 1].X, level, P.p, Y.p, s));
    if (nnz > 0) SPHC_CK(cudaMemcpyAsync(out, Y.p, sizeof(float) * nnz, cudaMemcpyDefault, s));
    SPHC_CK(cudaStreamSynchronize(s));
    return SPHC_OK;
}

const char* sphc_last_error(void) { return sphc::last_error(); }

}  // extern "C"
