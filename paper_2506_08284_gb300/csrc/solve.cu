// Solve phase: V-cycle with one pre- and one post symmetric Hiptmair sweep on every level but
// the coarsest, which is solved directly (Sec. 6.1), inside FP64 conjugate gradients with x0 = 0
// and the stopping test ||r|| <= tol ||b|| (Sec. 6.1).  The V-cycle runs in FP32 or FP64.
#include <chrono>
#include <cmath>
#include <cstring>

#include "sphc_level.cuh"

namespace sphc {

static constexpr int DOT_PARTS = 1024;

// ------------------------------------------------------------------ section timers
int Profiler::find(const char* name, double bytes) {
    for (size_t i = 0; i < timers.size(); ++i)
        if (timers[i].name == name) return (int)i;
    timers.emplace_back();
    timers.back().name = name;
    timers.back().bytes = bytes;
    return (int)timers.size() - 1;
}
void Profiler::begin(int id, cudaStream_t s) {
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, s);
    timers[id].pending.push_back({a, b});
}
void Profiler::end(int id, cudaStream_t s) {
    cudaEventRecord(timers[id].pending.back().second, s);
    timers[id].calls++;
}
int Profiler::resolve() {
    for (auto& t : timers) {
        for (auto& pr : t.pending) {
            float ms = 0.f;
            cudaEventSynchronize(pr.second);
            cudaEventElapsedTime(&ms, pr.first, pr.second);
            t.ms += ms;
            cudaEventDestroy(pr.first);
            cudaEventDestroy(pr.second);
        }
        t.pending.clear();
    }
    return SPHC_OK;
}
Profiler::~Profiler() {
    for (auto& t : timers)
        for (auto& pr : t.pending) {
            cudaEventDestroy(pr.first);
            cudaEventDestroy(pr.second);
        }
}

// ------------------------------------------------------------------ stable colour partition
static constexpr int PART_BLOCK = 1024;
static constexpr int PART_MAXC = 256;

__global__ void k_part_count(const int32_t* color, int64_t n, int ncolor, int32_t* table, int64_t nblocks) {
    __shared__ int32_t cnt[PART_MAXC];
    for (int c = threadIdx.x; c < ncolor; c += blockDim.x) cnt[c] = 0;
    __syncthreads();
    int64_t i = (int64_t)blockIdx.x * PART_BLOCK + threadIdx.x;
    if (i < n) atomicAdd(&cnt[color[i]], 1);
    __syncthreads();
    for (int c = threadIdx.x; c < ncolor; c += blockDim.x) table[(int64_t)c * nblocks + blockIdx.x] = cnt[c];
}
// rows keep their natural order inside a colour
__global__ void k_part_place(const int32_t* color, int64_t n, int ncolor, const int64_t* off, int64_t nblocks,
                             int32_t* perm) {
    __shared__ int32_t wcnt[PART_BLOCK / 32][PART_MAXC];
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int q = threadIdx.x; q < (PART_BLOCK / 32) * PART_MAXC; q += blockDim.x) (&wcnt[0][0])[q] = 0;
    __syncthreads();
    int64_t i = (int64_t)blockIdx.x * PART_BLOCK + threadIdx.x;
    int c = i < n ? color[i] : -1;
    unsigned m = __match_any_sync(0xffffffffu, c);
    int rank = __popc(m & ((1u << lane) - 1u));
    if (c >= 0 && rank == 0) wcnt[w][c] = __popc(m);
    __syncthreads();
    if (c >= 0) {
        int before = 0;
        for (int q = 0; q < w; ++q) before += wcnt[q][c];
        perm[off[(int64_t)c * nblocks + blockIdx.x] + before + rank] = (int32_t)i;
    }
}

static int colour_partition(const int32_t* color, int64_t n, int ncolor, DBuf<int32_t>& perm,
                            std::vector<int64_t>& cstart, cudaStream_t s) {
    if (ncolor > PART_MAXC) { set_error("too many colours (%d)", ncolor); return SPHC_ELIMIT; }
    SPHC_TRY(perm.alloc(n, s));
    int64_t nb = (n + PART_BLOCK - 1) / PART_BLOCK;
    if (nb < 1) nb = 1;
    DBuf<int32_t> table;
    DBuf<int64_t> table64, off;
    SPHC_TRY(table.alloc(ncolor * nb, s));
    SPHC_TRY(off.alloc(ncolor * nb + 1, s));
    if (n > 0) SPHC_LAUNCH(k_part_count<<<(unsigned)nb, PART_BLOCK, 0, s>>>(color, n, ncolor, table.p, nb));
    SPHC_TRY(table64.alloc(ncolor * nb, s));
    // widen to int64 for the scan
    {
        std::vector<int32_t> h(ncolor * nb);
        SPHC_CK(cudaMemcpyAsync(h.data(), table.p, sizeof(int32_t) * h.size(), cudaMemcpyDeviceToHost, s));
        SPHC_CK(cudaStreamSynchronize(s));
        std::vector<int64_t> o(ncolor * nb + 1);
        int64_t run = 0;
        cstart.assign(ncolor + 1, 0);
        for (int c = 0; c < ncolor; ++c) {
            cstart[c] = run;
            for (int64_t b = 0; b < nb; ++b) { o[c * nb + b] = run; run += h[c * nb + b]; }
        }
        cstart[ncolor] = run;
        o[ncolor * nb] = run;
        SPHC_CK(cudaMemcpyAsync(off.p, o.data(), sizeof(int64_t) * o.size(), cudaMemcpyHostToDevice, s));
        SPHC_CK(cudaStreamSynchronize(s));
    }
    if (n > 0) SPHC_LAUNCH(k_part_place<<<(unsigned)nb, PART_BLOCK, 0, s>>>(color, n, ncolor, off.p, nb, perm.p));
    SPHC_CK(cudaGetLastError());
    return SPHC_OK;
}

__global__ void k_perm_rowlen(const int64_t* rp, const int32_t* perm, int64_t n, int64_t* len) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) len[k] = rp[perm[k] + 1] - rp[perm[k]];
}
__global__ void k_rp_narrow(const int64_t* a, int32_t* b, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (int32_t)a[i];
}
template <typename T>
__global__ void k_perm_copy(const int64_t* rp, const int32_t* ci, const double* v, const int32_t* perm, int64_t n,
                            const int32_t* nrp, int32_t* nci, T* nv, T* dinv) {
    int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (k >= n) return;
    int64_t i = perm[k];
    int64_t b = rp[i], len = rp[i + 1] - b;
    int32_t o = nrp[k];
    for (int64_t q = lane; q < len; q += 32) {
        int32_t c = ci[b + q];
        nci[o + q] = c;
        nv[o + q] = (T)v[b + q];
        if (c == i) dinv[k] = (T)(1.0 / v[b + q]);
    }
}

template <typename T>
static int build_smooth_op(const DCSR& A, const int32_t* color, int ncolor, SmoothOp<T>& op, cudaStream_t s) {
    op.n = A.nr;
    op.nnz = A.nnz;
    op.ncolor = ncolor;
    if (A.nnz >= (1LL << 31)) { set_error("operator with %lld nonzeros exceeds int32 row pointers", (long long)A.nnz); return SPHC_ELIMIT; }
    SPHC_TRY(colour_partition(color, A.nr, ncolor, op.perm, op.cstart, s));
    SPHC_TRY(op.cstart_dev.alloc(ncolor + 1, s));
    SPHC_CK(cudaMemcpyAsync(op.cstart_dev.p, op.cstart.data(), sizeof(int64_t) * (ncolor + 1), cudaMemcpyHostToDevice, s));
    SPHC_CK(cudaStreamSynchronize(s));
    DBuf<int64_t> len, rp64;
    SPHC_TRY(len.alloc(A.nr + 1, s));
    SPHC_TRY(rp64.alloc(A.nr + 1, s));
    if (A.nr > 0) SPHC_LAUNCH(k_perm_rowlen<<<grid_for(A.nr, 256), 256, 0, s>>>(A.rp.p, op.perm.p, A.nr, len.p));
    SPHC_TRY(exclusive_scan_i64(len.p, rp64.p, A.nr, s, nullptr));
    SPHC_TRY(op.rp.alloc(A.nr + 1, s));
    SPHC_LAUNCH(k_rp_narrow<<<grid_for(A.nr + 1, 256), 256, 0, s>>>(rp64.p, op.rp.p, A.nr + 1));
    SPHC_TRY(op.ci.alloc(A.nnz, s));
    SPHC_TRY(op.v.alloc(A.nnz, s));
    SPHC_TRY(op.dinv.alloc(A.nr, s));
    if (A.nr > 0)
        SPHC_LAUNCH(k_perm_copy<T><<<grid_for(A.nr * 32, 256), 256, 0, s>>>(A.rp.p, A.ci.p, A.v.p, op.perm.p, A.nr, op.rp.p,
                                                                 op.ci.p, op.v.p, op.dinv.p));
    SPHC_CK(cudaGetLastError());
    return SPHC_OK;
}

template <typename T>
__global__ void k_csr_narrow(const int64_t* rp, const double* v, int64_t nr, int64_t nnz, int32_t* nrp, T* nv) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i <= nr) nrp[i] = (int32_t)rp[i];
    if (i < nnz) nv[i] = (T)v[i];
}
template <typename T>
static int build_vcsr(const DCSR& A, VCSR<T>& B, cudaStream_t s) {
    if (A.nnz >= (1LL << 31)) { set_error("transfer with %lld nonzeros exceeds int32 row pointers", (long long)A.nnz); return SPHC_ELIMIT; }
    B.nr = A.nr; B.nc = A.nc; B.nnz = A.nnz;
    SPHC_TRY(B.rp.alloc(A.nr + 1, s));
    SPHC_TRY(B.ci.alloc(A.nnz, s));
    SPHC_TRY(B.v.alloc(A.nnz, s));
    int64_t m = A.nnz > A.nr + 1 ? A.nnz : A.nr + 1;
    SPHC_LAUNCH(k_csr_narrow<T><<<grid_for(m, 256), 256, 0, s>>>(A.rp.p, A.v.p, A.nr, A.nnz, B.rp.p, B.v.p));
    if (A.nnz > 0) SPHC_CK(cudaMemcpyAsync(B.ci.p, A.ci.p, sizeof(int32_t) * A.nnz, cudaMemcpyDeviceToDevice, s));
    SPHC_CK(cudaGetLastError());
    return SPHC_OK;
}

__global__ void k_d_pairs(const int64_t* rp, const int32_t* ci, const double* v, int64_t ne, int2* D) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ne) return;
    int2 d = make_int2(-1, -1);
    for (int64_t k = rp[e]; k < rp[e + 1]; ++k) {
        if (v[k] < 0) d.x = ci[k]; else d.y = ci[k];
    }
    D[e] = d;
}
__global__ void k_dt_encode(const int64_t* rp, const int32_t* ci, const double* v, int64_t nv, int64_t nnz,
                            int32_t* nrp, int32_t* enc) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i <= nv) nrp[i] = (int32_t)rp[i];
    if (i < nnz) enc[i] = (ci[i] << 1) | (v[i] < 0 ? 1 : 0);
}

template <typename T>
static int build_vlevel(Hierarchy& H, int l, VLevel<T>& V, bool split, cudaStream_t s) {
    Level& L = H.L[l];
    int64_t ne = L.A.nr, nv = L.An.nr;
    SPHC_TRY(V.x.alloc(ne, s));
    SPHC_TRY(V.b.alloc(ne, s));
    SPHC_TRY(V.r.alloc(ne, s));
    if (split) {
        SPHC_TRY(V.c.alloc(nv, s));
        SPHC_TRY(V.dc.alloc(nv, s));
        SPHC_TRY(V.bp.alloc(ne, s));
        SPHC_TRY(V.D.alloc(ne, s));
        if (ne > 0) SPHC_LAUNCH(k_d_pairs<<<grid_for(ne, 256), 256, 0, s>>>(L.D.rp.p, L.D.ci.p, L.D.v.p, ne, V.D.p));
        SPHC_TRY(V.Dt_rp.alloc(nv + 1, s));
        SPHC_TRY(V.Dt_e.alloc(L.Dt.nnz, s));
        int64_t m0 = L.Dt.nnz > nv + 1 ? L.Dt.nnz : nv + 1;
        SPHC_LAUNCH(k_dt_encode<<<grid_for(m0, 256), 256, 0, s>>>(L.Dt.rp.p, L.Dt.ci.p, L.Dt.v.p, nv, L.Dt.nnz, V.Dt_rp.p, V.Dt_e.p));
    }
    if (l == H.nlev - 1) return SPHC_OK;
    if (split) {
        if (L.AD.nr != L.A.nr) SPHC_TRY(spgemm(L.A, L.D, L.AD, s));   // FP64: the curl-curl part cancels here
        SPHC_TRY(build_vcsr<T>(L.AD, V.AD, s));
        SPHC_TRY(build_vcsr<T>(L.Pn, V.Pn, s));
        L.AD = DCSR();
    }
    SPHC_TRY(build_smooth_op<T>(L.A, L.col_e.p, L.ncol_e, V.A, s));
    SPHC_TRY(build_smooth_op<T>(L.An, L.col_n.p, L.ncol_n, V.An, s));
    SPHC_TRY(V.g.alloc(nv, s));
    if (!split) {
        SPHC_TRY(V.c.alloc(nv, s));
        SPHC_TRY(V.D.alloc(ne, s));
        if (ne > 0) SPHC_LAUNCH(k_d_pairs<<<grid_for(ne, 256), 256, 0, s>>>(L.D.rp.p, L.D.ci.p, L.D.v.p, ne, V.D.p));
        SPHC_TRY(V.Dt_rp.alloc(nv + 1, s));
        SPHC_TRY(V.Dt_e.alloc(L.Dt.nnz, s));
        int64_t m = L.Dt.nnz > nv + 1 ? L.Dt.nnz : nv + 1;
        SPHC_LAUNCH(k_dt_encode<<<grid_for(m, 256), 256, 0, s>>>(L.Dt.rp.p, L.Dt.ci.p, L.Dt.v.p, nv, L.Dt.nnz, V.Dt_rp.p, V.Dt_e.p));
    }
    SPHC_TRY(build_vcsr<T>(L.Pe, V.Pe, s));
    SPHC_TRY(build_vcsr<T>(L.PeT, V.PeT, s));
    SPHC_CK(cudaGetLastError());
    return SPHC_OK;
}

int build_vcycle_ops(Hierarchy& H, cudaStream_t s) {
    if (H.opts.vcycle_fp32) {
        H.V32.clear();
        H.V32.resize(H.nlev);
        for (int l = 0; l < H.nlev; ++l) SPHC_TRY(build_vlevel<float>(H, l, H.V32[l], true, s));
    } else {
        H.V64.clear();
        H.V64.resize(H.nlev);
        for (int l = 0; l < H.nlev; ++l) SPHC_TRY(build_vlevel<double>(H, l, H.V64[l], false, s));
    }
    int64_t n0 = H.L[0].A.nr;
    SPHC_TRY(H.x.alloc(n0, s));
    SPHC_TRY(H.r.alloc(n0, s));
    SPHC_TRY(H.z.alloc(n0, s));
    SPHC_TRY(H.p.alloc(n0, s));
    SPHC_TRY(H.q.alloc(n0, s));
    SPHC_TRY(H.rold.alloc(n0, s));
    SPHC_TRY(H.scal.alloc(16, s));
    SPHC_TRY(H.cb.alloc(H.n_coarse, s));
    SPHC_TRY(H.cx.alloc(H.n_coarse, s));
    SPHC_TRY(H.cgn.alloc(H.n_coarse_nodes, s));
    SPHC_TRY(H.ccn.alloc(H.n_coarse_nodes, s));
    SPHC_TRY(H.dpart.alloc(DOT_PARTS, s));
    SPHC_TRY(H.itc.alloc(4, s));
    SPHC_TRY(H.bin.alloc(n0, s));

    return SPHC_OK;
}

// ------------------------------------------------------------------ dot products into persistent partials
__global__ void k_dot_part_b(const double* a, const double* b, int64_t n, double* part) {
    __shared__ double sw[32];
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        s += a[i] * b[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < (blockDim.x >> 5) ? sw[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) part[blockIdx.x] = s;
    }
}
__global__ void k_dot_final_b(const double* part, int np, double* out) {
    __shared__ double sw[32];
    double s = 0.0;
    for (int i = threadIdx.x; i < np; i += blockDim.x) s += part[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < (blockDim.x >> 5) ? sw[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) *out = s;
    }
}
static void dot_buf(Hierarchy& H, const double* a, const double* b, int64_t n, double* out, cudaStream_t s) {
    SPHC_LAUNCH(k_dot_part_b<<<DOT_PARTS, 256, 0, s>>>(a, b, n, H.dpart.p));
    SPHC_LAUNCH(k_dot_final_b<<<1, 1024, 0, s>>>(H.dpart.p, DOT_PARTS, out));
}

// ------------------------------------------------------------------ V-cycle kernels
template <typename T, int SUB>
__global__ void k_sgs_color(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci, const T* __restrict__ v,
                            const int32_t* __restrict__ perm, const T* __restrict__ dinv, int64_t k0, int64_t k1,
                            const T* __restrict__ b, T* x) {
    int64_t k = k0 + (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / SUB);
    int q = threadIdx.x & (SUB - 1);
    bool valid = k < k1;
    T sum = 0;
    if (valid)
        for (int32_t e = rp[k] + q; e < rp[k + 1]; e += SUB) sum += v[e] * x[ci[e]];
#pragma unroll
    for (int o = SUB / 2; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o, SUB);
    if (valid && q == 0) {
        int32_t i = perm[k];
        x[i] += (b[i] - sum) * dinv[k];
    }
}

template <typename T, int SUB>
__global__ void k_resid(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci, const T* __restrict__ v,
                        const int32_t* __restrict__ perm, int64_t n, const T* __restrict__ b, const T* __restrict__ x,
                        T* __restrict__ r) {
    int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / SUB;
    int q = threadIdx.x & (SUB - 1);
    bool valid = k < n;
    T sum = 0;
    if (valid)
        for (int32_t e = rp[k] + q; e < rp[k + 1]; e += SUB) sum += v[e] * x[ci[e]];
#pragma unroll
    for (int o = SUB / 2; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o, SUB);
    if (valid && q == 0) {
        int32_t i = perm[k];
        r[i] = b[i] - sum;
    }
}

template <typename T, int SUB>
__global__ void k_spmv_v(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci, const T* __restrict__ v,
                         int64_t n, const T* __restrict__ x, T* y, int accumulate, T alpha) {
    int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / SUB;
    int q = threadIdx.x & (SUB - 1);
    bool valid = i < n;
    T sum = 0;
    if (valid)
        for (int32_t e = rp[i] + q; e < rp[i + 1]; e += SUB) sum += v[e] * x[ci[e]];
#pragma unroll
    for (int o = SUB / 2; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o, SUB);
    if (valid && q == 0) y[i] = accumulate ? y[i] + alpha * sum : alpha * sum;
}

template <typename T>
__global__ void k_dt_gather(const int32_t* __restrict__ rp, const int32_t* __restrict__ enc, int64_t nv,
                            const T* __restrict__ r, T* __restrict__ g) {
    int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= nv) return;
    T s = 0;
    for (int32_t k = rp[u]; k < rp[u + 1]; ++k) {
        int32_t e = enc[k];
        T val = r[e >> 1];
        s += (e & 1) ? -val : val;
    }
    g[u] = s;
}
template <typename T>
__global__ void k_d_apply(const int2* __restrict__ D, int64_t ne, const T* __restrict__ c, T* __restrict__ x) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ne) return;
    int2 d = D[e];
    T v = 0;
    if (d.y >= 0) v += c[d.y];
    if (d.x >= 0) v -= c[d.x];
    x[e] += v;
}
template <typename T>
__global__ void k_zero(T* a, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = 0;
}
template <typename A, typename B>
__global__ void k_cast(const A* a, B* b, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (B)a[i];
}
// x = Ainv b on the coarsest level (FP64 arithmetic)
template <typename T>
__global__ void k_dense_solve(const double* __restrict__ Ainv, int64_t n, const T* __restrict__ b, T* __restrict__ x) {
    int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (i >= n) return;
    double s = 0.0;
    for (int64_t j = lane; j < n; j += 32) s += Ainv[i * n + j] * (double)b[j];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) x[i] = (T)s;
}

static int sub_for(int64_t nnz, int64_t n) {
    double avg = n > 0 ? (double)nnz / (double)n : 0.0;
    if (avg <= 6) return 4;
    if (avg <= 20) return 8;
    if (avg <= 48) return 16;
    return 32;
}

template <typename T>
static void launch_rows_sgs(const SmoothOp<T>& op, int64_t k0, int64_t k1, const T* b, T* x, cudaStream_t s) {
    int64_t rows = k1 - k0;
    if (rows <= 0) return;
    int sub = op.sub > 0 ? op.sub : sub_for(op.nnz, op.n);
    int64_t th = rows * sub;
    switch (sub) {
        case 4: SPHC_LAUNCH(k_sgs_color<T, 4><<<grid_for(th, 256), 256, 0, s>>>(op.rp.p, op.ci.p, op.v.p, op.perm.p, op.dinv.p, k0, k1, b, x)); break;
        case 8: SPHC_LAUNCH(k_sgs_color<T, 8><<<grid_for(th, 256), 256, 0, s>>>(op.rp.p, op.ci.p, op.v.p, op.perm.p, op.dinv.p, k0, k1, b, x)); break;
        case 16: SPHC_LAUNCH(k_sgs_color<T, 16><<<grid_for(th, 256), 256, 0, s>>>(op.rp.p, op.ci.p, op.v.p, op.perm.p, op.dinv.p, k0, k1, b, x)); break;
        default: SPHC_LAUNCH(k_sgs_color<T, 32><<<grid_for(th, 256), 256, 0, s>>>(op.rp.p, op.ci.p, op.v.p, op.perm.p, op.dinv.p, k0, k1, b, x)); break;
    }
}
// A whole forward + backward sweep of a small operator in one block: colours are separated by
// block barriers instead of kernel boundaries (the coarse levels are launch-bound otherwise).
static constexpr int SGS_BLOCK_MAX_ROWS = 2048;
template <typename T, int SUB>
__global__ void __launch_bounds__(1024)
k_sgs_block(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci, const T* __restrict__ v,
            const int32_t* __restrict__ perm, const T* __restrict__ dinv, const int64_t* __restrict__ cstart,
            int ncolor, const T* __restrict__ b, T* x) {
    int q = threadIdx.x & (SUB - 1);
    int slot = threadIdx.x / SUB, nslot = blockDim.x / SUB;
    for (int step = 0; step < 2 * ncolor; ++step) {
        int c = step < ncolor ? step : 2 * ncolor - 1 - step;
        int64_t k0 = cstart[c], k1 = cstart[c + 1];
        for (int64_t base = k0; base < k1; base += nslot) {
            int64_t k = base + slot;
            bool valid = k < k1;
            T sum = 0;
            if (valid)
                for (int32_t e = rp[k] + q; e < rp[k + 1]; e += SUB) sum += v[e] * x[ci[e]];
#pragma unroll
            for (int o = SUB / 2; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o, SUB);
            if (valid && q == 0) {
                int32_t i = perm[k];
                x[i] += (b[i] - sum) * dinv[k];
            }
        }
        __syncthreads();
    }
}

template <typename T>
static void sgs(const SmoothOp<T>& op, const T* b, T* x, cudaStream_t s) {
    if (op.n <= SGS_BLOCK_MAX_ROWS && op.cstart_dev.p) {
        int sub = sub_for(op.nnz, op.n);
        switch (sub) {
            case 4: SPHC_LAUNCH(k_sgs_block<T, 4><<<1, 1024, 0, s>>>(op.rp.p, op.ci.p, op.v.p, op.perm.p, op.dinv.p, op.cstart_dev.p, op.ncolor, b, x)); break;
            case 8: SPHC_LAUNCH(k_sgs_block<T, 8><<<1, 1024, 0, s>>>(op.rp.p, op.ci.p, op.v.p, op.perm.p, op.dinv.p, op.cstart_dev.p, op.ncolor, b, x)); break;
            case 16: SPHC_LAUNCH(k_sgs_block<T, 16><<<1, 1024, 0, s>>>(op.rp.p, op.ci.p, op.v.p, op.perm.p, op.dinv.p, op.cstart_dev.p, op.ncolor, b, x)); break;
            default: SPHC_LAUNCH(k_sgs_block<T, 32><<<1, 1024, 0, s>>>(op.rp.p, op.ci.p, op.v.p, op.perm.p, op.dinv.p, op.cstart_dev.p, op.ncolor, b, x)); break;
        }
        return;
    }
    for (int c = 0; c < op.ncolor; ++c) launch_rows_sgs(op, op.cstart[c], op.cstart[c + 1], b, x, s);
    for (int c = op.ncolor - 1; c >= 0; --c) launch_rows_sgs(op, op.cstart[c], op.cstart[c + 1], b, x, s);
}
template <typename T>
static void resid(const SmoothOp<T>& op, const T* b, const T* x, T* r, cudaStream_t s) {
    if (op.n == 0) return;
    int sub = op.sub > 0 ? op.sub : sub_for(op.nnz, op.n);
    int64_t th = op.n * sub;
    switch (sub) {
        case 4: SPHC_LAUNCH(k_resid<T, 4><<<grid_for(th, 256), 256, 0, s>>>(op.rp.p, op.ci.p, op.v.p, op.perm.p, op.n, b, x, r)); break;
        case 8: SPHC_LAUNCH(k_resid<T, 8><<<grid_for(th, 256), 256, 0, s>>>(op.rp.p, op.ci.p, op.v.p, op.perm.p, op.n, b, x, r)); break;
        case 16: SPHC_LAUNCH(k_resid<T, 16><<<grid_for(th, 256), 256, 0, s>>>(op.rp.p, op.ci.p, op.v.p, op.perm.p, op.n, b, x, r)); break;
        default: SPHC_LAUNCH(k_resid<T, 32><<<grid_for(th, 256), 256, 0, s>>>(op.rp.p, op.ci.p, op.v.p, op.perm.p, op.n, b, x, r)); break;
    }
}
template <typename T>
static void spmv_v(const VCSR<T>& A, const T* x, T* y, int acc, cudaStream_t s, T alpha = T(1)) {
    if (A.nr == 0) return;
    int sub = sub_for(A.nnz, A.nr);
    int64_t th = A.nr * sub;
    switch (sub) {
        case 4: SPHC_LAUNCH(k_spmv_v<T, 4><<<grid_for(th, 256), 256, 0, s>>>(A.rp.p, A.ci.p, A.v.p, A.nr, x, y, acc, alpha)); break;
        case 8: SPHC_LAUNCH(k_spmv_v<T, 8><<<grid_for(th, 256), 256, 0, s>>>(A.rp.p, A.ci.p, A.v.p, A.nr, x, y, acc, alpha)); break;
        case 16: SPHC_LAUNCH(k_spmv_v<T, 16><<<grid_for(th, 256), 256, 0, s>>>(A.rp.p, A.ci.p, A.v.p, A.nr, x, y, acc, alpha)); break;
        default: SPHC_LAUNCH(k_spmv_v<T, 32><<<grid_for(th, 256), 256, 0, s>>>(A.rp.p, A.ci.p, A.v.p, A.nr, x, y, acc, alpha)); break;
    }
}

// algorithmic bytes of one forward + backward sweep: the matrix once per direction and, per
// row, its pointer, permutation, inverse diagonal, right side and one read and write of x
template <typename T>
static double sgs_bytes(const SmoothOp<T>& op) {
    return 2.0 * ((double)op.nnz * (sizeof(T) + 4) + (double)op.n * (4 + 4 + 3 * sizeof(T) + sizeof(T)));
}

template <typename T>
static void timed_sgs(Hierarchy& H, int lev, const SmoothOp<T>& op, const T* b, T* x, cudaStream_t s) {
    int id = -1;
    if (H.prof.on && lev == 0 && !H.capturing) {
        id = H.prof.find("sgs_A_level0", sgs_bytes(op));
        H.prof.begin(id, s);
    }
    sgs(op, b, x, s);
    if (id >= 0) H.prof.end(id, s);
}

template <typename T>
static void hiptmair(Hierarchy& H, int lev, VLevel<T>& V, int64_t ne, int64_t nv, cudaStream_t s) {
    timed_sgs(H, lev, V.A, V.b.p, V.x.p, s);
    resid(V.A, V.b.p, V.x.p, V.r.p, s);
    if (nv > 0) {
        SPHC_LAUNCH(k_dt_gather<T><<<grid_for(nv, 256), 256, 0, s>>>(V.Dt_rp.p, V.Dt_e.p, nv, V.r.p, V.g.p));
        SPHC_LAUNCH(k_zero<T><<<grid_for(nv, 256), 256, 0, s>>>(V.c.p, nv));
        sgs(V.An, V.g.p, V.c.p, s);
        SPHC_LAUNCH(k_d_apply<T><<<grid_for(ne, 256), 256, 0, s>>>(V.D.p, ne, V.c.p, V.x.p));
    }
    timed_sgs(H, lev, V.A, V.b.p, V.x.p, s);
}

template <typename T>
static void vcycle_level(Hierarchy& H, std::vector<VLevel<T>>& V, int l, cudaStream_t s) {
    int64_t ne = H.L[l].A.nr, nv = H.L[l].An.nr;
    if (l == H.nlev - 1) {
        if (ne > 0) SPHC_LAUNCH(k_dense_solve<T><<<grid_for(ne * 32, 256), 256, 0, s>>>(H.coarse_inv.p, ne, V[l].b.p, V[l].x.p));
        return;
    }
    SPHC_LAUNCH(k_zero<T><<<grid_for(ne, 256), 256, 0, s>>>(V[l].x.p, ne));
    hiptmair(H, l, V[l], ne, nv, s);
    resid(V[l].A, V[l].b.p, V[l].x.p, V[l].r.p, s);
    spmv_v(V[l].PeT, V[l].r.p, V[l + 1].b.p, 0, s);
    vcycle_level(H, V, l + 1, s);
    spmv_v(V[l].Pe, V[l + 1].x.p, V[l].x.p, 1, s);
    hiptmair(H, l, V[l], ne, nv, s);
}

// ------------------------------------------------------------------ split V-cycle (FP32)
// The FP32 V-cycle keeps its iterate as x = y + D c.  Stored in FP32, the curl-curl part of A no
// longer annihilates gradients exactly (K D = O(eps32 |K|)), so a large gradient component of x
// would swamp the sigma-scale residual.  Here every gradient correction (the nodal step of the
// Hiptmair sweep and, through the commuting relation P_e D_H = D_h P_n, the gradient part of the
// coarse correction) is kept in the nodal potential c, and its effect on the residual is applied
// through A D, formed in FP64 (where K D cancels) and stored in FP32: b' = b - (A D) c.
template <typename T>
__global__ void k_axpy(T* y, const T* x, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] += x[i];
}
template <typename T>
__global__ void k_copy(T* y, const T* x, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = x[i];
}
// z = y + D c in FP64
template <typename T>
__global__ void k_combine(const T* __restrict__ y, const int2* __restrict__ D, const T* __restrict__ c, int64_t n,
                          double* __restrict__ z) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    int2 d = D[e];
    double v = (double)y[e];
    if (d.y >= 0) v += (double)c[d.y];
    if (d.x >= 0) v -= (double)c[d.x];
    z[e] = v;
}
__global__ void k_dense_mv64(const double* __restrict__ M, int64_t n, const double* __restrict__ b, double* __restrict__ x) {
    int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (i >= n) return;
    double s = 0.0;
    for (int64_t j = lane; j < n; j += 32) s += M[i * n + j] * b[j];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) x[i] = s;
}
// coarsest split: y = A^-1 b - D c, c = A_n^-1 D^T b (FP64), so that y is A-orthogonal to gradients
template <typename T>
__global__ void k_split_out(const double* __restrict__ xb, const int2* __restrict__ D, const double* __restrict__ cc,
                            int64_t ne, int64_t nv, T* __restrict__ y, T* __restrict__ c) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < ne) {
        int2 d = D[i];
        double g = 0.0;
        if (d.y >= 0) g += cc[d.y];
        if (d.x >= 0) g -= cc[d.x];
        y[i] = (T)(xb[i] - g);
    }
    if (i < nv) c[i] = (T)cc[i];
}

template <typename T>
static void coarse_split(Hierarchy& H, VLevel<T>& V, int64_t ne, int64_t nv, cudaStream_t s) {
    if (ne == 0) return;
    SPHC_LAUNCH(k_cast<T, double><<<grid_for(ne, 256), 256, 0, s>>>(V.b.p, H.cb.p, ne));
    SPHC_LAUNCH(k_dense_mv64<<<grid_for(ne * 32, 256), 256, 0, s>>>(H.coarse_inv.p, ne, H.cb.p, H.cx.p));
    if (nv > 0) {
        SPHC_LAUNCH(k_dt_gather<double><<<grid_for(nv, 256), 256, 0, s>>>(V.Dt_rp.p, V.Dt_e.p, nv, H.cb.p, H.cgn.p));
        SPHC_LAUNCH(k_dense_mv64<<<grid_for(nv * 32, 256), 256, 0, s>>>(H.coarse_inv_n.p, nv, H.cgn.p, H.ccn.p));
    }
    int64_t m = ne > nv ? ne : nv;
    SPHC_LAUNCH(k_split_out<T><<<grid_for(m, 256), 256, 0, s>>>(H.cx.p, V.D.p, H.ccn.p, ne, nv, V.x.p, V.c.p));
}

template <typename T>
static void hiptmair_split(Hierarchy& H, int lev, VLevel<T>& V, int64_t ne, int64_t nv, cudaStream_t s) {
    timed_sgs(H, lev, V.A, V.bp.p, V.x.p, s);
    if (nv > 0) {
        resid(V.A, V.bp.p, V.x.p, V.r.p, s);
        SPHC_LAUNCH(k_dt_gather<T><<<grid_for(nv, 256), 256, 0, s>>>(V.Dt_rp.p, V.Dt_e.p, nv, V.r.p, V.g.p));
        SPHC_LAUNCH(k_zero<T><<<grid_for(nv, 256), 256, 0, s>>>(V.dc.p, nv));
        sgs(V.An, V.g.p, V.dc.p, s);
        SPHC_LAUNCH(k_axpy<T><<<grid_for(nv, 256), 256, 0, s>>>(V.c.p, V.dc.p, nv));
        spmv_v(V.AD, V.dc.p, V.bp.p, 1, s, T(-1));
    }
    timed_sgs(H, lev, V.A, V.bp.p, V.x.p, s);
}

template <typename T>
static void vcycle_split(Hierarchy& H, std::vector<VLevel<T>>& V, int l, cudaStream_t s) {
    int64_t ne = H.L[l].A.nr, nv = H.L[l].An.nr;
    if (l == H.nlev - 1) {
        coarse_split(H, V[l], ne, nv, s);
        return;
    }
    SPHC_LAUNCH(k_zero<T><<<grid_for(ne, 256), 256, 0, s>>>(V[l].x.p, ne));
    if (nv > 0) SPHC_LAUNCH(k_zero<T><<<grid_for(nv, 256), 256, 0, s>>>(V[l].c.p, nv));
    SPHC_LAUNCH(k_copy<T><<<grid_for(ne, 256), 256, 0, s>>>(V[l].bp.p, V[l].b.p, ne));
    hiptmair_split(H, l, V[l], ne, nv, s);
    resid(V[l].A, V[l].bp.p, V[l].x.p, V[l].r.p, s);
    spmv_v(V[l].PeT, V[l].r.p, V[l + 1].b.p, 0, s);
    vcycle_split(H, V, l + 1, s);
    spmv_v(V[l].Pe, V[l + 1].x.p, V[l].x.p, 1, s);           // y += P_e y_H
    if (nv > 0) {
        spmv_v(V[l].Pn, V[l + 1].c.p, V[l].dc.p, 0, s);      // c += P_n c_H  (P_e D_H = D_h P_n)
        SPHC_LAUNCH(k_axpy<T><<<grid_for(nv, 256), 256, 0, s>>>(V[l].c.p, V[l].dc.p, nv));
        spmv_v(V[l].AD, V[l].dc.p, V[l].bp.p, 1, s, T(-1));
    }
    hiptmair_split(H, l, V[l], ne, nv, s);
}

int apply_vcycle(Hierarchy& H, const double* r, double* z, cudaStream_t s) {
    int64_t n = H.L[0].A.nr;
    if (H.opts.vcycle_fp32) {
        SPHC_LAUNCH(k_cast<double, float><<<grid_for(n, 256), 256, 0, s>>>(r, H.V32[0].b.p, n));
        vcycle_split<float>(H, H.V32, 0, s);
        SPHC_LAUNCH(k_combine<float><<<grid_for(n, 256), 256, 0, s>>>(H.V32[0].x.p, H.V32[0].D.p, H.V32[0].c.p, n, z));
    } else {
        SPHC_CK(cudaMemcpyAsync(H.V64[0].b.p, r, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
        vcycle_level<double>(H, H.V64, 0, s);
        SPHC_CK(cudaMemcpyAsync(z, H.V64[0].x.p, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    }
    SPHC_CK(cudaGetLastError());
    return SPHC_OK;
}

// Autotuner: time one forward + backward sweep for each lanes-per-row width and keep the fastest
// (the operators are stored in CSR with rows grouped by colour, so the tunable shape is the
// number of lanes that share a row).
template <typename T>
static int autotune_op(SmoothOp<T>& op, DBuf<T>& bvec, DBuf<T>& xvec, cudaStream_t s) {
    if (op.n <= SGS_BLOCK_MAX_ROWS || op.n > bvec.n || op.n > xvec.n) return SPHC_OK;
    cudaEvent_t e0, e1;
    SPHC_CK(cudaEventCreate(&e0));
    SPHC_CK(cudaEventCreate(&e1));
    SPHC_LAUNCH(k_zero<T><<<grid_for(op.n, 256), 256, 0, s>>>(bvec.p, op.n));
    float best = 1e30f;
    int best_sub = 0;
    for (int sub : {4, 8, 16, 32}) {
        op.sub = sub;
        sgs(op, bvec.p, xvec.p, s);                   // warm-up
        cudaEventRecord(e0, s);
        for (int rep = 0; rep < 3; ++rep) sgs(op, bvec.p, xvec.p, s);
        cudaEventRecord(e1, s);
        SPHC_CK(cudaEventSynchronize(e1));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) { best = ms; best_sub = sub; }
    }
    op.sub = best_sub;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return SPHC_OK;
}

int autotune_vcycle(Hierarchy& H, cudaStream_t s) {
    for (int l = 0; l + 1 < H.nlev; ++l) {
        if (H.opts.vcycle_fp32) {
            SPHC_TRY(autotune_op(H.V32[l].A, H.V32[l].b, H.V32[l].x, s));
            SPHC_TRY(autotune_op(H.V32[l].An, H.V32[l].g, H.V32[l].c, s));
        } else {
            SPHC_TRY(autotune_op(H.V64[l].A, H.V64[l].b, H.V64[l].x, s));
            SPHC_TRY(autotune_op(H.V64[l].An, H.V64[l].g, H.V64[l].c, s));
        }
    }
    return SPHC_OK;
}

// ------------------------------------------------------------------ CG
// scal: 0 rz, 1 pq, 2 rr, 3 rz_new, 4 z.r_old, 5 bb
__global__ void k_cg_xr(double* x, double* r, double* rold, const double* p, const double* q, const double* sc,
                        int64_t n, int flexible) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double alpha = sc[1] > 0.0 ? sc[0] / sc[1] : 0.0;     // breakdown: leave x unchanged
    x[i] += alpha * p[i];
    if (flexible) rold[i] = r[i];
    r[i] -= alpha * q[i];
}
__global__ void k_cg_p(double* p, const double* z, const double* sc, int64_t n, int flexible) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double beta = flexible ? (sc[3] - sc[4]) / sc[0] : sc[3] / sc[0];
    p[i] = z[i] + beta * p[i];
}
__global__ void k_cg_shift(double* sc) { sc[0] = sc[3]; }
__global__ void k_sub(const double* b, double* q, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) q[i] = b[i] - q[i];
}

// end of one graph iteration: count it and keep looping while not converged, not broken down
// and below the iteration cap.  itc[1]: 0 converged, 1 breakdown, 2 cap reached.
__global__ void k_cg_check(cudaGraphConditionalHandle hnd, const double* sc, int* itc, int max_iter) {
    int it = itc[0] + 1;
    itc[0] = it;
    double pq = sc[1], rr = sc[2], lim = sc[7];
    unsigned cont = 1;
    if (!(pq > 0.0) || !isfinite(rr)) { itc[1] = 1; cont = 0; }
    else if (rr <= lim) { itc[1] = 0; cont = 0; }
    else if (it >= max_iter) { itc[1] = 2; cont = 0; }
    cudaGraphSetConditional(hnd, cont);
}
__global__ void k_set_limit(double* sc, double tol2) { sc[7] = tol2 * sc[5]; }

// one CG iteration after the first: z = M^-1 r, p = z + beta p, q = A p, x += alpha p, r -= alpha q
static int cg_body(Hierarchy& H, cudaGraphConditionalHandle hnd, cudaStream_t s) {
    const DCSR& A = H.L[0].A;
    int64_t n = A.nr;
    int flexible = H.opts.flexible;
    double* sc = H.scal.p;
    SPHC_TRY(apply_vcycle(H, H.r.p, H.z.p, s));
    dot_buf(H, H.r.p, H.z.p, n, sc + 3, s);
    if (flexible) dot_buf(H, H.z.p, H.rold.p, n, sc + 4, s);
    SPHC_LAUNCH(k_cg_p<<<grid_for(n, 256), 256, 0, s>>>(H.p.p, H.z.p, sc, n, flexible));
    SPHC_LAUNCH(k_cg_shift<<<1, 1, 0, s>>>(sc));
    SPHC_TRY(spmv64(A, H.p.p, H.q.p, s));
    dot_buf(H, H.p.p, H.q.p, n, sc + 1, s);
    SPHC_LAUNCH(k_cg_xr<<<grid_for(n, 256), 256, 0, s>>>(H.x.p, H.r.p, H.rold.p, H.p.p, H.q.p, sc, n, flexible));
    dot_buf(H, H.r.p, H.r.p, n, sc + 2, s);
    SPHC_LAUNCH(k_cg_check<<<1, 1, 0, s>>>(hnd, sc, H.itc.p, H.opts.max_iter));
    SPHC_CK(cudaGetLastError());
    return SPHC_OK;
}

static int build_cg_graph(Hierarchy& H) {
    if (H.cg_exec) return SPHC_OK;
    if (!H.cap_stream) SPHC_CK(cudaStreamCreateWithFlags(&H.cap_stream, cudaStreamNonBlocking));
    SPHC_CK(cudaGraphCreate(&H.cg_graph, 0));
    cudaGraphConditionalHandle hnd;
    SPHC_CK(cudaGraphConditionalHandleCreate(&hnd, H.cg_graph, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = hnd;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    SPHC_CK(cudaGraphAddNode(&node, H.cg_graph, nullptr, nullptr, 0, &np));
    cudaGraph_t body = np.conditional.phGraph_out[0];
    SPHC_CK(cudaStreamBeginCaptureToGraph(H.cap_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    H.capturing = true;
    long long l0 = g_launches.load();
    int rc = cg_body(H, hnd, H.cap_stream);
    H.body_launches = g_launches.load() - l0;
    g_launches.fetch_sub(H.body_launches);      // counted when the graph runs, not when captured
    H.capturing = false;
    cudaGraph_t captured = nullptr;
    cudaError_t e = cudaStreamEndCapture(H.cap_stream, &captured);
    if (rc != SPHC_OK) return rc;
    if (e != cudaSuccess) {
        set_error("CG graph capture failed: %s", cudaGetErrorString(e));
        return SPHC_ECUDA;
    }
    SPHC_CK(cudaGraphInstantiate(&H.cg_exec, H.cg_graph, 0));
    return SPHC_OK;
}

// CG on the device: the first iteration is enqueued directly, the rest run inside one graph
// launch whose while node repeats an iteration until the stopping test holds.
static int pcg_graph(Hierarchy& H, const double* b, double* x, double tol, cudaStream_t s, int* iters,
                     double* relres) {
    const DCSR& A = H.L[0].A;
    int64_t n = A.nr;
    int flexible = H.opts.flexible;
    double* sc = H.scal.p;
    SPHC_TRY(build_cg_graph(H));
    SPHC_CK(cudaMemsetAsync(H.x.p, 0, sizeof(double) * n, s));
    SPHC_CK(cudaMemcpyAsync(H.r.p, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    dot_buf(H, b, b, n, sc + 5, s);
    double hb = 0.0;
    SPHC_CK(cudaMemcpyAsync(&hb, sc + 5, sizeof(double), cudaMemcpyDeviceToHost, s));
    SPHC_CK(cudaStreamSynchronize(s));
    double bnorm = sqrt(hb);
    int status = SPHC_OK, it = 0;
    if (bnorm > 0.0) {
        SPHC_TRY(apply_vcycle(H, H.r.p, H.z.p, s));
        SPHC_CK(cudaMemcpyAsync(H.p.p, H.z.p, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
        dot_buf(H, H.r.p, H.z.p, n, sc + 0, s);
        {
            Section sec(H.prof.on ? &H.prof : nullptr, "spmv_A_fp64", s, (double)A.nnz * 12.0 + (double)n * 24.0);
            SPHC_TRY(spmv64(A, H.p.p, H.q.p, s));
        }
        dot_buf(H, H.p.p, H.q.p, n, sc + 1, s);
        SPHC_LAUNCH(k_cg_xr<<<grid_for(n, 256), 256, 0, s>>>(H.x.p, H.r.p, H.rold.p, H.p.p, H.q.p, sc, n, flexible));
        dot_buf(H, H.r.p, H.r.p, n, sc + 2, s);
        SPHC_LAUNCH(k_set_limit<<<1, 1, 0, s>>>(sc, tol * tol));
        int hi[2] = {1, 0};
        SPHC_CK(cudaMemcpyAsync(H.itc.p, hi, 2 * sizeof(int), cudaMemcpyHostToDevice, s));
        double hsc[8];
        SPHC_CK(cudaMemcpyAsync(hsc, sc, 8 * sizeof(double), cudaMemcpyDeviceToHost, s));
        SPHC_CK(cudaStreamSynchronize(s));
        it = 1;
        if (!(hsc[1] > 0.0) || !std::isfinite(hsc[2])) status = SPHC_EBREAKDOWN;
        else if (hsc[2] <= hsc[7]) status = SPHC_OK;
        else if (it >= H.opts.max_iter) status = SPHC_ENOTCONV;
        else {
            SPHC_CK(cudaGraphLaunch(H.cg_exec, s));
            SPHC_CK(cudaMemcpyAsync(hi, H.itc.p, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
            SPHC_CK(cudaStreamSynchronize(s));
            it = hi[0];
            status = hi[1] == 0 ? SPHC_OK : (hi[1] == 1 ? SPHC_EBREAKDOWN : SPHC_ENOTCONV);
            g_launches.fetch_add(H.body_launches * (long long)(it - 1));
        }
    }
    SPHC_CK(cudaMemcpyAsync(x, H.x.p, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    // true residual
    SPHC_TRY(spmv64(A, H.x.p, H.q.p, s));
    SPHC_LAUNCH(k_sub<<<grid_for(n, 256), 256, 0, s>>>(b, H.q.p, n));
    dot_buf(H, H.q.p, H.q.p, n, sc + 6, s);
    double hr = 0.0;
    SPHC_CK(cudaMemcpyAsync(&hr, sc + 6, sizeof(double), cudaMemcpyDeviceToHost, s));
    SPHC_CK(cudaStreamSynchronize(s));
    if (iters) *iters = it;
    if (relres) *relres = bnorm > 0 ? sqrt(hr) / bnorm : 0.0;
    if (status == SPHC_EBREAKDOWN) set_error("CG breakdown after %d iterations", it);
    else if (status == SPHC_ENOTCONV) set_error("CG did not reach the tolerance in %d iterations", it);
    return status;
}

// ------------------------------------------------------------------ CG captured whole (batched solves)
// The right side is read from H.bin and tol^2 from scal[8]; x stays in H.x.  Every iteration
// (V-cycle first) runs inside a while node whose condition a prologue kernel sets, so the whole
// solve needs no host decision and can be one branch of a larger graph.
__global__ void k_cg_prep(cudaGraphConditionalHandle hnd, double* sc, int* itc) {
    sc[7] = sc[8] * sc[5];
    sc[0] = 1.0;                         // rz of the previous iteration (p = 0 makes beta irrelevant)
    itc[0] = 0;
    itc[1] = sc[5] > 0.0 ? 3 : 0;        // 3: running; 0: converged (b = 0)
    cudaGraphSetConditional(hnd, sc[5] > 0.0 ? 1u : 0u);
}

static int cg_iter_body(Hierarchy& H, cudaGraphConditionalHandle hnd, cudaStream_t s) {
    const DCSR& A = H.L[0].A;
    int64_t n = A.nr;
    int flexible = H.opts.flexible;
    double* sc = H.scal.p;
    SPHC_TRY(apply_vcycle(H, H.r.p, H.z.p, s));
    dot_buf(H, H.r.p, H.z.p, n, sc + 3, s);
    if (flexible) dot_buf(H, H.z.p, H.rold.p, n, sc + 4, s);
    SPHC_LAUNCH(k_cg_p<<<grid_for(n, 256), 256, 0, s>>>(H.p.p, H.z.p, sc, n, flexible));
    SPHC_LAUNCH(k_cg_shift<<<1, 1, 0, s>>>(sc));
    SPHC_TRY(spmv64(A, H.p.p, H.q.p, s));
    dot_buf(H, H.p.p, H.q.p, n, sc + 1, s);
    SPHC_LAUNCH(k_cg_xr<<<grid_for(n, 256), 256, 0, s>>>(H.x.p, H.r.p, H.rold.p, H.p.p, H.q.p, sc, n, flexible));
    dot_buf(H, H.r.p, H.r.p, n, sc + 2, s);
    SPHC_LAUNCH(k_cg_check<<<1, 1, 0, s>>>(hnd, sc, H.itc.p, H.opts.max_iter));
    SPHC_CK(cudaGetLastError());
    return SPHC_OK;
}

// Append the whole CG of H to the graph being captured on stream s.
int capture_cg(Hierarchy& H, cudaStream_t s) {
    const DCSR& A = H.L[0].A;
    int64_t n = A.nr;
    double* sc = H.scal.p;
    if (!H.cap_stream) SPHC_CK(cudaStreamCreateWithFlags(&H.cap_stream, cudaStreamNonBlocking));
    H.capturing = true;
    long long lstart = g_launches.load();
    SPHC_CK(cudaMemcpyAsync(H.r.p, H.bin.p, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    SPHC_CK(cudaMemsetAsync(H.x.p, 0, sizeof(double) * n, s));
    SPHC_CK(cudaMemsetAsync(H.p.p, 0, sizeof(double) * n, s));
    SPHC_CK(cudaMemsetAsync(H.rold.p, 0, sizeof(double) * n, s));
    dot_buf(H, H.bin.p, H.bin.p, n, sc + 5, s);
    cudaStreamCaptureStatus st;
    cudaGraph_t g;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    SPHC_CK(cudaStreamGetCaptureInfo(s, &st, nullptr, &g, &deps, nullptr, &ndeps));
    cudaGraphConditionalHandle hnd;
    SPHC_CK(cudaGraphConditionalHandleCreate(&hnd, g, 0, 0));
    SPHC_LAUNCH(k_cg_prep<<<1, 1, 0, s>>>(hnd, sc, H.itc.p));
    SPHC_CK(cudaStreamGetCaptureInfo(s, &st, nullptr, &g, &deps, nullptr, &ndeps));
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = hnd;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    SPHC_CK(cudaGraphAddNode(&node, g, deps, nullptr, ndeps, &np));
    SPHC_CK(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    cudaGraph_t body = np.conditional.phGraph_out[0];
    SPHC_CK(cudaStreamBeginCaptureToGraph(H.cap_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    long long l0 = g_launches.load();
    int rc = cg_iter_body(H, hnd, H.cap_stream);
    H.body_launches = g_launches.load() - l0;
    g_launches.fetch_sub(H.body_launches);
    cudaGraph_t captured = nullptr;
    cudaError_t e = cudaStreamEndCapture(H.cap_stream, &captured);
    if (rc != SPHC_OK) { H.capturing = false; return rc; }
    if (e != cudaSuccess) {
        H.capturing = false;
        set_error("CG body capture failed: %s", cudaGetErrorString(e));
        return SPHC_ECUDA;
    }
    // true residual
    SPHC_TRY(spmv64(A, H.x.p, H.q.p, s));
    SPHC_LAUNCH(k_sub<<<grid_for(n, 256), 256, 0, s>>>(H.bin.p, H.q.p, n));
    dot_buf(H, H.q.p, H.q.p, n, sc + 6, s);
    H.capturing = false;
    H.branch_launches = g_launches.load() - lstart;   // counted when the graph runs
    g_launches.fetch_sub(H.branch_launches);
    SPHC_CK(cudaGetLastError());
    return SPHC_OK;
}

int pcg_solve(Hierarchy& H, const double* b, double* x, double tol, cudaStream_t s, int* iters, double* relres) {
    if (H.opts.cg_graph) return pcg_graph(H, b, x, tol, s, iters, relres);
    const DCSR& A = H.L[0].A;
    int64_t n = A.nr;
    int flexible = H.opts.flexible;
    double* sc = H.scal.p;
    SPHC_CK(cudaMemsetAsync(x, 0, sizeof(double) * n, s));
    SPHC_CK(cudaMemcpyAsync(H.r.p, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    SPHC_TRY(dot64(b, b, n, sc + 5, s));
    double hb = 0.0;
    SPHC_CK(cudaMemcpyAsync(&hb, sc + 5, sizeof(double), cudaMemcpyDeviceToHost, s));
    SPHC_CK(cudaStreamSynchronize(s));
    double bnorm = sqrt(hb);
    int status = SPHC_ENOTCONV, it = 0;
    if (bnorm == 0.0) status = SPHC_OK;
    if (status != SPHC_OK) {
        SPHC_TRY(apply_vcycle(H, H.r.p, H.z.p, s));
        SPHC_CK(cudaMemcpyAsync(H.p.p, H.z.p, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
        SPHC_TRY(dot64(H.r.p, H.z.p, n, sc + 0, s));
        double hsc[6];
        int tid = H.prof.on ? H.prof.find("spmv_A_fp64", (double)A.nnz * 12.0 + (double)n * 24.0) : -1;
        for (it = 0; it < H.opts.max_iter;) {
            if (tid >= 0) H.prof.begin(tid, s);
            SPHC_TRY(spmv64(A, H.p.p, H.q.p, s));
            if (tid >= 0) H.prof.end(tid, s);
            SPHC_TRY(dot64(H.p.p, H.q.p, n, sc + 1, s));
            SPHC_LAUNCH(k_cg_xr<<<grid_for(n, 256), 256, 0, s>>>(x, H.r.p, H.rold.p, H.p.p, H.q.p, sc, n, flexible));
            ++it;
            SPHC_TRY(dot64(H.r.p, H.r.p, n, sc + 2, s));
            SPHC_CK(cudaMemcpyAsync(hsc, sc, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
            SPHC_CK(cudaStreamSynchronize(s));
            if (!(hsc[1] > 0.0) || !std::isfinite(hsc[2])) { status = SPHC_EBREAKDOWN; break; }
            if (sqrt(hsc[2]) <= tol * bnorm) { status = SPHC_OK; break; }
            SPHC_TRY(apply_vcycle(H, H.r.p, H.z.p, s));
            SPHC_TRY(dot64(H.r.p, H.z.p, n, sc + 3, s));
            if (flexible) SPHC_TRY(dot64(H.z.p, H.rold.p, n, sc + 4, s));
            SPHC_LAUNCH(k_cg_p<<<grid_for(n, 256), 256, 0, s>>>(H.p.p, H.z.p, sc, n, flexible));
            SPHC_LAUNCH(k_cg_shift<<<1, 1, 0, s>>>(sc));
        }
    }
    // true residual
    SPHC_TRY(spmv64(A, x, H.q.p, s));
    SPHC_LAUNCH(k_sub<<<grid_for(n, 256), 256, 0, s>>>(b, H.q.p, n));
    SPHC_TRY(dot64(H.q.p, H.q.p, n, sc + 6, s));
    double hr = 0.0;
    SPHC_CK(cudaMemcpyAsync(&hr, sc + 6, sizeof(double), cudaMemcpyDeviceToHost, s));
    SPHC_CK(cudaStreamSynchronize(s));
    if (iters) *iters = it;
    if (relres) *relres = bnorm > 0 ? sqrt(hr) / bnorm : 0.0;
    if (status != SPHC_OK && status != SPHC_ENOTCONV)
        set_error("CG breakdown after %d iterations", it);
    else if (status == SPHC_ENOTCONV)
        set_error("CG did not reach the tolerance in %d iterations", it);
    return status;
}

}  // namespace sphc
