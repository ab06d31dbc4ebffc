// Block right-hand sides: NB systems A x_k = b_k (NB = 2, 4, 8 or 16) solved together by NB
// independent preconditioned CG iterations (Sec. 6.1) that share every operator read.
//
// Vectors of a block are interleaved: entry k of row i sits at i * NB + k, so one row of a SELL
// operator, read once, is applied to all NB vectors, and the NB values gathered for one column
// are one contiguous 8 * NB- or 4 * NB-byte load.  Per right-hand side the matrix traffic of a
// sweep drops by NB; the vectors' traffic is unchanged.  Each column keeps its own CG scalars and
// status; a column that has converged (or broken down, or stagnated) is frozen while the others
// continue.  The iterations after the first run as one CUDA graph whose while node repeats an
// iteration until no column is active, as in the single-vector solve.
#include <cmath>

#include "sell.cuh"

namespace sphc {

// ------------------------------------------------------------------ rows of NB values
__device__ __forceinline__ void load_row(const float* __restrict__ p, float (&v)[2]) {
    float2 t = *reinterpret_cast<const float2*>(p);
    v[0] = t.x; v[1] = t.y;
}
template <int NB>
__device__ __forceinline__ void load_row(const float* __restrict__ p, float (&v)[NB]) {
#pragma unroll
    for (int j = 0; j < NB / 4; ++j) {
        float4 t = reinterpret_cast<const float4*>(p)[j];
        v[4 * j] = t.x; v[4 * j + 1] = t.y; v[4 * j + 2] = t.z; v[4 * j + 3] = t.w;
    }
}
template <int NB>
__device__ __forceinline__ void load_row(const double* __restrict__ p, double (&v)[NB]) {
#pragma unroll
    for (int j = 0; j < NB / 2; ++j) {
        double2 t = reinterpret_cast<const double2*>(p)[j];
        v[2 * j] = t.x; v[2 * j + 1] = t.y;
    }
}
__device__ __forceinline__ void store_row(float* p, const float (&v)[2]) {
    *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
}
template <int NB>
__device__ __forceinline__ void store_row(float* p, const float (&v)[NB]) {
#pragma unroll
    for (int j = 0; j < NB / 4; ++j)
        reinterpret_cast<float4*>(p)[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
}
template <int NB>
__device__ __forceinline__ void store_row(double* p, const double (&v)[NB]) {
#pragma unroll
    for (int j = 0; j < NB / 2; ++j) reinterpret_cast<double2*>(p)[j] = make_double2(v[2 * j], v[2 * j + 1]);
}

// This lane's partial (A X)_r for all NB vectors over the slice starting at o.
template <typename T, int CH, int NB>
__device__ __forceinline__ void sell_part_nb(const int32_t* __restrict__ ci, const T* __restrict__ v, int64_t o,
                                             int64_t steps, int lane, const T* __restrict__ x, T (&acc)[NB]) {
#pragma unroll
    for (int k = 0; k < NB; ++k) acc[k] = T(0);
    const T* vp = v + o + lane * CH;
    const int32_t* cp = ci + o + lane * CH;
    for (int64_t q = 0; q < steps; ++q) {
        T a[CH];
        int32_t c[CH];
        Chunk<T, CH>::load(vp, a);
        IChunk<CH>::load(cp, c);
#pragma unroll
        for (int t = 0; t < CH; ++t) {
            T xv[NB];
            load_row(x + (int64_t)c[t] * NB, xv);
#pragma unroll
            for (int k = 0; k < NB; ++k) acc[k] += a[t] * xv[k];
        }
        vp += SELL_C * CH;
        cp += SELL_C * CH;
    }
}
template <typename T, int NB>
__device__ __forceinline__ void row_reduce_nb(T (&acc)[NB], int lpr) {
#pragma unroll
    for (int k = 0; k < NB; ++k) acc[k] = row_reduce(acc[k], lpr);
}

// Gauss-Seidel update of one colour's slices [s0, s1) for all NB vectors
template <typename T, int CH, int NB>
__global__ void __launch_bounds__(256)
k_bsgs(const int64_t* __restrict__ soff, const int32_t* __restrict__ srow, int64_t s0, int64_t s1, int lpr,
       const int32_t* __restrict__ ci, const T* __restrict__ v, const T* __restrict__ dinv, const T* __restrict__ b,
       T* x) {
    pdl_enter();
    const int64_t sl = s0 + (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (sl >= s1) return;
    const int lane = threadIdx.x & 31;
    const int64_t o = soff[sl];
    const SliceRow q = slice_row(srow, sl, lane, lpr);
    T acc[NB];
    sell_part_nb<T, CH, NB>(ci, v, o, (soff[sl + 1] - o) / (SELL_C * CH), lane, x, acc);
    row_reduce_nb(acc, lpr);
    if (q.write) {
        T bv[NB], xv[NB];
        load_row(b + (int64_t)q.r * NB, bv);
        load_row(x + (int64_t)q.r * NB, xv);
        const T d = dinv[q.r];
#pragma unroll
        for (int k = 0; k < NB; ++k) xv[k] += (bv[k] - acc[k]) * d;
        store_row(x + (int64_t)q.r * NB, xv);
    }
}
// R = B - A X
template <typename T, int CH, int NB>
__global__ void __launch_bounds__(256)
k_bresid(const int64_t* __restrict__ soff, const int32_t* __restrict__ srow, int64_t nslice, int lpr,
         const int32_t* __restrict__ ci, const T* __restrict__ v, const T* __restrict__ b, const T* __restrict__ x,
         T* __restrict__ r) {
    pdl_enter();
    const int64_t sl = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (sl >= nslice) return;
    const int lane = threadIdx.x & 31;
    const int64_t o = soff[sl];
    const SliceRow q = slice_row(srow, sl, lane, lpr);
    T acc[NB];
    sell_part_nb<T, CH, NB>(ci, v, o, (soff[sl + 1] - o) / (SELL_C * CH), lane, x, acc);
    row_reduce_nb(acc, lpr);
    if (q.write) {
        T bv[NB];
        load_row(b + (int64_t)q.r * NB, bv);
#pragma unroll
        for (int k = 0; k < NB; ++k) bv[k] -= acc[k];
        store_row(r + (int64_t)q.r * NB, bv);
    }
}
// Y = alpha A X (+ Y)
template <typename T, int CH, int NB>
__global__ void __launch_bounds__(256)
k_bspmv(const int64_t* __restrict__ soff, const int32_t* __restrict__ srow, int64_t nslice, int lpr,
        const int32_t* __restrict__ ci, const T* __restrict__ v, const T* __restrict__ x, T* y, int accumulate,
        T alpha) {
    pdl_enter();
    const int64_t sl = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (sl >= nslice) return;
    const int lane = threadIdx.x & 31;
    const int64_t o = soff[sl];
    const SliceRow q = slice_row(srow, sl, lane, lpr);
    T acc[NB];
    sell_part_nb<T, CH, NB>(ci, v, o, (soff[sl + 1] - o) / (SELL_C * CH), lane, x, acc);
    row_reduce_nb(acc, lpr);
    if (q.write) {
        T yv[NB];
        if (accumulate) load_row(y + (int64_t)q.r * NB, yv);
#pragma unroll
        for (int k = 0; k < NB; ++k) yv[k] = accumulate ? yv[k] + alpha * acc[k] : alpha * acc[k];
        store_row(y + (int64_t)q.r * NB, yv);
    }
}
// a whole forward + backward sweep of a small operator (at most SGS_BLOCK_MAX_ROWS rows) in one block
template <typename T, int CH, int NB>
__global__ void __launch_bounds__(256)
k_bsgs_block(const int64_t* __restrict__ soff, const int32_t* __restrict__ srow, const int64_t* __restrict__ cslice,
             int ncolor, int lpr, const int32_t* __restrict__ ci, const T* __restrict__ v,
             const T* __restrict__ dinv, const T* __restrict__ b, T* x) {
    pdl_enter();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    for (int step = 0; step < sweep_steps(ncolor); ++step) {
        const int c = sweep_colour(step, ncolor);
        for (int64_t sl = cslice[c] + warp; sl < cslice[c + 1]; sl += nwarp) {
            const int64_t o = soff[sl];
            const SliceRow q = slice_row(srow, sl, lane, lpr);
            T acc[NB];
            sell_part_nb<T, CH, NB>(ci, v, o, (soff[sl + 1] - o) / (SELL_C * CH), lane, x, acc);
            row_reduce_nb(acc, lpr);
            if (q.write) {
                T bv[NB], xv[NB];
                load_row(b + (int64_t)q.r * NB, bv);
                load_row(x + (int64_t)q.r * NB, xv);
                const T d = dinv[q.r];
#pragma unroll
                for (int k = 0; k < NB; ++k) xv[k] += (bv[k] - acc[k]) * d;
                store_row(x + (int64_t)q.r * NB, xv);
            }
        }
        __syncthreads();
    }
}
// Y = alpha A X (+ Y) for a CSR operator, SUB lanes per row
template <typename T, int SUB, int NB>
__global__ void k_bspmv_csr(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci, const T* __restrict__ v,
                            int64_t n, const T* __restrict__ x, T* y, int accumulate, T alpha) {
    pdl_enter();
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / SUB;
    const int q = threadIdx.x & (SUB - 1);
    const bool valid = i < n;
    T acc[NB];
#pragma unroll
    for (int k = 0; k < NB; ++k) acc[k] = T(0);
    if (valid)
        for (int32_t e = rp[i] + q; e < rp[i + 1]; e += SUB) {
            T xv[NB];
            load_row(x + (int64_t)ci[e] * NB, xv);
            const T a = v[e];
#pragma unroll
            for (int k = 0; k < NB; ++k) acc[k] += a * xv[k];
        }
#pragma unroll
    for (int k = 0; k < NB; ++k)
#pragma unroll
        for (int o = SUB / 2; o > 0; o >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], o, SUB);
    if (valid && q == 0) {
        T yv[NB];
        if (accumulate) load_row(y + i * NB, yv);
#pragma unroll
        for (int k = 0; k < NB; ++k) yv[k] = accumulate ? yv[k] + alpha * acc[k] : alpha * acc[k];
        store_row(y + i * NB, yv);
    }
}

// ------------------------------------------------------------------ elementwise and gradient operators
template <typename T>
__global__ void k_bzero(T* a, int64_t n) {
    pdl_enter();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = T(0);
}
template <typename T>
__global__ void k_bcopy(T* y, const T* x, int64_t n) {
    pdl_enter();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = x[i];
}
template <typename T>
__global__ void k_baxpy(T* y, const T* x, int64_t n) {
    pdl_enter();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] += x[i];
}
template <typename A, typename B>
__global__ void k_bcast(const A* a, B* b, int64_t n) {
    pdl_enter();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (B)a[i];
}
// G = D^T R (per node: the signed sum of its incident edges' rows)
template <typename T, int NB>
__global__ void k_bdt_gather(const int32_t* __restrict__ rp, const int32_t* __restrict__ enc, int64_t nv,
                             const T* __restrict__ r, T* __restrict__ g) {
    pdl_enter();
    const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= nv) return;
    T s[NB];
#pragma unroll
    for (int k = 0; k < NB; ++k) s[k] = T(0);
    for (int32_t q = rp[u]; q < rp[u + 1]; ++q) {
        const int32_t e = enc[q];
        T rv[NB];
        load_row(r + (int64_t)(e >> 1) * NB, rv);
#pragma unroll
        for (int k = 0; k < NB; ++k) s[k] += (e & 1) ? -rv[k] : rv[k];
    }
    store_row(g + u * NB, s);
}
// X += D C (per edge: head minus tail)
template <typename T, int NB>
__global__ void k_bd_apply(const int2* __restrict__ D, int64_t ne, const T* __restrict__ c, T* __restrict__ x) {
    pdl_enter();
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ne * NB) return;
    const int64_t e = t / NB;
    const int k = (int)(t % NB);
    const int2 d = D[e];
    T v = 0;
    if (d.y >= 0) v += c[(int64_t)d.y * NB + k];
    if (d.x >= 0) v -= c[(int64_t)d.x * NB + k];
    x[t] += v;
}
// Z = Y + D C in FP64 (the split iterate of the FP32 V-cycle)
template <typename T, int NB>
__global__ void k_bcombine(const T* __restrict__ y, const int2* __restrict__ D, const T* __restrict__ c, int64_t ne,
                           double* __restrict__ z) {
    pdl_enter();
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ne * NB) return;
    const int64_t e = t / NB;
    const int k = (int)(t % NB);
    const int2 d = D[e];
    double v = (double)y[t];
    if (d.y >= 0) v += (double)c[(int64_t)d.y * NB + k];
    if (d.x >= 0) v -= (double)c[(int64_t)d.x * NB + k];
    z[t] = v;
}
// X = M B for a dense n x n FP64 matrix M (the coarsest inverses); warp per row
template <typename T, int NB>
__global__ void k_bdense(const double* __restrict__ M, int64_t n, const T* __restrict__ b, T* __restrict__ x) {
    pdl_enter();
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= n) return;
    double s[NB];
#pragma unroll
    for (int k = 0; k < NB; ++k) s[k] = 0.0;
    for (int64_t j = lane; j < n; j += 32) {
        const double m = M[i * n + j];
#pragma unroll
        for (int k = 0; k < NB; ++k) s[k] += m * (double)b[j * NB + k];
    }
#pragma unroll
    for (int k = 0; k < NB; ++k)
        for (int o = 16; o > 0; o >>= 1) s[k] += __shfl_xor_sync(0xffffffffu, s[k], o);
    if (lane < NB) {
        double out = 0.0;
#pragma unroll
        for (int k = 0; k < NB; ++k)
            if (k == lane) out = s[k];
        x[i * NB + lane] = (T)out;
    }
}
// coarsest split: Y = A^-1 B - D C, C = A_n^-1 D^T B (FP64 inputs, cast to T)
template <typename T, int NB>
__global__ void k_bsplit_out(const double* __restrict__ xb, const int2* __restrict__ D, const double* __restrict__ cc,
                             int64_t ne, int64_t nv, T* __restrict__ y, T* __restrict__ c) {
    pdl_enter();
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < ne * NB) {
        const int64_t e = t / NB;
        const int k = (int)(t % NB);
        const int2 d = D[e];
        double g = 0.0;
        if (d.y >= 0) g += cc[(int64_t)d.y * NB + k];
        if (d.x >= 0) g -= cc[(int64_t)d.x * NB + k];
        y[t] = (T)(xb[t] - g);
    }
    if (t < nv * NB) c[t] = (T)cc[t];
}

// ------------------------------------------------------------------ per-column CG kernels
// Scalars of column k at sc[k * BSC + f]: f = 0 rz, 1 pq, 2 rr, 3 rz_new, 4 z.r_old, 5 bb, 6 true
// r.r, 7 limit.  Control of column k at st[k * BST + f]: f = 0 iterations, 1 status (3 running,
// 0 converged, 1 breakdown, 2 cap, 4 stagnation), 2 moved (x changed in this iteration).
// st[NB * BST] counts the graph iterations run.
constexpr int BSC = 8, BST = 4;
constexpr int BDOT_PARTS = 512;
// column sums of a .* b over n rows of NB: partials part[block * NB + k]
template <int NB>
__global__ void __launch_bounds__(256) k_bdot_part(const double* __restrict__ a, const double* __restrict__ b,
                                                   int64_t n_el, double* __restrict__ part) {
    pdl_enter();
    __shared__ double sw[8][NB];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;      // a multiple of NB: fixed column per thread
    double s = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n_el; e += stride) s += a[e] * b[e];
    for (int o = 16; o >= NB; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane < NB) sw[w][lane] = s;
    __syncthreads();
    if (threadIdx.x < NB) {
        double t = 0.0;
        for (int q = 0; q < 8; ++q) t += sw[q][threadIdx.x];
        part[(int64_t)blockIdx.x * NB + threadIdx.x] = t;
    }
}
template <int NB>
__global__ void k_bdot_final(const double* __restrict__ part, int np, double* sc, int field) {
    pdl_enter();
    const int k = threadIdx.x;
    if (k >= NB) return;
    double t = 0.0;
    for (int q = 0; q < np; ++q) t += part[(int64_t)q * NB + k];
    sc[k * BSC + field] = t;
}
// x += alpha p, r -= alpha q for running columns; marks the columns whose x changed
template <int NB>
__global__ void __launch_bounds__(256) k_bcg_xr(double* x, double* r, double* rold, const double* p, const double* q,
                                                const double* sc, int* st, int64_t n_el, int flexible) {
    pdl_enter();
    __shared__ int mv[NB];
    if (threadIdx.x < NB) mv[threadIdx.x] = 0;
    __syncthreads();
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n_el) {
        const int k = (int)(e % NB);
        if (st[k * BST + 1] == 3) {
            const double pq = sc[k * BSC + 1];
            const double alpha = pq > 0.0 ? sc[k * BSC + 0] / pq : 0.0;
            const double xo = x[e], xn = xo + alpha * p[e];
            if (xn != xo) mv[k] = 1;
            x[e] = xn;
            if (flexible) rold[e] = r[e];
            r[e] -= alpha * q[e];
        }
    }
    __syncthreads();
    if (threadIdx.x < NB && mv[threadIdx.x] && *(volatile int*)&st[threadIdx.x * BST + 2] == 0)
        st[threadIdx.x * BST + 2] = 1;
}
template <int NB>
__global__ void k_bcg_p(double* p, const double* z, const double* sc, const int* st, int64_t n_el, int flexible) {
    pdl_enter();
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_el) return;
    const int k = (int)(e % NB);
    if (st[k * BST + 1] != 3) return;
    const double* c = sc + k * BSC;
    const double beta = flexible ? (c[3] - c[4]) / c[0] : c[3] / c[0];
    p[e] = z[e] + beta * p[e];
}
template <int NB>
__global__ void k_bcg_shift(double* sc, const int* st) {
    pdl_enter();
    const int k = threadIdx.x;
    if (k < NB && st[k * BST + 1] == 3) sc[k * BSC + 0] = sc[k * BSC + 3];
}
// limits and initial status: b = 0 is converged at once (a non-finite b runs and breaks down)
template <int NB>
__global__ void k_bcg_init(double* sc, int* st, double tol2) {
    pdl_enter();
    const int k = threadIdx.x;
    if (k < NB) {
        double* c = sc + k * BSC;
        c[7] = tol2 * c[5];
        st[k * BST + 0] = 0;
        st[k * BST + 1] = c[5] == 0.0 ? 0 : 3;
        st[k * BST + 2] = 0;
    }
    if (k == 0) st[NB * BST] = 0;
}
// end of an iteration: per running column count it and test breakdown, convergence,
// stagnation (x unchanged, Sec. 7) and the cap; loop while any column still runs
template <int NB>
__global__ void k_bcg_check(cudaGraphConditionalHandle hnd, int use_cond, const double* sc, int* st, int max_iter) {
    pdl_enter();
    const int k = threadIdx.x;
    bool run = false;
    if (k < NB) {
        int* c = st + k * BST;
        if (c[1] == 3) {
            const int it = c[0] + 1;
            c[0] = it;
            const double pq = sc[k * BSC + 1], rr = sc[k * BSC + 2], lim = sc[k * BSC + 7];
            if (!(pq > 0.0) || !isfinite(rr)) c[1] = 1;
            else if (rr <= lim) c[1] = 0;
            else if (c[2] == 0) c[1] = 4;
            else if (it >= max_iter) c[1] = 2;
            run = c[1] == 3;
        }
        c[2] = 0;
    }
    const bool any = __syncthreads_or(run);
    if (k == 0) {
        st[NB * BST] += 1;
        if (use_cond) cudaGraphSetConditional(hnd, any ? 1u : 0u);
    }
}
// caller layout (column k of n at k * n + old row) <-> block layout (new row * NB + k), with the
// level-0 renumbering p (new -> old); columns at or beyond nrhs are zero
template <int NB>
__global__ void k_bgather(const double* __restrict__ b, const int32_t* __restrict__ p, int64_t n, int nrhs,
                          double* __restrict__ out) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * NB) return;
    const int64_t i = t / NB;
    const int k = (int)(t % NB);
    const int64_t src = p ? p[i] : i;
    out[t] = k < nrhs ? b[(int64_t)k * n + src] : 0.0;
}
template <int NB>
__global__ void k_bscatter(const double* __restrict__ x, const int32_t* __restrict__ p, int64_t n, int nrhs,
                           double* __restrict__ out) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * NB) return;
    const int64_t i = t / NB;
    const int k = (int)(t % NB);
    if (k < nrhs) out[(int64_t)k * n + (p ? p[i] : i)] = x[t];
}
template <int NB>
__global__ void k_bsub(const double* b, double* q, int64_t n_el) {
    pdl_enter();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_el) q[i] = b[i] - q[i];
}

// ------------------------------------------------------------------ host drivers
namespace {

unsigned bslice_grid(int64_t nslice) { return (unsigned)grid_for(nslice * 32, 256); }
int bsub_for(int64_t nnz, int64_t n) {
    const double avg = n > 0 ? (double)nnz / (double)n : 0.0;
    if (avg <= 6) return 4;
    if (avg <= 20) return 8;
    if (avg <= 48) return 16;
    return 32;
}
const Sell<double>& bcg_op(const Hierarchy& H) { return H.A0.nr == H.L[0].A.nr ? H.A0 : H.V64[0].A.m; }
const int32_t* bperm0(const Hierarchy& H) { return H.ord.empty() ? nullptr : H.ord[0].pe.p; }

#define SPHC_BCH(ch, F)       \
    switch (ch) {             \
        case 1: F(1); break;  \
        case 2: F(2); break;  \
        default: F(4); break; \
    }

template <typename T, int NB>
void bsgs(const SmoothOp<T>& op, const T* b, T* x, cudaStream_t s) {
    const Sell<T>& m = op.m;
    if (op.n == 0) return;
    if (op.n <= SGS_BLOCK_MAX_ROWS) {
#define F(C) launch_pdl(k_bsgs_block<T, C, NB>, 1, 256, 0, s, m.soff.p, m.srow.p, op.cslice_dev.p, op.ncolor, m.lpr, m.ci.p, m.v.p, op.dinv.p, b, x)
        SPHC_BCH(m.ch, F)
#undef F
        return;
    }
    for (int step = 0; step < sweep_steps(op.ncolor); ++step) {
        const int c = sweep_colour(step, op.ncolor);
        const int64_t s0 = op.cslice[c], s1 = op.cslice[c + 1];
        if (s1 <= s0) continue;
#define F(C) launch_pdl(k_bsgs<T, C, NB>, bslice_grid(s1 - s0), 256, 0, s, m.soff.p, m.srow.p, s0, s1, m.lpr, m.ci.p, m.v.p, op.dinv.p, b, x)
        SPHC_BCH(m.ch, F)
#undef F
    }
}
template <typename T, int NB>
void bresid(const SmoothOp<T>& op, const T* b, const T* x, T* r, cudaStream_t s) {
    const Sell<T>& m = op.m;
    if (m.nslice == 0) return;
#define F(C) launch_pdl(k_bresid<T, C, NB>, bslice_grid(m.nslice), 256, 0, s, m.soff.p, m.srow.p, m.nslice, m.lpr, m.ci.p, m.v.p, b, x, r)
    SPHC_BCH(m.ch, F)
#undef F
}
template <typename T, int NB>
void bsell_spmv(const Sell<T>& m, const T* x, T* y, int acc, cudaStream_t s, T alpha = T(1)) {
    if (m.nslice == 0) return;
#define F(C) launch_pdl(k_bspmv<T, C, NB>, bslice_grid(m.nslice), 256, 0, s, m.soff.p, m.srow.p, m.nslice, m.lpr, m.ci.p, m.v.p, x, y, acc, alpha)
    SPHC_BCH(m.ch, F)
#undef F
}
template <typename T, int NB>
void bspmv_x(const XOp<T>& X, const T* x, T* y, int acc, cudaStream_t s, T alpha = T(1)) {
    if (X.nr == 0) return;
    if (X.sell) {
        bsell_spmv<T, NB>(X.s, x, y, acc, s, alpha);
        return;
    }
    const VCSR<T>& A = X.c;
    const int sub = bsub_for(A.nnz, A.nr);
    const int64_t th = A.nr * sub;
    switch (sub) {
        case 4: launch_pdl(k_bspmv_csr<T, 4, NB>, grid_for(th, 256), 256, 0, s, A.rp.p, A.ci.p, A.v.p, A.nr, x, y, acc, alpha); break;
        case 8: launch_pdl(k_bspmv_csr<T, 8, NB>, grid_for(th, 256), 256, 0, s, A.rp.p, A.ci.p, A.v.p, A.nr, x, y, acc, alpha); break;
        case 16: launch_pdl(k_bspmv_csr<T, 16, NB>, grid_for(th, 256), 256, 0, s, A.rp.p, A.ci.p, A.v.p, A.nr, x, y, acc, alpha); break;
        default: launch_pdl(k_bspmv_csr<T, 32, NB>, grid_for(th, 256), 256, 0, s, A.rp.p, A.ci.p, A.v.p, A.nr, x, y, acc, alpha); break;
    }
}
template <typename T>
void bzero(T* a, int64_t n, cudaStream_t s) {
    if (n > 0) launch_pdl(k_bzero<T>, grid_for(n, 256), 256, 0, s, a, n);
}

// ---- split FP32 V-cycle (iterate y + D c), as vcycle_split of the single-vector path
template <typename T, int NB>
void bhiptmair_split(Hierarchy& H, BlockLevel<T>& V, const VLevel<T>& O, int64_t ne, int64_t nv, cudaStream_t s) {
    bsgs<T, NB>(O.A, V.bp.p, V.x.p, s);
    if (nv > 0) {
        bresid<T, NB>(O.A, V.bp.p, V.x.p, V.r.p, s);
        launch_pdl(k_bdt_gather<T, NB>, grid_for(nv, 256), 256, 0, s, O.Dt_rp.p, O.Dt_e.p, nv, V.r.p, V.g.p);
        bzero(V.dc.p, nv * NB, s);
        bsgs<T, NB>(O.An, V.g.p, V.dc.p, s);
        launch_pdl(k_baxpy<T>, grid_for(nv * NB, 256), 256, 0, s, V.c.p, V.dc.p, nv * NB);
        bspmv_x<T, NB>(O.AD, V.dc.p, V.bp.p, 1, s, T(-1));
    }
    bsgs<T, NB>(O.A, V.bp.p, V.x.p, s);
}
template <typename T, int NB>
void bcoarse_split(Hierarchy& H, BlockWork& W, BlockLevel<T>& V, const VLevel<T>& O, int64_t ne, int64_t nv,
                   cudaStream_t s) {
    if (ne == 0) return;
    launch_pdl(k_bcast<T, double>, grid_for(ne * NB, 256), 256, 0, s, V.b.p, W.cb.p, ne * NB);
    launch_pdl(k_bdense<double, NB>, grid_for(ne * 32, 256), 256, 0, s, H.coarse_inv.p, ne, W.cb.p, W.cx.p);
    if (nv > 0) {
        launch_pdl(k_bdt_gather<double, NB>, grid_for(nv, 256), 256, 0, s, O.Dt_rp.p, O.Dt_e.p, nv, W.cb.p, W.cgn.p);
        launch_pdl(k_bdense<double, NB>, grid_for(nv * 32, 256), 256, 0, s, H.coarse_inv_n.p, nv, W.cgn.p, W.ccn.p);
    } else {
        bzero(W.ccn.p, 1, s);
    }
    const int64_t m = (ne > nv ? ne : nv) * NB;
    launch_pdl(k_bsplit_out<T, NB>, grid_for(m, 256), 256, 0, s, W.cx.p, O.D.p, W.ccn.p, ne, nv, V.x.p, V.c.p);
}
template <typename T, int NB>
void bvcycle_split(Hierarchy& H, BlockWork& W, std::vector<BlockLevel<T>>& V, std::vector<VLevel<T>>& O, int l,
                   cudaStream_t s) {
    const int64_t ne = H.L[l].A.nr, nv = H.L[l].An.nr;
    if (l == H.nlev - 1) {
        bcoarse_split<T, NB>(H, W, V[l], O[l], ne, nv, s);
        return;
    }
    bzero(V[l].x.p, ne * NB, s);
    bzero(V[l].c.p, nv * NB, s);
    launch_pdl(k_bcopy<T>, grid_for(ne * NB, 256), 256, 0, s, V[l].bp.p, V[l].b.p, ne * NB);
    bhiptmair_split<T, NB>(H, V[l], O[l], ne, nv, s);
    bresid<T, NB>(O[l].A, V[l].bp.p, V[l].x.p, V[l].r.p, s);
    bspmv_x<T, NB>(O[l].PeT, V[l].r.p, V[l + 1].b.p, 0, s);
    bvcycle_split<T, NB>(H, W, V, O, l + 1, s);
    bspmv_x<T, NB>(O[l].Pe, V[l + 1].x.p, V[l].x.p, 1, s);
    if (nv > 0) {
        bspmv_x<T, NB>(O[l].Pn, V[l + 1].c.p, V[l].dc.p, 0, s);
        launch_pdl(k_baxpy<T>, grid_for(nv * NB, 256), 256, 0, s, V[l].c.p, V[l].dc.p, nv * NB);
        bspmv_x<T, NB>(O[l].AD, V[l].dc.p, V[l].bp.p, 1, s, T(-1));
    }
    bhiptmair_split<T, NB>(H, V[l], O[l], ne, nv, s);
}
// ---- plain FP64 V-cycle, as vcycle_level of the single-vector path
template <int NB>
void bhiptmair(BlockLevel<double>& V, const VLevel<double>& O, int64_t ne, int64_t nv, cudaStream_t s) {
    bsgs<double, NB>(O.A, V.b.p, V.x.p, s);
    bresid<double, NB>(O.A, V.b.p, V.x.p, V.r.p, s);
    if (nv > 0) {
        launch_pdl(k_bdt_gather<double, NB>, grid_for(nv, 256), 256, 0, s, O.Dt_rp.p, O.Dt_e.p, nv, V.r.p, V.g.p);
        bzero(V.c.p, nv * NB, s);
        bsgs<double, NB>(O.An, V.g.p, V.c.p, s);
        launch_pdl(k_bd_apply<double, NB>, grid_for(ne * NB, 256), 256, 0, s, O.D.p, ne, V.c.p, V.x.p);
    }
    bsgs<double, NB>(O.A, V.b.p, V.x.p, s);
}
template <int NB>
void bvcycle_level(Hierarchy& H, std::vector<BlockLevel<double>>& V, std::vector<VLevel<double>>& O, int l,
                   cudaStream_t s) {
    const int64_t ne = H.L[l].A.nr, nv = H.L[l].An.nr;
    if (l == H.nlev - 1) {
        if (ne > 0) launch_pdl(k_bdense<double, NB>, grid_for(ne * 32, 256), 256, 0, s, H.coarse_inv.p, ne, V[l].b.p, V[l].x.p);
        return;
    }
    bzero(V[l].x.p, ne * NB, s);
    bhiptmair<NB>(V[l], O[l], ne, nv, s);
    bresid<double, NB>(O[l].A, V[l].b.p, V[l].x.p, V[l].r.p, s);
    bspmv_x<double, NB>(O[l].PeT, V[l].r.p, V[l + 1].b.p, 0, s);
    bvcycle_level<NB>(H, V, O, l + 1, s);
    bspmv_x<double, NB>(O[l].Pe, V[l + 1].x.p, V[l].x.p, 1, s);
    bhiptmair<NB>(V[l], O[l], ne, nv, s);
}

// z = M^-1 r for the NB columns (block layout, level-0 numbering, FP64 in and out)
template <int NB>
int bapply_vcycle(Hierarchy& H, BlockWork& W, const double* r, double* z, cudaStream_t s) {
    const int64_t n = H.L[0].A.nr;
    if (H.opts.vcycle_fp32) {
        launch_pdl(k_bcast<double, float>, grid_for(n * NB, 256), 256, 0, s, r, W.V32[0].b.p, n * NB);
        bvcycle_split<float, NB>(H, W, W.V32, H.V32, 0, s);
        launch_pdl(k_bcombine<float, NB>, grid_for(n * NB, 256), 256, 0, s, W.V32[0].x.p, H.V32[0].D.p, W.V32[0].c.p, n, z);
    } else {
        launch_pdl(k_bcopy<double>, grid_for(n * NB, 256), 256, 0, s, W.V64[0].b.p, r, n * NB);
        bvcycle_level<NB>(H, W.V64, H.V64, 0, s);
        launch_pdl(k_bcopy<double>, grid_for(n * NB, 256), 256, 0, s, z, W.V64[0].x.p, n * NB);
    }
    SPHC_CK(cudaGetLastError());
    return SPHC_OK;
}

template <int NB>
void bdot(BlockWork& W, const double* a, const double* b, int64_t n, int field, cudaStream_t s) {
    launch_pdl(k_bdot_part<NB>, BDOT_PARTS, 256, 0, s, a, b, n * NB, W.part.p);
    launch_pdl(k_bdot_final<NB>, 1, 32, 0, s, W.part.p, BDOT_PARTS, W.sc.p, field);
}
template <int NB>
void bcg_spmv(const Hierarchy& H, const double* x, double* y, cudaStream_t s) {
    bsell_spmv<double, NB>(bcg_op(H), x, y, 0, s);
}

// one CG iteration after the first (the body of the graph's while node)
template <int NB>
int bcg_body(Hierarchy& H, BlockWork& W, cudaGraphConditionalHandle hnd, int use_cond, cudaStream_t s) {
    const int64_t n = H.L[0].A.nr;
    const int flexible = H.opts.flexible;
    SPHC_TRY(bapply_vcycle<NB>(H, W, W.R.p, W.Z.p, s));
    bdot<NB>(W, W.R.p, W.Z.p, n, 3, s);
    if (flexible) bdot<NB>(W, W.Z.p, W.Rold.p, n, 4, s);
    launch_pdl(k_bcg_p<NB>, grid_for(n * NB, 256), 256, 0, s, W.P.p, W.Z.p, W.sc.p, W.st.p, n * NB, flexible);
    launch_pdl(k_bcg_shift<NB>, 1, 32, 0, s, W.sc.p, W.st.p);
    bcg_spmv<NB>(H, W.P.p, W.Q.p, s);
    bdot<NB>(W, W.P.p, W.Q.p, n, 1, s);
    launch_pdl(k_bcg_xr<NB>, grid_for(n * NB, 256), 256, 0, s, W.X.p, W.R.p, W.Rold.p, W.P.p, W.Q.p, W.sc.p, W.st.p,
               n * NB, flexible);
    bdot<NB>(W, W.R.p, W.R.p, n, 2, s);
    launch_pdl(k_bcg_check<NB>, 1, 32, 0, s, hnd, use_cond, (const double*)W.sc.p, W.st.p, H.opts.max_iter);
    SPHC_CK(cudaGetLastError());
    return SPHC_OK;
}

template <typename T>
int alloc_blevel(BlockLevel<T>& V, int64_t ne, int64_t nv, int nb, bool split, cudaStream_t s) {
    SPHC_TRY(V.x.alloc(ne * nb, s));
    SPHC_TRY(V.b.alloc(ne * nb, s));
    SPHC_TRY(V.r.alloc(ne * nb, s));
    SPHC_TRY(V.c.alloc(nv * nb, s));
    SPHC_TRY(V.g.alloc(nv * nb, s));
    if (split) {
        SPHC_TRY(V.bp.alloc(ne * nb, s));
        SPHC_TRY(V.dc.alloc(nv * nb, s));
    }
    return SPHC_OK;
}

int block_work(Hierarchy& H, int nb, cudaStream_t s) {
    if (H.blk && H.blk->nb == nb) return SPHC_OK;
    H.blk.reset(new BlockWork());
    BlockWork& W = *H.blk;
    W.nb = nb;
    const int64_t n = H.L[0].A.nr;
    if (H.opts.vcycle_fp32) {
        W.V32.resize(H.nlev);
        for (int l = 0; l < H.nlev; ++l) SPHC_TRY(alloc_blevel(W.V32[l], H.L[l].A.nr, H.L[l].An.nr, nb, true, s));
    } else {
        W.V64.resize(H.nlev);
        for (int l = 0; l < H.nlev; ++l) SPHC_TRY(alloc_blevel(W.V64[l], H.L[l].A.nr, H.L[l].An.nr, nb, false, s));
    }
    for (DBuf<double>* v : {&W.X, &W.R, &W.Z, &W.P, &W.Q, &W.Rold, &W.B}) SPHC_TRY(v->alloc(n * nb, s));
    SPHC_TRY(W.cb.alloc(H.n_coarse * nb, s));
    SPHC_TRY(W.cx.alloc(H.n_coarse * nb, s));
    const int64_t ncn = H.n_coarse_nodes > 0 ? H.n_coarse_nodes : 1;
    SPHC_TRY(W.cgn.alloc(ncn * nb, s));
    SPHC_TRY(W.ccn.alloc(ncn * nb, s));
    SPHC_TRY(W.part.alloc((int64_t)BDOT_PARTS * nb, s));
    SPHC_TRY(W.sc.alloc(16 * BSC, s));
    SPHC_TRY(W.st.alloc(16 * BST + 4, s));
    return SPHC_OK;
}

template <int NB>
int build_bcg_graph(Hierarchy& H, BlockWork& W) {
    if (W.ge) return SPHC_OK;
    if (!H.cap_stream) SPHC_CK(cudaStreamCreateWithFlags(&H.cap_stream, cudaStreamNonBlocking));
    SPHC_CK(cudaGraphCreate(&W.g, 0));
    cudaGraphConditionalHandle hnd;
    SPHC_CK(cudaGraphConditionalHandleCreate(&hnd, W.g, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = hnd;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    SPHC_CK(cudaGraphAddNode(&node, W.g, nullptr, nullptr, 0, &np));
    cudaGraph_t body = np.conditional.phGraph_out[0];
    SPHC_CK(cudaStreamBeginCaptureToGraph(H.cap_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    H.capturing = true;
    const long long l0 = g_launches.load();
    const int rc = bcg_body<NB>(H, W, hnd, 1, H.cap_stream);
    W.body_launches = g_launches.load() - l0;
    g_launches.fetch_sub(W.body_launches);          // counted when the graph runs
    H.capturing = false;
    cudaGraph_t captured = nullptr;
    const cudaError_t e = cudaStreamEndCapture(H.cap_stream, &captured);
    if (rc != SPHC_OK || e != cudaSuccess) {
        W.g = nullptr;                              // left as the runtime leaves a failed capture
        if (rc != SPHC_OK) return rc;
        set_error("block CG graph capture failed: %s", cudaGetErrorString(e));
        return SPHC_ECUDA;
    }
    SPHC_CK(cudaGraphInstantiate(&W.ge, W.g, 0));
    return SPHC_OK;
}

template <int NB>
int pcg_block_nb(Hierarchy& H, const double* b, double* x, int nrhs, double tol, cudaStream_t s, int* iters,
                 double* relres) {
    SPHC_TRY(block_work(H, NB, s));
    BlockWork& W = *H.blk;
    const int64_t n = H.L[0].A.nr;
    const int flexible = H.opts.flexible;
    if (H.opts.cg_graph) SPHC_TRY(build_bcg_graph<NB>(H, W));
    SPHC_LAUNCH(k_bgather<NB><<<grid_for(n * NB, 256), 256, 0, s>>>(b, bperm0(H), n, nrhs, W.B.p));
    SPHC_CK(cudaMemsetAsync(W.X.p, 0, sizeof(double) * n * NB, s));
    SPHC_CK(cudaMemsetAsync(W.Rold.p, 0, sizeof(double) * n * NB, s));
    SPHC_CK(cudaMemcpyAsync(W.R.p, W.B.p, sizeof(double) * n * NB, cudaMemcpyDeviceToDevice, s));
    bdot<NB>(W, W.B.p, W.B.p, n, 5, s);
    launch_pdl(k_bcg_init<NB>, 1, 32, 0, s, W.sc.p, W.st.p, tol * tol);
    // first iteration: z = M^-1 r, p = z
    SPHC_TRY(bapply_vcycle<NB>(H, W, W.R.p, W.Z.p, s));
    SPHC_CK(cudaMemcpyAsync(W.P.p, W.Z.p, sizeof(double) * n * NB, cudaMemcpyDeviceToDevice, s));
    bdot<NB>(W, W.R.p, W.Z.p, n, 0, s);
    bcg_spmv<NB>(H, W.P.p, W.Q.p, s);
    bdot<NB>(W, W.P.p, W.Q.p, n, 1, s);
    launch_pdl(k_bcg_xr<NB>, grid_for(n * NB, 256), 256, 0, s, W.X.p, W.R.p, W.Rold.p, W.P.p, W.Q.p, W.sc.p, W.st.p,
               n * NB, flexible);
    bdot<NB>(W, W.R.p, W.R.p, n, 2, s);
    launch_pdl(k_bcg_check<NB>, 1, 32, 0, s, cudaGraphConditionalHandle(0), 0, (const double*)W.sc.p, W.st.p,
               H.opts.max_iter);
    int hst[16 * BST + 4];
    SPHC_CK(cudaMemcpyAsync(hst, W.st.p, sizeof(int) * (NB * BST + 1), cudaMemcpyDeviceToHost, s));
    SPHC_CK(cudaStreamSynchronize(s));
    bool any = false;
    for (int k = 0; k < NB; ++k) any = any || hst[k * BST + 1] == 3;
    if (any) {
        if (H.opts.cg_graph) {
            SPHC_CK(cudaGraphLaunch(W.ge, s));
            SPHC_CK(cudaMemcpyAsync(hst, W.st.p, sizeof(int) * (NB * BST + 1), cudaMemcpyDeviceToHost, s));
            SPHC_CK(cudaStreamSynchronize(s));
            g_launches.fetch_add(W.body_launches * (long long)(hst[NB * BST] - 1));
        } else {
            while (any) {
                SPHC_TRY(bcg_body<NB>(H, W, cudaGraphConditionalHandle(0), 0, s));
                SPHC_CK(cudaMemcpyAsync(hst, W.st.p, sizeof(int) * (NB * BST + 1), cudaMemcpyDeviceToHost, s));
                SPHC_CK(cudaStreamSynchronize(s));
                any = false;
                for (int k = 0; k < NB; ++k) any = any || hst[k * BST + 1] == 3;
            }
        }
    }
    // solution back to the caller's layout; true residuals per column
    SPHC_LAUNCH(k_bscatter<NB><<<grid_for(n * NB, 256), 256, 0, s>>>(W.X.p, bperm0(H), n, nrhs, x));
    bcg_spmv<NB>(H, W.X.p, W.Q.p, s);
    launch_pdl(k_bsub<NB>, grid_for(n * NB, 256), 256, 0, s, W.B.p, W.Q.p, n * NB);
    bdot<NB>(W, W.Q.p, W.Q.p, n, 6, s);
    double hsc[16 * BSC];
    SPHC_CK(cudaMemcpyAsync(hsc, W.sc.p, sizeof(double) * NB * BSC, cudaMemcpyDeviceToHost, s));
    SPHC_CK(cudaStreamSynchronize(s));
    SPHC_CK(cudaGetLastError());
    int status = SPHC_OK;
    for (int k = 0; k < nrhs; ++k) {
        const int st = hst[k * BST + 1];
        const int code = st == 0 ? SPHC_OK
                                 : (st == 1 ? SPHC_EBREAKDOWN : (st == 4 ? SPHC_ESTAGNATION : SPHC_ENOTCONV));
        const double bb = hsc[k * BSC + 5];
        if (iters) iters[k] = hst[k * BST + 0];
        if (relres) relres[k] = bb == 0.0 ? 0.0 : sqrt(hsc[k * BSC + 6]) / sqrt(bb);
        if (code != SPHC_OK && status == SPHC_OK) {
            status = code;
            set_error("block CG, right-hand side %d: %s after %d iterations", k,
                      code == SPHC_EBREAKDOWN ? "breakdown" : (code == SPHC_ESTAGNATION ? "stagnation" : "no convergence"),
                      hst[k * BST + 0]);
        }
    }
    return status;
}

}  // namespace

// Block solve of nrhs <= 16 right-hand sides; b and x are device arrays in the caller's layout
// (nrhs x n_e, row-major).
int pcg_block(Hierarchy& H, const double* b, double* x, int nrhs, double tol, cudaStream_t s, int* iters,
              double* relres) {
    if (nrhs <= 2) return pcg_block_nb<2>(H, b, x, nrhs, tol, s, iters, relres);
    if (nrhs <= 4) return pcg_block_nb<4>(H, b, x, nrhs, tol, s, iters, relres);
    if (nrhs <= 8) return pcg_block_nb<8>(H, b, x, nrhs, tol, s, iters, relres);
    return pcg_block_nb<16>(H, b, x, nrhs, tol, s, iters, relres);
}

BlockWork::~BlockWork() {
    if (ge) cudaGraphExecDestroy(ge);
    if (g) cudaGraphDestroy(g);
}

}  // namespace sphc
