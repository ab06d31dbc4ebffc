// Solve phase: V-cycle with one pre- and one post symmetric Hiptmair sweep on every level but
// the coarsest, which is solved directly (Sec. 6.1), inside FP64 conjugate gradients with x0 = 0
// and the stopping test ||r|| <= tol ||b|| (Sec. 6.1).  The V-cycle runs in FP32 or FP64.
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>

#include <cooperative_groups.h>

#include "sell.cuh"

namespace sphc {
namespace cg = cooperative_groups;

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

// ------------------------------------------------------------------ V-cycle operators
// Level l's copies live in the numbering of H.ord[l]: the smoothers and A D take rows and columns
// from it, P_e / P_n map the numbering of level l+1 to that of level l, P_e^T the reverse.
static int build_orders(Hierarchy& H, cudaStream_t s) {
    H.ord.clear();
    H.ord.resize(H.nlev);
    for (int l = 0; l + 1 < H.nlev; ++l) {
        Level& L = H.L[l];
        LevelOrder& O = H.ord[l];
        SPHC_TRY(level_order(L.A, L.col_e.p, L.ncol_e, O.pe, O.ie, O.ce, s));
        SPHC_TRY(level_order(L.An, L.col_n.p, L.ncol_n, O.pn, O.in, O.cn, s));
    }
    return SPHC_OK;
}

template <typename T>
static bool cluster_sgs_chosen(const SmoothOp<T>& op, int sweep_form);
template <typename T>
static int grid_sgs_chosen(const SmoothOp<T>& op, int sweep_form);

template <typename T>
static int build_vlevel(Hierarchy& H, int l, VLevel<T>& V, bool split, cudaStream_t s) {
    Level& L = H.L[l];
    const LevelOrder& O = H.ord[l];
    int64_t ne = L.A.nr, nv = L.An.nr;
    SPHC_TRY(V.x.alloc(ne, s));
    SPHC_TRY(V.b.alloc(ne, s));
    SPHC_TRY(V.r.alloc(ne, s));
    SPHC_TRY(V.c.alloc(nv, s));
    SPHC_TRY(V.g.alloc(nv, s));
    SPHC_TRY(build_d_pairs(L.D, O.pe.p, O.in.p, V.D, s));
    SPHC_TRY(build_dt_enc(L.Dt, O.pn.p, O.ie.p, V.Dt_rp, V.Dt_e, s));
    if (split) {
        SPHC_TRY(V.dc.alloc(nv, s));
        SPHC_TRY(V.bp.alloc(ne, s));
    }
    if (l == H.nlev - 1) return SPHC_OK;
    const LevelOrder& C = H.ord[l + 1];
    if (split) {
        if (L.AD.nr != L.A.nr) SPHC_TRY(amul_d(L.A, L.D, L.AD, s));   // FP64: the curl-curl part cancels here
        SPHC_TRY(build_xop<T>(L.AD, O.pe.p, O.in.p, V.AD, s));
        SPHC_TRY(build_xop<T>(L.Pn, O.pn.p, C.in.p, V.Pn, s));
        L.AD = DCSR();
    }
    SPHC_TRY(build_smooth<T>(L.A, O.pe.p, O.ie.p, O.ce, l == 0 ? H.opts.sell_ch0 : 0, l == 0 ? H.opts.sell_lpr0 : 0,
                             V.A, s));
    SPHC_TRY(build_smooth<T>(L.An, O.pn.p, O.in.p, O.cn, 0, 0, V.An, s));
    V.A.cluster = cluster_sgs_chosen(V.A, H.opts.sweep_form) ? 1 : 0;
    V.An.cluster = cluster_sgs_chosen(V.An, H.opts.sweep_form) ? 1 : 0;
    V.A.grid = grid_sgs_chosen(V.A, H.opts.sweep_form);
    V.An.grid = grid_sgs_chosen(V.An, H.opts.sweep_form);
    V.A.bar = V.An.bar = H.gbar.p;
    V.A.polls = V.An.polls = H.opts.grid_wait_polls > 0 ? (unsigned)H.opts.grid_wait_polls : GRID_BAR_POLLS;
    SPHC_TRY(build_xop<T>(L.Pe, O.pe.p, C.ie.p, V.Pe, s));
    SPHC_TRY(build_xop<T>(L.PeT, C.pe.p, O.ie.p, V.PeT, s));
    SPHC_CK(cudaGetLastError());
    return SPHC_OK;
}

int build_vcycle_ops(Hierarchy& H, cudaStream_t s) {
    SPHC_TRY(build_orders(H, s));
    SPHC_TRY(H.gbar.alloc(1, s));
    SPHC_TRY(H.gbar.zero(s));
    const LevelOrder& O = H.ord[0];
    if (H.opts.vcycle_fp32) {
        H.V32.clear();
        H.V32.resize(H.nlev);
        for (int l = 0; l < H.nlev; ++l) SPHC_TRY(build_vlevel<float>(H, l, H.V32[l], true, s));
    } else {
        H.V64.clear();
        H.V64.resize(H.nlev);
        for (int l = 0; l < H.nlev; ++l) SPHC_TRY(build_vlevel<double>(H, l, H.V64[l], false, s));
    }
    // CG operator: shared with the FP64 smoother of level 0 when there is one
    H.A0 = Sell<double>();
    if (H.opts.vcycle_fp32 || H.nlev == 1) {
        std::vector<int64_t> seg{0, H.L[0].A.nr};
        int ch = 4, lpr = sell_lpr_for(H.L[0].A, 1);
        SPHC_TRY(sell_pick_ch(H.L[0].A, O.pe.p, seg, lpr, s, &ch));
        SPHC_TRY(build_sell<double>(H.L[0].A, O.pe.p, O.ie.p, seg, ch, lpr, H.A0, nullptr, nullptr, s));
    }
    int64_t n0 = H.L[0].A.nr;
    SPHC_TRY(H.x.alloc(n0, s));
    SPHC_TRY(H.r.alloc(n0, s));
    SPHC_TRY(H.z.alloc(n0, s));
    SPHC_TRY(H.p.alloc(n0, s));
    SPHC_TRY(H.q.alloc(n0, s));
    SPHC_TRY(H.rold.alloc(n0, s));
    SPHC_TRY(H.bperm.alloc(n0, s));
    SPHC_TRY(H.xo.alloc(n0, s));
    SPHC_TRY(H.scal.alloc(16, s));
    SPHC_TRY(H.cb.alloc(H.n_coarse, s));
    SPHC_TRY(H.cx.alloc(H.n_coarse, s));
    SPHC_TRY(H.cgn.alloc(H.n_coarse_nodes, s));
    SPHC_TRY(H.ccn.alloc(H.n_coarse_nodes, s));
    SPHC_TRY(H.dpart.alloc(DOT_PARTS, s));
    SPHC_TRY(H.itc.alloc(4, s));
    SPHC_TRY(H.bin.alloc(n0, s));
    SPHC_CK(cudaStreamSynchronize(s));
    return SPHC_OK;
}

static const Sell<double>& cg_op(const Hierarchy& H) {
    return H.A0.nr == H.L[0].A.nr ? H.A0 : H.V64[0].A.m;
}
static const int32_t* perm0(const Hierarchy& H) { return H.ord.empty() ? nullptr : H.ord[0].pe.p; }

// ------------------------------------------------------------------ dot products into persistent partials
__global__ void k_dot_part_b(const double* a, const double* b, int64_t n, double* part) {
    pdl_enter();
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
    pdl_enter();
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
    launch_pdl(k_dot_part_b, DOT_PARTS, 256, 0, s, a, b, n, H.dpart.p);
    launch_pdl(k_dot_final_b, 1, 1024, 0, s, H.dpart.p, DOT_PARTS, out);
}

// ------------------------------------------------------------------ V-cycle kernels (helpers in sell.cuh)
// Gauss-Seidel update of the rows of slices [s0, s1) (one colour): x_r += (b_r - (A x)_r) / a_rr
template <typename T, int CH>
__global__ void __launch_bounds__(256)
k_sell_sgs(const int64_t* __restrict__ soff, const int32_t* __restrict__ srow, int64_t s0, int64_t s1, int lpr,
           const int32_t* __restrict__ ci, const T* __restrict__ v, const T* __restrict__ dinv,
           const T* __restrict__ b, T* x) {
    pdl_enter();
    int64_t sl = s0 + (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (sl >= s1) return;
    int lane = threadIdx.x & 31;
    int64_t o = soff[sl];
    SliceRow q = slice_row(srow, sl, lane, lpr);
    T br = q.write ? b[q.r] : T(0), dr = q.write ? dinv[q.r] : T(0);
    T sum = row_reduce(sell_part<T, CH>(ci, v, o, (soff[sl + 1] - o) / (SELL_C * CH), lane, x), lpr);
    if (q.write) x[q.r] += (br - sum) * dr;
}
// r = b - A x over all slices
template <typename T, int CH>
__global__ void __launch_bounds__(256)
k_sell_resid(const int64_t* __restrict__ soff, const int32_t* __restrict__ srow, int64_t nslice, int lpr,
             const int32_t* __restrict__ ci, const T* __restrict__ v, const T* __restrict__ b,
             const T* __restrict__ x, T* __restrict__ r) {
    pdl_enter();
    int64_t sl = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (sl >= nslice) return;
    int lane = threadIdx.x & 31;
    int64_t o = soff[sl];
    SliceRow q = slice_row(srow, sl, lane, lpr);
    T br = q.write ? b[q.r] : T(0);
    T sum = row_reduce(sell_part<T, CH>(ci, v, o, (soff[sl + 1] - o) / (SELL_C * CH), lane, x), lpr);
    if (q.write) r[q.r] = br - sum;
}
// y = alpha A x (+ y)
template <typename T, int CH>
__global__ void __launch_bounds__(256)
k_sell_spmv(const int64_t* __restrict__ soff, const int32_t* __restrict__ srow, int64_t nslice, int lpr,
            const int32_t* __restrict__ ci, const T* __restrict__ v, const T* __restrict__ x, T* y, int accumulate,
            T alpha) {
    pdl_enter();
    int64_t sl = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (sl >= nslice) return;
    int lane = threadIdx.x & 31;
    int64_t o = soff[sl];
    SliceRow q = slice_row(srow, sl, lane, lpr);
    T sum = row_reduce(sell_part<T, CH>(ci, v, o, (soff[sl + 1] - o) / (SELL_C * CH), lane, x), lpr);
    if (q.write) y[q.r] = accumulate ? y[q.r] + alpha * sum : alpha * sum;
}
// A whole forward + backward sweep of a small operator in one block: colours are separated by
// block barriers instead of kernel boundaries (the coarse levels are launch-bound otherwise).
template <typename T, int CH>
__global__ void __launch_bounds__(1024)
k_sell_sgs_block(const int64_t* __restrict__ soff, const int32_t* __restrict__ srow,
                 const int64_t* __restrict__ cslice, int ncolor, int lpr, const int32_t* __restrict__ ci,
                 const T* __restrict__ v, const T* __restrict__ dinv, const T* __restrict__ b, T* x) {
    pdl_enter();
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    for (int step = 0; step < sweep_steps(ncolor); ++step) {
        int c = sweep_colour(step, ncolor);
        for (int64_t sl = cslice[c] + warp; sl < cslice[c + 1]; sl += nwarp) {
            int64_t o = soff[sl];
            SliceRow q = slice_row(srow, sl, lane, lpr);
            T sum = row_reduce(sell_part<T, CH>(ci, v, o, (soff[sl + 1] - o) / (SELL_C * CH), lane, x), lpr);
            if (q.write) x[q.r] += (b[q.r] - sum) * dinv[q.r];
        }
        __syncthreads();
    }
}

// A whole forward + backward sweep of a mid-sized operator (x small enough for shared memory) on
// one thread-block cluster.  Every CTA keeps a copy of x in its shared memory; the new value of a
// row is stored into every copy through distributed shared memory, and a cluster barrier (release
// / acquire) separates the colours.  The gathers of x then hit shared memory and the colours cost
// a cluster barrier instead of a kernel boundary.  Warp gw of the cluster takes the slices
// gw, gw + nw, ... of each colour and loads the head of its next slice before the barrier.  At
// the end every copy holds the result; each CTA writes back a share.
// (A deeper per-warp pipeline, with the bounds of the slice after next also in flight, measured
// slower: 1.19 against 0.81 ms for the level-2 pre-smoothing of the 128^3 problem.)
static constexpr int SGS_CLUSTER = 8;
// threads per CTA: 1024 (64 registers) for FP32, 512 for FP64, which needs more registers
template <typename T>
struct SgsClusterThreads {
    static constexpr int value = sizeof(T) == 4 ? 1024 : 512;
};
static constexpr int64_t SGS_CLUSTER_MAX_BYTES = 200 * 1024;
template <typename T, int CH>
__global__ void __launch_bounds__(SgsClusterThreads<T>::value)
k_sell_sgs_cluster(const int64_t* __restrict__ soff, const int32_t* __restrict__ srow,
                   const int64_t* __restrict__ cslice, int ncolor, int lpr, int64_t n,
                   const int32_t* __restrict__ ci, const T* __restrict__ v, const T* __restrict__ dinv,
                   const T* __restrict__ b, T* __restrict__ x) {
    extern __shared__ __align__(16) unsigned char sgs_smem[];
    T* xs = reinterpret_cast<T*>(sgs_smem);
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank(), ncta = (int)cl.num_blocks();
    const int lane = threadIdx.x & 31;
    const int64_t gw = (int64_t)rank * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int64_t nw = (int64_t)ncta * (blockDim.x >> 5);
    // the warp's current slice: its head loads, its row, and (after the wait) b_r and 1 / a_rr
    int64_t sl = 0, end = 0, o = 0, steps = 0;
    int32_t r = 0;
    bool have = false, valid = false;
    T br = 0, dr = 0;
    SellHead<T, CH> h;
    h.n = 0;
    auto fetch = [&](int64_t s_, int64_t e_, bool rhs) {
        sl = s_;
        end = e_;
        have = sl < end;
        if (!have) return;
        o = soff[sl];
        steps = (soff[sl + 1] - o) / (SELL_C * CH);
        r = srow[sl] + lane / lpr;
        valid = r < srow[sl + 1];
        h.load(ci, v, o, steps, lane);
        if (rhs && valid) { br = b[r]; dr = dinv[r]; }
    };
    fetch(cslice[0] + gw, cslice[1], false);          // matrix only before the wait
    pdl_enter();
    if (have && valid) { br = b[r]; dr = dinv[r]; }
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) xs[i] = x[i];
    cl.sync();
    for (int step = 0; step < sweep_steps(ncolor); ++step) {
        while (have) {
            T sum = row_reduce(h.finish(ci, v, o, steps, lane, xs), lpr);
            if (valid) {
                T xn = xs[r] + (br - sum) * dr;
                for (int k = lane & (lpr - 1); k < ncta; k += lpr) *cl.map_shared_rank(xs + r, k) = xn;
            }
            fetch(sl + nw, end, true);
        }
        if (step + 1 < sweep_steps(ncolor)) {            // head of the next colour's first slice
            const int cn = sweep_colour(step + 1, ncolor);
            fetch(cslice[cn] + gw, cslice[cn + 1], true);
        }
        cl.sync();
    }
    for (int64_t i = (int64_t)rank * blockDim.x + threadIdx.x; i < n; i += (int64_t)ncta * blockDim.x) x[i] = xs[i];
}

// A whole forward + backward sweep of a large operator as one persistent kernel: every CTA of a
// co-resident (cooperative) grid works on each colour in turn, and a grid barrier replaces the
// kernel boundary between colours.  Mid-sized levels (tens of colours of a few thousand rows each)
// are latency-bound when every colour is its own launch: the launch, the drain of the previous
// kernel and the first loads of the matrix make up most of a colour.  Here the head of each warp's
// first slice of the next colour (matrix entries, b and 1 / a_rr) is loaded before the barrier, so
// a colour costs the gathers of x, the update and the barrier.  x stays in global memory (L2) and
// is read through L2 only; every CTA writes the rows it updates.
//
// The barrier counts arrivals in bar->count; the last CTA to arrive resets it and advances
// bar->gen (release); the others poll gen (acquire).  Every poll loop has an iteration limit: a
// CTA that gives up, or sees another CTA's give-up in bar->err, sets bar->err and leaves the
// kernel, so all CTAs return and the host reads the error word after the solve.
template <typename T>
struct SgsGridThreads {
    static constexpr int value = sizeof(T) == 4 ? 1024 : 512;
};
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// every thread of every CTA calls it; false when a wait gave up (the caller returns)
__device__ __forceinline__ bool grid_barrier(GridBar* bar, unsigned nblocks, unsigned max_polls) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned g = ld_acquire_u32(&bar->gen);      // cannot advance before this CTA arrives
        __threadfence();                                   // the CTA's writes (ordered by the block barrier)
        if (atomicAdd(&bar->count, 1u) == nblocks - 1) {
            atomicExch(&bar->count, 0u);
            st_release_u32(&bar->gen, g + 1);
        } else {
            for (unsigned polls = 0; ld_acquire_u32(&bar->gen) == g; ++polls) {
                if (*(volatile int*)&bar->err != 0 || polls >= max_polls) {
                    atomicExch(&bar->err, 1);
                    ok = 0;
                    break;
                }
                if (polls >= 1024) __nanosleep(64);
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}
template <typename T, int CH>
__global__ void __launch_bounds__(SgsGridThreads<T>::value)
k_sell_sgs_grid(const int64_t* __restrict__ soff, const int32_t* __restrict__ srow,
                const int64_t* __restrict__ cslice, int ncolor, int lpr, const int32_t* __restrict__ ci,
                const T* __restrict__ v, const T* __restrict__ dinv, const T* __restrict__ b, T* x, GridBar* bar,
                unsigned max_polls) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    const L2Read<T> xr{x};
    int64_t sl = 0, end = 0, o = 0, steps = 0;
    int32_t r = 0;
    bool have = false, valid = false;
    T br = 0, dr = 0;
    SellHead<T, CH> h;
    h.n = 0;
    auto fetch = [&](int64_t s_, int64_t e_) {
        sl = s_;
        end = e_;
        have = sl < end;
        if (!have) return;
        o = soff[sl];
        steps = (soff[sl + 1] - o) / (SELL_C * CH);
        r = srow[sl] + lane / lpr;
        valid = r < srow[sl + 1];
        h.load(ci, v, o, steps, lane);
        if (valid) { br = b[r]; dr = dinv[r]; }
    };
    fetch(cslice[0] + gw, cslice[1]);
    for (int step = 0; step < sweep_steps(ncolor); ++step) {
        while (have) {
            T sum = row_reduce(h.finish(ci, v, o, steps, lane, xr), lpr);
            if (valid && (lane & (lpr - 1)) == 0) x[r] = xr[r] + (br - sum) * dr;
            fetch(sl + nw, end);
        }
        if (step + 1 < sweep_steps(ncolor)) {            // head of the next colour's first slice
            const int cn = sweep_colour(step + 1, ncolor);
            fetch(cslice[cn] + gw, cslice[cn + 1]);
            if (!grid_barrier(bar, gridDim.x, max_polls)) return;
        }
    }
}

template <typename T, int SUB>
__global__ void k_spmv_v(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci, const T* __restrict__ v,
                         int64_t n, const T* __restrict__ x, T* y, int accumulate, T alpha) {
    pdl_enter();
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
// The same product for short rows (up to a few dozen entries): a warp takes 32 consecutive rows,
// whose entries are one contiguous range.  The warp streams that range in tiles of 32 * ROWS_U
// entries (coalesced loads, ROWS_U per lane in flight before the gathers), stages the products in
// shared memory, and lane k then sums row k's products in entry order.  Lanes per row with strided
// loops keep one load per lane in flight, which leaves the fine-level prolongation latency-bound.
static constexpr int ROWS_U = 16, ROWS_WARPS = 8;
template <typename T>
__global__ void __launch_bounds__(ROWS_WARPS * 32)
k_spmv_rows32(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci, const T* __restrict__ v, int64_t n,
              const T* __restrict__ x, T* y, int accumulate, T alpha) {
    constexpr int TILE = 32 * ROWS_U;
    __shared__ T sp[ROWS_WARPS][TILE];
    pdl_enter();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t r0 = ((int64_t)blockIdx.x * ROWS_WARPS + w) * 32;
    if (r0 >= n) return;                                   // uniform over the warp
    const int64_t r = r0 + lane;
    const int nrow = (int)(n - r0 < 32 ? n - r0 : 32);
    const bool valid = lane < nrow;
    const int32_t rs = valid ? rp[r] : 0, re = valid ? rp[r + 1] : 0;
    const int32_t e0 = __shfl_sync(0xffffffffu, rs, 0), e1 = __shfl_sync(0xffffffffu, re, nrow - 1);
    T* s = sp[w];
    T sum = 0;
    for (int32_t t0 = e0; t0 < e1; t0 += TILE) {
        const int32_t tn = e1 - t0 < TILE ? e1 - t0 : TILE;
        T a[ROWS_U];
        int32_t c[ROWS_U];
#pragma unroll
        for (int u = 0; u < ROWS_U; ++u)
            if (u * 32 + lane < tn) {
                a[u] = __ldcs(v + t0 + u * 32 + lane);
                c[u] = __ldcs(ci + t0 + u * 32 + lane);
            }
#pragma unroll
        for (int u = 0; u < ROWS_U; ++u)
            if (u * 32 + lane < tn) s[u * 32 + lane] = a[u] * x[c[u]];
        __syncwarp();
        const int32_t lo = (rs > t0 ? rs : t0) - t0, hi = (re < t0 + tn ? re : t0 + tn) - t0;
        for (int32_t k = lo; k < hi; ++k) sum += s[k];
        __syncwarp();
    }
    if (valid) y[r] = accumulate ? y[r] + alpha * sum : alpha * sum;
}

template <typename T>
__global__ void k_dt_gather(const int32_t* __restrict__ rp, const int32_t* __restrict__ enc, int64_t nv,
                            const T* __restrict__ r, T* __restrict__ g) {
    pdl_enter();
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
    pdl_enter();
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
    pdl_enter();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = 0;
}
template <typename A, typename B>
__global__ void k_cast(const A* a, B* b, int64_t n) {
    pdl_enter();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (B)a[i];
}
// x = Ainv b on the coarsest level (FP64 arithmetic)
template <typename T>
__global__ void k_dense_solve(const double* __restrict__ Ainv, int64_t n, const T* __restrict__ b, T* __restrict__ x) {
    pdl_enter();
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

static unsigned slice_grid(int64_t nslice) { return (unsigned)grid_for(nslice * 32, 256); }

#define SPHC_CH_SWITCH(ch, F) \
    switch (ch) {             \
        case 1: F(1); break;  \
        case 2: F(2); break;  \
        default: F(4); break; \
    }

// one launch of the cluster sweep (shared memory for x; programmatic launch outside capture)
template <typename T, int CH>
static cudaError_t launch_sgs_cluster(const SmoothOp<T>& op, const T* b, T* x, cudaStream_t s) {
    const Sell<T>& m = op.m;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(SGS_CLUSTER);
    cfg.blockDim = dim3(SgsClusterThreads<T>::value);
    cfg.dynamicSmemBytes = (size_t)op.n * sizeof(T);
    cfg.stream = s;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(s, &cap);
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = SGS_CLUSTER;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[1].val.programmaticStreamSerializationAllowed = cap == cudaStreamCaptureStatusNone ? 1 : 0;
    cfg.attrs = at;
    cfg.numAttrs = 2;
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaLaunchKernelEx(&cfg, k_sell_sgs_cluster<T, CH>, m.soff.p, m.srow.p, op.cslice_dev.p, op.ncolor, m.lpr,
                              op.n, m.ci.p, m.v.p, op.dinv.p, b, x);
}
// Whether the cluster sweep can run op on this device: x fits the shared memory of a CTA and a
// cluster of that shape can be resident (sets the kernels' shared-memory limit on the way).
template <typename T>
static bool cluster_sgs_fits(const SmoothOp<T>& op) {
    if (op.n <= SGS_BLOCK_MAX_ROWS || (int64_t)op.n * (int64_t)sizeof(T) > SGS_CLUSTER_MAX_BYTES) return false;
    void (*ks[3])(const int64_t*, const int32_t*, const int64_t*, int, int, int64_t, const int32_t*, const T*,
                  const T*, const T*, T*) = {k_sell_sgs_cluster<T, 1>, k_sell_sgs_cluster<T, 2>,
                                             k_sell_sgs_cluster<T, 4>};
    for (auto k : ks)
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SGS_CLUSTER_MAX_BYTES) !=
            cudaSuccess) {
            cudaGetLastError();
            return false;
        }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(SGS_CLUSTER);
    cfg.blockDim = dim3(SgsClusterThreads<T>::value);
    cfg.dynamicSmemBytes = (size_t)op.n * sizeof(T);
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = SGS_CLUSTER;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nclus = 0;
    if (cudaOccupancyMaxActiveClusters(&nclus, ks[0], &cfg) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return nclus > 0;
}
// Sweep cost model used without the autotuner (microseconds per forward + backward sweep), from
// the 128^3 level-2 smoother (6.6K rows, 73 colours): a colour launch costs about 4 us of latency
// and the launches stream at HBM speed; the cluster sweep pays about 2 us per colour and streams
// at the bandwidth of its 8 SMs.
template <typename T>
static bool cluster_sgs_preferred(const SmoothOp<T>& op) {
    double bytes = (double)op.m.stored * (sizeof(T) + 4);
    double t_launch = 2.0 * op.ncolor * 4.0 + 2.0 * bytes / 5.0e6;
    double t_cluster = 2.0 * op.ncolor * 2.0 + 2.0 * bytes / 0.5e6;
    return t_cluster < t_launch && cluster_sgs_fits(op);
}
// the sweep form of op under sphc_opts.sweep_form
template <typename T>
static bool cluster_sgs_chosen(const SmoothOp<T>& op, int sweep_form) {
    if (sweep_form == 1 || sweep_form == 3) return false;
    if (sweep_form == 2) return cluster_sgs_fits(op);
    return cluster_sgs_preferred(op);
}

// The grid barrier on its own: `rounds` barriers of a cooperative grid that counts `extra`
// arrivals more than it has CTAs (extra > 0: a wait nothing can end, so every CTA gives up after
// max_polls polls and sets bar->err).
__global__ void k_grid_barrier_check(GridBar* bar, unsigned extra, unsigned max_polls, int rounds) {
    for (int k = 0; k < rounds; ++k)
        if (!grid_barrier(bar, gridDim.x + extra, max_polls)) return;
}
int grid_barrier_check(int extra, unsigned max_polls, int* timed_out, cudaStream_t s) {
    int dev = 0, nsm = 0, coop = 0, per_sm = 0;
    SPHC_CK(cudaGetDevice(&dev));
    SPHC_CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    SPHC_CK(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
    SPHC_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_grid_barrier_check, 256, 0));
    if (!coop || per_sm < 1) {
        set_error("grid barrier check: the device does not run cooperative launches");
        return SPHC_EINVAL;
    }
    DBuf<GridBar> bar;
    SPHC_TRY(bar.alloc(1, s));
    SPHC_TRY(bar.zero(s));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nsm * per_sm);
    cfg.blockDim = dim3(256);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    g_launches.fetch_add(1, std::memory_order_relaxed);
    SPHC_CK(cudaLaunchKernelEx(&cfg, k_grid_barrier_check, bar.p, (unsigned)extra, max_polls, 3));
    GridBar hb = {};
    SPHC_CK(cudaMemcpyAsync(&hb, bar.p, sizeof(GridBar), cudaMemcpyDeviceToHost, s));
    SPHC_CK(cudaStreamSynchronize(s));
    *timed_out = hb.err != 0;
    return SPHC_OK;
}

// one cooperative launch of the grid sweep (one CTA per resident slot; the cooperative launch
// makes the runtime check that the whole grid is resident at once)
template <typename T, int CH>
static cudaError_t launch_sgs_grid(const SmoothOp<T>& op, const T* b, T* x, cudaStream_t s) {
    const Sell<T>& m = op.m;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(op.grid);
    cfg.blockDim = dim3(SgsGridThreads<T>::value);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaLaunchKernelEx(&cfg, k_sell_sgs_grid<T, CH>, m.soff.p, m.srow.p, op.cslice_dev.p, op.ncolor, m.lpr,
                              m.ci.p, m.v.p, op.dinv.p, b, x, op.bar, op.polls);
}
// CTAs of op's grid sweep that can be resident at once on this device (0: it cannot run)
template <typename T>
static int grid_sgs_blocks(const SmoothOp<T>& op) {
    void (*k)(const int64_t*, const int32_t*, const int64_t*, int, int, const int32_t*, const T*, const T*,
              const T*, T*, GridBar*, unsigned) =
        op.m.ch == 1 ? k_sell_sgs_grid<T, 1> : (op.m.ch == 2 ? k_sell_sgs_grid<T, 2> : k_sell_sgs_grid<T, 4>);
    int dev = 0, nsm = 0, coop = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, SgsGridThreads<T>::value, 0) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return coop ? nsm * per_sm : 0;
}
// Whether the grid sweep runs op: only where sphc_opts.sweep_form 3 asks for it, for every
// smoother above one block.  The cost model does not pick it: on the 128^3 problem's level 1
// (571K rows, 47 colours of about 8 MB of matrix each) a colour took about 12 us in the grid
// sweep against 8.7 us as its own launch.  The grid barrier alone costs 2.7 us (152 CTAs), and one
// CTA of 1024 threads per SM keeps fewer matrix loads in flight than a launch of the whole colour.
template <typename T>
static int grid_sgs_chosen(const SmoothOp<T>& op, int sweep_form) {
    if (sweep_form != 3 || op.n <= SGS_BLOCK_MAX_ROWS || op.ncolor < 2) return 0;
    return grid_sgs_blocks(op);
}

// Grid sweeps are not captured into the batched solve's multi-branch graph (its branches run
// concurrently and persistent grids would compete for the SMs): capture_cg turns them off on its
// thread while it captures.
static thread_local bool g_grid_sweep_off = false;

template <typename T>
static void sgs(const SmoothOp<T>& op, const T* b, T* x, cudaStream_t s) {
    const Sell<T>& m = op.m;
    if (op.n == 0) return;
    if (op.cluster) {
#define F(C) launch_sgs_cluster<T, C>(op, b, x, s)
        SPHC_CH_SWITCH(m.ch, F)
#undef F
        return;
    }
    if (op.grid && op.bar && !g_grid_sweep_off) {
#define F(C) launch_sgs_grid<T, C>(op, b, x, s)
        SPHC_CH_SWITCH(m.ch, F)
#undef F
        return;
    }
    if (op.n <= SGS_BLOCK_MAX_ROWS) {
#define F(C) launch_pdl(k_sell_sgs_block<T, C>, 1, 1024, 0, s, m.soff.p, m.srow.p, op.cslice_dev.p, op.ncolor, m.lpr, m.ci.p, m.v.p, op.dinv.p, b, x)
        SPHC_CH_SWITCH(m.ch, F)
#undef F
        return;
    }
    for (int step = 0; step < sweep_steps(op.ncolor); ++step) {
        int c = sweep_colour(step, op.ncolor);
        int64_t s0 = op.cslice[c], s1 = op.cslice[c + 1];
        if (s1 <= s0) continue;
#define F(C) launch_pdl(k_sell_sgs<T, C>, slice_grid(s1 - s0), 256, 0, s, m.soff.p, m.srow.p, s0, s1, m.lpr, m.ci.p, m.v.p, op.dinv.p, b, x)
        SPHC_CH_SWITCH(m.ch, F)
#undef F
    }
}
template <typename T>
static void resid(const SmoothOp<T>& op, const T* b, const T* x, T* r, cudaStream_t s) {
    const Sell<T>& m = op.m;
    if (m.nslice == 0) return;
#define F(C) launch_pdl(k_sell_resid<T, C>, slice_grid(m.nslice), 256, 0, s, m.soff.p, m.srow.p, m.nslice, m.lpr, m.ci.p, m.v.p, b, x, r)
    SPHC_CH_SWITCH(m.ch, F)
#undef F
}
template <typename T>
static void sell_spmv(const Sell<T>& m, const T* x, T* y, int acc, cudaStream_t s, T alpha = T(1)) {
    if (m.nslice == 0) return;
#define F(C) launch_pdl(k_sell_spmv<T, C>, slice_grid(m.nslice), 256, 0, s, m.soff.p, m.srow.p, m.nslice, m.lpr, m.ci.p, m.v.p, x, y, acc, alpha)
    SPHC_CH_SWITCH(m.ch, F)
#undef F
}
template <typename T>
static void spmv_v(const XOp<T>& X, const T* x, T* y, int acc, cudaStream_t s, T alpha = T(1)) {
    if (X.nr == 0) return;
    if (X.sell) {
        sell_spmv<T>(X.s, x, y, acc, s, alpha);
        return;
    }
    const VCSR<T>& A = X.c;
    if (A.rows32) {
        launch_pdl(k_spmv_rows32<T>, (unsigned)((A.nr + 32 * ROWS_WARPS - 1) / (32 * ROWS_WARPS)), ROWS_WARPS * 32, 0, s,
                   A.rp.p, A.ci.p, A.v.p, A.nr, x, y, acc, alpha);
        return;
    }
    int sub = sub_for(A.nnz, A.nr);
    int64_t th = A.nr * sub;
    switch (sub) {
        case 4: launch_pdl(k_spmv_v<T, 4>, grid_for(th, 256), 256, 0, s, A.rp.p, A.ci.p, A.v.p, A.nr, x, y, acc, alpha); break;
        case 8: launch_pdl(k_spmv_v<T, 8>, grid_for(th, 256), 256, 0, s, A.rp.p, A.ci.p, A.v.p, A.nr, x, y, acc, alpha); break;
        case 16: launch_pdl(k_spmv_v<T, 16>, grid_for(th, 256), 256, 0, s, A.rp.p, A.ci.p, A.v.p, A.nr, x, y, acc, alpha); break;
        default: launch_pdl(k_spmv_v<T, 32>, grid_for(th, 256), 256, 0, s, A.rp.p, A.ci.p, A.v.p, A.nr, x, y, acc, alpha); break;
    }
}
// y = A x for CG (FP64, level-0 V-cycle numbering)
static int cg_spmv(const Hierarchy& H, const double* x, double* y, cudaStream_t s) {
    sell_spmv<double>(cg_op(H), x, y, 0, s);
    SPHC_CK(cudaGetLastError());
    return SPHC_OK;
}

// algorithmic bytes of one forward + backward sweep: the matrix (values and column indices)
// once per direction and, per row, its right side, inverse diagonal and one read and write of x;
// the last colour is swept once
template <typename T>
static double sgs_bytes(const SmoothOp<T>& op) {
    return (2.0 * (double)op.nnz - (double)op.nnz_last) * (sizeof(T) + 4) +
           (2.0 * (double)op.n - (double)op.n_last) * 4.0 * sizeof(T);
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
        launch_pdl(k_dt_gather<T>, grid_for(nv, 256), 256, 0, s, V.Dt_rp.p, V.Dt_e.p, nv, V.r.p, V.g.p);
        launch_pdl(k_zero<T>, grid_for(nv, 256), 256, 0, s, V.c.p, nv);
        sgs(V.An, V.g.p, V.c.p, s);
        launch_pdl(k_d_apply<T>, grid_for(ne, 256), 256, 0, s, V.D.p, ne, V.c.p, V.x.p);
    }
    timed_sgs(H, lev, V.A, V.b.p, V.x.p, s);
}

template <typename T>
static void vcycle_level(Hierarchy& H, std::vector<VLevel<T>>& V, int l, cudaStream_t s) {
    int64_t ne = H.L[l].A.nr, nv = H.L[l].An.nr;
    if (l == H.nlev - 1) {
        if (ne > 0) launch_pdl(k_dense_solve<T>, grid_for(ne * 32, 256), 256, 0, s, H.coarse_inv.p, ne, V[l].b.p, V[l].x.p);
        return;
    }
    launch_pdl(k_zero<T>, grid_for(ne, 256), 256, 0, s, V[l].x.p, ne);
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
    pdl_enter();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] += x[i];
}
template <typename T>
__global__ void k_copy(T* y, const T* x, int64_t n) {
    pdl_enter();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = x[i];
}
// z = y + D c in FP64
template <typename T>
__global__ void k_combine(const T* __restrict__ y, const int2* __restrict__ D, const T* __restrict__ c, int64_t n,
                          double* __restrict__ z) {
    pdl_enter();
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    int2 d = D[e];
    double v = (double)y[e];
    if (d.y >= 0) v += (double)c[d.y];
    if (d.x >= 0) v -= (double)c[d.x];
    z[e] = v;
}
__global__ void k_dense_mv64(const double* __restrict__ M, int64_t n, const double* __restrict__ b, double* __restrict__ x) {
    pdl_enter();
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
    pdl_enter();
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
    launch_pdl(k_cast<T, double>, grid_for(ne, 256), 256, 0, s, V.b.p, H.cb.p, ne);
    launch_pdl(k_dense_mv64, grid_for(ne * 32, 256), 256, 0, s, H.coarse_inv.p, ne, H.cb.p, H.cx.p);
    if (nv > 0) {
        launch_pdl(k_dt_gather<double>, grid_for(nv, 256), 256, 0, s, V.Dt_rp.p, V.Dt_e.p, nv, H.cb.p, H.cgn.p);
        launch_pdl(k_dense_mv64, grid_for(nv * 32, 256), 256, 0, s, H.coarse_inv_n.p, nv, H.cgn.p, H.ccn.p);
    }
    int64_t m = ne > nv ? ne : nv;
    launch_pdl(k_split_out<T>, grid_for(m, 256), 256, 0, s, H.cx.p, V.D.p, H.ccn.p, ne, nv, V.x.p, V.c.p);
}

template <typename T>
static void hiptmair_split(Hierarchy& H, int lev, VLevel<T>& V, int64_t ne, int64_t nv, cudaStream_t s) {
    timed_sgs(H, lev, V.A, V.bp.p, V.x.p, s);
    if (nv > 0) {
        resid(V.A, V.bp.p, V.x.p, V.r.p, s);
        launch_pdl(k_dt_gather<T>, grid_for(nv, 256), 256, 0, s, V.Dt_rp.p, V.Dt_e.p, nv, V.r.p, V.g.p);
        launch_pdl(k_zero<T>, grid_for(nv, 256), 256, 0, s, V.dc.p, nv);
        sgs(V.An, V.g.p, V.dc.p, s);
        launch_pdl(k_axpy<T>, grid_for(nv, 256), 256, 0, s, V.c.p, V.dc.p, nv);
        spmv_v(V.AD, V.dc.p, V.bp.p, 1, s, T(-1));
    }
    timed_sgs(H, lev, V.A, V.bp.p, V.x.p, s);
}

// per-level section timers of the V-cycle (profile on, outside graph capture)
static Profiler* vc_prof(Hierarchy& H) { return H.prof.on && !H.capturing ? &H.prof : nullptr; }
static std::string vc_name(const char* what, int l) { return std::string(what) + "_l" + std::to_string(l); }

template <typename T>
static void vcycle_split(Hierarchy& H, std::vector<VLevel<T>>& V, int l, cudaStream_t s) {
    int64_t ne = H.L[l].A.nr, nv = H.L[l].An.nr;
    Profiler* pr = vc_prof(H);
    if (l == H.nlev - 1) {
        Section sec(pr, "vc_coarsest", s);
        coarse_split(H, V[l], ne, nv, s);
        return;
    }
    {
        Section sec(pr, vc_name("vc_pre", l).c_str(), s);
        launch_pdl(k_zero<T>, grid_for(ne, 256), 256, 0, s, V[l].x.p, ne);
        if (nv > 0) launch_pdl(k_zero<T>, grid_for(nv, 256), 256, 0, s, V[l].c.p, nv);
        launch_pdl(k_copy<T>, grid_for(ne, 256), 256, 0, s, V[l].bp.p, V[l].b.p, ne);
        hiptmair_split(H, l, V[l], ne, nv, s);
    }
    {
        Section sec(pr, vc_name("vc_restrict", l).c_str(), s);
        resid(V[l].A, V[l].bp.p, V[l].x.p, V[l].r.p, s);
        spmv_v(V[l].PeT, V[l].r.p, V[l + 1].b.p, 0, s);
    }
    vcycle_split(H, V, l + 1, s);
    {
        Section sec(pr, vc_name("vc_prolong", l).c_str(), s);
        spmv_v(V[l].Pe, V[l + 1].x.p, V[l].x.p, 1, s);           // y += P_e y_H
        if (nv > 0) {
            spmv_v(V[l].Pn, V[l + 1].c.p, V[l].dc.p, 0, s);      // c += P_n c_H  (P_e D_H = D_h P_n)
            launch_pdl(k_axpy<T>, grid_for(nv, 256), 256, 0, s, V[l].c.p, V[l].dc.p, nv);
            spmv_v(V[l].AD, V[l].dc.p, V[l].bp.p, 1, s, T(-1));
        }
    }
    {
        Section sec(pr, vc_name("vc_post", l).c_str(), s);
        hiptmair_split(H, l, V[l], ne, nv, s);
    }
}

int apply_vcycle(Hierarchy& H, const double* r, double* z, cudaStream_t s) {
    int64_t n = H.L[0].A.nr;
    if (H.opts.vcycle_fp32) {
        launch_pdl(k_cast<double, float>, grid_for(n, 256), 256, 0, s, r, H.V32[0].b.p, n);
        vcycle_split<float>(H, H.V32, 0, s);
        launch_pdl(k_combine<float>, grid_for(n, 256), 256, 0, s, H.V32[0].x.p, H.V32[0].D.p, H.V32[0].c.p, n, z);
    } else {
        SPHC_CK(cudaMemcpyAsync(H.V64[0].b.p, r, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
        vcycle_level<double>(H, H.V64, 0, s);
        SPHC_CK(cudaMemcpyAsync(z, H.V64[0].x.p, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    }
    SPHC_CK(cudaGetLastError());
    return SPHC_OK;
}

// Autotuner: for every smoother too large for the one-block sweep, build its SELL copy with
// lanes per row in {l/2, l, 2l} (l from the mean row length) and 1, 2 or 4 entries per lane load,
// time three forward + backward sweeps of each and keep the fastest shape.
template <typename T>
static int autotune_op(const DCSR& A, const int32_t* rmap, const int32_t* cmap, const std::vector<int64_t>& cstart,
                       SmoothOp<T>& op, DBuf<T>& bvec, DBuf<T>& xvec, cudaStream_t s) {
    if (op.n <= SGS_BLOCK_MAX_ROWS || op.n > bvec.n || op.n > xvec.n) return SPHC_OK;
    cudaEvent_t e0, e1;
    SPHC_CK(cudaEventCreate(&e0));
    SPHC_CK(cudaEventCreate(&e1));
    launch_pdl(k_zero<T>, grid_for(op.n, 256), 256, 0, s, bvec.p, op.n);
    launch_pdl(k_zero<T>, grid_for(op.n, 256), 256, 0, s, xvec.p, op.n);
    int l0 = sell_lpr_for(A, (int)cstart.size() - 1);
    float best = 1e30f;
    op.grid = 0;                                      // the tuner chooses between the other forms
    int best_ch = op.m.ch, best_lpr = op.m.lpr, best_cluster = op.cluster;
    int rc = SPHC_OK;
    for (int lpr : {l0 / 2, l0, 2 * l0}) {
        if (lpr < 1 || lpr > SELL_C) continue;
        for (int ch : {1, 2, 4}) {
            if ((ch != op.m.ch || lpr != op.m.lpr) &&
                (rc = build_smooth<T>(A, rmap, cmap, cstart, ch, lpr, op, s)) != SPHC_OK)
                break;
            bool fits = cluster_sgs_fits(op);
            for (int cl = 0; cl <= (fits ? 1 : 0); ++cl) {
                op.cluster = cl;
                sgs(op, bvec.p, xvec.p, s);               // warm-up
                cudaEventRecord(e0, s);
                for (int rep = 0; rep < 3; ++rep) sgs(op, bvec.p, xvec.p, s);
                cudaEventRecord(e1, s);
                if (cudaEventSynchronize(e1) != cudaSuccess) { rc = SPHC_ECUDA; break; }
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (ms < best) { best = ms; best_ch = ch; best_lpr = lpr; best_cluster = cl; }
            }
            if (rc != SPHC_OK) break;
        }
        if (rc != SPHC_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != SPHC_OK) return rc;
    if (op.m.ch != best_ch || op.m.lpr != best_lpr)
        SPHC_TRY(build_smooth<T>(A, rmap, cmap, cstart, best_ch, best_lpr, op, s));
    op.cluster = best_cluster;
    return SPHC_OK;
}

template <typename T>
static int autotune_levels(Hierarchy& H, std::vector<VLevel<T>>& V, cudaStream_t s) {
    for (int l = 0; l + 1 < H.nlev; ++l) {
        const Level& L = H.L[l];
        const LevelOrder& O = H.ord[l];
        SPHC_TRY(autotune_op<T>(L.A, O.pe.p, O.ie.p, O.ce, V[l].A, V[l].b, V[l].x, s));
        SPHC_TRY(autotune_op<T>(L.An, O.pn.p, O.in.p, O.cn, V[l].An, V[l].g, V[l].c, s));
    }
    return SPHC_OK;
}

int autotune_vcycle(Hierarchy& H, cudaStream_t s) {
    if (H.opts.vcycle_fp32) return autotune_levels<float>(H, H.V32, s);
    return autotune_levels<double>(H, H.V64, s);
}

// ------------------------------------------------------------------ CG
// scal: 0 rz, 1 pq, 2 rr, 3 rz_new, 4 z.r_old, 5 bb
// x += alpha p, r -= alpha q.  *moved is set when some entry of x changed: an iteration that
// leaves every entry unchanged is the stagnation of Sec. 7 (two consecutive iterations with the
// same solution), which k_cg_check reports.
__global__ void k_cg_xr(double* x, double* r, double* rold, const double* p, const double* q, const double* sc,
                        int64_t n, int flexible, int* moved) {
    pdl_enter();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool changed = false;
    if (i < n) {
        double alpha = sc[1] > 0.0 ? sc[0] / sc[1] : 0.0;     // breakdown: leave x unchanged
        double xo = x[i], xn = xo + alpha * p[i];
        changed = xn != xo;
        x[i] = xn;
        if (flexible) rold[i] = r[i];
        r[i] -= alpha * q[i];
    }
    if (__syncthreads_or(changed) && threadIdx.x == 0 && *(volatile int*)moved == 0) *moved = 1;
}
__global__ void k_cg_p(double* p, const double* z, const double* sc, int64_t n, int flexible) {
    pdl_enter();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double beta = flexible ? (sc[3] - sc[4]) / sc[0] : sc[3] / sc[0];
    p[i] = z[i] + beta * p[i];
}
__global__ void k_cg_shift(double* sc) {
    pdl_enter();
    sc[0] = sc[3];
}
__global__ void k_sub(const double* b, double* q, int64_t n) {
    pdl_enter();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) q[i] = b[i] - q[i];
}

// end of one graph iteration: count it and keep looping while not converged, not broken down,
// not stagnated and below the iteration cap.  itc[1]: 0 converged, 1 breakdown, 2 cap reached,
// 4 stagnation (itc[2], set by k_cg_xr, was not: x did not change); itc[2] is cleared for the
// next iteration.
__global__ void k_cg_check(cudaGraphConditionalHandle hnd, const double* sc, int* itc, int max_iter) {
    pdl_enter();
    int it = itc[0] + 1;
    itc[0] = it;
    double pq = sc[1], rr = sc[2], lim = sc[7];
    unsigned cont = 1;
    if (!(pq > 0.0) || !isfinite(rr)) { itc[1] = 1; cont = 0; }
    else if (rr <= lim) { itc[1] = 0; cont = 0; }
    else if (itc[2] == 0) { itc[1] = 4; cont = 0; }
    else if (it >= max_iter) { itc[1] = 2; cont = 0; }
    itc[2] = 0;
    cudaGraphSetConditional(hnd, cont);
}
// status code of the CG control word itc[1]
static int cg_status(int code) {
    switch (code) {
        case 0: return SPHC_OK;
        case 1: return SPHC_EBREAKDOWN;
        case 4: return SPHC_ESTAGNATION;
        default: return SPHC_ENOTCONV;
    }
}
__global__ void k_set_limit(double* sc, double tol2) {
    pdl_enter();
    sc[7] = tol2 * sc[5];
}

// one CG iteration after the first: z = M^-1 r, p = z + beta p, q = A p, x += alpha p, r -= alpha q
static int cg_body(Hierarchy& H, cudaGraphConditionalHandle hnd, cudaStream_t s) {
    int64_t n = H.L[0].A.nr;
    int flexible = H.opts.flexible;
    double* sc = H.scal.p;
    SPHC_TRY(apply_vcycle(H, H.r.p, H.z.p, s));
    dot_buf(H, H.r.p, H.z.p, n, sc + 3, s);
    if (flexible) dot_buf(H, H.z.p, H.rold.p, n, sc + 4, s);
    launch_pdl(k_cg_p, grid_for(n, 256), 256, 0, s, H.p.p, H.z.p, sc, n, flexible);
    launch_pdl(k_cg_shift, 1, 1, 0, s, sc);
    SPHC_TRY(cg_spmv(H, H.p.p, H.q.p, s));
    dot_buf(H, H.p.p, H.q.p, n, sc + 1, s);
    launch_pdl(k_cg_xr, grid_for(n, 256), 256, 0, s, H.x.p, H.r.p, H.rold.p, H.p.p, H.q.p, sc, n, flexible, H.itc.p + 2);
    dot_buf(H, H.r.p, H.r.p, n, sc + 2, s);
    launch_pdl(k_cg_check, 1, 1, 0, s, hnd, sc, H.itc.p, H.opts.max_iter);
    SPHC_CK(cudaGetLastError());
    return SPHC_OK;
}

// Whether some smoother of H runs the grid sweep, and turning them all back into per-colour
// launches (the CG graph is then captured again).
template <typename T>
static bool any_grid(const std::vector<VLevel<T>>& V) {
    for (const auto& v : V)
        if (v.A.grid || v.An.grid) return true;
    return false;
}
template <typename T>
static void grid_off(std::vector<VLevel<T>>& V) {
    for (auto& v : V) v.A.grid = v.An.grid = 0;
}
static bool has_grid_sweeps(const Hierarchy& H) { return any_grid(H.V32) || any_grid(H.V64); }

// SPHC_ETIMEOUT when a grid sweep gave up at its barrier since the last check (the barrier is then
// reset for the next solve), else SPHC_OK.  Synchronises s.
int grid_sweep_status(Hierarchy& H, cudaStream_t s) {
    if (!H.gbar.p || !has_grid_sweeps(H)) return SPHC_OK;
    GridBar hb = {};
    SPHC_CK(cudaMemcpyAsync(&hb, H.gbar.p, sizeof(GridBar), cudaMemcpyDeviceToHost, s));
    SPHC_CK(cudaStreamSynchronize(s));
    if (hb.err == 0) return SPHC_OK;
    SPHC_TRY(H.gbar.zero(s));
    set_error("a smoother sweep gave up waiting at its grid barrier (%u polls): the V-cycle result is invalid",
              H.opts.grid_wait_polls > 0 ? (unsigned)H.opts.grid_wait_polls : GRID_BAR_POLLS);
    return SPHC_ETIMEOUT;
}

static int build_cg_graph_once(Hierarchy& H);
// The CG graph; if capturing the cooperative grid sweeps into it fails, they become per-colour
// launches and the graph is captured again.
static int build_cg_graph(Hierarchy& H) {
    const int rc = build_cg_graph_once(H);
    if (rc != SPHC_ECUDA || !has_grid_sweeps(H)) return rc;
    cudaGetLastError();
    if (H.cg_graph && !H.cg_exec) cudaGraphDestroy(H.cg_graph);
    H.cg_graph = nullptr;
    grid_off(H.V32);
    grid_off(H.V64);
    return build_cg_graph_once(H);
}

static int build_cg_graph_once(Hierarchy& H) {
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
    if (rc != SPHC_OK || e != cudaSuccess) {
        // the body graph of a failed capture is left as the runtime leaves it: the handle drops its
        // reference instead of destroying a graph whose state it does not know (a one-off leak)
        H.cg_graph = nullptr;
        if (rc != SPHC_OK) return rc;
        set_error("CG graph capture failed: %s", cudaGetErrorString(e));
        return SPHC_ECUDA;
    }
    SPHC_CK(cudaGraphInstantiate(&H.cg_exec, H.cg_graph, 0));
    return SPHC_OK;
}

// ||b - A x||^2 into scal[6]; x and bperm in the V-cycle numbering
static int true_residual(Hierarchy& H, const double* xp, cudaStream_t s) {
    int64_t n = H.L[0].A.nr;
    SPHC_TRY(cg_spmv(H, xp, H.q.p, s));
    launch_pdl(k_sub, grid_for(n, 256), 256, 0, s, H.bperm.p, H.q.p, n);
    dot_buf(H, H.q.p, H.q.p, n, H.scal.p + 6, s);
    return SPHC_OK;
}
static double read_relres(Hierarchy& H, double bnorm, cudaStream_t s) {
    double hr = 0.0;
    cudaMemcpyAsync(&hr, H.scal.p + 6, sizeof(double), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    return bnorm == 0.0 ? 0.0 : sqrt(hr) / bnorm;   // NaN for a non-finite b
}

static void cg_error(int status, int it) {
    if (status == SPHC_EBREAKDOWN) set_error("CG breakdown after %d iterations", it);
    else if (status == SPHC_ENOTCONV) set_error("CG did not reach the tolerance in %d iterations", it);
    else if (status == SPHC_ESTAGNATION)
        set_error("CG stagnated after %d iterations: an iteration left x unchanged (tolerance below the "
                  "FP64 rounding floor of this system)", it);
}

// CG on the device: the first iteration is enqueued directly, the rest run inside one graph
// launch whose while node repeats an iteration until the stopping test holds.  b and x are in
// the caller's numbering; the iteration runs in the level-0 V-cycle numbering.
static int pcg_graph(Hierarchy& H, const double* b, double* x, double tol, cudaStream_t s, int* iters,
                     double* relres) {
    int64_t n = H.L[0].A.nr;
    int flexible = H.opts.flexible;
    double* sc = H.scal.p;
    SPHC_TRY(build_cg_graph(H));
    SPHC_TRY(gather64(b, perm0(H), n, H.bperm.p, s));
    SPHC_CK(cudaMemsetAsync(H.x.p, 0, sizeof(double) * n, s));
    SPHC_CK(cudaMemcpyAsync(H.r.p, H.bperm.p, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    dot_buf(H, H.bperm.p, H.bperm.p, n, sc + 5, s);
    double hb = 0.0;
    SPHC_CK(cudaMemcpyAsync(&hb, sc + 5, sizeof(double), cudaMemcpyDeviceToHost, s));
    SPHC_CK(cudaStreamSynchronize(s));
    double bnorm = sqrt(hb);
    int status = SPHC_OK, it = 0;
    if (!(bnorm == 0.0)) {               // a non-finite b runs into the breakdown test of iteration 1
        SPHC_TRY(apply_vcycle(H, H.r.p, H.z.p, s));
        SPHC_CK(cudaMemcpyAsync(H.p.p, H.z.p, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
        dot_buf(H, H.r.p, H.z.p, n, sc + 0, s);
        {
            const Sell<double>& A = cg_op(H);
            Section sec(H.prof.on ? &H.prof : nullptr, "spmv_A_fp64", s, (double)A.nnz * 12.0 + (double)n * 16.0);
            SPHC_TRY(cg_spmv(H, H.p.p, H.q.p, s));
        }
        dot_buf(H, H.p.p, H.q.p, n, sc + 1, s);
        SPHC_CK(cudaMemsetAsync(H.itc.p + 2, 0, sizeof(int), s));
        launch_pdl(k_cg_xr, grid_for(n, 256), 256, 0, s, H.x.p, H.r.p, H.rold.p, H.p.p, H.q.p, sc, n, flexible,
                   H.itc.p + 2);
        dot_buf(H, H.r.p, H.r.p, n, sc + 2, s);
        launch_pdl(k_set_limit, 1, 1, 0, s, sc, tol * tol);
        int hmoved = 0;
        SPHC_CK(cudaMemcpyAsync(&hmoved, H.itc.p + 2, sizeof(int), cudaMemcpyDeviceToHost, s));
        int hi[3] = {1, 0, 0};
        SPHC_CK(cudaMemcpyAsync(H.itc.p, hi, 3 * sizeof(int), cudaMemcpyHostToDevice, s));
        double hsc[8];
        SPHC_CK(cudaMemcpyAsync(hsc, sc, 8 * sizeof(double), cudaMemcpyDeviceToHost, s));
        SPHC_CK(cudaStreamSynchronize(s));
        it = 1;
        if (!(hsc[1] > 0.0) || !std::isfinite(hsc[2])) status = SPHC_EBREAKDOWN;
        else if (hsc[2] <= hsc[7]) status = SPHC_OK;
        else if (!hmoved) status = SPHC_ESTAGNATION;
        else if (it >= H.opts.max_iter) status = SPHC_ENOTCONV;
        else {
            SPHC_CK(cudaGraphLaunch(H.cg_exec, s));
            SPHC_CK(cudaMemcpyAsync(hi, H.itc.p, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
            SPHC_CK(cudaStreamSynchronize(s));
            it = hi[0];
            status = cg_status(hi[1]);
            g_launches.fetch_add(H.body_launches * (long long)(it - 1));
        }
    }
    SPHC_TRY(scatter64(H.x.p, perm0(H), n, x, s));
    SPHC_TRY(true_residual(H, H.x.p, s));
    double rr = read_relres(H, bnorm, s);
    SPHC_CK(cudaGetLastError());
    if (iters) *iters = it;
    if (relres) *relres = rr;
    cg_error(status, it);
    SPHC_TRY(grid_sweep_status(H, s));
    return status;
}

// ------------------------------------------------------------------ CG captured whole (batched solves)
// The right side is read from H.bin and tol^2 from scal[8]; the solution is left in H.xo (both
// in the caller's numbering).  Every iteration (V-cycle first) runs inside a while node whose
// condition a prologue kernel sets, so the whole solve needs no host decision and can be one
// branch of a larger graph.
__global__ void k_cg_prep(cudaGraphConditionalHandle hnd, double* sc, int* itc) {
    pdl_enter();
    sc[7] = sc[8] * sc[5];
    sc[0] = 1.0;                         // rz of the previous iteration (p = 0 makes beta irrelevant)
    itc[0] = 0;
    const bool run = !(sc[5] == 0.0);    // b = 0 is converged; a non-finite b breaks down in iteration 1
    itc[1] = run ? 3 : 0;                // 3: running; 0: converged
    itc[2] = 0;
    cudaGraphSetConditional(hnd, run ? 1u : 0u);
}

static int cg_iter_body(Hierarchy& H, cudaGraphConditionalHandle hnd, cudaStream_t s) {
    int64_t n = H.L[0].A.nr;
    int flexible = H.opts.flexible;
    double* sc = H.scal.p;
    SPHC_TRY(apply_vcycle(H, H.r.p, H.z.p, s));
    dot_buf(H, H.r.p, H.z.p, n, sc + 3, s);
    if (flexible) dot_buf(H, H.z.p, H.rold.p, n, sc + 4, s);
    launch_pdl(k_cg_p, grid_for(n, 256), 256, 0, s, H.p.p, H.z.p, sc, n, flexible);
    launch_pdl(k_cg_shift, 1, 1, 0, s, sc);
    SPHC_TRY(cg_spmv(H, H.p.p, H.q.p, s));
    dot_buf(H, H.p.p, H.q.p, n, sc + 1, s);
    launch_pdl(k_cg_xr, grid_for(n, 256), 256, 0, s, H.x.p, H.r.p, H.rold.p, H.p.p, H.q.p, sc, n, flexible, H.itc.p + 2);
    dot_buf(H, H.r.p, H.r.p, n, sc + 2, s);
    launch_pdl(k_cg_check, 1, 1, 0, s, hnd, sc, H.itc.p, H.opts.max_iter);
    SPHC_CK(cudaGetLastError());
    return SPHC_OK;
}

// Append the whole CG of H to the graph being captured on stream s.
static int capture_cg_impl(Hierarchy& H, cudaStream_t s);
int capture_cg(Hierarchy& H, cudaStream_t s) {
    g_grid_sweep_off = true;
    const int rc = capture_cg_impl(H, s);
    g_grid_sweep_off = false;
    return rc;
}
static int capture_cg_impl(Hierarchy& H, cudaStream_t s) {
    int64_t n = H.L[0].A.nr;
    double* sc = H.scal.p;
    if (!H.cap_stream) SPHC_CK(cudaStreamCreateWithFlags(&H.cap_stream, cudaStreamNonBlocking));
    H.capturing = true;
    long long lstart = g_launches.load();
    SPHC_TRY(gather64(H.bin.p, perm0(H), n, H.bperm.p, s));
    SPHC_CK(cudaMemcpyAsync(H.r.p, H.bperm.p, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    SPHC_CK(cudaMemsetAsync(H.x.p, 0, sizeof(double) * n, s));
    SPHC_CK(cudaMemsetAsync(H.p.p, 0, sizeof(double) * n, s));
    SPHC_CK(cudaMemsetAsync(H.rold.p, 0, sizeof(double) * n, s));
    dot_buf(H, H.bperm.p, H.bperm.p, n, sc + 5, s);
    cudaStreamCaptureStatus st;
    cudaGraph_t g;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    SPHC_CK(cudaStreamGetCaptureInfo(s, &st, nullptr, &g, &deps, nullptr, &ndeps));
    cudaGraphConditionalHandle hnd;
    SPHC_CK(cudaGraphConditionalHandleCreate(&hnd, g, 0, 0));
    launch_pdl(k_cg_prep, 1, 1, 0, s, hnd, sc, H.itc.p);
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
    SPHC_TRY(scatter64(H.x.p, perm0(H), n, H.xo.p, s));
    SPHC_TRY(true_residual(H, H.x.p, s));
    H.capturing = false;
    H.branch_launches = g_launches.load() - lstart;   // counted when the graph runs
    g_launches.fetch_sub(H.branch_launches);
    SPHC_CK(cudaGetLastError());
    return SPHC_OK;
}

// CG with a host decision per iteration (no graph)
int pcg_solve(Hierarchy& H, const double* b, double* x, double tol, cudaStream_t s, int* iters, double* relres) {
    if (H.opts.cg_graph) return pcg_graph(H, b, x, tol, s, iters, relres);
    int64_t n = H.L[0].A.nr;
    int flexible = H.opts.flexible;
    double* sc = H.scal.p;
    SPHC_TRY(gather64(b, perm0(H), n, H.bperm.p, s));
    SPHC_CK(cudaMemsetAsync(H.x.p, 0, sizeof(double) * n, s));
    SPHC_CK(cudaMemcpyAsync(H.r.p, H.bperm.p, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    SPHC_TRY(dot64(H.bperm.p, H.bperm.p, n, sc + 5, s));
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
        const Sell<double>& A = cg_op(H);
        int tid = H.prof.on ? H.prof.find("spmv_A_fp64", (double)A.nnz * 12.0 + (double)n * 16.0) : -1;
        for (it = 0; it < H.opts.max_iter;) {
            if (tid >= 0) H.prof.begin(tid, s);
            SPHC_TRY(cg_spmv(H, H.p.p, H.q.p, s));
            if (tid >= 0) H.prof.end(tid, s);
            SPHC_TRY(dot64(H.p.p, H.q.p, n, sc + 1, s));
            SPHC_CK(cudaMemsetAsync(H.itc.p + 2, 0, sizeof(int), s));
            launch_pdl(k_cg_xr, grid_for(n, 256), 256, 0, s, H.x.p, H.r.p, H.rold.p, H.p.p, H.q.p, sc, n, flexible,
                       H.itc.p + 2);
            ++it;
            SPHC_TRY(dot64(H.r.p, H.r.p, n, sc + 2, s));
            int hmoved = 0;
            SPHC_CK(cudaMemcpyAsync(&hmoved, H.itc.p + 2, sizeof(int), cudaMemcpyDeviceToHost, s));
            SPHC_CK(cudaMemcpyAsync(hsc, sc, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
            SPHC_CK(cudaStreamSynchronize(s));
            if (!(hsc[1] > 0.0) || !std::isfinite(hsc[2])) { status = SPHC_EBREAKDOWN; break; }
            if (sqrt(hsc[2]) <= tol * bnorm) { status = SPHC_OK; break; }
            if (!hmoved) { status = SPHC_ESTAGNATION; break; }
            SPHC_TRY(apply_vcycle(H, H.r.p, H.z.p, s));
            SPHC_TRY(dot64(H.r.p, H.z.p, n, sc + 3, s));
            if (flexible) SPHC_TRY(dot64(H.z.p, H.rold.p, n, sc + 4, s));
            launch_pdl(k_cg_p, grid_for(n, 256), 256, 0, s, H.p.p, H.z.p, sc, n, flexible);
            launch_pdl(k_cg_shift, 1, 1, 0, s, sc);
        }
    }
    SPHC_TRY(scatter64(H.x.p, perm0(H), n, x, s));
    SPHC_TRY(true_residual(H, H.x.p, s));
    double rr = read_relres(H, bnorm, s);
    SPHC_CK(cudaGetLastError());
    if (iters) *iters = it;
    if (relres) *relres = rr;
    cg_error(status, it);
    SPHC_TRY(grid_sweep_status(H, s));
    return status;
}

// z = M^-1 r with r and z in the caller's numbering
int apply_vcycle_user(Hierarchy& H, const double* r, double* z, cudaStream_t s) {
    int64_t n = H.L[0].A.nr;
    SPHC_TRY(gather64(r, perm0(H), n, H.q.p, s));
    SPHC_TRY(apply_vcycle(H, H.q.p, H.z.p, s));
    SPHC_TRY(scatter64(H.z.p, perm0(H), n, z, s));
    return grid_sweep_status(H, s);
}

}  // namespace sphc
