// Device helpers of the sliced-ELLPACK (SELL-32) kernels, shared by the single-vector V-cycle
// (solve.cu) and the block right-hand-side path (block.cu).
#pragma once
#include "sphc_level.cuh"

namespace sphc {

// ------------------------------------------------------------------ V-cycle kernels
// Streaming loads of ch matrix entries (evict-first: the matrix is read once per sweep and should
// not push the iterate out of L2).
template <typename T, int CH> struct Chunk;
template <> struct Chunk<float, 1> {
    static __device__ __forceinline__ void load(const float* p, float* a) { a[0] = __ldcs(p); }
};
template <> struct Chunk<float, 2> {
    static __device__ __forceinline__ void load(const float* p, float* a) {
        float2 t = __ldcs(reinterpret_cast<const float2*>(p));
        a[0] = t.x; a[1] = t.y;
    }
};
template <> struct Chunk<float, 4> {
    static __device__ __forceinline__ void load(const float* p, float* a) {
        float4 t = __ldcs(reinterpret_cast<const float4*>(p));
        a[0] = t.x; a[1] = t.y; a[2] = t.z; a[3] = t.w;
    }
};
template <> struct Chunk<double, 1> {
    static __device__ __forceinline__ void load(const double* p, double* a) { a[0] = __ldcs(p); }
};
template <> struct Chunk<double, 2> {
    static __device__ __forceinline__ void load(const double* p, double* a) {
        double2 t = __ldcs(reinterpret_cast<const double2*>(p));
        a[0] = t.x; a[1] = t.y;
    }
};
template <> struct Chunk<double, 4> {
    static __device__ __forceinline__ void load(const double* p, double* a) {
        double2 t = __ldcs(reinterpret_cast<const double2*>(p));
        double2 u = __ldcs(reinterpret_cast<const double2*>(p) + 1);
        a[0] = t.x; a[1] = t.y; a[2] = u.x; a[3] = u.y;
    }
};
template <int CH> struct IChunk;
template <> struct IChunk<1> {
    static __device__ __forceinline__ void load(const int32_t* p, int32_t* c) { c[0] = __ldcs(p); }
};
template <> struct IChunk<2> {
    static __device__ __forceinline__ void load(const int32_t* p, int32_t* c) {
        int2 t = __ldcs(reinterpret_cast<const int2*>(p));
        c[0] = t.x; c[1] = t.y;
    }
};
template <> struct IChunk<4> {
    static __device__ __forceinline__ void load(const int32_t* p, int32_t* c) {
        int4 t = __ldcs(reinterpret_cast<const int4*>(p));
        c[0] = t.x; c[1] = t.y; c[2] = t.z; c[3] = t.w;
    }
};

// x read through L2 only (ld.global.cg).  The persistent grid sweep rewrites x between its colours
// and other SMs' L1 caches may still hold the old lines; L2 is coherent across the GPU.
template <typename T>
struct L2Read {
    const T* p;
    __device__ __forceinline__ T operator[](int64_t i) const { return __ldcg(p + i); }
};

// This lane's partial (A x)_r over the slice starting at o: `steps` loads of CH entries.  Four
// steps of matrix loads are issued before their gathers, so a row costs about steps / 4 memory
// round trips instead of steps / 2 (the small coarse-level colours are latency-bound).
template <typename T, int CH, typename X>
__device__ __forceinline__ T sell_part(const int32_t* __restrict__ ci, const T* __restrict__ v, int64_t o,
                                       int64_t steps, int lane, X x) {
    constexpr int U = 4;
    const T* vp = v + o + lane * CH;
    const int32_t* cp = ci + o + lane * CH;
    T sum = 0;
    int64_t q = 0;
    for (; q + U <= steps; q += U) {
        T a[U][CH];
        int32_t c[U][CH];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            Chunk<T, CH>::load(vp + u * SELL_C * CH, a[u]);
            IChunk<CH>::load(cp + u * SELL_C * CH, c[u]);
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int t = 0; t < CH; ++t) sum += a[u][t] * x[c[u][t]];
        vp += U * SELL_C * CH;
        cp += U * SELL_C * CH;
    }
    // The last steps - q < U steps: all their matrix loads are issued before the first gather, so
    // the tail costs one more round trip, not one per step (a coarse level's lanes often hold only
    // 2 or 3 steps).  The sum takes the products in the same order as a step-by-step loop.
    const int rem = (int)(steps - q);
    if (rem > 0) {
        T a[U - 1][CH];
        int32_t c[U - 1][CH];
#pragma unroll
        for (int u = 0; u < U - 1; ++u)
            if (u < rem) {
                Chunk<T, CH>::load(vp + u * SELL_C * CH, a[u]);
                IChunk<CH>::load(cp + u * SELL_C * CH, c[u]);
            }
#pragma unroll
        for (int u = 0; u < U - 1; ++u)
            if (u < rem)
#pragma unroll
                for (int t = 0; t < CH; ++t) sum += a[u][t] * x[c[u][t]];
    }
    return sum;
}
// sum over the lpr lanes of a row (every lane of the warp must call it)
template <typename T>
__device__ __forceinline__ T row_reduce(T sum, int lpr) {
    for (int d = lpr >> 1; d > 0; d >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, d);
    return sum;
}
// the row of this lane in slice sl and whether this lane writes it
struct SliceRow {
    int32_t r;
    bool write;
};
__device__ __forceinline__ SliceRow slice_row(const int32_t* __restrict__ srow, int64_t sl, int lane, int lpr) {
    SliceRow q;
    q.r = srow[sl] + lane / lpr;
    q.write = (lane & (lpr - 1)) == 0 && q.r < srow[sl + 1];
    return q;
}

// The first batch (up to four steps) of a lane's loads of one slice, loaded ahead of the barrier
// that precedes its gathers (the cluster sweep).
template <typename T, int CH>
struct SellHead {
    static constexpr int U = 4;
    T a[U][CH];
    int32_t c[U][CH];
    int n;
    __device__ __forceinline__ void load(const int32_t* __restrict__ ci, const T* __restrict__ v, int64_t o,
                                         int64_t steps, int lane) {
        n = steps < U ? (int)steps : U;
        const T* vp = v + o + lane * CH;
        const int32_t* cp = ci + o + lane * CH;
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (u < n) {
                Chunk<T, CH>::load(vp + u * SELL_C * CH, a[u]);
                IChunk<CH>::load(cp + u * SELL_C * CH, c[u]);
            }
    }
    template <typename X>
    __device__ __forceinline__ T finish(const int32_t* __restrict__ ci, const T* __restrict__ v, int64_t o,
                                        int64_t steps, int lane, X x) const {
        T sum = 0;
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (u < n)
#pragma unroll
                for (int t = 0; t < CH; ++t) sum += a[u][t] * x[c[u][t]];
        if (steps > n) sum += sell_part<T, CH>(ci, v, o + (int64_t)n * SELL_C * CH, steps - n, lane, x);
        return sum;
    }
};
// Colour order of a symmetric sweep: forward 0 .. C-1, then backward C-2 .. 0.  The backward
// sweep's first colour, C-1, would repeat the update just made: a Gauss-Seidel step leaves its own
// rows with zero residual, and rows of one colour do not couple, so that step changes nothing
// (beyond rounding) and is left out.
__host__ __device__ __forceinline__ int sweep_steps(int ncolor) { return ncolor > 0 ? 2 * ncolor - 1 : 0; }
__host__ __device__ __forceinline__ int sweep_colour(int step, int ncolor) {
    return step < ncolor ? step : 2 * ncolor - 2 - step;
}

}  // namespace sphc
