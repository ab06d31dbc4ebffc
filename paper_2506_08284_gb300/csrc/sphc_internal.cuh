// Internal declarations of the sm_103a SpHcurlAMG library (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <vector>

#include "../../include/sphc.h"

namespace sphc {

// ------------------------------------------------------------------ errors
void set_error(const char* fmt, ...);
const char* last_error();

#define SPHC_CK(call)                                                                       \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) {                                                            \
            ::sphc::set_error("%s:%d: %s: %s", __FILE__, __LINE__, #call,                  \
                              cudaGetErrorString(e_));                                     \
            return SPHC_ECUDA;                                                              \
        }                                                                                   \
    } while (0)

#define SPHC_TRY(call)                \
    do {                              \
        int rc_ = (call);             \
        if (rc_ != SPHC_OK) return rc_; \
    } while (0)

// ------------------------------------------------------------------ launch accounting
// Process-wide count of kernel launches made by the library (read by sphc_launch_count).
extern std::atomic<long long> g_launches;
#define SPHC_LAUNCH(...)                                                   \
    do {                                                                   \
        ::sphc::g_launches.fetch_add(1, std::memory_order_relaxed);       \
        __VA_ARGS__;                                                       \
    } while (0)

// Programmatic dependent launch: a kernel launched this way may be scheduled while the previous
// kernel of the stream drains, hiding the launch latency of the short kernels of a V-cycle.
// Every kernel launched with launch_pdl calls pdl_enter() first: it waits until the previous
// kernel has completed and its writes are visible, then lets the next kernel be scheduled.
// Inside stream capture the attribute is left off: in the CG graph (whose kernel nodes the GPU
// already launches back to back) programmatic edges measured slower, 476 vs 464 ms per 128^3
// solve, and with smoother kernels that issued their matrix loads ahead of the wait, repeated
// executions of the captured batched solve no longer agreed.
__device__ __forceinline__ void pdl_enter() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
template <typename... P, typename... A>
inline void launch_pdl(void (*k)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, A&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(s, &cap);
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = cap == cudaStreamCaptureStatusNone ? 1 : 0;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    ::sphc::g_launches.fetch_add(1, std::memory_order_relaxed);
    cudaLaunchKernelEx(&cfg, k, std::forward<A>(args)...);
}

// ------------------------------------------------------------------ stream-ordered buffers
// Every device buffer of the library comes from the library's own memory pool of the current
// device (cudaMallocFromPoolAsync on the caller's stream) and is released with cudaFreeAsync on
// the same stream.  The pool keeps freed memory mapped (release threshold: unlimited), so a
// setup that follows another reuses its memory instead of mapping it again; sphc_trim_memory
// returns it to the driver.
// When set (only while a handle is destroyed), buffers are released with the synchronous
// cudaFree so that no stream of the caller needs to be alive at that point.
extern bool g_sync_free;
// the library's pool of the current device (null if it could not be created)
cudaMemPool_t device_pool();

template <typename T>
struct DBuf {
    T* p = nullptr;
    int64_t n = 0;
    cudaStream_t s = 0;
    DBuf() = default;
    DBuf(const DBuf&) = delete;
    DBuf& operator=(const DBuf&) = delete;
    DBuf(DBuf&& o) noexcept { *this = std::move(o); }
    DBuf& operator=(DBuf&& o) noexcept {
        if (this != &o) {
            release();
            p = o.p; n = o.n; s = o.s;
            o.p = nullptr; o.n = 0;
        }
        return *this;
    }
    ~DBuf() { release(); }
    void release() {
        if (p) {
            if (g_sync_free) cudaFree(p);
            else cudaFreeAsync(p, s);
        }
        p = nullptr;
        n = 0;
    }
    int alloc(int64_t count, cudaStream_t stream) {
        release();
        s = stream;
        n = count;
        if (count <= 0) return SPHC_OK;
        cudaMemPool_t pool = device_pool();
        cudaError_t e = pool ? cudaMallocFromPoolAsync((void**)&p, sizeof(T) * (size_t)count, pool, stream)
                             : cudaMallocAsync((void**)&p, sizeof(T) * (size_t)count, stream);
        if (e != cudaSuccess) {
            p = nullptr;
            n = 0;
            set_error("cudaMallocAsync(%lld bytes): %s", (long long)(sizeof(T) * count), cudaGetErrorString(e));
            return SPHC_ENOMEM;
        }
        return SPHC_OK;
    }
    int zero(cudaStream_t stream) {
        if (n > 0) {
            cudaError_t e = cudaMemsetAsync(p, 0, sizeof(T) * (size_t)n, stream);
            if (e != cudaSuccess) {
                set_error("cudaMemsetAsync: %s", cudaGetErrorString(e));
                return SPHC_ECUDA;
            }
        }
        return SPHC_OK;
    }
};

// ------------------------------------------------------------------ device CSR
// rowptr int64, col int32 (sorted within rows), values FP64.
struct DCSR {
    int64_t nr = 0, nc = 0, nnz = 0;
    DBuf<int64_t> rp;
    DBuf<int32_t> ci;
    DBuf<double> v;
    int alloc(int64_t rows, int64_t cols, int64_t nz, cudaStream_t s) {
        nr = rows; nc = cols; nnz = nz;
        SPHC_TRY(rp.alloc(rows + 1, s));
        SPHC_TRY(ci.alloc(nz, s));
        SPHC_TRY(v.alloc(nz, s));
        return SPHC_OK;
    }
};

// ------------------------------------------------------------------ sparse primitives (sparse.cu)
int exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t s, int64_t* total_host);
// out[0..n] = exclusive prefix of int32 counts (out[n] = total)
int scan_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, cudaStream_t s, int64_t* total_host);
// C = A * B, structural (every reached entry kept), columns sorted, FP64 values.
int spgemm(const DCSR& A, const DCSR& B, DCSR& C, cudaStream_t s);
// The same for a product known to be symmetric (a Galerkin product): only the upper triangle is
// formed, the lower one is its exact mirror.
int spgemm_sym(const DCSR& A, const DCSR& B, DCSR& C, cudaStream_t s);
// C = D B for D with at most two entries per row (thread-per-row merge; spgemm otherwise),
// same result as spgemm
int dmul(const DCSR& D, const DCSR& B, DCSR& C, cudaStream_t s);
// C = A D for a D with at most two entries per row and A rows of at most 32 entries (warp-per-row
// sort; spgemm otherwise), same entries as spgemm
int amul_d(const DCSR& A, const DCSR& D, DCSR& C, cudaStream_t s);
// At = A^T, rows sorted.
int transpose(const DCSR& A, DCSR& At, cudaStream_t s);
// copy a CSR
int csr_copy(const DCSR& A, DCSR& B, cudaStream_t s);
// diag(A) into d (FP64)
int csr_diag(const DCSR& A, double* d, cudaStream_t s);
// y = A x (FP64)
int spmv64(const DCSR& A, const double* x, double* y, cudaStream_t s);
// deterministic dot product into a device scalar
int dot64(const double* a, const double* b, int64_t n, double* result_dev, cudaStream_t s);
// sort each row segment [rp[i], rp[i+1]) of (key, val) pairs by key (keys unique per row)
int segmented_sort(const int64_t* rp, int64_t nrows, int32_t* keys, double* vals, int64_t max_len,
                   cudaStream_t s);
int max_row_length(const int64_t* rp, int64_t nrows, cudaStream_t s, int64_t* out_host);

// ------------------------------------------------------------------ misc device helpers
__host__ __device__ inline uint64_t splitmix64(uint64_t seed, uint64_t counter) {
    uint64_t z = seed + (counter + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
// priority comparison: larger hash wins, ties -> smaller id wins
__device__ inline bool prio_greater(uint64_t ha, int64_t a, uint64_t hb, int64_t b) {
    return ha > hb || (ha == hb && a < b);
}

// Warp-aggregated atomic increment: the lanes active at the call reserve consecutive slots with
// one atomic per warp.  Returns this lane's slot.
__device__ inline int warp_reserve(int* ctr) {
    unsigned m = __activemask();
    int lane = threadIdx.x & 31;
    int leader = __ffs(m) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(ctr, __popc(m));
    base = __shfl_sync(m, base, leader);
    return base + __popc(m & ((1u << lane) - 1u));
}
// Add the number of lanes (of the full warp) with pred set: one atomic per warp.  Every lane of
// the warp must call it.
__device__ inline void warp_count(int* ctr, bool pred) {
    unsigned m = __ballot_sync(0xffffffffu, pred);
    if ((threadIdx.x & 31) == 0 && m) atomicAdd(ctr, __popc(m));
}

inline int grid_for(int64_t n, int block) {
    int64_t g = (n + block - 1) / block;
    if (g < 1) g = 1;
    if (g > 2147483647LL) g = 2147483647;
    return (int)g;
}

}  // namespace sphc
