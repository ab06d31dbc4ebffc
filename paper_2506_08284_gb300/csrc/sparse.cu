// Sparse building blocks of the setup phase: scans, transposes, segmented sorts, the
// structural sparse matrix product (used for D_h^T A_e D_h, A_n Pbar, D_h P_n and the Galerkin
// products P_e^T A_e P_e, P_n^T A_n P_n of Sec. 2), FP64 SpMV and deterministic dots.
#include <algorithm>
#include <cstdlib>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <mutex>

#include "sphc_internal.cuh"

namespace sphc {

bool g_sync_free = false;
std::atomic<long long> g_launches{0};

static std::mutex g_pool_mutex;
static cudaMemPool_t g_pools[64] = {};
cudaMemPool_t device_pool() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(g_pool_mutex);
    if (!g_pools[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        uint64_t keep = ~0ULL;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        g_pools[dev] = pool;
    }
    return g_pools[dev];
}
static thread_local std::string g_err;
void set_error(const char* fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
}
const char* last_error() { return g_err.c_str(); }

// ------------------------------------------------------------------ scans
static constexpr int SCAN_BLOCK = 1024;
static constexpr int SCAN_ITEMS = 4;
static constexpr int SCAN_TILE = SCAN_BLOCK * SCAN_ITEMS;

__device__ inline int64_t warp_incl_scan(int64_t v) {
    int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// inclusive block scan of one value per thread; returns inclusive prefix, *total = block sum
__device__ inline int64_t block_incl_scan(int64_t v, int64_t* smem_warps, int64_t* total) {
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int64_t x = warp_incl_scan(v);
    if (lane == 31) smem_warps[w] = x;
    __syncthreads();
    if (w == 0) {
        int64_t y = lane < nw ? smem_warps[lane] : 0;
        y = warp_incl_scan(y);
        if (lane < nw) smem_warps[lane] = y;
    }
    __syncthreads();
    int64_t off = w > 0 ? smem_warps[w - 1] : 0;
    if (total) *total = smem_warps[nw - 1];
    __syncthreads();
    return x + off;
}

template <typename TI>
__global__ void k_scan_tiles(const TI* in, int64_t n, int64_t* tile_sums) {
    __shared__ int64_t sw[32];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    int64_t s = 0;
#pragma unroll
    for (int q = 0; q < SCAN_ITEMS; ++q)
        if (base + q < n) s += (int64_t)in[base + q];
    int64_t tot;
    block_incl_scan(s, sw, &tot);
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = tot;
}

__global__ void k_scan_sums(int64_t* sums, int64_t nt, int64_t* total) {
    __shared__ int64_t sw[32];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t b = 0; b < nt; b += blockDim.x) {
        int64_t i = b + threadIdx.x;
        int64_t v = i < nt ? sums[i] : 0;
        int64_t tot;
        int64_t inc = block_incl_scan(v, sw, &tot);
        if (i < nt) sums[i] = carry + inc - v;   // exclusive
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

template <typename TI>
__global__ void k_scan_apply(const TI* in, int64_t n, const int64_t* tile_off, int64_t* out) {
    __shared__ int64_t sw[32];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    int64_t v[SCAN_ITEMS];
    int64_t s = 0;
#pragma unroll
    for (int q = 0; q < SCAN_ITEMS; ++q) {
        v[q] = (base + q < n) ? (int64_t)in[base + q] : 0;
        s += v[q];
    }
    int64_t inc = block_incl_scan(s, sw, nullptr);
    int64_t run = tile_off[blockIdx.x] + inc - s;
#pragma unroll
    for (int q = 0; q < SCAN_ITEMS; ++q) {
        if (base + q < n) out[base + q] = run;
        run += v[q];
    }
}

// out[0..n) = exclusive prefix of in; out[n] = total (out must hold n+1 entries)
template <typename TI>
static int scan_impl(const TI* in, int64_t* out, int64_t n, cudaStream_t s, int64_t* total_host) {
    int64_t nt = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (nt < 1) nt = 1;
    DBuf<int64_t> sums;
    SPHC_TRY(sums.alloc(nt + 1, s));
    if (n > 0) SPHC_LAUNCH(k_scan_tiles<TI><<<(unsigned)nt, SCAN_BLOCK, 0, s>>>(in, n, sums.p));
    else SPHC_CK(cudaMemsetAsync(sums.p, 0, sizeof(int64_t) * nt, s));
    SPHC_LAUNCH(k_scan_sums<<<1, SCAN_BLOCK, 0, s>>>(sums.p, nt, out + n));
    if (n > 0) SPHC_LAUNCH(k_scan_apply<TI><<<(unsigned)nt, SCAN_BLOCK, 0, s>>>(in, n, sums.p, out));
    SPHC_CK(cudaGetLastError());
    if (total_host) {
        SPHC_CK(cudaMemcpyAsync(total_host, out + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        SPHC_CK(cudaStreamSynchronize(s));
    }
    return SPHC_OK;
}
int exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t s, int64_t* total_host) {
    return scan_impl<int64_t>(in, out, n, s, total_host);
}
int scan_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, cudaStream_t s, int64_t* total_host) {
    return scan_impl<int32_t>(in, out, n, s, total_host);
}

// ------------------------------------------------------------------ row-length helpers
__global__ void k_row_len_max(const int64_t* rp, int64_t n, unsigned long long* mx) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long v = 0;
    if (i < n) v = (unsigned long long)(rp[i + 1] - rp[i]);
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long t = __shfl_down_sync(0xffffffffu, v, o);
        v = t > v ? t : v;
    }
    if ((threadIdx.x & 31) == 0 && v > 0) atomicMax(mx, v);
}
int max_row_length(const int64_t* rp, int64_t nrows, cudaStream_t s, int64_t* out_host) {
    DBuf<unsigned long long> m;
    SPHC_TRY(m.alloc(1, s));
    SPHC_TRY(m.zero(s));
    if (nrows > 0) SPHC_LAUNCH(k_row_len_max<<<grid_for(nrows, 256), 256, 0, s>>>(rp, nrows, m.p));
    unsigned long long h = 0;
    SPHC_CK(cudaMemcpyAsync(&h, m.p, sizeof(h), cudaMemcpyDeviceToHost, s));
    SPHC_CK(cudaStreamSynchronize(s));
    *out_host = (int64_t)h;
    return SPHC_OK;
}

// ------------------------------------------------------------------ segmented sort
// rows of length <= 32: one warp per row, bitonic network over lanes
__global__ void k_segsort_warp(const int64_t* rp, int64_t nrows, int32_t* keys, double* vals) {
    int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (row >= nrows) return;
    int64_t b = rp[row];
    int len = (int)(rp[row + 1] - b);
    if (len <= 1 || len > 32) return;
    int32_t k = lane < len ? keys[b + lane] : 0x7fffffff;
    double v = lane < len && vals ? vals[b + lane] : 0.0;
    for (int size = 2; size <= 32; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            int32_t ok = __shfl_xor_sync(0xffffffffu, k, stride);
            double ov = __shfl_xor_sync(0xffffffffu, v, stride);
            bool up = ((lane & size) == 0);
            bool lower = (lane & stride) == 0;
            bool take_min = (up == lower);
            bool swap = take_min ? (ok < k) : (ok > k);
            if (swap) { k = ok; v = ov; }
        }
    }
    if (lane < len) {
        keys[b + lane] = k;
        if (vals) vals[b + lane] = v;
    }
}

// rows of length <= cap (power of two): one block per row, bitonic network in shared memory
__global__ void k_segsort_block(const int64_t* rp, int64_t nrows, int32_t* keys, double* vals, int cap) {
    extern __shared__ unsigned char smem_raw[];
    int32_t* sk = (int32_t*)smem_raw;
    double* sv = (double*)(smem_raw + sizeof(int32_t) * cap);
    for (int64_t row = blockIdx.x; row < nrows; row += gridDim.x) {
        int64_t b = rp[row];
        int len = (int)(rp[row + 1] - b);
        if (len <= 32) continue;   // handled by the warp kernel
        int n2 = 64;
        while (n2 < len) n2 <<= 1;
        for (int t = threadIdx.x; t < n2; t += blockDim.x) {
            sk[t] = t < len ? keys[b + t] : 0x7fffffff;
            sv[t] = (t < len && vals) ? vals[b + t] : 0.0;
        }
        __syncthreads();
        for (int size = 2; size <= n2; size <<= 1)
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                for (int t = threadIdx.x; t < n2; t += blockDim.x) {
                    int p = t ^ stride;
                    if (p > t) {
                        bool up = ((t & size) == 0);
                        int32_t a = sk[t], c = sk[p];
                        if ((a > c) == up) {
                            sk[t] = c; sk[p] = a;
                            double tv = sv[t]; sv[t] = sv[p]; sv[p] = tv;
                        }
                    }
                }
                __syncthreads();
            }
        for (int t = threadIdx.x; t < len; t += blockDim.x) {
            keys[b + t] = sk[t];
            if (vals) vals[b + t] = sv[t];
        }
        __syncthreads();
    }
}

int segmented_sort(const int64_t* rp, int64_t nrows, int32_t* keys, double* vals, int64_t max_len,
                   cudaStream_t s) {
    if (nrows <= 0) return SPHC_OK;
    SPHC_LAUNCH(k_segsort_warp<<<grid_for(nrows * 32, 256), 256, 0, s>>>(rp, nrows, keys, vals));
    if (max_len > 32) {
        int cap = 64;
        while (cap < max_len) cap <<= 1;
        if (cap > 8192) {
            set_error("segmented_sort: row of %lld entries exceeds 8192", (long long)max_len);
            return SPHC_ELIMIT;
        }
        size_t sm = (size_t)cap * (sizeof(int32_t) + sizeof(double));
        SPHC_CK(cudaFuncSetAttribute(k_segsort_block, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        int grid = (int)(nrows < 65536 ? nrows : 65536);
        SPHC_LAUNCH(k_segsort_block<<<grid, 256, sm, s>>>(rp, nrows, keys, vals, cap));
    }
    SPHC_CK(cudaGetLastError());
    return SPHC_OK;
}

// ------------------------------------------------------------------ transpose
__global__ void k_col_count(const int32_t* ci, int64_t nnz, int32_t* cnt) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < nnz) atomicAdd(&cnt[ci[k]], 1);
}
__global__ void k_transpose_scatter(const int64_t* rp, const int32_t* ci, const double* v, int64_t nr,
                                    unsigned long long* cursor, int32_t* tci, double* tv) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nr) return;
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
        unsigned long long pos = atomicAdd(&cursor[ci[k]], 1ULL);
        tci[pos] = (int32_t)i;
        if (tv) tv[pos] = v[k];
    }
}
__global__ void k_i64_to_u64(const int64_t* a, unsigned long long* b, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (unsigned long long)a[i];
}

// Test switches of the path choices of the sparse products and the transpose, read from the
// environment variable SPHC_SPGEMM_PATHS (a bit mask, 0 when unset): 1 the small bin's counting
// and writing passes instead of its one pass into temporary slots; 2 the numeric pass binned by
// row length whatever the number of rows; 4 never binned by row length; 8 the hash bins through
// counting and numeric passes instead of their one pass into an arena (bits 2 and 4 apply then);
// 16 sub-arenas of 64 entries, so that most one-pass rows take the overflow path; 32 every
// transpose by the radix sort; 64 the 256-slot one-pass tables for every upper-triangle product.
// Every path gives the same matrix.
static int spgemm_path_flags() {
    const char* e = getenv("SPHC_SPGEMM_PATHS");
    return e ? atoi(e) : 0;
}

// ------------------------------------------------------------------ transpose by stable radix sort
// The entries of A, in row-major order, are sorted by column with a stable least-significant-digit
// radix sort of (column, entry index) pairs, RX_BITS bits a pass: per pass, per-block digit
// histograms, one scan of them (digit-major, block-minor), and a stable scatter (warp match for the
// rank inside a warp, per-warp counts for the warps before it).  Equal columns keep their entries'
// order, so every row of A^T comes out sorted by A's row index: the segmented sort of the
// scatter-based transpose is not needed.  Then A^T's row index and value of each sorted entry are
// gathered.
static constexpr int RX_BLOCK = 1024, RX_BITS = 8, RX_KEYS = 1 << RX_BITS;
static constexpr int64_t TRANSPOSE_RADIX_MIN_NNZ = 1 << 20;     // smaller: scatter + segmented sort
static constexpr double TRANSPOSE_RADIX_MIN_MEAN = 24.0;         // mean row length of A^T
__global__ void k_rx_init(const int32_t* ci, int64_t nnz, int2* it) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < nnz) it[e] = make_int2(ci[e], (int32_t)e);
}
__global__ void k_rx_count(const int2* it, int64_t n, int shift, int32_t* table, int64_t nb) {
    __shared__ int32_t cnt[RX_KEYS];
    for (int c = threadIdx.x; c < RX_KEYS; c += blockDim.x) cnt[c] = 0;
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * RX_BLOCK + threadIdx.x;
    const int c = i < n ? (it[i].x >> shift) & (RX_KEYS - 1) : -1;
    const unsigned m = __match_any_sync(0xffffffffu, c);     // one add per digit and warp
    if (c >= 0 && (threadIdx.x & 31) == __ffs(m) - 1) atomicAdd(&cnt[c], __popc(m));
    __syncthreads();
    for (int c = threadIdx.x; c < RX_KEYS; c += blockDim.x) table[(int64_t)c * nb + blockIdx.x] = cnt[c];
}
__global__ void __launch_bounds__(RX_BLOCK)
k_rx_place(const int2* in, int64_t n, int shift, const int64_t* off, int64_t nb, int2* out) {
    __shared__ int32_t wcnt[RX_BLOCK / 32][RX_KEYS];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int q = threadIdx.x; q < (RX_BLOCK / 32) * RX_KEYS; q += blockDim.x) (&wcnt[0][0])[q] = 0;
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * RX_BLOCK + threadIdx.x;
    const int2 item = i < n ? in[i] : make_int2(0, 0);
    const int c = i < n ? (item.x >> shift) & (RX_KEYS - 1) : -1;
    const unsigned m = __match_any_sync(0xffffffffu, c);
    const int rank = __popc(m & ((1u << lane) - 1u));
    if (c >= 0 && rank == 0) wcnt[w][c] = __popc(m);
    __syncthreads();
    if (c >= 0) {
        int before = 0;
        for (int q = 0; q < w; ++q) before += wcnt[q][c];
        out[off[(int64_t)c * nb + blockIdx.x] + before + rank] = item;
    }
}
// row index of every entry (G lanes per row)
template <int G>
__global__ void k_entry_rows(const int64_t* rp, int64_t nr, int32_t* rowof) {
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
    if (i >= nr) return;
    for (int64_t k = rp[i] + (threadIdx.x & (G - 1)); k < rp[i + 1]; k += G) rowof[k] = (int32_t)i;
}
// row pointers of A^T from the sorted keys: row c starts at the first key >= c
__global__ void k_rx_rowptr(const int2* it, int64_t nnz, int64_t nc, int64_t* trp) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c > nc) return;
    int64_t lo = 0, hi = nnz;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (it[mid].x < c) lo = mid + 1; else hi = mid;
    }
    trp[c] = lo;
}
__global__ void k_rx_gather(const int2* it, int64_t nnz, const int32_t* rowof, const double* v, int32_t* tci,
                            double* tv) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nnz) return;
    const int32_t e = it[k].y;
    tci[k] = rowof[e];
    tv[k] = v[e];
}
static int transpose_radix(const DCSR& A, DCSR& At, cudaStream_t s) {
    const int64_t nnz = A.nnz, nb = (nnz + RX_BLOCK - 1) / RX_BLOCK;
    int bits = 1;
    while (bits < 31 && (1LL << bits) < A.nc) ++bits;
    const int passes = (bits + RX_BITS - 1) / RX_BITS;
    DBuf<int2> it0, it1;
    DBuf<int32_t> table, rowof;
    DBuf<int64_t> off;
    SPHC_TRY(it0.alloc(nnz, s));
    SPHC_TRY(it1.alloc(nnz, s));
    SPHC_TRY(table.alloc((int64_t)RX_KEYS * nb, s));
    SPHC_TRY(off.alloc((int64_t)RX_KEYS * nb + 1, s));
    SPHC_LAUNCH(k_rx_init<<<grid_for(nnz, 256), 256, 0, s>>>(A.ci.p, nnz, it0.p));
    int2* in = it0.p;
    int2* out = it1.p;
    for (int ps = 0; ps < passes; ++ps) {
        const int shift = ps * RX_BITS;
        SPHC_LAUNCH(k_rx_count<<<(unsigned)nb, RX_BLOCK, 0, s>>>(in, nnz, shift, table.p, nb));
        SPHC_TRY(scan_i32_to_i64(table.p, off.p, (int64_t)RX_KEYS * nb, s, nullptr));
        SPHC_LAUNCH(k_rx_place<<<(unsigned)nb, RX_BLOCK, 0, s>>>(in, nnz, shift, off.p, nb, out));
        std::swap(in, out);
    }
    SPHC_TRY(rowof.alloc(nnz, s));
    const double avg = (double)nnz / (double)(A.nr > 0 ? A.nr : 1);
    if (A.nr > 0) {
        if (avg <= 6) SPHC_LAUNCH(k_entry_rows<4><<<grid_for(A.nr * 4, 256), 256, 0, s>>>(A.rp.p, A.nr, rowof.p));
        else if (avg <= 12) SPHC_LAUNCH(k_entry_rows<8><<<grid_for(A.nr * 8, 256), 256, 0, s>>>(A.rp.p, A.nr, rowof.p));
        else SPHC_LAUNCH(k_entry_rows<32><<<grid_for(A.nr * 32, 256), 256, 0, s>>>(A.rp.p, A.nr, rowof.p));
    }
    SPHC_LAUNCH(k_rx_gather<<<grid_for(nnz, 256), 256, 0, s>>>(in, nnz, rowof.p, A.v.p, At.ci.p, At.v.p));
    SPHC_LAUNCH(k_rx_rowptr<<<grid_for(A.nc + 1, 256), 256, 0, s>>>(in, nnz, A.nc, At.rp.p));
    SPHC_CK(cudaGetLastError());
    return SPHC_OK;
}

int transpose(const DCSR& A, DCSR& At, cudaStream_t s) {
    // long rows of A^T (whose segmented sort takes a block per row) by the radix sort, which also
    // gives A^T's row pointers: chosen by the mean row length of A^T
    if (A.nnz > 0 && A.nnz < (1LL << 31) &&
        ((spgemm_path_flags() & 32) ||
         (A.nnz >= TRANSPOSE_RADIX_MIN_NNZ && (double)A.nnz > TRANSPOSE_RADIX_MIN_MEAN * (double)A.nc))) {
        SPHC_TRY(At.alloc(A.nc, A.nr, A.nnz, s));
        return transpose_radix(A, At, s);
    }
    DBuf<int32_t> cnt;
    SPHC_TRY(cnt.alloc(A.nc + 1, s));
    SPHC_TRY(cnt.zero(s));
    if (A.nnz > 0) SPHC_LAUNCH(k_col_count<<<grid_for(A.nnz, 256), 256, 0, s>>>(A.ci.p, A.nnz, cnt.p));
    SPHC_TRY(At.alloc(A.nc, A.nr, A.nnz, s));
    int64_t tot = 0;
    SPHC_TRY(scan_i32_to_i64(cnt.p, At.rp.p, A.nc, s, &tot));
    int64_t mx = 0;
    SPHC_TRY(max_row_length(At.rp.p, At.nr, s, &mx));
    DBuf<unsigned long long> cur;
    SPHC_TRY(cur.alloc(A.nc + 1, s));
    SPHC_LAUNCH(k_i64_to_u64<<<grid_for(A.nc + 1, 256), 256, 0, s>>>(At.rp.p, cur.p, A.nc + 1));
    if (A.nr > 0)
        SPHC_LAUNCH(k_transpose_scatter<<<grid_for(A.nr, 256), 256, 0, s>>>(A.rp.p, A.ci.p, A.v.p, A.nr, cur.p, At.ci.p, At.v.p));
    SPHC_CK(cudaGetLastError());
    SPHC_TRY(segmented_sort(At.rp.p, At.nr, At.ci.p, At.v.p, mx, s));
    return SPHC_OK;
}

int csr_copy(const DCSR& A, DCSR& B, cudaStream_t s) {
    SPHC_TRY(B.alloc(A.nr, A.nc, A.nnz, s));
    SPHC_CK(cudaMemcpyAsync(B.rp.p, A.rp.p, sizeof(int64_t) * (A.nr + 1), cudaMemcpyDeviceToDevice, s));
    if (A.nnz > 0) {
        SPHC_CK(cudaMemcpyAsync(B.ci.p, A.ci.p, sizeof(int32_t) * A.nnz, cudaMemcpyDeviceToDevice, s));
        SPHC_CK(cudaMemcpyAsync(B.v.p, A.v.p, sizeof(double) * A.nnz, cudaMemcpyDeviceToDevice, s));
    }
    return SPHC_OK;
}

__global__ void k_diag(const int64_t* rp, const int32_t* ci, const double* v, int64_t n, double* d) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double r = 0.0;
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k)
        if (ci[k] == i) r = v[k];
    d[i] = r;
}
int csr_diag(const DCSR& A, double* d, cudaStream_t s) {
    if (A.nr > 0) SPHC_LAUNCH(k_diag<<<grid_for(A.nr, 256), 256, 0, s>>>(A.rp.p, A.ci.p, A.v.p, A.nr, d));
    SPHC_CK(cudaGetLastError());
    return SPHC_OK;
}

// ------------------------------------------------------------------ gradient times matrix
// C = D B for a D with at most two entries per row (a discrete gradient): row i of C is the sorted
// union of B's rows at D's columns, the values combined with D's coefficients.  Structural like
// spgemm: every reached column is kept, even where the two contributions cancel, and a column
// reached twice gets the sum of two products (exact in either order, as in spgemm).  Thread per
// row; mode 0 counts, mode 1 writes.
__global__ void k_dmul(const int64_t* __restrict__ drp, const int32_t* __restrict__ dci, const double* __restrict__ dv,
                       int64_t n, const int64_t* __restrict__ brp, const int32_t* __restrict__ bci,
                       const double* __restrict__ bv, int mode, int64_t* cnt, const int64_t* __restrict__ crp,
                       int32_t* __restrict__ cci, double* __restrict__ cv) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t d0 = drp[i], dl = drp[i + 1] - d0;
    int64_t a0 = 0, a1 = 0, b0 = 0, b1 = 0;
    double ca = 0.0, cb = 0.0;
    if (dl >= 1) { int32_t u = dci[d0]; a0 = brp[u]; a1 = brp[u + 1]; ca = dv[d0]; }
    if (dl >= 2) { int32_t w = dci[d0 + 1]; b0 = brp[w]; b1 = brp[w + 1]; cb = dv[d0 + 1]; }
    int64_t out = mode ? crp[i] : 0, c = 0;
    int64_t ka = a0, kb = b0;
    while (ka < a1 || kb < b1) {
        int32_t ja = ka < a1 ? bci[ka] : INT32_MAX, jb = kb < b1 ? bci[kb] : INT32_MAX;
        int32_t col;
        double val;
        if (ja < jb) { col = ja; val = ca * bv[ka]; ++ka; }
        else if (jb < ja) { col = jb; val = cb * bv[kb]; ++kb; }
        else { col = ja; val = ca * bv[ka] + cb * bv[kb]; ++ka; ++kb; }
        if (mode) { cci[out + c] = col; cv[out + c] = val; }
        ++c;
    }
    if (!mode) cnt[i] = c;
}

// ------------------------------------------------------------------ matrix times gradient
// C = A D for D with at most two entries per row and A rows of at most 32 entries: warp per row.
// Lane k takes A's entry k (column f) and the one or two node ids of D's row f.  The distinct
// nodes of the row come out in ascending order from a warp min-reduction over the lanes' ids
// (one round per node, which then leaves the candidate set); two ballots per round record the
// lanes that reach it, kept by lane c % 32 for the c-th node.  In the fill pass each lane then
// adds up its node's products a_if d_fn over those lanes in ascending lane order, i.e. in A's row
// order, the order a sparse accumulator walking A's row uses.  Mode 0 counts the nodes of each
// row, mode 1 writes them.
constexpr int AD_WARPS = 8;
// a * d, by a sign flip when d is +1 or -1 (every entry of a discrete gradient), compared and
// flipped on the bit patterns so that the FP64 pipe only sees the rare other values
__device__ __forceinline__ double times_unit(double a, double d) {
    const unsigned long long db = (unsigned long long)__double_as_longlong(d);
    if (db == 0x3FF0000000000000ULL) return a;
    if (db == 0xBFF0000000000000ULL) return __longlong_as_double(__double_as_longlong(a) ^ (long long)(1ULL << 63));
    return a * d;
}
__global__ void __launch_bounds__(AD_WARPS * 32)
k_amul_d(const int64_t* __restrict__ arp, const int32_t* __restrict__ aci, const double* __restrict__ av, int64_t n,
         const int64_t* __restrict__ drp, const int32_t* __restrict__ dci, const double* __restrict__ dv, int mode,
         int64_t* __restrict__ cnt, const int64_t* __restrict__ crp, int32_t* __restrict__ cci,
         double* __restrict__ cv) {
    __shared__ double s_val[AD_WARPS][64];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t i = (int64_t)blockIdx.x * AD_WARPS + w;
    if (i >= n) return;
    const int NONE = 0x7fffffff;
    int k0 = NONE, k1 = NONE;
    const int64_t a0 = arp[i];
    if (lane < arp[i + 1] - a0) {
        const int32_t f = aci[a0 + lane];
        const int64_t d0 = drp[f], dl = drp[f + 1] - d0;
        if (dl > 0) k0 = dci[d0];
        if (dl > 1) k1 = dci[d0 + 1];
        if (mode != 0) {
            const double a = av[a0 + lane];
            s_val[w][lane] = dl > 0 ? times_unit(a, dv[d0]) : 0.0;
            s_val[w][32 + lane] = dl > 1 ? times_unit(a, dv[d0 + 1]) : 0.0;
        }
    }
    unsigned lo0 = 0, lo1 = 0, hi0 = 0, hi1 = 0;     // ballots of node lane and node lane + 32
    int node_lo = NONE, node_hi = NONE;
    int c = 0;
    for (;;) {
        const int m = __reduce_min_sync(0xffffffffu, k0 < k1 ? k0 : k1);
        if (m == NONE) break;
        const unsigned b0 = __ballot_sync(0xffffffffu, k0 == m), b1 = __ballot_sync(0xffffffffu, k1 == m);
        if (lane == (c & 31)) {
            if (c < 32) { lo0 = b0; lo1 = b1; node_lo = m; }
            else { hi0 = b0; hi1 = b1; node_hi = m; }
        }
        if (k0 == m) k0 = NONE;
        if (k1 == m) k1 = NONE;
        ++c;
    }
    if (mode == 0) {
        if (lane == 0) cnt[i] = c;
        return;
    }
    __syncwarp();
    const int64_t out = crp[i];
    for (int r = 0; r < 2; ++r) {
        const int slot = lane + 32 * r;
        if (slot >= c) break;
        const unsigned b0 = r ? hi0 : lo0, b1 = r ? hi1 : lo1;
        // a lane reaches a node through one of its two D entries (the two nodes of an edge
        // differ): pick that product, then one FP64 add per further lane, the first term as is
        unsigned any = b0 | b1;
        int l = __ffs(any) - 1;
        any &= any - 1;
        double sum = s_val[w][((b0 >> l) & 1u) ? l : 32 + l];
        while (any) {
            l = __ffs(any) - 1;
            any &= any - 1;
            sum += s_val[w][((b0 >> l) & 1u) ? l : 32 + l];
        }
        cci[out + slot] = r ? node_hi : node_lo;
        cv[out + slot] = sum;
    }
}

int amul_d(const DCSR& A, const DCSR& D, DCSR& C, cudaStream_t s) {
    int64_t amax = 0, dmax = 0;
    SPHC_TRY(max_row_length(A.rp.p, A.nr, s, &amax));
    SPHC_TRY(max_row_length(D.rp.p, D.nr, s, &dmax));
    if (amax > 32 || dmax > 2) return spgemm(A, D, C, s);
    const int64_t n = A.nr;
    DBuf<int64_t> cnt;
    SPHC_TRY(cnt.alloc(n + 1, s));
    const int g = grid_for(n, AD_WARPS);
    if (n > 0)
        SPHC_LAUNCH(k_amul_d<<<g, AD_WARPS * 32, 0, s>>>(A.rp.p, A.ci.p, A.v.p, n, D.rp.p, D.ci.p, D.v.p, 0, cnt.p,
                                                        nullptr, nullptr, nullptr));
    C = DCSR();
    C.nr = n;
    C.nc = D.nc;
    SPHC_TRY(C.rp.alloc(n + 1, s));
    SPHC_TRY(exclusive_scan_i64(cnt.p, C.rp.p, n, s, &C.nnz));
    SPHC_TRY(C.ci.alloc(C.nnz, s));
    SPHC_TRY(C.v.alloc(C.nnz, s));
    if (n > 0)
        SPHC_LAUNCH(k_amul_d<<<g, AD_WARPS * 32, 0, s>>>(A.rp.p, A.ci.p, A.v.p, n, D.rp.p, D.ci.p, D.v.p, 1, nullptr,
                                                        C.rp.p, C.ci.p, C.v.p));
    SPHC_CK(cudaGetLastError());
    return SPHC_OK;
}

int dmul(const DCSR& D, const DCSR& B, DCSR& C, cudaStream_t s) {
    int64_t dmax = 0;
    SPHC_TRY(max_row_length(D.rp.p, D.nr, s, &dmax));
    if (dmax > 2) return spgemm(D, B, C, s);
    int64_t n = D.nr;
    DBuf<int64_t> cnt;
    SPHC_TRY(cnt.alloc(n + 1, s));
    if (n > 0)
        SPHC_LAUNCH(k_dmul<<<grid_for(n, 256), 256, 0, s>>>(D.rp.p, D.ci.p, D.v.p, n, B.rp.p, B.ci.p, B.v.p, 0, cnt.p,
                                                           nullptr, nullptr, nullptr));
    C = DCSR();
    C.nr = n;
    C.nc = B.nc;
    SPHC_TRY(C.rp.alloc(n + 1, s));
    SPHC_TRY(exclusive_scan_i64(cnt.p, C.rp.p, n, s, &C.nnz));
    SPHC_TRY(C.ci.alloc(C.nnz, s));
    SPHC_TRY(C.v.alloc(C.nnz, s));
    if (n > 0)
        SPHC_LAUNCH(k_dmul<<<grid_for(n, 256), 256, 0, s>>>(D.rp.p, D.ci.p, D.v.p, n, B.rp.p, B.ci.p, B.v.p, 1, nullptr,
                                                           C.rp.p, C.ci.p, C.v.p));
    SPHC_CK(cudaGetLastError());
    return SPHC_OK;
}

// ------------------------------------------------------------------ structural SpGEMM
// Row-wise: every product a_ik * b_kj of row i is inserted into a per-warp open-addressing
// table in shared memory.  Rows are binned by their product count so that a row touches a table
// of matching size (small tables also give more resident warps); rows with more than
// BIG_FILL-capable output go to a block-per-row path.  The symbolic pass counts distinct columns,
// the numeric pass accumulates, compacts and writes each row sorted by column.
static constexpr int MED_SLOTS = 1024;       // largest per-warp table
static constexpr int MED_FILL = 768;         // rows with more distinct columns go to the big path
static constexpr int BIG_SLOTS = 8192;       // per block on the big path
static constexpr int BIG_FILL = 6144;
static constexpr int NBINS = 4;

__device__ inline uint32_t hslot(int32_t key, int mask) {
    return ((uint32_t)key * 2654435761u) & (uint32_t)mask;
}

// First position of B's row k whose column is >= floor (floor < 0: the row start).  A product
// restricted to the upper triangle (floor = the output row) only visits these entries.
__device__ inline int64_t row_floor(const int64_t* brp, const int32_t* bci, int32_t k, int32_t floor) {
    int64_t lo = brp[k], hi = brp[k + 1];
    if (floor < 0) return lo;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (bci[mid] < floor) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// bins: 0 at most 64 products and 64 A entries (register sort), 1 at most 128 products
// (256-slot tables), 2 at most 256 (512-slot tables), 3 the rest (1024-slot tables / big path)
__device__ inline int spgemm_bin_of(int64_t ub, int64_t alen) {
    return (ub <= 64 && alen <= 64) ? 0 : (ub <= 128 ? 1 : (ub <= 256 ? 2 : 3));
}
// Product count (restricted to the upper triangle when `upper`) of every row, G lanes per row
// (rows of long A rows, such as the P^T factors of coarse Galerkin products, would otherwise
// walk their entries' binary searches one after the other); bin sizes counted per block.
template <int G>
__global__ void k_spgemm_ub(const int64_t* arp, const int32_t* aci, const int64_t* brp, const int32_t* bci, int64_t n,
                            int upper, int64_t* ub, int* bin_cnt) {
    const int lane = threadIdx.x & 31, sub = lane & (G - 1);
    const unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
    int bin = -1;
    if (i < n) {                                     // uniform over the group
        int64_t sum = 0;
        const int32_t floor = upper ? (int32_t)i : -1;
        for (int64_t k = arp[i] + sub; k < arp[i + 1]; k += G) sum += brp[aci[k] + 1] - row_floor(brp, bci, aci[k], floor);
#pragma unroll
        for (int d = G / 2; d > 0; d >>= 1) sum += __shfl_xor_sync(gmask, sum, d);
        if (sub == 0) {
            ub[i] = sum;
            bin = spgemm_bin_of(sum, arp[i + 1] - arp[i]);
        }
    }
    for (int b = 0; b < NBINS; ++b) {
        int c = __syncthreads_count(bin == b);
        if (threadIdx.x == 0 && c) atomicAdd(&bin_cnt[b], c);
    }
}
__global__ void k_spgemm_bin(const int64_t* arp, const int64_t* ub, int64_t n, const int* bin_off, int* bin_fill,
                             int32_t* rows) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int bin = spgemm_bin_of(ub[i], arp[i + 1] - arp[i]);
    unsigned m = __match_any_sync(__activemask(), bin);
    int lane = threadIdx.x & 31;
    int leader = __ffs(m) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(&bin_fill[bin], __popc(m));
    base = __shfl_sync(m, base, leader);
    rows[bin_off[bin] + base + __popc(m & ((1u << lane) - 1u))] = (int32_t)i;
}

// Rows with at most 64 products (and 64 A entries): one warp per row, the products held two per
// lane; the distinct columns are taken in ascending order by warp min-reductions.  mode 0 counts
// distinct columns, mode 1 writes the row at its place in C, mode 2 writes it (and its count) to
// a temporary slot of the listed row.
static constexpr int SMALL_WARPS = 8;
__global__ void __launch_bounds__(SMALL_WARPS * 32)
k_spgemm_small(const int64_t* arp, const int32_t* aci, const double* av, const int64_t* brp, const int32_t* bci,
               const double* bv, const int32_t* rows, int nrows, int mode, int upper, int64_t* cnt, const int64_t* crp,
               int32_t* cci, double* cv) {
    __shared__ int64_t s_off[SMALL_WARPS][64];
    __shared__ int64_t s_bst[SMALL_WARPS][64];
    __shared__ double s_val[SMALL_WARPS][64];
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int64_t li = (int64_t)blockIdx.x * SMALL_WARPS + w;
    if (li >= nrows) return;
    int64_t i = rows[li];
    int64_t a0 = arp[i];
    int alen = (int)(arp[i + 1] - a0);
    // product offsets of the (at most 64) A entries
    int64_t len[2] = {0, 0};
    int32_t floor = upper ? (int32_t)i : -1;
    for (int q = 0; q < 2; ++q) {
        int e = lane + 32 * q;
        if (e < alen) {
            int32_t k = aci[a0 + e];
            int64_t b0 = row_floor(brp, bci, k, floor);
            s_bst[w][e] = b0;
            len[q] = brp[k + 1] - b0;
        }
    }
    int64_t inc0 = warp_incl_scan(len[0]);
    int64_t tot0 = __shfl_sync(0xffffffffu, inc0, 31);
    int64_t inc1 = warp_incl_scan(len[1]) + tot0;
    s_off[w][lane] = inc0 - len[0];
    s_off[w][lane + 32] = inc1 - len[1];
    int64_t total = __shfl_sync(0xffffffffu, inc1, 31);
    __syncwarp();
    // element e = 2 * lane + q holds product e (column key, value); padding keys are INT_MAX
    int32_t key[2];
    double val[2];
    for (int q = 0; q < 2; ++q) {
        int e = 2 * lane + q;
        key[q] = 0x7fffffff;
        val[q] = 0.0;
        if (e < total) {
            int lo = 0, hi = (alen < 64 ? alen : 64) - 1;
            while (lo < hi) {
                int mid = (lo + hi + 1) >> 1;
                if (s_off[w][mid] <= e) lo = mid; else hi = mid - 1;
            }
            int64_t kb = s_bst[w][lo] + (e - s_off[w][lo]);
            key[q] = bci[kb];
            if (mode != 0) val[q] = av[a0 + lo] * bv[kb];
        }
    }
    // The distinct columns come out in ascending order from warp min-reductions over the lanes'
    // two keys (one round per column, which then leaves the candidates); two ballots per round
    // record the lanes that hold it, kept by lane c % 32 for the c-th column.  Each owner lane then
    // adds its column's products in product order (element 2 lane + q), the order a sparse
    // accumulator walking A's row and B's rows uses.
    if (mode != 0) {
        s_val[w][2 * lane] = val[0];
        s_val[w][2 * lane + 1] = val[1];
    }
    int32_t k0 = key[0], k1 = key[1];
    unsigned lo0 = 0, lo1 = 0, hi0 = 0, hi1 = 0;
    int32_t col_lo = 0, col_hi = 0;
    int distinct = 0;
    for (;;) {
        const int32_t m = __reduce_min_sync(0xffffffffu, k0 < k1 ? k0 : k1);
        if (m == 0x7fffffff) break;
        const unsigned b0 = __ballot_sync(0xffffffffu, k0 == m), b1 = __ballot_sync(0xffffffffu, k1 == m);
        if (lane == (distinct & 31)) {
            if (distinct < 32) { lo0 = b0; lo1 = b1; col_lo = m; }
            else { hi0 = b0; hi1 = b1; col_hi = m; }
        }
        if (k0 == m) k0 = 0x7fffffff;
        if (k1 == m) k1 = 0x7fffffff;
        ++distinct;
    }
    if (mode == 0) {
        if (lane == 0) cnt[i] = distinct;
        return;
    }
    // mode 1: the row at crp[i]; mode 2: at crp[li] (a temporary slot of the listed row), and the
    // count too (the one pass of the small bin, copied into place once the row pointers exist)
    if (mode == 2 && lane == 0) cnt[i] = distinct;
    const int64_t c0 = mode == 2 ? crp[li] : crp[i];
    __syncwarp();
    for (int r = 0; r < 2; ++r) {
        const int slot = lane + 32 * r;
        if (slot >= distinct) break;
        const unsigned b0 = r ? hi0 : lo0, b1 = r ? hi1 : lo1;
        unsigned any = b0 | b1;
        double sum = 0.0;
        while (any) {
            const int l = __ffs(any) - 1;
            any &= any - 1;
            if ((b0 >> l) & 1u) sum += s_val[w][2 * l];
            if ((b1 >> l) & 1u) sum += s_val[w][2 * l + 1];
        }
        cci[c0 + slot] = r ? col_hi : col_lo;
        cv[c0 + slot] = sum;
    }
}

// slot offsets of the listed rows: ub[rows[li]] (at most 64 each)
__global__ void k_list_ub(const int32_t* rows, int nrows, const int64_t* ub, int64_t* out) {
    int64_t li = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (li < nrows) out[li] = ub[rows[li]];
}
// copy the listed rows from their temporary slots into C (warp per row)
__global__ void k_copy_listed(const int32_t* rows, int nrows, const int64_t* toff, const int32_t* tci,
                              const double* tv, const int64_t* crp, int32_t* cci, double* cv) {
    int64_t li = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (li >= nrows) return;
    int64_t i = rows[li], c0 = crp[i], len = crp[i + 1] - c0, t0 = toff[li];
    for (int64_t e = lane; e < len; e += 32) {
        cci[c0 + e] = tci[t0 + e];
        cv[c0 + e] = tv[t0 + e];
    }
}

// flattened enumeration of the products of row i, 32 A-entries at a time
struct ProdWindow {
    int64_t off[32];
    int64_t bst[32];
    double av[32];
};

__device__ inline int64_t window_load(ProdWindow& W, const int32_t* bci, int32_t floor, int64_t base, int64_t a1,
                                      const int32_t* aci, const double* av, const int64_t* brp, int lane) {
    int64_t ka = base + lane;
    int64_t len = 0, bstart = 0;
    double aval = 0.0;
    if (ka < a1) {
        int32_t k = aci[ka];
        bstart = row_floor(brp, bci, k, floor);
        len = brp[k + 1] - bstart;
        aval = av ? av[ka] : 0.0;
    }
    int64_t inc = warp_incl_scan(len);
    W.off[lane] = inc - len;
    W.bst[lane] = bstart;
    W.av[lane] = aval;
    __syncwarp();
    return __shfl_sync(0xffffffffu, inc, 31);
}
__device__ inline int window_find(const ProdWindow& W, int64_t t) {
    int lo = 0, hi = 31;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (W.off[mid] <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// symbolic: distinct column count per listed row (0 and appended to big_list on overflow)
template <int SLOTS, int WARPS>
__global__ void __launch_bounds__(WARPS * 32)
k_spgemm_symbolic(const int64_t* arp, const int32_t* aci, const int64_t* brp, const int32_t* bci,
                  const int32_t* rows, int nrows, int upper, const int64_t* ub, int64_t* cnt, int32_t* big_list,
                  int* big_n) {
    __shared__ int32_t s_keys[WARPS][SLOTS];
    __shared__ ProdWindow s_win[WARPS];
    __shared__ int s_cnt[WARPS];
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int64_t li = (int64_t)blockIdx.x * WARPS + w;
    if (li >= nrows) return;
    int64_t i = rows[li];
    int32_t floor = upper ? (int32_t)i : -1;
    int32_t* keys = s_keys[w];
    int64_t ubi = ub[i];
    int tsize = 32;
    while (tsize < SLOTS && tsize < 2 * ubi) tsize <<= 1;
    int tmask = tsize - 1;
    int fill = SLOTS == MED_SLOTS ? MED_FILL : SLOTS;
    for (int t = lane; t < tsize; t += 32) keys[t] = -1;
    if (lane == 0) s_cnt[w] = 0;
    __syncwarp();
    bool overflow = false;
    int64_t a0 = arp[i], a1 = arp[i + 1];
    for (int64_t base = a0; base < a1 && !overflow; base += 32) {
        int64_t total = window_load(s_win[w], bci, floor, base, a1, aci, nullptr, brp, lane);
        for (int64_t t0 = 0; t0 < total; t0 += 32) {
            int64_t t = t0 + lane;
            if (t < total) {
                int lo = window_find(s_win[w], t);
                int32_t col = bci[s_win[w].bst[lo] + (t - s_win[w].off[lo])];
                uint32_t h = hslot(col, tmask);
                for (int probe = 0; probe < tsize; ++probe) {
                    int32_t cur = keys[h];
                    if (cur == col) break;
                    if (cur == -1) {
                        int32_t old = atomicCAS(&keys[h], -1, col);
                        if (old == -1) { atomicAdd(&s_cnt[w], 1); break; }
                        if (old == col) break;
                    }
                    h = (h + 1) & tmask;
                }
            }
            __syncwarp();
            if (s_cnt[w] > fill) { overflow = true; break; }
        }
        __syncwarp();
    }
    if (lane == 0) {
        if (overflow) {
            cnt[i] = 0;
            big_list[atomicAdd(big_n, 1)] = (int32_t)i;
        } else {
            cnt[i] = s_cnt[w];
        }
    }
}

// big path symbolic: one block per listed row
__global__ void k_spgemm_symbolic_big(const int64_t* arp, const int32_t* aci, const int64_t* brp,
                                      const int32_t* bci, const int32_t* list, int nlist, int upper, int64_t* cnt,
                                      int* fail) {
    extern __shared__ int32_t s_big[];
    __shared__ int s_n;
    for (int li = blockIdx.x; li < nlist; li += gridDim.x) {
        int64_t i = list[li];
        for (int t = threadIdx.x; t < BIG_SLOTS; t += blockDim.x) s_big[t] = -1;
        if (threadIdx.x == 0) s_n = 0;
        __syncthreads();
        int32_t floor = upper ? (int32_t)i : -1;
        for (int64_t ka = arp[i]; ka < arp[i + 1]; ++ka) {
            int32_t k = aci[ka];
            for (int64_t kb = row_floor(brp, bci, k, floor) + threadIdx.x; kb < brp[k + 1]; kb += blockDim.x) {
                int32_t col = bci[kb];
                uint32_t h = hslot(col, BIG_SLOTS - 1);
                for (int probe = 0; probe < BIG_SLOTS; ++probe) {
                    int32_t old = atomicCAS(&s_big[h], -1, col);
                    if (old == -1) { atomicAdd(&s_n, 1); break; }
                    if (old == col) break;
                    h = (h + 1) & (BIG_SLOTS - 1);
                }
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            cnt[i] = s_n;
            if (s_n > BIG_FILL) atomicExch(fail, 1);
        }
        __syncthreads();
    }
}

// Accumulate row i's products into a warp's table (keys, vals; tsize slots, all empty).  Products
// go round by round, 32 at a time in product order (A's row, then each B row).  A lane finds (or
// claims) its column's slot; the lanes of one slot are matched, and the lowest of them adds their
// a_ik b_kj to the slot with fused multiply-adds in lane order.  No FP64 atomics, and each
// column's sum is taken in product order.  Returns the number of columns, or -1 as soon as it
// exceeds `limit` (the table then stops growing: limit + 32 <= tsize).
__device__ inline int accumulate_row(int64_t i, int32_t floor, const int64_t* arp, const int32_t* aci,
                                     const double* av, const int64_t* brp, const int32_t* bci, const double* bv,
                                     int32_t* keys, double* vals, int tsize, int limit, ProdWindow& win,
                                     double* fa_s, double* fb_s, int lane) {
    const int tmask = tsize - 1;
    int count = 0;
    const int64_t a0 = arp[i], a1 = arp[i + 1];
    for (int64_t base = a0; base < a1; base += 32) {
        const int64_t total = window_load(win, bci, floor, base, a1, aci, av, brp, lane);
        for (int64_t t0 = 0; t0 < total; t0 += 32) {
            const int64_t t = t0 + lane;
            int slot = -1;
            bool ins = false;
            double fa = 0.0, fb = 0.0;
            if (t < total) {
                const int lo = window_find(win, t);
                const int64_t kb = win.bst[lo] + (t - win.off[lo]);
                const int32_t col = bci[kb];
                fa = win.av[lo];
                fb = bv[kb];
                uint32_t h = hslot(col, tmask);
                for (int probe = 0; probe < tsize; ++probe) {
                    const int32_t cur = keys[h];
                    if (cur == col) { slot = (int)h; break; }
                    if (cur == -1) {
                        const int32_t old = atomicCAS(&keys[h], -1, col);
                        if (old == -1 || old == col) { slot = (int)h; ins = old == -1; break; }
                    }
                    h = (h + 1) & tmask;
                }
            }
            fa_s[lane] = fa;
            fb_s[lane] = fb;
            const unsigned act = __ballot_sync(0xffffffffu, slot >= 0);
            count += __popc(__ballot_sync(0xffffffffu, ins));
            __syncwarp();
            if (slot >= 0) {
                const unsigned grp = __match_any_sync(act, slot);
                if (lane == __ffs(grp) - 1) {
                    double v = vals[slot];
                    for (unsigned g = grp; g; g &= g - 1) {
                        const int l = __ffs(g) - 1;
                        v = fma(fa_s[l], fb_s[l], v);
                    }
                    vals[slot] = v;
                }
            }
            __syncwarp();
            if (count > limit) return -1;
        }
        __syncwarp();
    }
    return count;
}
// Move the table's keys to its front (order kept); returns the count.
__device__ inline int compact_keys(int32_t* keys, double* vals, int tsize, int lane) {
    int count = 0;
    for (int t0 = 0; t0 < tsize; t0 += 32) {
        const int32_t k = keys[t0 + lane];
        const double vv = vals[t0 + lane];
        const unsigned m = __ballot_sync(0xffffffffu, k >= 0);
        const int pos = count + __popc(m & ((1u << lane) - 1u));
        __syncwarp();
        if (k >= 0) { keys[pos] = k; vals[pos] = vv; }
        count += __popc(m);
        __syncwarp();
    }
    return count;
}
// Write the count distinct keys (compacted, unsorted) and their values in ascending key order:
// a key's place is the number of smaller keys (broadcast reads of the list), cheaper than a
// sorting network for the few dozen to few hundred columns of a product row.
__device__ inline void write_ranked(const int32_t* keys, const double* vals, int count, int lane, int32_t* oc,
                                    double* ov) {
    for (int e = lane; e < count; e += 32) {
        const int32_t k = keys[e];
        int rank = 0;
        for (int j = 0; j < count; ++j) rank += keys[j] < k ? 1 : 0;
        oc[rank] = k;
        ov[rank] = vals[e];
    }
}
// numeric: accumulate in the table, compact in place, write the row in column order
template <int SLOTS, int WARPS>
__global__ void __launch_bounds__(WARPS * 32)
k_spgemm_numeric(const int64_t* arp, const int32_t* aci, const double* av, const int64_t* brp,
                 const int32_t* bci, const double* bv, const int32_t* rows, int nrows, int upper, const int64_t* crp,
                 int32_t* cci, double* cv) {
    __shared__ int32_t s_keys[WARPS][SLOTS];
    __shared__ double s_vals[WARPS][SLOTS];
    __shared__ ProdWindow s_win[WARPS];
    __shared__ double s_fa[WARPS][32], s_fb[WARPS][32];     // this round's factors, per lane
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int64_t li = (int64_t)blockIdx.x * WARPS + w;
    if (li >= nrows) return;
    int64_t i = rows[li];
    int32_t floor = upper ? (int32_t)i : -1;
    int32_t* keys = s_keys[w];
    double* vals = s_vals[w];
    int64_t c0 = crp[i];
    int clen = (int)(crp[i + 1] - c0);
    int fill = SLOTS == MED_SLOTS ? MED_FILL : SLOTS;
    if (clen > fill) return;  // big path
    int tsize = 32;                              // at most half full: the row's length is known
    while (tsize < SLOTS && tsize < 2 * clen) tsize <<= 1;
    for (int t = lane; t < tsize; t += 32) { keys[t] = -1; vals[t] = 0.0; }
    __syncwarp();
    accumulate_row(i, floor, arp, aci, av, brp, bci, bv, keys, vals, tsize, tsize, s_win[w], s_fa[w], s_fb[w], lane);
    const int count = compact_keys(keys, vals, tsize, lane);
    __syncwarp();
    write_ranked(keys, vals, count, lane, cci + c0, cv + c0);
}

// One pass for rows whose product count exceeds the register-sort bin: accumulate in a table of TS
// slots; a row of at most TS / 2 columns is written in column order to a temporary arena (sub-arena
// blockIdx % SPG_SUBS, reserved by that sub-arena's bump counter; its offset goes to moff[li], its
// length to cnt[i]).  A row with more columns, or one its sub-arena has no room for, gets
// moff[li] = -1 and joins the overflow list for the counting and numeric passes.
static constexpr int SPG_SUBS = 64;
template <int TS, int WARPS>
__global__ void __launch_bounds__(WARPS * 32)
k_spgemm_onepass(const int64_t* arp, const int32_t* aci, const double* av, const int64_t* brp, const int32_t* bci,
                 const double* bv, const int32_t* rows, int nrows, int upper, int64_t* cnt, int64_t* moff,
                 int32_t* tci, double* tv, unsigned long long* cursors, int64_t sub_cap, int32_t* ovf, int* novf) {
    __shared__ int32_t s_keys[WARPS][TS];
    __shared__ double s_vals[WARPS][TS];
    __shared__ ProdWindow s_win[WARPS];
    __shared__ double s_fa[WARPS][32], s_fb[WARPS][32];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t li = (int64_t)blockIdx.x * WARPS + w;
    if (li >= nrows) return;
    const int32_t i = rows[li];
    int32_t* keys = s_keys[w];
    double* vals = s_vals[w];
    for (int t = lane; t < TS; t += 32) { keys[t] = -1; vals[t] = 0.0; }
    __syncwarp();
    int count = accumulate_row(i, upper ? i : -1, arp, aci, av, brp, bci, bv, keys, vals, TS, TS / 2, s_win[w],
                               s_fa[w], s_fb[w], lane);
    int64_t dst = -1;
    if (count >= 0) {
        count = compact_keys(keys, vals, TS, lane);
        __syncwarp();
        const int sub = blockIdx.x % SPG_SUBS;
        unsigned long long at = 0;
        if (lane == 0) at = atomicAdd(&cursors[sub], (unsigned long long)count);
        at = __shfl_sync(0xffffffffu, at, 0);
        if ((int64_t)at + count <= sub_cap) dst = (int64_t)sub * sub_cap + (int64_t)at;
    }
    if (dst < 0) {
        if (lane == 0) {
            moff[li] = -1;
            ovf[atomicAdd(novf, 1)] = i;
        }
        return;
    }
    write_ranked(keys, vals, count, lane, tci + dst, tv + dst);
    if (lane == 0) {
        moff[li] = dst;
        cnt[i] = count;
    }
}
// copy the one-pass rows (moff >= 0) from the arena into C (G lanes per row)
template <int G>
__global__ void k_copy_arena(const int32_t* rows, int nrows, const int64_t* moff, const int32_t* tci, const double* tv,
                             const int64_t* crp, int32_t* cci, double* cv) {
    const int64_t li = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
    const int lane = threadIdx.x & (G - 1);
    if (li >= nrows) return;
    const int64_t t0 = moff[li];
    if (t0 < 0) return;
    const int64_t i = rows[li], c0 = crp[i], len = crp[i + 1] - c0;
    for (int64_t e = lane; e < len; e += G) {
        cci[c0 + e] = tci[t0 + e];
        cv[c0 + e] = tv[t0 + e];
    }
}
// bound on the columns of the listed rows that the one pass keeps: sum of min(products, cap)
__global__ void k_sum_capped(const int32_t* rows, int nrows, const int64_t* ub, int64_t cap_small, int64_t cap_big,
                             int64_t big_from, unsigned long long* out) {
    const int64_t li = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long v = 0;
    if (li < nrows) {
        const int64_t u = ub[rows[li]];
        const int64_t cap = u > big_from ? cap_big : cap_small;
        v = (unsigned long long)(u < cap ? u : cap);
    }
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(out, v);
}

__global__ void k_spgemm_numeric_big(const int64_t* arp, const int32_t* aci, const double* av,
                                     const int64_t* brp, const int32_t* bci, const double* bv,
                                     const int32_t* list, int nlist, int upper, const int64_t* crp, int32_t* cci,
                                     double* cv) {
    extern __shared__ unsigned char smem_raw[];
    int32_t* keys = (int32_t*)smem_raw;
    double* vals = (double*)(smem_raw + sizeof(int32_t) * BIG_SLOTS);
    __shared__ int32_t s_ck[1024];
    for (int li = blockIdx.x; li < nlist; li += gridDim.x) {
        int64_t i = list[li];
        for (int t = threadIdx.x; t < BIG_SLOTS; t += blockDim.x) { keys[t] = -1; vals[t] = 0.0; }
        __syncthreads();
        int32_t floor = upper ? (int32_t)i : -1;
        for (int64_t ka = arp[i]; ka < arp[i + 1]; ++ka) {
            int32_t k = aci[ka];
            double a = av[ka];
            for (int64_t kb = row_floor(brp, bci, k, floor) + threadIdx.x; kb < brp[k + 1]; kb += blockDim.x) {
                int32_t col = bci[kb];
                uint32_t h = hslot(col, BIG_SLOTS - 1);
                for (int probe = 0; probe < BIG_SLOTS; ++probe) {
                    int32_t old = atomicCAS(&keys[h], -1, col);
                    if (old == -1 || old == col) { atomicAdd(&vals[h], a * bv[kb]); break; }
                    h = (h + 1) & (BIG_SLOTS - 1);
                }
            }
        }
        __syncthreads();
        int64_t c0 = crp[i];
        for (int t0 = 0; t0 < BIG_SLOTS; t0 += blockDim.x) {
            int t = t0 + threadIdx.x;
            int32_t k = t < BIG_SLOTS ? keys[t] : -1;
            int rank = 0;
            for (int u0 = 0; u0 < BIG_SLOTS; u0 += 1024) {
                __syncthreads();
                for (int q = threadIdx.x; q < 1024; q += blockDim.x) s_ck[q] = keys[u0 + q];
                __syncthreads();
                if (k >= 0)
                    for (int q = 0; q < 1024; ++q) rank += (s_ck[q] >= 0 && s_ck[q] < k);
            }
            if (k >= 0) {
                cci[c0 + rank] = k;
                cv[c0 + rank] = vals[t];
            }
        }
        __syncthreads();
    }
}

template <int SLOTS, int WARPS>
static void launch_symbolic(const DCSR& A, const DCSR& B, const int32_t* rows, int nrows, int upper, const int64_t* ub,
                            int64_t* cnt, int32_t* big, int* bign, cudaStream_t s) {
    if (nrows <= 0) return;
    SPHC_LAUNCH((k_spgemm_symbolic<SLOTS, WARPS><<<(nrows + WARPS - 1) / WARPS, WARPS * 32, 0, s>>>(
        A.rp.p, A.ci.p, B.rp.p, B.ci.p, rows, nrows, upper, ub, cnt, big, bign)));
}
template <int SLOTS, int WARPS>
static void launch_numeric(const DCSR& A, const DCSR& B, DCSR& C, const int32_t* rows, int nrows, int upper,
                           cudaStream_t s) {
    if (nrows <= 0) return;
    SPHC_LAUNCH((k_spgemm_numeric<SLOTS, WARPS><<<(nrows + WARPS - 1) / WARPS, WARPS * 32, 0, s>>>(
        A.rp.p, A.ci.p, A.v.p, B.rp.p, B.ci.p, B.v.p, rows, nrows, upper, C.rp.p, C.ci.p, C.v.p)));
}

// Numeric bins by output row length (known once the symbolic pass has run): a row's table holds
// at most twice its columns, so rows with many products but few columns (the P^T (A P) rows of a
// Galerkin product: thousands of products, tens of columns) take small tables and many warps
// share an SM.  Bin b holds rows of at most 32 << b columns (tables of 64 << b slots); rows above
// MED_FILL columns are on the big path.
static constexpr int NUM_BINS = 5;
static constexpr int NUM_REBIN_MIN_ROWS = 1 << 16;
__device__ inline int numeric_bin_of(int64_t clen) {
    if (clen > MED_FILL) return -1;
    int b = 0;
    while (b < NUM_BINS - 1 && clen > (32 << b)) ++b;
    return b;
}
__global__ void k_numeric_bin_count(const int32_t* rows, int nrows, const int64_t* crp, int* bin_cnt) {
    const int64_t li = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int bin = -1;
    if (li < nrows) {
        const int32_t i = rows[li];
        bin = numeric_bin_of(crp[i + 1] - crp[i]);
    }
    for (int b = 0; b < NUM_BINS; ++b) {
        const int c = __syncthreads_count(bin == b);
        if (threadIdx.x == 0 && c) atomicAdd(&bin_cnt[b], c);
    }
}
__global__ void k_numeric_bin_fill(const int32_t* rows, int nrows, const int64_t* crp, const int* bin_off,
                                   int* bin_fill, int32_t* out) {
    const int64_t li = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (li >= nrows) return;
    const int32_t i = rows[li];
    const int bin = numeric_bin_of(crp[i + 1] - crp[i]);
    if (bin < 0) return;
    const unsigned m = __match_any_sync(__activemask(), bin);
    const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(&bin_fill[bin], __popc(m));
    base = __shfl_sync(m, base, leader);
    out[bin_off[bin] + base + __popc(m & ((1u << lane) - 1u))] = i;
}
// the numeric pass of the listed rows (their row pointers in C already set), binned by length
static int numeric_by_length(const DCSR& A, const DCSR& B, DCSR& C, const int32_t* rows, int nrows, int upper,
                             cudaStream_t s) {
    if (nrows <= 0) return SPHC_OK;
    DBuf<int> cnt;                       // 0..4 counts, 5..9 offsets, 10..14 fill
    DBuf<int32_t> list;
    SPHC_TRY(cnt.alloc(3 * NUM_BINS, s));
    SPHC_TRY(cnt.zero(s));
    SPHC_TRY(list.alloc(nrows, s));
    SPHC_LAUNCH(k_numeric_bin_count<<<grid_for(nrows, 256), 256, 0, s>>>(rows, nrows, C.rp.p, cnt.p));
    int h[NUM_BINS] = {0};
    SPHC_CK(cudaMemcpyAsync(h, cnt.p, sizeof(h), cudaMemcpyDeviceToHost, s));
    SPHC_CK(cudaStreamSynchronize(s));
    int off[NUM_BINS];
    off[0] = 0;
    for (int b = 1; b < NUM_BINS; ++b) off[b] = off[b - 1] + h[b - 1];
    SPHC_CK(cudaMemcpyAsync(cnt.p + NUM_BINS, off, sizeof(off), cudaMemcpyHostToDevice, s));
    SPHC_LAUNCH(k_numeric_bin_fill<<<grid_for(nrows, 256), 256, 0, s>>>(rows, nrows, C.rp.p, cnt.p + NUM_BINS,
                                                                         cnt.p + 2 * NUM_BINS, list.p));
    launch_numeric<64, 16>(A, B, C, list.p + off[0], h[0], upper, s);
    launch_numeric<128, 16>(A, B, C, list.p + off[1], h[1], upper, s);
    launch_numeric<256, 8>(A, B, C, list.p + off[2], h[2], upper, s);
    launch_numeric<512, 4>(A, B, C, list.p + off[3], h[3], upper, s);
    launch_numeric<1024, 2>(A, B, C, list.p + off[4], h[4], upper, s);
    SPHC_CK(cudaGetLastError());
    return SPHC_OK;
}


static int spgemm_impl(const DCSR& A, const DCSR& B, DCSR& C, int upper, cudaStream_t s) {
    const int paths = spgemm_path_flags();
    if (A.nc != B.nr) {
        set_error("spgemm: inner dimensions %lld vs %lld", (long long)A.nc, (long long)B.nr);
        return SPHC_EINVAL;
    }
    int64_t n = A.nr;
    if (n >= (1LL << 31)) { set_error("spgemm: %lld rows exceed int32 row lists", (long long)n); return SPHC_ELIMIT; }
    DBuf<int64_t> ub, cnt;
    DBuf<int32_t> big, rows;
    DBuf<int> flags;                 // 0 bign, 1 fail, 2..5 bin counts, 6..9 bin offsets, 10..13 bin fill
    DBuf<int64_t> toff;              // small bin: temporary slot offsets, then its rows
    DBuf<int32_t> tci;
    DBuf<double> tv;
    int64_t tslots = 0;
    bool small_one_pass = false;
    // rows of the hash bins in one pass into an arena (k_spgemm_onepass), overflow rows listed
    DBuf<int64_t> moff;
    DBuf<int32_t> mci, ovf;
    DBuf<double> mv;
    DBuf<unsigned long long> curs;
    bool med_one_pass = false;
    SPHC_TRY(ub.alloc(n + 1, s));
    SPHC_TRY(cnt.alloc(n + 1, s));
    SPHC_TRY(big.alloc(n + 1, s));
    SPHC_TRY(rows.alloc(n + 1, s));
    SPHC_TRY(flags.alloc(16, s));
    SPHC_TRY(flags.zero(s));
    int h[16] = {0};
    if (n > 0) {
        // lanes per row of the count: the mean A row length over 4, a power of two from 1 to 32
        double avg = (double)A.nnz / (double)n;
        int g = 1;
        while (g < 32 && 4 * g < avg) g <<= 1;
        switch (g) {
#define UB(G) SPHC_LAUNCH(k_spgemm_ub<G><<<grid_for(n * G, 256), 256, 0, s>>>(A.rp.p, A.ci.p, B.rp.p, B.ci.p, n, upper, ub.p, flags.p + 2))
            case 1: UB(1); break;
            case 2: UB(2); break;
            case 4: UB(4); break;
            case 8: UB(8); break;
            case 16: UB(16); break;
            default: UB(32); break;
#undef UB
        }
        SPHC_CK(cudaMemcpyAsync(h, flags.p, 16 * sizeof(int), cudaMemcpyDeviceToHost, s));
        SPHC_CK(cudaStreamSynchronize(s));
        int off[NBINS] = {0, h[2], h[2] + h[3], h[2] + h[3] + h[4]};
        SPHC_CK(cudaMemcpyAsync(flags.p + 6, off, NBINS * sizeof(int), cudaMemcpyHostToDevice, s));
        SPHC_LAUNCH(k_spgemm_bin<<<grid_for(n, 256), 256, 0, s>>>(A.rp.p, ub.p, n, flags.p + 6, flags.p + 10, rows.p));
        if (h[2] > 0) {
            // small bin in one pass: sorted rows into temporary slots of ub entries each, while
            // those slots take at most a quarter of the free device memory; else a counting pass
            // and a writing pass
            DBuf<int64_t> lub;
            SPHC_TRY(lub.alloc(h[2], s));
            SPHC_TRY(toff.alloc(h[2] + 1, s));               // the scan also writes the total
            SPHC_LAUNCH(k_list_ub<<<grid_for(h[2], 256), 256, 0, s>>>(rows.p, h[2], ub.p, lub.p));
            SPHC_TRY(exclusive_scan_i64(lub.p, toff.p, h[2], s, &tslots));
            size_t fr = 0, tt = 0;
            small_one_pass = !(paths & 1) && cudaMemGetInfo(&fr, &tt) == cudaSuccess &&
                             (double)tslots * (sizeof(int32_t) + sizeof(double)) <= 0.25 * (double)fr;
            cudaGetLastError();
            if (small_one_pass) {
                SPHC_TRY(tci.alloc(tslots > 0 ? tslots : 1, s));
                SPHC_TRY(tv.alloc(tslots > 0 ? tslots : 1, s));
                SPHC_LAUNCH(k_spgemm_small<<<(h[2] + SMALL_WARPS - 1) / SMALL_WARPS, SMALL_WARPS * 32, 0, s>>>(
                    A.rp.p, A.ci.p, A.v.p, B.rp.p, B.ci.p, B.v.p, rows.p, h[2], 2, upper, cnt.p, toff.p, tci.p, tv.p));
            } else {
                SPHC_LAUNCH(k_spgemm_small<<<(h[2] + SMALL_WARPS - 1) / SMALL_WARPS, SMALL_WARPS * 32, 0, s>>>(
                    A.rp.p, A.ci.p, A.v.p, B.rp.p, B.ci.p, B.v.p, rows.p, h[2], 0, upper, cnt.p, nullptr, nullptr,
                    nullptr));
            }
        }
        // The hash bins in one pass where the arena fits a quarter of the free memory: its size is
        // the sum over the rows of min(products, columns a table keeps), at most four times the
        // larger operand's nonzeros (rows that find their sub-arena full fall back).  Otherwise,
        // and for the overflow rows, a counting pass first.
        const int nmed = h[3] + h[4] + h[5];
        if (nmed > 0 && !(paths & 8)) {
            DBuf<unsigned long long> bsum;
            SPHC_TRY(bsum.alloc(1, s));
            SPHC_TRY(bsum.zero(s));
            // Upper triangles keep about half of a row's columns: on products with many long rows
            // (the Galerkin product of the finest level) tables of 256 slots (at most 128 columns)
            // let twice the warps hide the latency of the gathered B rows; a mid level's few long
            // rows overflow them more often than that gains.
            const bool small_tables = upper && ((paths & 64) || h[5] >= NUM_REBIN_MIN_ROWS);
            SPHC_LAUNCH(k_sum_capped<<<grid_for(nmed, 256), 256, 0, s>>>(rows.p + off[1], nmed, ub.p, 64,
                                                                          small_tables ? 128 : 256, 256, bsum.p));
            unsigned long long hb = 0;
            SPHC_CK(cudaMemcpyAsync(&hb, bsum.p, sizeof(hb), cudaMemcpyDeviceToHost, s));
            SPHC_CK(cudaStreamSynchronize(s));
            const int64_t cap_total = std::min<int64_t>((int64_t)hb, 4 * std::max<int64_t>(A.nnz, B.nnz));
            const int64_t sub_cap = (paths & 16) ? 64 : (cap_total + SPG_SUBS - 1) / SPG_SUBS + 512;
            size_t fr = 0, tt = 0;
            med_one_pass = cudaMemGetInfo(&fr, &tt) == cudaSuccess &&
                           (double)SPG_SUBS * (double)sub_cap * (sizeof(int32_t) + sizeof(double)) <= 0.25 * (double)fr;
            cudaGetLastError();
            if (med_one_pass) {
                SPHC_TRY(moff.alloc(nmed, s));
                SPHC_TRY(ovf.alloc(nmed, s));
                SPHC_TRY(mci.alloc((int64_t)SPG_SUBS * sub_cap, s));
                SPHC_TRY(mv.alloc((int64_t)SPG_SUBS * sub_cap, s));
                SPHC_TRY(curs.alloc(SPG_SUBS, s));
                SPHC_TRY(curs.zero(s));
                const int part[3] = {h[3], h[4], h[5]};
                int64_t first = 0;
                for (int b = 0; b < 3; ++b) {
                    const int nr = part[b];
                    if (nr > 0) {
                        const int32_t* rl = rows.p + off[1] + first;
                        if (b < 2)
                            SPHC_LAUNCH((k_spgemm_onepass<128, 16><<<(nr + 15) / 16, 512, 0, s>>>(
                                A.rp.p, A.ci.p, A.v.p, B.rp.p, B.ci.p, B.v.p, rl, nr, upper, cnt.p, moff.p + first,
                                mci.p, mv.p, curs.p, sub_cap, ovf.p, flags.p + 14)));
                        else if (small_tables)  // see below
                            SPHC_LAUNCH((k_spgemm_onepass<256, 8><<<(nr + 7) / 8, 256, 0, s>>>(
                                A.rp.p, A.ci.p, A.v.p, B.rp.p, B.ci.p, B.v.p, rl, nr, upper, cnt.p, moff.p + first,
                                mci.p, mv.p, curs.p, sub_cap, ovf.p, flags.p + 14)));
                        else
                            SPHC_LAUNCH((k_spgemm_onepass<512, 4><<<(nr + 3) / 4, 128, 0, s>>>(
                                A.rp.p, A.ci.p, A.v.p, B.rp.p, B.ci.p, B.v.p, rl, nr, upper, cnt.p, moff.p + first,
                                mci.p, mv.p, curs.p, sub_cap, ovf.p, flags.p + 14)));
                    }
                    first += nr;
                }
            }
        }
        if (!med_one_pass) {
            launch_symbolic<256, 8>(A, B, rows.p + off[1], h[3], upper, ub.p, cnt.p, big.p, flags.p, s);
            launch_symbolic<512, 8>(A, B, rows.p + off[2], h[4], upper, ub.p, cnt.p, big.p, flags.p, s);
            launch_symbolic<1024, 8>(A, B, rows.p + off[3], h[5], upper, ub.p, cnt.p, big.p, flags.p, s);
        }
    }
    SPHC_CK(cudaGetLastError());
    int novf = 0;
    if (med_one_pass) {
        SPHC_CK(cudaMemcpyAsync(&novf, flags.p + 14, sizeof(int), cudaMemcpyDeviceToHost, s));
        SPHC_CK(cudaStreamSynchronize(s));
        if (novf > 0) launch_symbolic<1024, 8>(A, B, ovf.p, novf, upper, ub.p, cnt.p, big.p, flags.p, s);
    }
    int nbig = 0;
    SPHC_CK(cudaMemcpyAsync(&nbig, flags.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    SPHC_CK(cudaStreamSynchronize(s));
    size_t big_sym_sm = sizeof(int32_t) * BIG_SLOTS;
    size_t big_num_sm = (sizeof(int32_t) + sizeof(double)) * BIG_SLOTS;
    if (nbig > 0) {
        SPHC_CK(cudaFuncSetAttribute(k_spgemm_symbolic_big, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)big_sym_sm));
        SPHC_LAUNCH(k_spgemm_symbolic_big<<<nbig < 4096 ? nbig : 4096, 512, big_sym_sm, s>>>(
            A.rp.p, A.ci.p, B.rp.p, B.ci.p, big.p, nbig, upper, cnt.p, flags.p + 1));
        int f = 0;
        SPHC_CK(cudaMemcpyAsync(&f, flags.p + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
        SPHC_CK(cudaStreamSynchronize(s));
        if (f) {
            set_error("spgemm: a product row has more than %d columns", BIG_FILL);
            return SPHC_ELIMIT;
        }
    }
    int64_t nnz = 0;
    SPHC_TRY(C.alloc(n, B.nc, 0, s));
    SPHC_TRY(exclusive_scan_i64(cnt.p, C.rp.p, n, s, &nnz));
    C.nnz = nnz;
    SPHC_TRY(C.ci.alloc(nnz, s));
    SPHC_TRY(C.v.alloc(nnz, s));
    if (n > 0) {
        int off[NBINS] = {0, h[2], h[2] + h[3], h[2] + h[3] + h[4]};
        if (h[2] > 0 && small_one_pass)
            SPHC_LAUNCH(k_copy_listed<<<grid_for((int64_t)h[2] * 32, 256), 256, 0, s>>>(rows.p, h[2], toff.p, tci.p, tv.p,
                                                                                      C.rp.p, C.ci.p, C.v.p));
        else if (h[2] > 0)
            SPHC_LAUNCH(k_spgemm_small<<<(h[2] + SMALL_WARPS - 1) / SMALL_WARPS, SMALL_WARPS * 32, 0, s>>>(
                A.rp.p, A.ci.p, A.v.p, B.rp.p, B.ci.p, B.v.p, rows.p, h[2], 1, upper, nullptr, C.rp.p, C.ci.p, C.v.p));
        // Re-binned by length where the rows fill the GPU many times over; a few thousand rows
        // of long product lists (the Galerkin product of a mid level) run better as one launch
        // per product-count bin than split over length bins that each wait for their longest row.
        const int nmed = h[3] + h[4] + h[5];
        if (med_one_pass) {
            if (nmed > 0) {
                // lanes per row from the mean output row
                const double avg = (double)nnz / (double)(n > 0 ? n : 1);
#define CA(G) SPHC_LAUNCH((k_copy_arena<G><<<grid_for((int64_t)nmed * G, 256), 256, 0, s>>>( \
                    rows.p + off[1], nmed, moff.p, mci.p, mv.p, C.rp.p, C.ci.p, C.v.p)))
                if (avg <= 12) CA(8);
                else if (avg <= 24) CA(16);
                else CA(32);
#undef CA
            }
            if (novf > 0) SPHC_TRY(numeric_by_length(A, B, C, ovf.p, novf, upper, s));
        } else if ((paths & 2) || (!(paths & 4) && nmed >= NUM_REBIN_MIN_ROWS)) {
            SPHC_TRY(numeric_by_length(A, B, C, rows.p + off[1], nmed, upper, s));
        } else {
            launch_numeric<256, 4>(A, B, C, rows.p + off[1], h[3], upper, s);
            launch_numeric<512, 4>(A, B, C, rows.p + off[2], h[4], upper, s);
            launch_numeric<1024, 2>(A, B, C, rows.p + off[3], h[5], upper, s);
        }
    }
    if (nbig > 0) {
        SPHC_CK(cudaFuncSetAttribute(k_spgemm_numeric_big, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)big_num_sm));
        SPHC_LAUNCH(k_spgemm_numeric_big<<<nbig < 4096 ? nbig : 4096, 512, big_num_sm, s>>>(
            A.rp.p, A.ci.p, A.v.p, B.rp.p, B.ci.p, B.v.p, big.p, nbig, upper, C.rp.p, C.ci.p, C.v.p));
    }
    SPHC_CK(cudaGetLastError());
    return SPHC_OK;
}

int spgemm(const DCSR& A, const DCSR& B, DCSR& C, cudaStream_t s) { return spgemm_impl(A, B, C, 0, s); }

// Full symmetric matrix from its upper triangle U (diagonal included): row i is row i of U^T
// without its diagonal (the columns below i), then row i of U.  Both parts are sorted and
// disjoint, so the row is their concatenation; the lower triangle holds exact copies.
__global__ void k_sym_count(const int64_t* urp, const int64_t* trp, const int32_t* tci, int64_t n, int64_t* cnt) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t t0 = trp[i], t1 = trp[i + 1];
    int64_t below = t1 - t0 - ((t1 > t0 && tci[t1 - 1] == i) ? 1 : 0);
    cnt[i] = below + (urp[i + 1] - urp[i]);
}
__global__ void k_sym_fill(const int64_t* urp, const int32_t* uci, const double* uv, const int64_t* trp,
                           const int32_t* tci, const double* tv, int64_t n, const int64_t* crp, int32_t* cci,
                           double* cv) {
    int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (i >= n) return;
    int64_t t0 = trp[i], t1 = trp[i + 1];
    int64_t below = t1 - t0 - ((t1 > t0 && tci[t1 - 1] == i) ? 1 : 0);
    int64_t c0 = crp[i];
    for (int64_t q = lane; q < below; q += 32) { cci[c0 + q] = tci[t0 + q]; cv[c0 + q] = tv[t0 + q]; }
    int64_t u0 = urp[i], ul = urp[i + 1] - u0;
    for (int64_t q = lane; q < ul; q += 32) { cci[c0 + below + q] = uci[u0 + q]; cv[c0 + below + q] = uv[u0 + q]; }
}

int spgemm_sym(const DCSR& A, const DCSR& B, DCSR& C, cudaStream_t s) {
    DCSR U, Ut;
    SPHC_TRY(spgemm_impl(A, B, U, 1, s));
    if (U.nr != U.nc) { set_error("spgemm_sym: product is %lld x %lld", (long long)U.nr, (long long)U.nc); return SPHC_EINVAL; }
    SPHC_TRY(transpose(U, Ut, s));
    int64_t n = U.nr;
    DBuf<int64_t> cnt;
    SPHC_TRY(cnt.alloc(n + 1, s));
    if (n > 0) SPHC_LAUNCH(k_sym_count<<<grid_for(n, 256), 256, 0, s>>>(U.rp.p, Ut.rp.p, Ut.ci.p, n, cnt.p));
    C = DCSR();
    C.nr = n;
    C.nc = n;
    SPHC_TRY(C.rp.alloc(n + 1, s));
    SPHC_TRY(exclusive_scan_i64(cnt.p, C.rp.p, n, s, &C.nnz));
    SPHC_TRY(C.ci.alloc(C.nnz, s));
    SPHC_TRY(C.v.alloc(C.nnz, s));
    if (n > 0)
        SPHC_LAUNCH(k_sym_fill<<<grid_for(n * 32, 256), 256, 0, s>>>(U.rp.p, U.ci.p, U.v.p, Ut.rp.p, Ut.ci.p, Ut.v.p, n,
                                                                    C.rp.p, C.ci.p, C.v.p));
    SPHC_CK(cudaGetLastError());
    return SPHC_OK;
}

// ------------------------------------------------------------------ FP64 SpMV, dots
__global__ void k_spmv64(const int64_t* rp, const int32_t* ci, const double* v, int64_t n, const double* x,
                         double* y) {
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t i = g >> 3;
    int sub = threadIdx.x & 7;
    bool valid = i < n;
    double s = 0.0;
    if (valid)
        for (int64_t k = rp[i] + sub; k < rp[i + 1]; k += 8) s += v[k] * x[ci[k]];
    s += __shfl_xor_sync(0xffffffffu, s, 4);
    s += __shfl_xor_sync(0xffffffffu, s, 2);
    s += __shfl_xor_sync(0xffffffffu, s, 1);
    if (valid && sub == 0) y[i] = s;
}
int spmv64(const DCSR& A, const double* x, double* y, cudaStream_t s) {
    if (A.nr > 0) SPHC_LAUNCH(k_spmv64<<<grid_for(A.nr * 8, 256), 256, 0, s>>>(A.rp.p, A.ci.p, A.v.p, A.nr, x, y));
    SPHC_CK(cudaGetLastError());
    return SPHC_OK;
}

static constexpr int DOT_BLOCKS = 1024;
__global__ void k_dot_part(const double* a, const double* b, int64_t n, double* part) {
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
__global__ void k_dot_final(const double* part, int np, double* out) {
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
int dot64(const double* a, const double* b, int64_t n, double* result_dev, cudaStream_t s) {
    DBuf<double> part;
    SPHC_TRY(part.alloc(DOT_BLOCKS, s));
    SPHC_LAUNCH(k_dot_part<<<DOT_BLOCKS, 256, 0, s>>>(a, b, n, part.p));
    SPHC_LAUNCH(k_dot_final<<<1, 1024, 0, s>>>(part.p, DOT_BLOCKS, result_dev));
    SPHC_CK(cudaGetLastError());
    return SPHC_OK;
}

}  // namespace sphc
