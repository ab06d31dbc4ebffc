// sphc_relres_noalloc: the true relative residual ||b - A_e x|| / ||b|| of up to
// SPHC_NOALLOC_MAX_RHS right-hand sides, computed without allocating any memory.
//
// Some callers cannot call cudaMalloc: code that runs while a memory pool is being resized or
// from inside another allocator's callbacks, processes whose device memory is fully reserved
// by a framework, or real-time loops that forbid allocation after start-up.  The residual check
// that sphc_solve performs needs per-block partial sums; here they live in a fixed, file-scope
// device array instead of memory obtained at call time.
#include <cmath>
#include <mutex>

#include "sphc_level.cuh"

using namespace sphc;

namespace {

constexpr int NA_BLOCKS = 256;       // partial sums per right-hand side
constexpr int NA_THREADS = 256;
constexpr int NA_STRIDE = 2 * NA_BLOCKS + 1;   // per RHS: r.r partials, b.b partials, result
constexpr int NA_MAX_DEVICES = 64;

// Shared by every call on a device and kept until the process exits (about 257 KB).
static __device__ __align__(256) double g_noalloc_scratch[SPHC_NOALLOC_MAX_RHS * NA_STRIDE];

// Device address of g_noalloc_scratch for each device, resolved once with that device current.
std::mutex g_na_mutex;
double* g_na_ptr[NA_MAX_DEVICES] = {nullptr};

int scratch_for_device(int dev, double** out) {
    if (dev < 0 || dev >= NA_MAX_DEVICES) {
        set_error("sphc_relres_noalloc: device %d is beyond the %d devices supported", dev, NA_MAX_DEVICES);
        return SPHC_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) {
            set_error("sphc_relres_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
            return SPHC_ECUDA;
        }
        g_na_ptr[dev] = (double*)p;
    }
    *out = g_na_ptr[dev];
    return SPHC_OK;
}

// Where p lives: 0 host (or unknown to CUDA), 1 device memory of `dev` or managed memory, -1
// device memory of another GPU (a kernel here would read a peer address: rejected).
int placement(const void* p, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (a.type == cudaMemoryTypeManaged) return 1;
    if (a.type == cudaMemoryTypeDevice) return a.device == dev ? 1 : -1;
    return 0;
}

// grid (NA_BLOCKS, nrhs): block partial sums of (b - A x)_i^2 and b_i^2 for one right-hand side
__global__ void __launch_bounds__(NA_THREADS)
k_na_partial(const int64_t* __restrict__ rp, const int32_t* __restrict__ ci, const double* __restrict__ v, int64_t n,
             const double* __restrict__ b, const double* __restrict__ x, double* scratch) {
    __shared__ double s_rr[NA_THREADS / 32], s_bb[NA_THREADS / 32];
    int k = blockIdx.y;
    const double* bk = b + (int64_t)k * n;
    const double* xk = x + (int64_t)k * n;
    int sub = threadIdx.x & 7;
    double rr = 0.0, bb = 0.0;
    int64_t rows_per_pass = (int64_t)gridDim.x * (NA_THREADS / 8);
    for (int64_t base = (int64_t)blockIdx.x * (NA_THREADS / 8); base < n; base += rows_per_pass) {
        int64_t i = base + (threadIdx.x >> 3);
        bool valid = i < n;
        double s = 0.0;
        if (valid)
            for (int64_t e = rp[i] + sub; e < rp[i + 1]; e += 8) s += v[e] * xk[ci[e]];
        s += __shfl_xor_sync(0xffffffffu, s, 4);
        s += __shfl_xor_sync(0xffffffffu, s, 2);
        s += __shfl_xor_sync(0xffffffffu, s, 1);
        if (valid && sub == 0) {
            double r = bk[i] - s;
            rr += r * r;
            bb += bk[i] * bk[i];
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        rr += __shfl_down_sync(0xffffffffu, rr, o);
        bb += __shfl_down_sync(0xffffffffu, bb, o);
    }
    if ((threadIdx.x & 31) == 0) {
        s_rr[threadIdx.x >> 5] = rr;
        s_bb[threadIdx.x >> 5] = bb;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, c = 0.0;
        for (int w = 0; w < NA_THREADS / 32; ++w) { a += s_rr[w]; c += s_bb[w]; }
        double* part = scratch + (int64_t)k * NA_STRIDE;
        part[blockIdx.x] = a;
        part[NA_BLOCKS + blockIdx.x] = c;
    }
}

// one block per right-hand side: reduce the partials in a fixed order
__global__ void k_na_final(double* scratch) {
    __shared__ double s_rr[NA_BLOCKS], s_bb[NA_BLOCKS];
    double* part = scratch + (int64_t)blockIdx.x * NA_STRIDE;
    for (int t = threadIdx.x; t < NA_BLOCKS; t += blockDim.x) {
        s_rr[t] = part[t];
        s_bb[t] = part[NA_BLOCKS + t];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double rr = 0.0, bb = 0.0;
        for (int t = 0; t < NA_BLOCKS; ++t) { rr += s_rr[t]; bb += s_bb[t]; }
        part[2 * NA_BLOCKS] = bb > 0.0 ? sqrt(rr) / sqrt(bb) : 0.0;
    }
}

__global__ void k_na_gather(const double* scratch, int nrhs, double* out) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < nrhs) out[k] = scratch[(int64_t)k * NA_STRIDE + 2 * NA_BLOCKS];
}

}  // namespace

extern "C" int sphc_relres_noalloc(const sphc_handle* h, const double* b, const double* x, int nrhs, double* relres,
                                   void* stream) {
    if (!h || !b || !x || !relres) {
        set_error("sphc_relres_noalloc: NULL argument");
        return SPHC_EINVAL;
    }
    if (nrhs < 1 || nrhs > SPHC_NOALLOC_MAX_RHS) {
        set_error("sphc_relres_noalloc: nrhs = %d is outside 1..%d, the right-hand sides its fixed scratch holds",
                  nrhs, SPHC_NOALLOC_MAX_RHS);
        return SPHC_EINVAL;
    }
    int dev = 0;
    SPHC_CK(cudaGetDevice(&dev));
    if (dev != h->device) {
        set_error("sphc_relres_noalloc: the current device %d is not the handle's device %d", dev, h->device);
        return SPHC_EINVAL;
    }
    int pb = placement(b, dev), px = placement(x, dev), pr = placement(relres, dev);
    if (pb != 1 || px != 1) {
        set_error("sphc_relres_noalloc: b and x must be memory of the handle's device %d (host data would need a "
                  "staging copy; another GPU's memory is not read)", dev);
        return SPHC_EINVAL;
    }
    if (pr < 0) {
        set_error("sphc_relres_noalloc: relres is memory of another GPU than the handle's device %d", dev);
        return SPHC_EINVAL;
    }
    double* scratch = nullptr;
    SPHC_TRY(scratch_for_device(dev, &scratch));
    const DCSR& A = h->H.L[0].A;
    cudaStream_t s = (cudaStream_t)stream;
    SPHC_LAUNCH(k_na_partial<<<dim3(NA_BLOCKS, nrhs), NA_THREADS, 0, s>>>(A.rp.p, A.ci.p, A.v.p, A.nr, b, x, scratch));
    SPHC_LAUNCH(k_na_final<<<nrhs, 256, 0, s>>>(scratch));
    if (pr == 1) {
        SPHC_LAUNCH(k_na_gather<<<1, 64, 0, s>>>(scratch, nrhs, relres));
    } else {
        for (int k = 0; k < nrhs; ++k)
            SPHC_CK(cudaMemcpyAsync(relres + k, scratch + (int64_t)k * NA_STRIDE + 2 * NA_BLOCKS, sizeof(double),
                                    cudaMemcpyDeviceToHost, s));
    }
    SPHC_CK(cudaGetLastError());
    SPHC_CK(cudaStreamSynchronize(s));
    return SPHC_OK;
}
