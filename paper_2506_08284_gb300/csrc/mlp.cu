// The learned warm start of the edge prolongator (not part of the paper): a multilayer perceptron
// of SPHC_MLP_NFEAT inputs, two hidden ReLU layers of SPHC_MLP_HIDDEN units and one output,
// which predicts the correction (P_e after several energy-minimisation steps) - (least-norm P0)
// of one pattern entry from local features.  Its output always passes through the exact
// constraint projection before use, so the commuting relation P_e D_H = D_h P_n still holds.
//
// Inference: bf16 weights and activations on the fifth-generation tensor cores (tcgen05 MMAs,
// FP32 accumulators in tensor memory).  Training: FP32 forward / backward GEMM kernels and Adam.
#include <cmath>
#include <cstring>
#include <vector>

#include <cuda_bf16.h>

#include "features.cuh"
#include "sphc_level.cuh"
#include "tc.cuh"

using namespace sphc;

namespace sphc {

constexpr int NF = SPHC_MLP_NFEAT;     // 32
constexpr int NH = SPHC_MLP_HIDDEN;    // 128
// parameter block offsets (floats)
constexpr int P_MU = 0, P_SD = NF, P_W1 = 2 * NF, P_B1 = P_W1 + NF * NH, P_W2 = P_B1 + NH, P_B2 = P_W2 + NH * NH,
              P_W3 = P_B2 + NH, P_B3 = P_W3 + NH, P_TOTAL = P_B3 + 1;
static_assert(P_TOTAL == SPHC_MLP_NPARAM, "parameter layout");

// ------------------------------------------------------------------ inference on tensor cores
// Two blocks per SM walk tiles of 128 pattern entries.  Per tile: the normalised features go to
// shared memory as the bf16 A operand (K = 32); one thread issues the first layer as tcgen05 MMAs
// (M = 128, N = 128, FP32 accumulator D1 in tensor memory); eight warps read D1 back (warp w:
// rows 32 (w % 4) .., columns 64 (w / 4) ..), add the bias, apply ReLU and store the bf16 hidden
// layer as the A operand of the second layer (K = 128, accumulator D2); the output layer is a dot
// product of ReLU(D2 + b2) with w3 in the same epilogue pattern.  Weights are staged once per block.
constexpr int TILE_M = 128;           // pattern entries per tile (MMA M)
constexpr int TC_THREADS = 256;       // 8 warps; two threads per tile row compute its features
static_assert(TC_THREADS == 2 * TILE_M, "two threads per tile row compute its features");
constexpr uint32_t TC_COLS = 256;     // half of tensor memory: D1 at column 0, D2 at column 128
constexpr uint32_t TC_D2 = 128;
constexpr int TC_WAIT = 1 << 20;      // polls of an MMA-completion wait before the kernel gives up
// Dynamic shared memory per block: more than a third of an SM's, so at most two blocks share an
// SM and their two 256-column allocations never wait for each other.
constexpr size_t TC_SMEM = 100 * 1024;
constexpr int TC_BLOCKS_PER_SM = 2;

// Operands start on 1 KB boundaries, each followed by 1 KB that no descriptor of the layout
// reaches (a margin should a descriptor field be read as a swizzled layout).
struct __align__(1024) TcSmem {
    __nv_bfloat16 a1[TILE_M * NF];    // features, K-major core matrices
    unsigned char g0[1024];
    __nv_bfloat16 w1[NH * NF];        // W1 transposed ([out][in]), K-major core matrices
    unsigned char g1[1024];
    __nv_bfloat16 a2[TILE_M * NH];    // hidden layer
    unsigned char g2[1024];
    __nv_bfloat16 w2[NH * NH];        // W2 transposed
    unsigned char g3[1024];
    float b1[NH], b2[NH], w3[NH], mu[NF], isd[NF], part[TILE_M];
    uint64_t bar;
    uint32_t tmem;
};
static_assert(sizeof(TcSmem) <= TC_SMEM, "shared memory layout");

// element offset of (row r, column k) in a K-major bf16 operand of K columns: core matrix
// (r / 8, k / 8) at ((r / 8) (K / 8) + k / 8) * 64 elements, rows of 8 elements inside
__device__ __forceinline__ int cm_off(int r, int k, int K) {
    return (((r >> 3) * (K >> 3) + (k >> 3)) << 6) + ((r & 7) << 3) + (k & 7);
}
// descriptor of K-step ks (16 columns) of a K-major operand: adjacent core matrices are 128 bytes
// apart along K and (K / 8) * 128 bytes apart along the rows
__device__ __forceinline__ uint64_t op_desc(const __nv_bfloat16* M, int K, int ks) {
    return tc_desc(reinterpret_cast<const unsigned char*>(M) + 256 * ks, 128u, (uint32_t)(K / 8) * 128u);
}

// FUSED: the features of tile row r (pattern entry base + r, in fine row rowof[base + r]) are
// computed in place from the level's operators instead of being read from X.
template <bool FUSED>
__global__ void __launch_bounds__(TC_THREADS, TC_BLOCKS_PER_SM)
k_mlp_infer(const float* __restrict__ params, const float* __restrict__ X, int64_t m, FeatArgs g,
            const int32_t* __restrict__ rowof, float* __restrict__ out, int* err, int polls) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    TcSmem& S = *reinterpret_cast<TcSmem*>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    for (int q = tid; q < NF; q += blockDim.x) {
        S.mu[q] = params[P_MU + q];
        float sd = params[P_SD + q];
        S.isd[q] = sd > 0.f ? 1.f / sd : 0.f;
    }
    for (int q = tid; q < NH; q += blockDim.x) {
        S.b1[q] = params[P_B1 + q];
        S.b2[q] = params[P_B2 + q];
        S.w3[q] = params[P_W3 + q];
    }
    for (int q = tid; q < NF * NH; q += blockDim.x) {
        int i = q / NH, o = q % NH;                    // W1[i][o]
        S.w1[cm_off(o, i, NF)] = __float2bfloat16(params[P_W1 + q]);
    }
    for (int q = tid; q < NH * NH; q += blockDim.x) {
        int i = q / NH, o = q % NH;                    // W2[i][o]
        S.w2[cm_off(o, i, NH)] = __float2bfloat16(params[P_W2 + q]);
    }
    const float b3 = params[P_B3];
    if (tid == 0) tc_bar_init(&S.bar, 1);
    if (w == 0) {
        tc_alloc(&S.tmem, TC_COLS);
        tc_relinquish();
    }
    tc_fence_smem_to_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = S.tmem;
    const uint32_t idesc = tc_idesc_bf16(TILE_M, NH);
    const int q4 = w & 3, half = w >> 2, row = 32 * q4 + lane;
    const uint32_t lane_off = (uint32_t)(32 * q4) << 16;
    uint32_t phase = 0;
    bool failed = false;
    for (int64_t base = (int64_t)blockIdx.x * TILE_M; base < m && !failed; base += (int64_t)gridDim.x * TILE_M) {
        // normalised features of the tile (rows past m are zero)
        if (FUSED) {
            // two threads per entry: part 0 (geometry, row quantities) and part 1 (row lookups)
            int r = tid % TILE_M, part = tid / TILE_M;
            int64_t e = base + r;
            float f[NF];
            if (e < m) entry_features(g, rowof[e], e, f, part);
            for (int c = 0; c < NF; ++c)
                if (feat_part(c) == part)
                    S.a1[cm_off(r, c, NF)] = __float2bfloat16(e < m ? (f[c] - S.mu[c]) * S.isd[c] : 0.f);
        } else {
            for (int q = tid; q < TILE_M * NF; q += blockDim.x) {
                int r = q / NF, c = q % NF;
                int64_t e = base + r;
                float v = e < m ? (X[e * NF + c] - S.mu[c]) * S.isd[c] : 0.f;
                S.a1[cm_off(r, c, NF)] = __float2bfloat16(v);
            }
        }
        // layer 1: D1 = x W1
        tc_fence_smem_to_async();
        tc_fence_before();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
#pragma unroll
            for (int ks = 0; ks < NF / 16; ++ks) tc_mma(tmem, op_desc(S.a1, NF, ks), op_desc(S.w1, NF, ks), idesc, ks > 0);
            tc_commit(&S.bar);
        }
        bool ok = polls > 0 ? tc_bar_poll(&S.bar, phase, polls) : tc_bar_wait(&S.bar, phase, TC_WAIT);
        phase ^= 1u;
        if (__syncthreads_or(!ok)) { failed = true; break; }
        tc_fence_after();
        // h1 = relu(D1 + b1) -> bf16 A operand of layer 2
#pragma unroll
        for (int cc = 0; cc < 2; ++cc) {
            float v[32];
            tc_ld32(tmem + lane_off + (uint32_t)(64 * half + 32 * cc), v);
#pragma unroll
            for (int j8 = 0; j8 < 32; j8 += 8) {         // 8 columns = one 16-byte row of a core matrix
                const int n0 = 64 * half + 32 * cc + j8;
                uint32_t pk[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const __nv_bfloat16 lo = __float2bfloat16(fmaxf(v[j8 + 2 * q] + S.b1[n0 + 2 * q], 0.f));
                    const __nv_bfloat16 hi = __float2bfloat16(fmaxf(v[j8 + 2 * q + 1] + S.b1[n0 + 2 * q + 1], 0.f));
                    pk[q] = (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
                }
                *reinterpret_cast<uint4*>(&S.a2[cm_off(row, n0, NH)]) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
            }
        }
        // layer 2: D2 = h1 W2
        tc_fence_smem_to_async();
        tc_fence_before();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
#pragma unroll
            for (int ks = 0; ks < NH / 16; ++ks)
                tc_mma(tmem + TC_D2, op_desc(S.a2, NH, ks), op_desc(S.w2, NH, ks), idesc, ks > 0);
            tc_commit(&S.bar);
        }
        ok = polls > 0 ? tc_bar_poll(&S.bar, phase, polls) : tc_bar_wait(&S.bar, phase, TC_WAIT);
        phase ^= 1u;
        if (__syncthreads_or(!ok)) { failed = true; break; }
        tc_fence_after();
        // y = relu(D2 + b2) . w3 + b3, each half of the columns by its own warps
        float y = 0.f;
#pragma unroll
        for (int cc = 0; cc < 2; ++cc) {
            float v[32];
            tc_ld32(tmem + lane_off + TC_D2 + (uint32_t)(64 * half + 32 * cc), v);
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const int n = 64 * half + 32 * cc + j;
                y += fmaxf(v[j] + S.b2[n], 0.f) * S.w3[n];
            }
        }
        if (half == 1) S.part[row] = y;
        tc_fence_before();                   // tensor-memory reads done before the next tile's MMAs
        __syncthreads();
        if (half == 0 && base + row < m) out[base + row] = y + S.part[row] + b3;
    }
    if (failed) {
        // a completion wait gave up: report, give the MMA in flight one more wait with the full
        // limit (it must complete before its tensor memory is freed), and release the memory
        if (tid == 0) atomicExch(err, 1);
        if (!tc_bar_wait(&S.bar, phase ^ 1u, TC_WAIT) && tid == 0) atomicExch(err, 2);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (w == 0) tc_dealloc(tmem, TC_COLS);
}

static int infer_grid(int64_t m) {
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (nsm <= 0) nsm = 1;
    int64_t tiles = (m + TILE_M - 1) / TILE_M;
    int64_t cap = (int64_t)nsm * TC_BLOCKS_PER_SM;
    return (int)(tiles < cap ? tiles : cap);
}

// launch one of the inference kernels (as clusters of one CTA: the MMA commit addresses its
// mbarrier in the cluster window) and report a completion wait that gave up
template <bool FUSED>
static int launch_infer(const float* params_dev, const float* X, int64_t m, const FeatArgs& g, const int32_t* rowof,
                        float* out, cudaStream_t s, int polls) {
    SPHC_CK(cudaFuncSetAttribute(k_mlp_infer<FUSED>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM));
    DBuf<int> err;
    SPHC_TRY(err.alloc(1, s));
    SPHC_TRY(err.zero(s));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(infer_grid(m));
    cfg.blockDim = dim3(TC_THREADS);
    cfg.dynamicSmemBytes = TC_SMEM;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 1;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    g_launches.fetch_add(1, std::memory_order_relaxed);
    SPHC_CK(cudaLaunchKernelEx(&cfg, k_mlp_infer<FUSED>, params_dev, X, m, g, rowof, out, err.p, polls));
    int h = 0;
    SPHC_CK(cudaMemcpyAsync(&h, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    SPHC_CK(cudaStreamSynchronize(s));
    if (h) {
        set_error("MLP inference: a tensor-core completion wait exceeded its limit of %d %s polls%s",
                  polls > 0 ? polls : TC_WAIT, polls > 0 ? "non-blocking" : "blocking",
                  h == 2 ? " (and the drain wait before freeing tensor memory gave up too)" : "");
        return SPHC_ETIMEOUT;
    }
    return SPHC_OK;
}

int mlp_predict(const float* params_dev, const float* X, int64_t m, float* out, cudaStream_t s) {
    if (m <= 0) return SPHC_OK;
    return launch_infer<false>(params_dev, X, m, FeatArgs(), nullptr, out, s, 0);
}

// row of every pattern entry (warp per row)
__global__ void k_row_of(const int64_t* nrp, int64_t ne, int32_t* rowof) {
    int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (i >= ne) return;
    for (int64_t q = nrp[i] + lane; q < nrp[i + 1]; q += 32) rowof[q] = (int32_t)i;
}

int mlp_predict_level(const float* params_dev, const FeatArgs& g, float* out, cudaStream_t s, int polls) {
    int64_t m = g.nnzN;
    if (m <= 0) return SPHC_OK;
    DBuf<int32_t> rowof;
    SPHC_TRY(rowof.alloc(m, s));
    SPHC_LAUNCH(k_row_of<<<grid_for(g.ne * 32, 256), 256, 0, s>>>(g.nrp, g.ne, rowof.p));
    return launch_infer<true>(params_dev, nullptr, m, g, rowof.p, out, s, polls);
}

// ------------------------------------------------------------------ training (FP32)
// C[M x N] = op(A) op(B) (+ C if beta), row-major; op = transpose when the flag is set.
// A is M x K (or K x M transposed), B is K x N (or N x K transposed).
constexpr int GT = 32;
__global__ void k_gemm(int M, int N, int K, const float* A, int lda, int ta, const float* B, int ldb, int tb, float* C,
                       int ldc, int beta) {
    __shared__ float As[GT][GT + 1], Bs[GT][GT + 1];
    int tx = threadIdx.x % GT, ty = threadIdx.x / GT;   // 32 x 8 threads, 4 rows each
    int row0 = blockIdx.y * GT, col0 = blockIdx.x * GT;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int k0 = 0; k0 < K; k0 += GT) {
        for (int q = 0; q < 4; ++q) {
            int r = ty + 8 * q;
            int gr = row0 + r, gk = k0 + tx;
            float va = 0.f;
            if (gr < M && gk < K) va = ta ? A[(int64_t)gk * lda + gr] : A[(int64_t)gr * lda + gk];
            As[r][tx] = va;
            int bk = k0 + r, bc = col0 + tx;
            float vb = 0.f;
            if (bk < K && bc < N) vb = tb ? B[(int64_t)bc * ldb + bk] : B[(int64_t)bk * ldb + bc];
            Bs[r][tx] = vb;
        }
        __syncthreads();
        for (int kk = 0; kk < GT; ++kk) {
            float b = Bs[kk][tx];
            for (int q = 0; q < 4; ++q) acc[q] += As[ty + 8 * q][kk] * b;
        }
        __syncthreads();
    }
    for (int q = 0; q < 4; ++q) {
        int r = row0 + ty + 8 * q, c = col0 + tx;
        if (r < M && c < N) {
            float* p = C + (int64_t)r * ldc + c;
            *p = beta ? *p + acc[q] : acc[q];
        }
    }
}
static void gemm(int M, int N, int K, const float* A, int lda, int ta, const float* B, int ldb, int tb, float* C, int ldc,
                 int beta, cudaStream_t s) {
    dim3 grid((N + GT - 1) / GT, (M + GT - 1) / GT);
    SPHC_LAUNCH(k_gemm<<<grid, 256, 0, s>>>(M, N, K, A, lda, ta, B, ldb, tb, C, ldc, beta));
}

// gather a minibatch: rows idx[b] of X, normalised with (mu, sd); targets y
__global__ void k_gather_batch(const float* X, const float* y, const int64_t* idx, int B, const float* params, float* xb,
                               float* yb) {
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= B * NF) return;
    int b = q / NF, c = q % NF;
    int64_t r = idx[b];
    float sd = params[P_SD + c];
    xb[q] = sd > 0.f ? (X[r * NF + c] - params[P_MU + c]) / sd : 0.f;
    if (c == 0) yb[b] = y[r];
}
__global__ void k_batch_index(int64_t m, int B, uint64_t seed, uint64_t step, int64_t* idx) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < B) idx[b] = (int64_t)(splitmix64(seed ^ (step * 0x9E3779B97F4A7C15ULL), (uint64_t)b) % (uint64_t)m);
}
__global__ void k_bias_relu(float* Z, const float* bias, int B, int N, float* H) {
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= B * N) return;
    float z = Z[q] + bias[q % N];
    Z[q] = z;
    H[q] = z > 0.f ? z : 0.f;
}
// output layer, loss and its gradient: y = H2 w3 + b3, dy = 2 (y - t) / B
__global__ void k_out_loss(const float* H2, const float* w3, const float* b3, const float* t, int B, float* dy,
                           float* loss) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    float l = 0.f;
    if (b < B) {
        float y = b3[0];
        for (int c = 0; c < NH; ++c) y += H2[(int64_t)b * NH + c] * w3[c];
        float e = y - t[b];
        dy[b] = 2.f * e / B;
        l = e * e / B;
    }
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, l);
}
// dH2[b][c] = dy[b] w3[c] masked by relu'(Z2);  grad w3 = H2^T dy and b3 = sum dy (block sums)
__global__ void k_back_out(const float* H2, const float* Z2, const float* w3, const float* dy, int B, float* dZ2) {
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= B * NH) return;
    int b = q / NH, c = q % NH;
    dZ2[q] = Z2[q] > 0.f ? dy[b] * w3[c] : 0.f;
}
__global__ void k_colsum(const float* M, int B, int N, float* out) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    float s = 0.f;
    for (int b = 0; b < B; ++b) s += M[(int64_t)b * N + c];
    out[c] = s;
}
__global__ void k_relu_mask(float* dH, const float* Z, int n) {
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < n && !(Z[q] > 0.f)) dH[q] = 0.f;
}
// Adam on the weights (normalisation constants are not trained)
__global__ void k_adam(float* p, const float* g, float* m1, float* m2, int n, int first, float lr, float b1, float b2,
                       float eps, float bc1, float bc2, float wd) {
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    int k = first + q;
    float gr = g[k] + wd * p[k];
    m1[k] = b1 * m1[k] + (1.f - b1) * gr;
    m2[k] = b2 * m2[k] + (1.f - b2) * gr * gr;
    p[k] -= lr * (m1[k] / bc1) / (sqrtf(m2[k] / bc2) + eps);
}

// gradient of the mean squared error of one batch (params on the device); grad[P_TOTAL]
struct TrainWork {
    DBuf<float> xb, yb, z1, h1, z2, h2, dy, dz2, dh1, loss;
    int alloc(int B, cudaStream_t s) {
        SPHC_TRY(xb.alloc((int64_t)B * NF, s));
        SPHC_TRY(yb.alloc(B, s));
        SPHC_TRY(z1.alloc((int64_t)B * NH, s));
        SPHC_TRY(h1.alloc((int64_t)B * NH, s));
        SPHC_TRY(z2.alloc((int64_t)B * NH, s));
        SPHC_TRY(h2.alloc((int64_t)B * NH, s));
        SPHC_TRY(dy.alloc(B, s));
        SPHC_TRY(dz2.alloc((int64_t)B * NH, s));
        SPHC_TRY(dh1.alloc((int64_t)B * NH, s));
        SPHC_TRY(loss.alloc(1, s));
        return SPHC_OK;
    }
};

static void batch_gradient(const float* params, TrainWork& W, int B, float* grad, cudaStream_t s) {
    const float* W1 = params + P_W1;
    const float* W2 = params + P_W2;
    // forward
    gemm(B, NH, NF, W.xb.p, NF, 0, W1, NH, 0, W.z1.p, NH, 0, s);
    SPHC_LAUNCH(k_bias_relu<<<grid_for((int64_t)B * NH, 256), 256, 0, s>>>(W.z1.p, params + P_B1, B, NH, W.h1.p));
    gemm(B, NH, NH, W.h1.p, NH, 0, W2, NH, 0, W.z2.p, NH, 0, s);
    SPHC_LAUNCH(k_bias_relu<<<grid_for((int64_t)B * NH, 256), 256, 0, s>>>(W.z2.p, params + P_B2, B, NH, W.h2.p));
    cudaMemsetAsync(W.loss.p, 0, sizeof(float), s);
    SPHC_LAUNCH(k_out_loss<<<grid_for(B, 256), 256, 0, s>>>(W.h2.p, params + P_W3, params + P_B3, W.yb.p, B, W.dy.p,
                                                            W.loss.p));
    // backward
    gemm(NH, 1, B, W.h2.p, NH, 1, W.dy.p, 1, 0, grad + P_W3, 1, 0, s);            // w3 = H2^T dy
    SPHC_LAUNCH(k_colsum<<<1, 32, 0, s>>>(W.dy.p, B, 1, grad + P_B3));
    SPHC_LAUNCH(k_back_out<<<grid_for((int64_t)B * NH, 256), 256, 0, s>>>(W.h2.p, W.z2.p, params + P_W3, W.dy.p, B,
                                                                          W.dz2.p));
    gemm(NH, NH, B, W.h1.p, NH, 1, W.dz2.p, NH, 0, grad + P_W2, NH, 0, s);       // W2 = H1^T dZ2
    SPHC_LAUNCH(k_colsum<<<1, NH, 0, s>>>(W.dz2.p, B, NH, grad + P_B2));
    gemm(B, NH, NH, W.dz2.p, NH, 0, W2, NH, 1, W.dh1.p, NH, 0, s);               // dH1 = dZ2 W2^T
    SPHC_LAUNCH(k_relu_mask<<<grid_for((int64_t)B * NH, 256), 256, 0, s>>>(W.dh1.p, W.z1.p, B * NH));
    gemm(NF, NH, B, W.xb.p, NF, 1, W.dh1.p, NH, 0, grad + P_W1, NH, 0, s);       // W1 = X^T dZ1
    SPHC_LAUNCH(k_colsum<<<1, NH, 0, s>>>(W.dh1.p, B, NH, grad + P_B1));
}

}  // namespace sphc

extern "C" {

int sphc_default_train_opts(sphc_train_opts* o) {
    if (!o) return SPHC_EINVAL;
    memset(o, 0, sizeof(*o));
    o->steps = 3000;
    o->batch = 4096;
    o->lr = 1e-3f;
    o->beta1 = 0.9f;
    o->beta2 = 0.999f;
    o->eps = 1e-8f;
    o->weight_decay = 0.f;
    o->seed = 1;
    return SPHC_OK;
}

int sphc_mlp_predict(const float* params, const float* X, int64_t m, float* out, void* stream) {
    if (!params || (m > 0 && (!X || !out)) || m < 0) {
        set_error("sphc_mlp_predict: invalid argument");
        return SPHC_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    DBuf<float> P, Xd, Od;
    SPHC_TRY(P.alloc(SPHC_MLP_NPARAM, s));
    SPHC_CK(cudaMemcpyAsync(P.p, params, sizeof(float) * SPHC_MLP_NPARAM, cudaMemcpyDefault, s));
    const float* xp = X;
    float* op = out;
    cudaPointerAttributes a;
    bool xdev = cudaPointerGetAttributes(&a, X) == cudaSuccess && (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged);
    cudaGetLastError();
    bool odev = cudaPointerGetAttributes(&a, out) == cudaSuccess && (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged);
    cudaGetLastError();
    if (!xdev) {
        SPHC_TRY(Xd.alloc(m * SPHC_MLP_NFEAT, s));
        SPHC_CK(cudaMemcpyAsync(Xd.p, X, sizeof(float) * m * SPHC_MLP_NFEAT, cudaMemcpyDefault, s));
        xp = Xd.p;
    }
    if (!odev) {
        SPHC_TRY(Od.alloc(m, s));
        op = Od.p;
    }
    SPHC_TRY(mlp_predict(P.p, xp, m, op, s));
    if (!odev) SPHC_CK(cudaMemcpyAsync(out, Od.p, sizeof(float) * m, cudaMemcpyDefault, s));
    SPHC_CK(cudaStreamSynchronize(s));
    return SPHC_OK;
}

int sphc_mlp_gradient(const float* params, const float* X, const float* y, int B, float* grad, float* loss,
                      void* stream) {
    if (!params || !X || !y || !grad || B < 1) {
        set_error("sphc_mlp_gradient: invalid argument");
        return SPHC_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    DBuf<float> P, G;
    DBuf<int64_t> idx;
    TrainWork W;
    SPHC_TRY(P.alloc(SPHC_MLP_NPARAM, s));
    SPHC_TRY(G.alloc(SPHC_MLP_NPARAM, s));
    SPHC_TRY(G.zero(s));
    SPHC_TRY(W.alloc(B, s));
    SPHC_CK(cudaMemcpyAsync(P.p, params, sizeof(float) * SPHC_MLP_NPARAM, cudaMemcpyDefault, s));
    DBuf<float> Xd, yd;
    SPHC_TRY(Xd.alloc((int64_t)B * NF, s));
    SPHC_TRY(yd.alloc(B, s));
    SPHC_CK(cudaMemcpyAsync(Xd.p, X, sizeof(float) * B * NF, cudaMemcpyDefault, s));
    SPHC_CK(cudaMemcpyAsync(yd.p, y, sizeof(float) * B, cudaMemcpyDefault, s));
    SPHC_TRY(idx.alloc(B, s));
    std::vector<int64_t> hidx(B);
    for (int b = 0; b < B; ++b) hidx[b] = b;
    SPHC_CK(cudaMemcpyAsync(idx.p, hidx.data(), sizeof(int64_t) * B, cudaMemcpyHostToDevice, s));
    SPHC_LAUNCH(k_gather_batch<<<grid_for((int64_t)B * NF, 256), 256, 0, s>>>(Xd.p, yd.p, idx.p, B, P.p, W.xb.p, W.yb.p));
    batch_gradient(P.p, W, B, G.p, s);
    SPHC_CK(cudaMemcpyAsync(grad, G.p, sizeof(float) * SPHC_MLP_NPARAM, cudaMemcpyDefault, s));
    if (loss) SPHC_CK(cudaMemcpyAsync(loss, W.loss.p, sizeof(float), cudaMemcpyDefault, s));
    SPHC_CK(cudaStreamSynchronize(s));
    return SPHC_OK;
}

int sphc_mlp_train(const float* X, const float* y, int64_t m, const sphc_train_opts* opts, float* params,
                   float* loss_history, void* stream) {
    if (!X || !y || !params || m < 1) {
        set_error("sphc_mlp_train: invalid argument");
        return SPHC_EINVAL;
    }
    sphc_train_opts o;
    if (opts) o = *opts;
    else sphc_default_train_opts(&o);
    if (o.steps < 0 || o.batch < 1 || !(o.lr > 0.f)) {
        set_error("sphc_mlp_train: invalid options");
        return SPHC_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    DBuf<float> Xd, yd, P, G, M1, M2, L;
    SPHC_TRY(Xd.alloc(m * NF, s));
    SPHC_TRY(yd.alloc(m, s));
    SPHC_CK(cudaMemcpyAsync(Xd.p, X, sizeof(float) * m * NF, cudaMemcpyDefault, s));
    SPHC_CK(cudaMemcpyAsync(yd.p, y, sizeof(float) * m, cudaMemcpyDefault, s));
    SPHC_TRY(P.alloc(SPHC_MLP_NPARAM, s));
    SPHC_TRY(G.alloc(SPHC_MLP_NPARAM, s));
    SPHC_TRY(M1.alloc(SPHC_MLP_NPARAM, s));
    SPHC_TRY(M2.alloc(SPHC_MLP_NPARAM, s));
    SPHC_TRY(M1.zero(s));
    SPHC_TRY(M2.zero(s));
    SPHC_TRY(L.alloc(o.steps > 0 ? o.steps : 1, s));
    SPHC_CK(cudaMemcpyAsync(P.p, params, sizeof(float) * SPHC_MLP_NPARAM, cudaMemcpyDefault, s));
    TrainWork W;
    SPHC_TRY(W.alloc(o.batch, s));
    DBuf<int64_t> idx;
    SPHC_TRY(idx.alloc(o.batch, s));
    int nw = P_TOTAL - P_W1;
    for (int step = 0; step < o.steps; ++step) {
        SPHC_LAUNCH(k_batch_index<<<grid_for(o.batch, 256), 256, 0, s>>>(m, o.batch, o.seed, (uint64_t)step, idx.p));
        SPHC_LAUNCH(k_gather_batch<<<grid_for((int64_t)o.batch * NF, 256), 256, 0, s>>>(Xd.p, yd.p, idx.p, o.batch, P.p,
                                                                                       W.xb.p, W.yb.p));
        batch_gradient(P.p, W, o.batch, G.p, s);
        SPHC_CK(cudaMemcpyAsync(L.p + step, W.loss.p, sizeof(float), cudaMemcpyDeviceToDevice, s));
        float bc1 = 1.f - powf(o.beta1, (float)(step + 1)), bc2 = 1.f - powf(o.beta2, (float)(step + 1));
        SPHC_LAUNCH(k_adam<<<grid_for(nw, 256), 256, 0, s>>>(P.p, G.p, M1.p, M2.p, nw, P_W1, o.lr, o.beta1, o.beta2,
                                                            o.eps, bc1, bc2, o.weight_decay));
    }
    SPHC_CK(cudaMemcpyAsync(params, P.p, sizeof(float) * SPHC_MLP_NPARAM, cudaMemcpyDefault, s));
    if (loss_history && o.steps > 0)
        SPHC_CK(cudaMemcpyAsync(loss_history, L.p, sizeof(float) * o.steps, cudaMemcpyDefault, s));
    SPHC_CK(cudaGetLastError());
    SPHC_CK(cudaStreamSynchronize(s));
    return SPHC_OK;
}

}  // extern "C"
