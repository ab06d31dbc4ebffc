// The learned warm start of the edge prolongator (not part of the paper): a multilayer perceptron
// of SPHC_MLP_NFEAT inputs, two hidden ReLU layers of SPHC_MLP_HIDDEN units and one output,
// which predicts the correction (P_e after several energy-minimisation steps) - (least-norm P0)
// of one pattern entry from local features.  Its output always passes through the exact
// constraint projection before use, so the commuting relation P_e D_H = D_h P_n still holds.
//
// Inference: BF16 weights and activations on the tensor cores (mma.sync m16n8k16, FP32
// accumulate).  Training: FP32 forward / backward GEMM kernels and Adam.
#include <cmath>
#include <cstring>
#include <vector>

#include <cuda_bf16.h>

#include "features.cuh"
#include "sphc_level.cuh"

using namespace sphc;

namespace sphc {

constexpr int NF = SPHC_MLP_NFEAT;     // 32
constexpr int NH = SPHC_MLP_HIDDEN;    // 128
// parameter block offsets (floats)
constexpr int P_MU = 0, P_SD = NF, P_W1 = 2 * NF, P_B1 = P_W1 + NF * NH, P_W2 = P_B1 + NH, P_B2 = P_W2 + NH * NH,
              P_W3 = P_B2 + NH, P_B3 = P_W3 + NH, P_TOTAL = P_B3 + 1;
static_assert(P_TOTAL == SPHC_MLP_NPARAM, "parameter layout");

// ------------------------------------------------------------------ inference on tensor cores
constexpr int TILE_M = 128;           // rows (pattern entries) per block
constexpr int INF_WARPS = 8;          // each warp owns 16 rows
constexpr int XS = NF + 8;            // padded shared-memory row strides (bf16 elements)
static_assert(INF_WARPS * 32 == 2 * TILE_M, "two threads per tile row compute its features");
constexpr int HS = NH + 8;

struct InferSmem {
    __nv_bfloat16 x[TILE_M * XS];
    __nv_bfloat16 w1t[NH * XS];       // W1 transposed: [out][in]
    __nv_bfloat16 w2t[NH * HS];       // W2 transposed: [out][in]
    __nv_bfloat16 h1[TILE_M * HS];
    float b1[NH], b2[NH], w3[NH], mu[NF], isd[NF];
};

__device__ inline uint32_t pack_bf16(__nv_bfloat16 lo, __nv_bfloat16 hi) {
    uint32_t a = (uint32_t)__bfloat16_as_ushort(lo), b = (uint32_t)__bfloat16_as_ushort(hi);
    return a | (b << 16);
}
__device__ inline uint32_t ld_pair(const __nv_bfloat16* p) { return *(const uint32_t*)p; }

// D(16x8, f32) += A(16x16, bf16, row) * B(16x8, bf16, col)
__device__ inline void mma_bf16(float d[4], const uint32_t a[4], const uint32_t b[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// A fragment of rows [r0, r0+16), columns [k0, k0+16) of a row-major bf16 matrix (stride ld)
__device__ inline void load_a(uint32_t a[4], const __nv_bfloat16* M, int ld, int r0, int k0, int lane) {
    int g = lane >> 2, t = lane & 3;
    a[0] = ld_pair(M + (r0 + g) * ld + k0 + 2 * t);
    a[1] = ld_pair(M + (r0 + g + 8) * ld + k0 + 2 * t);
    a[2] = ld_pair(M + (r0 + g) * ld + k0 + 8 + 2 * t);
    a[3] = ld_pair(M + (r0 + g + 8) * ld + k0 + 8 + 2 * t);
}
// B fragment of k rows [k0, k0+16), n columns [n0, n0+8) from a transposed ([n][k]) matrix
__device__ inline void load_b(uint32_t b[2], const __nv_bfloat16* Mt, int ld, int n0, int k0, int lane) {
    int g = lane >> 2, t = lane & 3;
    b[0] = ld_pair(Mt + (n0 + g) * ld + k0 + 2 * t);
    b[1] = ld_pair(Mt + (n0 + g) * ld + k0 + 8 + 2 * t);
}

// FUSED: the features of tile row r (pattern entry base + r, in fine row rowof[base + r]) are
// computed in place from the level's operators instead of being read from X.
template <bool FUSED>
__global__ void __launch_bounds__(INF_WARPS * 32)
k_mlp_infer(const float* __restrict__ params, const float* __restrict__ X, int64_t m, FeatArgs g,
            const int32_t* __restrict__ rowof, float* __restrict__ out) {
    extern __shared__ unsigned char smem_raw[];
    InferSmem& S = *(InferSmem*)smem_raw;
    int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
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
        S.w1t[o * XS + i] = __float2bfloat16(params[P_W1 + q]);
    }
    for (int q = tid; q < NH * NH; q += blockDim.x) {
        int i = q / NH, o = q % NH;                    // W2[i][o]
        S.w2t[o * HS + i] = __float2bfloat16(params[P_W2 + q]);
    }
    float b3 = params[P_B3];
    __syncthreads();
    for (int64_t base = (int64_t)blockIdx.x * TILE_M; base < m; base += (int64_t)gridDim.x * TILE_M) {
        // normalised features of the tile (rows past m are zero)
        if (FUSED) {
            // two threads per entry: part 0 (geometry, row quantities) and part 1 (row lookups)
            int r = tid % TILE_M, part = tid / TILE_M;
            int64_t row = base + r;
            float f[NF];
            if (row < m) entry_features(g, rowof[row], row, f, part);
            for (int c = 0; c < NF; ++c)
                if (feat_part(c) == part)
                    S.x[r * XS + c] = __float2bfloat16(row < m ? (f[c] - S.mu[c]) * S.isd[c] : 0.f);
        } else {
            for (int q = tid; q < TILE_M * NF; q += blockDim.x) {
                int r = q / NF, c = q % NF;
                int64_t row = base + r;
                float v = row < m ? (X[row * NF + c] - S.mu[c]) * S.isd[c] : 0.f;
                S.x[r * XS + c] = __float2bfloat16(v);
            }
        }
        __syncthreads();
        int r0 = 16 * w;
        // layer 1: h1 = relu(x W1 + b1)
        uint32_t a1[2][4];
        load_a(a1[0], S.x, XS, r0, 0, lane);
        load_a(a1[1], S.x, XS, r0, 16, lane);
        int g = lane >> 2, t = lane & 3;
        for (int nt = 0; nt < NH / 8; ++nt) {
            float d[4] = {0.f, 0.f, 0.f, 0.f};
            for (int ks = 0; ks < NF / 16; ++ks) {
                uint32_t b[2];
                load_b(b, S.w1t, XS, nt * 8, ks * 16, lane);
                mma_bf16(d, a1[ks], b);
            }
            int c = nt * 8 + 2 * t;
            float h00 = fmaxf(d[0] + S.b1[c], 0.f), h01 = fmaxf(d[1] + S.b1[c + 1], 0.f);
            float h10 = fmaxf(d[2] + S.b1[c], 0.f), h11 = fmaxf(d[3] + S.b1[c + 1], 0.f);
            *(uint32_t*)(S.h1 + (r0 + g) * HS + c) = pack_bf16(__float2bfloat16(h00), __float2bfloat16(h01));
            *(uint32_t*)(S.h1 + (r0 + g + 8) * HS + c) = pack_bf16(__float2bfloat16(h10), __float2bfloat16(h11));
        }
        __syncwarp();
        // layer 2 and the output layer: y = relu(h1 W2 + b2) . w3 + b3
        float y0 = 0.f, y1 = 0.f;             // rows r0+g and r0+g+8, partial over this lane's columns
        uint32_t a2[NH / 16][4];
        for (int ks = 0; ks < NH / 16; ++ks) load_a(a2[ks], S.h1, HS, r0, ks * 16, lane);
        for (int nt = 0; nt < NH / 8; ++nt) {
            float d[4] = {0.f, 0.f, 0.f, 0.f};
            for (int ks = 0; ks < NH / 16; ++ks) {
                uint32_t b[2];
                load_b(b, S.w2t, HS, nt * 8, ks * 16, lane);
                mma_bf16(d, a2[ks], b);
            }
            int c = nt * 8 + 2 * t;
            y0 += fmaxf(d[0] + S.b2[c], 0.f) * S.w3[c] + fmaxf(d[1] + S.b2[c + 1], 0.f) * S.w3[c + 1];
            y1 += fmaxf(d[2] + S.b2[c], 0.f) * S.w3[c] + fmaxf(d[3] + S.b2[c + 1], 0.f) * S.w3[c + 1];
        }
        y0 += __shfl_xor_sync(0xffffffffu, y0, 1);
        y0 += __shfl_xor_sync(0xffffffffu, y0, 2);
        y1 += __shfl_xor_sync(0xffffffffu, y1, 1);
        y1 += __shfl_xor_sync(0xffffffffu, y1, 2);
        if (t == 0) {
            int64_t ra = base + r0 + g, rb = base + r0 + g + 8;
            if (ra < m) out[ra] = y0 + b3;
            if (rb < m) out[rb] = y1 + b3;
        }
        __syncthreads();
    }
}

static int infer_grid(int64_t m) {
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (nsm <= 0) nsm = 1;
    int64_t tiles = (m + TILE_M - 1) / TILE_M;
    int64_t cap = (int64_t)nsm * 2;                   // two 92 KB blocks fit one SM
    return (int)(tiles < cap ? tiles : cap);
}

int mlp_predict(const float* params_dev, const float* X, int64_t m, float* out, cudaStream_t s) {
    if (m <= 0) return SPHC_OK;
    size_t sm = sizeof(InferSmem);
    SPHC_CK(cudaFuncSetAttribute(k_mlp_infer<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    SPHC_LAUNCH(k_mlp_infer<false><<<infer_grid(m), INF_WARPS * 32, sm, s>>>(params_dev, X, m, FeatArgs(), nullptr, out));
    SPHC_CK(cudaGetLastError());
    return SPHC_OK;
}

// row of every pattern entry (warp per row)
__global__ void k_row_of(const int64_t* nrp, int64_t ne, int32_t* rowof) {
    int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (i >= ne) return;
    for (int64_t q = nrp[i] + lane; q < nrp[i + 1]; q += 32) rowof[q] = (int32_t)i;
}

int mlp_predict_level(const float* params_dev, const FeatArgs& g, float* out, cudaStream_t s) {
    int64_t m = g.nnzN;
    if (m <= 0) return SPHC_OK;
    DBuf<int32_t> rowof;
    SPHC_TRY(rowof.alloc(m, s));
    SPHC_LAUNCH(k_row_of<<<grid_for(g.ne * 32, 256), 256, 0, s>>>(g.nrp, g.ne, rowof.p));
    size_t sm = sizeof(InferSmem);
    SPHC_CK(cudaFuncSetAttribute(k_mlp_infer<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    SPHC_LAUNCH(k_mlp_infer<true><<<infer_grid(m), INF_WARPS * 32, sm, s>>>(params_dev, nullptr, m, g, rowof.p, out));
    SPHC_CK(cudaGetLastError());
    return SPHC_OK;
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
