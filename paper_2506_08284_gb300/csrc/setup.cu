// Setup phase of SpHcurlAMG on the GPU: one level of Alg. 3 at a time.
//   colouring (Gauss-Seidel order), aggregation (tentative Pbar), smoothed nodal prolongator
//   P_n (Sec. 4.1, Sec. 6.1), coarse gradient D_H from Pbar (eqs. (4), (11)), pattern T / N of
//   Alg. 2, least-norm initial guess (Sec. 6.1), projected-Jacobi energy minimisation (eq. (9))
//   with per-row commuting-constraint projections (Sec. 3, Sec. 4.2), Galerkin products (Sec. 2)
//   and the dense coarsest factor.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <string>

#include "features.cuh"
#include "sphc_level.cuh"

namespace sphc {

// ------------------------------------------------------------------ greedy colouring in
// priority order, computed as Jones-Plassmann rounds: an uncoloured row whose priority beats
// every uncoloured neighbour takes the smallest colour absent from its coloured neighbours.
static constexpr int MAX_COLORS = 256;

// The rounds run inside one CUDA graph: a conditional while node repeats {JP_UNROLL rounds,
// advance} on the device, so no round waits for the host (an iteration of the while node costs
// far more than a round of a small graph; rounds after the last colour has been given only
// return).  ctrl holds {colour overflow, iterations, then one "rows still waiting" flag per round
// of an iteration}.  A round visits every row; coloured rows are skipped at once, so no worklist
// (and no contended counter to append to it) is needed.
enum { JP_OVERFLOW = 0, JP_ITERS = 1, JP_WAITING = 2 };
static constexpr int JP_UNROLL = 8;
// blocks of a round per SM (eight waves of resident blocks): a waiting row's re-check is a chain of
// dependent loads, so more rows in flight pay for the extra block scheduling (level-0 edge graph
// at 128^3: 8 blocks/SM 28.1 ms, 32 22.1, 64 20.0, 128 21.2, 256 24.5 ms over its 37 rounds)
static constexpr int JP_BLOCKS_PER_SM = 64;
static constexpr int JP_MAX_ITERS = 1 << 17;

__global__ void k_prio(int64_t n, uint64_t seed, uint64_t* prio) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) prio[v] = splitmix64(seed, (uint64_t)v);
}

// One round; a group of G lanes handles a row (rows of coarse levels are long, and one thread
// walking them is latency-bound).  Decisions read colours in place: a row only colours itself
// once every higher-priority neighbour is coloured, so the result equals the greedy colouring in
// priority order whatever the interleaving inside a round.  A waiting row remembers where its
// scan stopped (pos, the first blocking neighbour): the neighbours before it are coloured or of
// lower priority, which stays true, so the next round resumes there and the scans of all rounds
// add up to one pass over the row.
template <int G>
__global__ void k_jp_round(const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                           const uint64_t* __restrict__ prio, int64_t n, int* ctrl, int slot, int32_t* pos,
                           int32_t* color) {
    int lane = threadIdx.x & 31;
    int sub = lane & (G - 1);
    unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
    const int64_t stride = ((int64_t)gridDim.x * blockDim.x) / G;
    volatile int32_t* col = color;
    bool waiting = false;
    for (int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G; v < n; v += stride) {
        if (col[v] >= 0) continue;                 // uniform over the group
        bool wv = false;
        uint64_t hv = prio[v];
        int64_t b = rp[v], e = rp[v + 1];
        for (int64_t k0 = b + pos[v]; k0 < e; k0 += G) {
            int64_t k = k0 + sub;
            bool blocks = false;
            if (k < e) {
                int32_t w = ci[k];
                blocks = w != v && col[w] < 0 && prio_greater(prio[w], w, hv, v);
            }
            unsigned bal = (__ballot_sync(gmask, blocks) & gmask) >> (lane & ~(G - 1));
            if (bal) {
                wv = true;
                if (sub == 0) pos[v] = (int32_t)(k0 + (__ffs(bal) - 1) - b);
                break;
            }
        }
        if (wv) {
            waiting = true;
            continue;
        }
        uint64_t used[MAX_COLORS / 64] = {0, 0, 0, 0};
        for (int64_t k = b + sub; k < e; k += G) {
            int32_t w = ci[k];
            if (w == v) continue;
            int32_t c = col[w];
            if (c >= 0 && c < MAX_COLORS) {
                if (c < 64) used[0] |= 1ULL << c;
                else if (c < 128) used[1] |= 1ULL << (c - 64);
                else if (c < 192) used[2] |= 1ULL << (c - 128);
                else used[3] |= 1ULL << (c - 192);
            }
        }
#pragma unroll
        for (int d = G / 2; d > 0; d >>= 1)
#pragma unroll
            for (int q = 0; q < MAX_COLORS / 64; ++q) used[q] |= __shfl_xor_sync(gmask, used[q], d);
        if (sub == 0) {
            int c = MAX_COLORS;
#pragma unroll
            for (int q = MAX_COLORS / 64 - 1; q >= 0; --q)
                if (~used[q]) c = 64 * q + __ffsll((long long)~used[q]) - 1;
            if (c >= MAX_COLORS) { atomicExch(&ctrl[JP_OVERFLOW], 1); c = MAX_COLORS - 1; }
            color[v] = c;
        }
    }
    if (__syncthreads_or(waiting) && threadIdx.x == 0) ctrl[JP_WAITING + slot] = 1;
}
// another iteration while a row waited in the last round
__global__ void k_jp_advance(cudaGraphConditionalHandle hnd, int* ctrl) {
    int waiting = ctrl[JP_WAITING + JP_UNROLL - 1];
    for (int q = 0; q < JP_UNROLL; ++q) ctrl[JP_WAITING + q] = 0;
    int it = ++ctrl[JP_ITERS];
    cudaGraphSetConditional(hnd, (waiting && it < JP_MAX_ITERS) ? 1u : 0u);
}

__global__ void k_fill_i32(int32_t* a, int64_t n, int32_t v) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = v;
}
__global__ void k_max_i32(const int32_t* a, int64_t n, int* mx) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) atomicMax(mx, a[i]);
}

int color_graph(const DCSR& G, uint64_t seed, DBuf<int32_t>& color, int* ncolors, cudaStream_t s, int* rounds,
                Profiler* prof, const char* tag) {
    const std::string tg = tag ? tag : "";
    Profiler* pr = tag ? prof : nullptr;
    std::unique_ptr<Section> sec_build(new Section(pr, ("colour_build_" + tg).c_str(), s));
    int64_t n = G.nr;
    SPHC_TRY(color.alloc(n, s));
    if (n == 0) { *ncolors = 0; return SPHC_OK; }
    if (n >= (1LL << 31)) { set_error("colouring: %lld rows exceed int32", (long long)n); return SPHC_ELIMIT; }
    SPHC_LAUNCH(k_fill_i32<<<grid_for(n, 256), 256, 0, s>>>(color.p, n, -1));
    DBuf<int32_t> pos;
    DBuf<uint64_t> prio;
    DBuf<int> ctrl;
    SPHC_TRY(pos.alloc(n, s));
    SPHC_TRY(pos.zero(s));
    SPHC_TRY(prio.alloc(n, s));
    SPHC_TRY(ctrl.alloc(JP_WAITING + JP_UNROLL, s));
    SPHC_TRY(ctrl.zero(s));
    SPHC_LAUNCH(k_prio<<<grid_for(n, 256), 256, 0, s>>>(n, seed, prio.p));
    // graph: while (rows waiting) { round; advance }
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    cudaStream_t cs = nullptr;
    int rc = SPHC_OK;
    auto fail = [&](cudaError_t e, const char* what) {
        set_error("colouring graph: %s: %s", what, cudaGetErrorString(e));
        rc = SPHC_ECUDA;
    };
    cudaError_t e = cudaGraphCreate(&g, 0);
    if (e != cudaSuccess) fail(e, "create");
    cudaGraphConditionalHandle hnd;
    if (rc == SPHC_OK && (e = cudaGraphConditionalHandleCreate(&hnd, g, 1, cudaGraphCondAssignDefault)) != cudaSuccess)
        fail(e, "handle");
    cudaGraphNodeParams np = {};
    if (rc == SPHC_OK) {
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = hnd;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        cudaGraphNode_t node;
        if ((e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np)) != cudaSuccess) fail(e, "while node");
    }
    if (rc == SPHC_OK && (e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) != cudaSuccess) fail(e, "stream");
    // rounds loop over the rows with a grid capped at JP_BLOCKS_PER_SM blocks per SM: a round
    // colours only about 6 % of the rows of a mesh graph (37 rounds at level 0 of the 128^3
    // problem), and every waiting row re-checks its blocking neighbour each round (an appended
    // list of waiting rows measured slower: its counter is contended)
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (nsm <= 0) nsm = 1;
    if (rc == SPHC_OK) {
        cudaGraph_t body = np.conditional.phGraph_out[0];
        if ((e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
            fail(e, "capture");
        else {
            // lanes per row: one on large graphs (every round visits every row, so the thread
            // count sets its fixed cost), else the mean row length rounded up to a power of two
            double avg = (double)G.nnz / (double)n;
            int lanes = 1;
            if (n <= (1 << 20)) {
                lanes = 4;
                while (lanes < 32 && lanes < avg) lanes *= 2;
            }
            for (int q = 0; q < JP_UNROLL; ++q) {
                unsigned blocks = (unsigned)std::min<int64_t>(grid_for(n * lanes, 256), (int64_t)nsm * JP_BLOCKS_PER_SM);
                switch (lanes) {
                    case 1: k_jp_round<1><<<blocks, 256, 0, cs>>>(G.rp.p, G.ci.p, prio.p, n, ctrl.p, q, pos.p, color.p); break;
                    case 4: k_jp_round<4><<<blocks, 256, 0, cs>>>(G.rp.p, G.ci.p, prio.p, n, ctrl.p, q, pos.p, color.p); break;
                    case 8: k_jp_round<8><<<blocks, 256, 0, cs>>>(G.rp.p, G.ci.p, prio.p, n, ctrl.p, q, pos.p, color.p); break;
                    case 16: k_jp_round<16><<<blocks, 256, 0, cs>>>(G.rp.p, G.ci.p, prio.p, n, ctrl.p, q, pos.p, color.p); break;
                    default: k_jp_round<32><<<blocks, 256, 0, cs>>>(G.rp.p, G.ci.p, prio.p, n, ctrl.p, q, pos.p, color.p); break;
                }
            }
            k_jp_advance<<<1, 1, 0, cs>>>(hnd, ctrl.p);
            cudaGraph_t captured = nullptr;
            if ((e = cudaStreamEndCapture(cs, &captured)) != cudaSuccess) fail(e, "end capture");
        }
    }
    if (rc == SPHC_OK && (e = cudaGraphInstantiate(&ge, g, 0)) != cudaSuccess) fail(e, "instantiate");
    sec_build.reset();
    Section sec_rounds(pr, ("colour_rounds_" + tg).c_str(), s);
    if (rc == SPHC_OK && (e = cudaGraphLaunch(ge, s)) != cudaSuccess) fail(e, "launch");
    if (ge) cudaGraphExecDestroy(ge);
    if (g) cudaGraphDestroy(g);
    if (cs) cudaStreamDestroy(cs);
    if (rc != SPHC_OK) return rc;
    int h[JP_WAITING + JP_UNROLL];
    SPHC_CK(cudaMemcpyAsync(h, ctrl.p, sizeof(h), cudaMemcpyDeviceToHost, s));
    SPHC_CK(cudaStreamSynchronize(s));
    g_launches.fetch_add((long long)(JP_UNROLL + 1) * h[JP_ITERS]);
    if (rounds) *rounds = JP_UNROLL * h[JP_ITERS];
    if (h[JP_OVERFLOW]) { set_error("colouring needs more than %d colours", MAX_COLORS); return SPHC_ELIMIT; }
    if (h[JP_ITERS] >= JP_MAX_ITERS) {
        set_error("colouring did not finish in %d rounds", JP_UNROLL * JP_MAX_ITERS);
        return SPHC_ELIMIT;
    }
    SPHC_CK(cudaMemsetAsync(ctrl.p, 0, sizeof(int), s));
    SPHC_LAUNCH(k_max_i32<<<grid_for(n, 256), 256, 0, s>>>(color.p, n, ctrl.p));
    SPHC_CK(cudaMemcpyAsync(h, ctrl.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    SPHC_CK(cudaStreamSynchronize(s));
    *ncolors = h[0] + 1;
    return SPHC_OK;
}

// ------------------------------------------------------------------ aggregation
// state: 0 undecided, 1 root, 2 decided, 3 root chosen in the current round
// G lanes per node split its neighbours w; each lane walks w and w's neighbours.  After every
// stripe of G neighbours the group's ballot ends the walk once any lane met a blocking node, so the
// group's trip count stays uniform.
template <int G>
__global__ void k_mis2_select(const int64_t* rp, const int32_t* ci, int64_t n, uint64_t seed, int8_t* state) {
    const int lane = threadIdx.x & 31, sub = lane & (G - 1);
    const unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
    const int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
    if (v >= n) return;                              // uniform over the group
    volatile int8_t* st = state;
    if (st[v] != 0) return;
    const uint64_t hv = splitmix64(seed, (uint64_t)v);
    const int64_t b0 = rp[v], e0 = rp[v + 1];
    for (int64_t k0 = b0; k0 < e0; k0 += G) {
        bool blocked = false;
        const int64_t k = k0 + sub;
        if (k < e0) {
            const int32_t w = ci[k];
            if (w != v) {
                for (int q = 0; q < 2 && !blocked; ++q) {
                    // q = 0: w itself, q = 1: w's neighbours
                    const int64_t b = q == 0 ? 0 : rp[w], e = q == 0 ? 1 : rp[w + 1];
                    for (int64_t k2 = b; k2 < e; ++k2) {
                        const int32_t u = q == 0 ? w : ci[k2];
                        if (u == v) continue;
                        const int8_t su = st[u];
                        if (su == 1 || su == 3 ||
                            (su == 0 && prio_greater(splitmix64(seed, (uint64_t)u), u, hv, v))) {
                            blocked = true;
                            break;
                        }
                    }
                }
            }
        }
        if (__any_sync(gmask, blocked)) return;
    }
    if (sub == 0) state[v] = 3;
}

template <int G>
__global__ void k_mis2_mark(const int64_t* rp, const int32_t* ci, int64_t n, int8_t* state) {
    const int sub = threadIdx.x & (G - 1);
    const int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
    if (v >= n) return;
    if (state[v] != 3) return;
    for (int64_t k = rp[v] + sub; k < rp[v + 1]; k += G) {
        const int32_t w = ci[k];
        if (w != v && state[w] == 0) state[w] = 2;
        for (int64_t k2 = rp[w]; k2 < rp[w + 1]; ++k2) {
            const int32_t u = ci[k2];
            if (u != v && state[u] == 0) state[u] = 2;
        }
    }
}
__global__ void k_mis2_commit(int8_t* state, int64_t n, int* left) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool undecided = false;
    if (v < n) {
        if (state[v] == 3) state[v] = 1;
        else undecided = state[v] == 0;
    }
    warp_count(left, undecided);
}
__global__ void k_root_flags(const int8_t* state, int64_t n, int64_t* flag) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) flag[v] = state[v] == 1 ? 1 : 0;
}
__global__ void k_agg_phase2(const int64_t* rp, const int32_t* ci, int64_t n, const int8_t* state,
                             const int64_t* rid, int32_t* agg) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    if (state[v] == 1) { agg[v] = (int32_t)rid[v]; return; }
    int32_t a = -1;
    for (int64_t k = rp[v]; k < rp[v + 1]; ++k) {
        int32_t w = ci[k];
        if (w != v && state[w] == 1) { a = (int32_t)rid[w]; break; }
    }
    agg[v] = a;
}
// one synchronous round: join the aggregate with the most edges (ties -> lowest id)
__global__ void k_agg_phase3(const int64_t* rp, const int32_t* ci, int64_t n, const int32_t* cur, int32_t* nxt,
                             int* left, int* changed) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool open = v < n && cur[v] < 0;
    warp_count(left, open);
    if (v >= n) return;
    int32_t a = cur[v];
    if (a >= 0) { nxt[v] = a; return; }
    int32_t best = -1, bestc = 0;
    for (int64_t k = rp[v]; k < rp[v + 1]; ++k) {
        int32_t w = ci[k];
        if (w == v) continue;
        int32_t g = cur[w];
        if (g < 0) continue;
        // count edges of v into aggregate g (first occurrence only)
        bool first = true;
        for (int64_t k2 = rp[v]; k2 < k; ++k2) {
            int32_t w2 = ci[k2];
            if (w2 != v && cur[w2] == g) { first = false; break; }
        }
        if (!first) continue;
        int32_t c = 0;
        for (int64_t k2 = k; k2 < rp[v + 1]; ++k2) {
            int32_t w2 = ci[k2];
            if (w2 != v && cur[w2] == g) ++c;
        }
        if (c > bestc || (c == bestc && g < best)) { best = g; bestc = c; }
    }
    nxt[v] = best;
    if (best >= 0) atomicAdd(changed, 1);   // rare: only nodes left after the root neighbourhoods
}

int aggregate(const DCSR& G, uint64_t seed, DBuf<int32_t>& agg, int64_t* nagg, cudaStream_t s) {
    int64_t n = G.nr;
    SPHC_TRY(agg.alloc(n, s));
    if (n == 0) { *nagg = 0; return SPHC_OK; }
    DBuf<int8_t> state;
    SPHC_TRY(state.alloc(n, s));
    SPHC_TRY(state.zero(s));
    DBuf<int> flags;
    SPHC_TRY(flags.alloc(2, s));
    int h[2];
    // lanes per node: the mean degree rounded up to a power of two (at most 32) on graphs of up to
    // 2^20 nodes, whose distance-2 walks are long and few; 4 on larger graphs
    const double deg = (double)G.nnz / (double)n;
    int lanes = 4;
    if (n <= (1 << 20)) {
        lanes = 1;
        while (lanes < 32 && lanes < deg) lanes *= 2;
    }
    for (int round = 0; round < 100000; ++round) {
        switch (lanes) {
#define MIS(L) SPHC_LAUNCH(k_mis2_select<L><<<grid_for(n * L, 256), 256, 0, s>>>(G.rp.p, G.ci.p, n, seed, state.p)); \
               SPHC_LAUNCH(k_mis2_mark<L><<<grid_for(n * L, 256), 256, 0, s>>>(G.rp.p, G.ci.p, n, state.p)); break;
            case 1: MIS(1)
            case 2: MIS(2)
            case 4: MIS(4)
            case 8: MIS(8)
            case 16: MIS(16)
            default: MIS(32)
#undef MIS
        }
        SPHC_CK(cudaMemsetAsync(flags.p, 0, sizeof(int), s));
        SPHC_LAUNCH(k_mis2_commit<<<grid_for(n, 256), 256, 0, s>>>(state.p, n, flags.p));
        SPHC_CK(cudaMemcpyAsync(h, flags.p, sizeof(int), cudaMemcpyDeviceToHost, s));
        SPHC_CK(cudaStreamSynchronize(s));
        if (h[0] == 0) break;
    }
    DBuf<int64_t> flag, rid;
    SPHC_TRY(flag.alloc(n, s));
    SPHC_TRY(rid.alloc(n + 1, s));
    SPHC_LAUNCH(k_root_flags<<<grid_for(n, 256), 256, 0, s>>>(state.p, n, flag.p));
    SPHC_TRY(exclusive_scan_i64(flag.p, rid.p, n, s, nagg));
    DBuf<int32_t> tmp;
    SPHC_TRY(tmp.alloc(n, s));
    SPHC_LAUNCH(k_agg_phase2<<<grid_for(n, 256), 256, 0, s>>>(G.rp.p, G.ci.p, n, state.p, rid.p, agg.p));
    for (int round = 0; round < 64; ++round) {
        SPHC_CK(cudaMemsetAsync(flags.p, 0, 2 * sizeof(int), s));
        SPHC_LAUNCH(k_agg_phase3<<<grid_for(n, 256), 256, 0, s>>>(G.rp.p, G.ci.p, n, agg.p, tmp.p, flags.p, flags.p + 1));
        std::swap(agg.p, tmp.p);
        SPHC_CK(cudaMemcpyAsync(h, flags.p, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
        SPHC_CK(cudaStreamSynchronize(s));
        if (h[0] == 0) break;
        if (h[1] == 0) { set_error("aggregation left isolated nodes"); return SPHC_ENUMERIC; }
    }
    SPHC_CK(cudaGetLastError());
    return SPHC_OK;
}

// ------------------------------------------------------------------ nodal prolongator
__global__ void k_uniform_vec(double* v, int64_t n, uint64_t seed) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] = (double)(splitmix64(seed, (uint64_t)i) >> 11) * (1.0 / 9007199254740992.0);
}
__global__ void k_scale_dinv(double* w, const double* d, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) w[i] /= d[i];
}
__global__ void k_normalise(double* v, const double* w, const double* ww, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double nw = sqrt(*ww);
    if (i < n) v[i] = w[i] / nw;
}

int power_rho(const DCSR& A, const double* diag, uint64_t seed, int iters, double* rho, cudaStream_t s) {
    int64_t n = A.nr;
    if (n == 0) { *rho = 1.0; return SPHC_OK; }
    DBuf<double> v, w, sc;
    SPHC_TRY(v.alloc(n, s));
    SPHC_TRY(w.alloc(n, s));
    SPHC_TRY(sc.alloc(2, s));
    SPHC_LAUNCH(k_uniform_vec<<<grid_for(n, 256), 256, 0, s>>>(v.p, n, seed));
    double h[2] = {1.0, 1.0};
    // only the last iteration's v . v is read.  (Dividing by the diagonal inside the SpMV's store
    // measured slower: there one lane in eight runs the FP64 division sequence, so the thin FP64
    // pipe executes it once per four rows instead of once per 32.)
    for (int it = 0; it < iters; ++it) {
        SPHC_TRY(spmv64(A, v.p, w.p, s));
        SPHC_LAUNCH(k_scale_dinv<<<grid_for(n, 256), 256, 0, s>>>(w.p, diag, n));
        if (it + 1 == iters) SPHC_TRY(dot64(v.p, v.p, n, sc.p, s));
        SPHC_TRY(dot64(w.p, w.p, n, sc.p + 1, s));
        SPHC_LAUNCH(k_normalise<<<grid_for(n, 256), 256, 0, s>>>(v.p, w.p, sc.p + 1, n));
    }
    SPHC_CK(cudaMemcpyAsync(h, sc.p, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    SPHC_CK(cudaStreamSynchronize(s));
    *rho = sqrt(h[1]) / sqrt(h[0]);
    return SPHC_OK;
}

__global__ void k_pbar(int64_t n, const int32_t* agg, int64_t* rp, int32_t* ci, double* v) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) { rp[i] = i; ci[i] = agg[i]; v[i] = 1.0; }
    if (i == n) rp[n] = n;
}

// P_n row u = rowscale(e_agg(u) - w/a_uu (A_n Pbar)_u), or the tentative row when the sum is small
__global__ void k_pn_finish(const int64_t* rp, const int32_t* ci, double* v, int64_t n, const int32_t* agg,
                            const double* diag, double omega, int smooth, int* n_fallback, int* bad) {
    int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n) return;
    int32_t a = agg[u];
    double d = diag[u];
    double rs = 0.0;
    for (int64_t k = rp[u]; k < rp[u + 1]; ++k) {
        double p = (ci[k] == a ? 1.0 : 0.0);
        if (smooth) p -= omega / d * v[k];
        v[k] = p;
        rs += p;
    }
    if (!isfinite(rs)) { atomicExch(bad, 1); return; }
    if (rs <= SA_MIN_ROWSUM) {
        for (int64_t k = rp[u]; k < rp[u + 1]; ++k) v[k] = ci[k] == a ? 1.0 : 0.0;
        atomicAdd(n_fallback, 1);
        return;
    }
    for (int64_t k = rp[u]; k < rp[u + 1]; ++k) v[k] /= rs;
}

// ------------------------------------------------------------------ coarse gradient
__global__ void k_count_agg(const int32_t* agg, int64_t n, int32_t* cnt) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) atomicAdd(&cnt[agg[i]], 1);
}
__global__ void k_scatter_agg(const int32_t* agg, int64_t n, unsigned long long* cur, int32_t* members) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) members[atomicAdd(&cur[agg[i]], 1ULL)] = (int32_t)i;
}
__global__ void k_i64_to_u64b(const int64_t* a, unsigned long long* b, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (unsigned long long)a[i];
}

static constexpr int DH_SET = 1024;
static constexpr int DH_WARPS = 4;
// warp per aggregate U: the set of aggregates V > U joined to U by a fine edge.  mode 0
// counts, mode 1 writes the sorted rows of D_H (tail U: -1, head V: +1).
__global__ void k_dh_rows(int64_t nagg, const int64_t* mptr, const int32_t* members, const int64_t* dtrp,
                          const int32_t* dtci, const int64_t* drp, const int32_t* dci, const int32_t* agg,
                          int mode, int64_t* cnt, const int64_t* off, int32_t* hci, double* hv, int* fail) {
    __shared__ int32_t s_set[DH_WARPS][DH_SET];
    __shared__ int s_n[DH_WARPS];
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int64_t U = (int64_t)blockIdx.x * DH_WARPS + w;
    if (U >= nagg) return;
    int32_t* set = s_set[w];
    for (int t = lane; t < DH_SET; t += 32) set[t] = -1;
    if (lane == 0) s_n[w] = 0;
    __syncwarp();
    for (int64_t m = mptr[U]; m < mptr[U + 1]; ++m) {
        int32_t u = members[m];
        for (int64_t k = dtrp[u] + lane; k < dtrp[u + 1]; k += 32) {
            int32_t e = dtci[k];
            if (drp[e + 1] - drp[e] != 2) continue;
            int32_t o = dci[drp[e]] == u ? dci[drp[e] + 1] : dci[drp[e]];
            int32_t V = agg[o];
            if (V <= U) continue;
            uint32_t h = ((uint32_t)V * 2654435761u) & (DH_SET - 1);
            for (int probe = 0; probe < DH_SET; ++probe) {
                int32_t old = atomicCAS(&set[h], -1, V);
                if (old == -1) { atomicAdd(&s_n[w], 1); break; }
                if (old == V) break;
                h = (h + 1) & (DH_SET - 1);
            }
        }
    }
    __syncwarp();
    int nset = s_n[w];
    if (nset > DH_SET / 2) { if (lane == 0) atomicExch(fail, 1); return; }
    if (mode == 0) { if (lane == 0) cnt[U] = nset; return; }
    int64_t base = off[U];
    for (int t = lane; t < DH_SET; t += 32) {
        int32_t V = set[t];
        if (V < 0) continue;
        int rank = 0;
        for (int q = 0; q < DH_SET; ++q) rank += (set[q] >= 0 && set[q] < V);
        int64_t e = base + rank;
        hci[2 * e] = (int32_t)U; hv[2 * e] = -1.0;
        hci[2 * e + 1] = V;      hv[2 * e + 1] = 1.0;
    }
}
__global__ void k_single_flags(const int64_t* drp, const int32_t* dci, int64_t ne, const int32_t* agg, int64_t* flag) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ne) return;
    if (drp[e + 1] - drp[e] == 1) flag[agg[dci[drp[e]]]] = 1;
}
__global__ void k_dh_singles(const int64_t* flag, const int64_t* sid, int64_t nagg, int64_t n2, int32_t* hci,
                             double* hv) {
    int64_t U = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (U >= nagg || !flag[U]) return;
    int64_t q = 2 * n2 + sid[U];
    hci[q] = (int32_t)U;
    hv[q] = 1.0;
}
__global__ void k_dh_rowptr(int64_t n2, int64_t n1, int64_t* rp) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e > n2 + n1) return;
    rp[e] = e <= n2 ? 2 * e : 2 * n2 + (e - n2);
}

int coarse_gradient(const DCSR& D, const DCSR& Dt, const int32_t* agg, int64_t nagg, DCSR& DH, cudaStream_t s) {
    int64_t nv = D.nc, ne = D.nr;
    DBuf<int32_t> cnt, members;
    DBuf<int64_t> mptr;
    DBuf<unsigned long long> cur;
    SPHC_TRY(cnt.alloc(nagg + 1, s));
    SPHC_TRY(cnt.zero(s));
    SPHC_TRY(mptr.alloc(nagg + 1, s));
    SPHC_TRY(members.alloc(nv, s));
    SPHC_TRY(cur.alloc(nagg + 1, s));
    if (nv > 0) SPHC_LAUNCH(k_count_agg<<<grid_for(nv, 256), 256, 0, s>>>(agg, nv, cnt.p));
    SPHC_TRY(scan_i32_to_i64(cnt.p, mptr.p, nagg, s, nullptr));
    SPHC_LAUNCH(k_i64_to_u64b<<<grid_for(nagg + 1, 256), 256, 0, s>>>(mptr.p, cur.p, nagg + 1));
    if (nv > 0) SPHC_LAUNCH(k_scatter_agg<<<grid_for(nv, 256), 256, 0, s>>>(agg, nv, cur.p, members.p));
    DBuf<int64_t> c2, off2;
    DBuf<int> fail;
    SPHC_TRY(c2.alloc(nagg + 1, s));
    SPHC_TRY(off2.alloc(nagg + 1, s));
    SPHC_TRY(fail.alloc(1, s));
    SPHC_TRY(fail.zero(s));
    if (nagg > 0)
        SPHC_LAUNCH(k_dh_rows<<<grid_for(nagg, DH_WARPS), DH_WARPS * 32, 0, s>>>(nagg, mptr.p, members.p, Dt.rp.p, Dt.ci.p, D.rp.p,
                                                                    D.ci.p, agg, 0, c2.p, nullptr, nullptr, nullptr,
                                                                    fail.p));
    int64_t n2 = 0;
    SPHC_TRY(exclusive_scan_i64(c2.p, off2.p, nagg, s, &n2));
    int f = 0;
    SPHC_CK(cudaMemcpyAsync(&f, fail.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    SPHC_CK(cudaStreamSynchronize(s));
    if (f) { set_error("coarse gradient: an aggregate has more than %d neighbours", DH_SET / 2); return SPHC_ELIMIT; }
    DBuf<int64_t> sflag, sid;
    SPHC_TRY(sflag.alloc(nagg + 1, s));
    SPHC_TRY(sflag.zero(s));
    SPHC_TRY(sid.alloc(nagg + 1, s));
    if (ne > 0) SPHC_LAUNCH(k_single_flags<<<grid_for(ne, 256), 256, 0, s>>>(D.rp.p, D.ci.p, ne, agg, sflag.p));
    int64_t n1 = 0;
    SPHC_TRY(exclusive_scan_i64(sflag.p, sid.p, nagg, s, &n1));
    SPHC_TRY(DH.alloc(n2 + n1, nagg, 2 * n2 + n1, s));
    SPHC_LAUNCH(k_dh_rowptr<<<grid_for(n2 + n1 + 1, 256), 256, 0, s>>>(n2, n1, DH.rp.p));
    if (nagg > 0) {
        SPHC_LAUNCH(k_dh_rows<<<grid_for(nagg, DH_WARPS), DH_WARPS * 32, 0, s>>>(nagg, mptr.p, members.p, Dt.rp.p, Dt.ci.p, D.rp.p,
                                                                    D.ci.p, agg, 1, nullptr, off2.p, DH.ci.p, DH.v.p,
                                                                    fail.p));
        SPHC_LAUNCH(k_dh_singles<<<grid_for(nagg, 256), 256, 0, s>>>(sflag.p, sid.p, nagg, n2, DH.ci.p, DH.v.p));
    }
    SPHC_CK(cudaGetLastError());
    return SPHC_OK;
}

// ------------------------------------------------------------------ pattern N (Alg. 2)
// Warp per fine row i: N_i = coarse edges whose every node lies in T_i.  mode 0 counts and
// checks the local graph (nodes T_i, two-node edges of N_i) for connectivity; mode 1 writes
// the sorted row.
__global__ void k_pattern(const int64_t* trp, const int32_t* tci, int64_t ne, const int32_t* rows, const int64_t* htrp,
                          const int32_t* htci, const int64_t* hrp, const int32_t* hci, int mode, int64_t* cnt,
                          const int64_t* nrp, int32_t* nci, int* stats /*0 too big T, 1 too big N, 2 disconnected*/,
                          int32_t* bad /* disconnected rows (mode 0), or null */) {
    __shared__ int32_t s_T[PAT_WARPS][MAX_T];
    __shared__ int32_t s_N[PAT_WARPS][MAX_NP];
    __shared__ int s_n[PAT_WARPS];
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int64_t i = (int64_t)blockIdx.x * PAT_WARPS + w;
    if (i >= ne) return;
    if (rows) i = rows[i];
    int64_t t0 = trp[i];
    int m = (int)(trp[i + 1] - t0);
    if (m > MAX_T) { if (lane == 0) { atomicExch(&stats[0], 1); if (mode == 0) cnt[i] = 0; } return; }
    if (lane < m) s_T[w][lane] = tci[t0 + lane];
    if (lane == 0) s_n[w] = 0;
    __syncwarp();
    if (lane < m) {
        int32_t J = s_T[w][lane];
        for (int64_t k = htrp[J]; k < htrp[J + 1]; ++k) {
            int32_t e = htci[k];
            int64_t b = hrp[e];
            int len = (int)(hrp[e + 1] - b);
            bool take = false;
            if (len == 1) take = true;
            else if (hci[b] == J) {
                int32_t o = hci[b + 1];
                for (int q = 0; q < m; ++q) if (s_T[w][q] == o) { take = true; break; }
            }
            if (take) {
                int pos = atomicAdd(&s_n[w], 1);
                if (pos < MAX_NP) s_N[w][pos] = e;
            }
        }
    }
    __syncwarp();
    int np = s_n[w];
    if (np > MAX_NP) { if (lane == 0) { atomicExch(&stats[1], 1); if (mode == 0) cnt[i] = 0; } return; }
    if (mode == 0) {
        if (lane == 0) {
            cnt[i] = np;
            // connectivity of the local graph
            if (m > 1) {
                int par[MAX_T];
                for (int q = 0; q < m; ++q) par[q] = q;
                for (int t = 0; t < np; ++t) {
                    int32_t e = s_N[w][t];
                    int64_t b = hrp[e];
                    if (hrp[e + 1] - b != 2) continue;
                    int a = -1, c = -1;
                    for (int q = 0; q < m; ++q) {
                        if (s_T[w][q] == hci[b]) a = q;
                        if (s_T[w][q] == hci[b + 1]) c = q;
                    }
                    while (par[a] != a) a = par[a];
                    while (par[c] != c) c = par[c];
                    if (a != c) par[a > c ? a : c] = a > c ? c : a;
                }
                int roots = 0;
                for (int q = 0; q < m; ++q) roots += (par[q] == q);
                if (roots > 1) {
                    int pos = atomicAdd(&stats[2], 1);
                    if (bad) bad[pos] = (int32_t)i;
                }
            }
        }
        return;
    }
    int64_t base = nrp[i];
    for (int t = lane; t < np; t += 32) {
        int32_t e = s_N[w][t];
        int rank = 0;
        for (int q = 0; q < np; ++q) rank += (s_N[w][q] < e);
        nci[base + rank] = e;
    }
}

// Thread per fine row for rows whose T_i has at most PT_K coarse nodes (larger rows go to
// k_pattern through a row list): the same N_i, enumerated from the incidence lists of T_i's nodes
// (each two-node edge once, from its first node).  A coarse edge's nodes come from E2 (first node,
// second node or -1), one load per incidence; each node's list is read four entries at a time.
// mode 0 counts N_i and checks that the local graph is connected (reachability over an 8 x 8
// adjacency bitmask); mode 1 collects N_i (up to PT_NMAX edges) and writes each edge at its rank,
// so the row comes out sorted; a longer N_i is written by merging the per-node lists (each sorted
// by edge id).
constexpr int PT_K = 8;
constexpr int PT_NMAX = 48;
__global__ void k_edge_pairs(const int64_t* __restrict__ hrp, const int32_t* __restrict__ hci, int64_t nE,
                             int2* __restrict__ E2) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nE) return;
    int64_t b = hrp[e];
    int len = (int)(hrp[e + 1] - b);
    E2[e] = make_int2(len >= 1 ? hci[b] : -1, len == 2 ? hci[b + 1] : -1);
}
__device__ __forceinline__ int pat_local(const int32_t T[PT_K], int m, int32_t u) {
    int c = -1;
#pragma unroll
    for (int a = 0; a < PT_K; ++a)
        if (a < m && T[a] == u) c = a;
    return c;
}
// is coarse edge e with nodes p (listed under node J) in N_i, counted from this list?
__device__ __forceinline__ bool pat_take(int2 p, const int32_t T[PT_K], int m, int32_t J, int* other) {
    *other = -1;
    if (p.y < 0) return true;
    if (p.x != J) return false;
    int c = pat_local(T, m, p.y);
    *other = c;
    return c >= 0;
}
__global__ void __launch_bounds__(128)
k_pattern_rows(const int64_t* __restrict__ trp, const int32_t* __restrict__ tci, int64_t ne,
               const int64_t* __restrict__ htrp, const int32_t* __restrict__ htci, const int2* __restrict__ E2,
               int mode, int64_t* cnt, const int64_t* __restrict__ nrp, int32_t* __restrict__ nci, int* stats,
               int32_t* big, int* nbig, int32_t* bad) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ne) return;
    int64_t t0 = trp[i];
    int m = (int)(trp[i + 1] - t0);
    if (m > PT_K) {
        if (mode == 0) big[warp_reserve(nbig)] = (int32_t)i;
        return;
    }
    int32_t T[PT_K];
#pragma unroll
    for (int a = 0; a < PT_K; ++a) T[a] = a < m ? tci[t0 + a] : -1;
    int64_t kb[PT_K], ke[PT_K];
#pragma unroll
    for (int a = 0; a < PT_K; ++a) {
        kb[a] = a < m ? htrp[T[a]] : 0;
        ke[a] = a < m ? htrp[T[a] + 1] : 0;
    }
    int32_t N[PT_NMAX];
    int np = 0;
    uint64_t adj = 0;
#pragma unroll
    for (int a = 0; a < PT_K; ++a) {
        for (int64_t k0 = kb[a]; k0 < ke[a]; k0 += 4) {
            int32_t e[4];
            int2 pr[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) e[u] = k0 + u < ke[a] ? htci[k0 + u] : -1;
#pragma unroll
            for (int u = 0; u < 4; ++u) pr[u] = e[u] >= 0 ? E2[e[u]] : make_int2(-1, -1);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                int c;
                if (e[u] >= 0 && pat_take(pr[u], T, m, T[a], &c)) {
                    if (np < PT_NMAX) N[np] = e[u];
                    ++np;
                    if (c >= 0) adj |= (1ull << (8 * a + c)) | (1ull << (8 * c + a));
                }
            }
        }
    }
    if (mode == 0) {
        if (np > MAX_NP) { atomicExch(&stats[1], 1); cnt[i] = 0; return; }
        cnt[i] = np;
        if (m > 1) {
            uint32_t reach = 1u;
            for (int it = 0; it < m; ++it) {
                uint32_t nr = reach;
#pragma unroll
                for (int a = 0; a < PT_K; ++a)
                    if ((reach >> a) & 1u) nr |= (uint32_t)((adj >> (8 * a)) & 0xffull);
                reach = nr;
            }
            if (reach != (1u << m) - 1u) {
                int pos = atomicAdd(&stats[2], 1);
                if (bad) bad[pos] = (int32_t)i;
            }
        }
        return;
    }
    int64_t out = nrp[i];
    if (np <= PT_NMAX) {
        for (int t = 0; t < np; ++t) {
            int rank = 0;
            for (int q = 0; q < np; ++q) rank += N[q] < N[t];
            nci[out + rank] = N[t];
        }
        return;
    }
    // a long N_i: merge the per-node lists
    int64_t cur[PT_K];
#pragma unroll
    for (int a = 0; a < PT_K; ++a) {
        cur[a] = kb[a];
        int c;
        while (cur[a] < ke[a] && !pat_take(E2[htci[cur[a]]], T, m, T[a], &c)) ++cur[a];
    }
    for (;;) {
        int32_t best = INT32_MAX;
        int bi = -1;
#pragma unroll
        for (int a = 0; a < PT_K; ++a)
            if (cur[a] < ke[a] && htci[cur[a]] < best) { best = htci[cur[a]]; bi = a; }
        if (bi < 0) break;
        nci[out++] = best;
#pragma unroll
        for (int a = 0; a < PT_K; ++a)
            if (a == bi) {
                ++cur[a];
                int c;
                while (cur[a] < ke[a] && !pat_take(E2[htci[cur[a]]], T, m, T[a], &c)) ++cur[a];
            }
    }
}

// ------------------------------------------------------------------ make_irreducible (Alg. 2)
// For every row whose local graph (nodes T_i, two-node coarse edges of N_i) is disconnected: join
// two components by the pair of coarse nodes (u, v) in different components with the largest
// |Z_uv|, Z = P_n^T D_h^T D_h P_n (the columns of D_h P_n are the rows of T^T), values within a
// relative 1e-9 of the largest counting as ties (the first pair in (a, b) order wins), until the
// row is connected.  Z_uv is summed in increasing fine-edge order without fused multiply-add.
// The new pairs are merged into D_H (sorted pairs first, then the single-node rows) and the
// pattern is rebuilt; at most 8 passes.
constexpr int IRR_WARPS = 4;
constexpr int IRR_MAXP = MAX_T * (MAX_T - 1) / 2;
constexpr int IRR_CAP = 4096;              // new pairs one pass may add (before removing duplicates)

__global__ void __launch_bounds__(IRR_WARPS * 32)
k_irreducible(const int32_t* __restrict__ bad, int nbad, const int64_t* __restrict__ trp,
              const int32_t* __restrict__ tci, const int64_t* __restrict__ htrp, const int32_t* __restrict__ htci,
              const int64_t* __restrict__ hrp, const int32_t* __restrict__ hci, const int64_t* __restrict__ mrp,
              const int32_t* __restrict__ mci, const double* __restrict__ mv, uint64_t* pairs, int* npairs,
              int* overflow) {
    __shared__ int32_t s_J[IRR_WARPS][MAX_T];
    __shared__ int32_t s_comp[IRR_WARPS][MAX_T];
    __shared__ double s_z[IRR_WARPS][IRR_MAXP];
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int li = blockIdx.x * IRR_WARPS + w;
    if (li >= nbad) return;
    int64_t i = bad[li];
    int64_t t0 = trp[i];
    int m = (int)(trp[i + 1] - t0);
    if (m > MAX_T) return;                 // rejected by the pattern step already
    if (lane < m) s_J[w][lane] = tci[t0 + lane];
    __syncwarp();
    // components of the local graph (lane 0; union by the smaller index)
    int nc = 0;
    if (lane == 0) {
        int par[MAX_T];
        for (int q = 0; q < m; ++q) par[q] = q;
        for (int a = 0; a < m; ++a) {
            int32_t J = s_J[w][a];
            for (int64_t k = htrp[J]; k < htrp[J + 1]; ++k) {
                int32_t e = htci[k];
                int64_t b = hrp[e];
                if (hrp[e + 1] - b != 2 || hci[b] != J) continue;
                int c = -1;
                for (int q = 0; q < m; ++q) if (s_J[w][q] == hci[b + 1]) c = q;
                if (c < 0) continue;
                int ra = a, rc = c;
                while (par[ra] != ra) ra = par[ra];
                while (par[rc] != rc) rc = par[rc];
                if (ra != rc) par[ra > rc ? ra : rc] = ra > rc ? rc : ra;
            }
        }
        for (int q = 0; q < m; ++q) {
            int r = q;
            while (par[r] != r) r = par[r];
            s_comp[w][q] = r;
            nc += (r == q);
        }
    }
    nc = __shfl_sync(0xffffffffu, nc, 0);
    // |Z_uv| of every pair (a < b), in (a, b) order
    int npair = m * (m - 1) / 2;
    for (int p = lane; p < npair; p += 32) {
        int a = 0, rem = p;
        while (rem >= m - 1 - a) { rem -= m - 1 - a; ++a; }
        int b = a + 1 + rem;
        int32_t u = s_J[w][a], v = s_J[w][b];
        int64_t x = mrp[u], xe = mrp[u + 1], y = mrp[v], ye = mrp[v + 1];
        double z = 0.0;
        while (x < xe && y < ye) {
            if (mci[x] < mci[y]) ++x;
            else if (mci[y] < mci[x]) ++y;
            else { z = __dadd_rn(z, __dmul_rn(mv[x], mv[y])); ++x; ++y; }
        }
        s_z[w][p] = fabs(z);
    }
    __syncwarp();
    while (nc > 1) {
        double best = -1.0;
        for (int p = lane; p < npair; p += 32) {
            int a = 0, rem = p;
            while (rem >= m - 1 - a) { rem -= m - 1 - a; ++a; }
            int b = a + 1 + rem;
            if (s_comp[w][a] != s_comp[w][b] && s_z[w][p] > best) best = s_z[w][p];
        }
        for (int o = 16; o > 0; o >>= 1) best = fmax(best, __shfl_xor_sync(0xffffffffu, best, o));
        double thr = best * (1.0 - 1e-9);
        int first = INT32_MAX;
        for (int p = lane; p < npair; p += 32) {
            int a = 0, rem = p;
            while (rem >= m - 1 - a) { rem -= m - 1 - a; ++a; }
            int b = a + 1 + rem;
            if (s_comp[w][a] != s_comp[w][b] && s_z[w][p] >= thr) { first = p; break; }
        }
        for (int o = 16; o > 0; o >>= 1) first = min(first, __shfl_xor_sync(0xffffffffu, first, o));
        if (first == INT32_MAX) break;     // cannot happen while nc > 1
        if (lane == 0) {
            int a = 0, rem = first;
            while (rem >= m - 1 - a) { rem -= m - 1 - a; ++a; }
            int b = a + 1 + rem;
            int slot = atomicAdd(npairs, 1);
            if (slot < IRR_CAP) pairs[slot] = ((uint64_t)(uint32_t)s_J[w][a] << 32) | (uint32_t)s_J[w][b];
            else atomicExch(overflow, 1);
            int ca = s_comp[w][a], cb = s_comp[w][b];
            int lo = ca < cb ? ca : cb, hi = ca < cb ? cb : ca;
            for (int q = 0; q < m; ++q) if (s_comp[w][q] == hi) s_comp[w][q] = lo;
        }
        --nc;
        __syncwarp();
    }
}

// key of a two-node coarse edge (rows [0, n2) of D_H are those edges, sorted by key)
__device__ __forceinline__ uint64_t dh_key(const int64_t* hrp, const int32_t* hci, int64_t j) {
    int64_t b = hrp[j];
    return ((uint64_t)(uint32_t)hci[b] << 32) | (uint32_t)hci[b + 1];
}
__device__ __forceinline__ int64_t key_lower_bound(const int64_t* hrp, const int32_t* hci, int64_t n2, uint64_t key) {
    int64_t lo = 0, hi = n2;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (dh_key(hrp, hci, mid) < key) lo = mid + 1; else hi = mid;
    }
    return lo;
}
// One block: sort the new pairs, drop repeats and pairs already in D_H, count the rest (*nu)
__global__ void __launch_bounds__(1024)
k_pairs_unique(uint64_t* pairs, int n, const int64_t* hrp, const int32_t* hci, int64_t n2, int* nu) {
    __shared__ uint64_t s_k[IRR_CAP];
    int n2pow = 1;
    while (n2pow < n) n2pow <<= 1;
    for (int t = threadIdx.x; t < n2pow; t += blockDim.x) s_k[t] = t < n ? pairs[t] : ~0ull;
    __syncthreads();
    for (int size = 2; size <= n2pow; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = threadIdx.x; t < n2pow; t += blockDim.x) {
                int o = t ^ stride;
                if (o > t) {
                    bool up = (t & size) == 0;
                    if ((s_k[t] > s_k[o]) == up) { uint64_t x = s_k[t]; s_k[t] = s_k[o]; s_k[o] = x; }
                }
            }
            __syncthreads();
        }
    if (threadIdx.x == 0) {
        int q = 0;
        for (int t = 0; t < n; ++t) {
            uint64_t k = s_k[t];
            if (q > 0 && pairs[q - 1] == k) continue;
            int64_t pos = key_lower_bound(hrp, hci, n2, k);
            if (pos < n2 && dh_key(hrp, hci, pos) == k) continue;
            pairs[q++] = k;
        }
        *nu = q;
    }
}
// D_H with the nu new pairs merged: pair rows at their sorted positions, single rows after
__global__ void k_dh_merge(const int64_t* hrp, const int32_t* hci, const double* hv, int64_t nr, int64_t n2,
                           const uint64_t* pairs, int nu, int64_t* nrp, int32_t* nci, double* nv) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t total = nr + nu;
    if (t > total) return;
    int64_t npair = n2 + nu;
    nrp[t] = t <= npair ? 2 * t : 2 * npair + (t - npair);
    if (t == total) return;
    if (t < nr) {
        int64_t r;
        if (t < n2) {
            uint64_t k = dh_key(hrp, hci, t);
            int lo = 0, hi = nu;                     // new pairs below k
            while (lo < hi) { int mid = (lo + hi) >> 1; if (pairs[mid] < k) lo = mid + 1; else hi = mid; }
            r = t + lo;
            nci[2 * r] = hci[hrp[t]];
            nci[2 * r + 1] = hci[hrp[t] + 1];
            nv[2 * r] = hv[hrp[t]];
            nv[2 * r + 1] = hv[hrp[t] + 1];
        } else {
            r = t + nu;
            int64_t o = 2 * npair + (r - npair);
            nci[o] = hci[hrp[t]];
            nv[o] = hv[hrp[t]];
        }
    } else {
        int64_t q = t - nr;                          // new pair q
        uint64_t k = pairs[q];
        int64_t r = q + key_lower_bound(hrp, hci, n2, k);
        nci[2 * r] = (int32_t)(k >> 32);
        nci[2 * r + 1] = (int32_t)(k & 0xffffffffull);
        nv[2 * r] = -1.0;
        nv[2 * r + 1] = 1.0;
    }
}

// ------------------------------------------------------------------ local least-norm systems
// Per-warp view of the local system of fine row i: nodes T_i (m <= MAX_T), pattern entries N_i
// (np <= MAX_NP) with the local indices of their coarse nodes and the signs of D_H.
//
// The normal matrix G~^T G~ of a row is a small integer matrix (a grounded graph Laplacian).
// FP64 throughput is scarce on this GPU, so it is factored in FP32 (LDL^T) and every solve is
// refined twice against FP64 residuals evaluated exactly through the +-1 entries of G~; each
// step multiplies the error by about eps32 * cond (cond is at most a few hundred for these
// graphs), which brings the solution to FP64 accuracy.
constexpr int REFINE_STEPS = 2;
struct LocalSys {
    int32_t T[MAX_T];
    double r[MAX_T];
    int32_t N[MAX_NP];
    int8_t la[MAX_NP], lb[MAX_NP];    // local node (or -1) carrying -1 (la) / +1 (lb)
    double w[MAX_NP];                 // per-entry work values
    double z[MAX_T];                  // solution being refined
    double rhs[MAX_T];                // right side of the normal equations
    double res[MAX_T];                // its FP64 residual
    int16_t inc[2 * MAX_NP];          // node incidence lists: (entry << 1) | (coefficient < 0)
    int inc_ptr[MAX_T + 1];
    float xs[MAX_T];                  // FP32 right side / solution of the factored solve
    int G[MAX_T * MAX_T];             // integer G~^T G~
    float L[MAX_T * MAX_T];           // FP32 LDL^T (unit lower triangle below the diagonal)
    float dinv[MAX_T];
};

// Load the row, build G~^T G~ and factor it; returns k (columns kept) or -1 on failure.
__device__ int local_setup(LocalSys& S, int64_t i, const int64_t* trp, const int32_t* tci, const double* tv,
                           const int64_t* nrp, const int32_t* nci, const int64_t* hrp, const int32_t* hci,
                           const double* hv, int* m_out, int* np_out) {
    int lane = threadIdx.x & 31;
    int64_t t0 = trp[i], n0 = nrp[i];
    int m = (int)(trp[i + 1] - t0), np = (int)(nrp[i + 1] - n0);
    *m_out = m;
    *np_out = np;
    if (lane < m) { S.T[lane] = tci[t0 + lane]; S.r[lane] = tv[t0 + lane]; }
    __syncwarp();
    int single = 0;
    for (int t = lane; t < np; t += 32) {
        int32_t e = nci[n0 + t];
        S.N[t] = e;
        int64_t b = hrp[e];
        int len = (int)(hrp[e + 1] - b);
        int8_t la = -1, lb = -1;
        for (int q = 0; q < len; ++q) {
            int32_t u = hci[b + q];
            int loc = -1;
            for (int zz = 0; zz < m; ++zz) if (S.T[zz] == u) loc = zz;
            if (hv[b + q] < 0) la = (int8_t)loc; else lb = (int8_t)loc;
        }
        S.la[t] = la;
        S.lb[t] = lb;
        if (len == 1) single = 1;
    }
    single = __any_sync(0xffffffffu, single);
    int k = single ? m : m - 1;     // Reduce_Dimension drops the largest coarse node
    if (k < 0) k = 0;
    for (int q = lane; q < k * k; q += 32) S.G[q] = 0;
    __syncwarp();
    for (int t = lane; t < np; t += 32) {
        int a = S.la[t], b = S.lb[t];
        bool ia = a >= 0 && a < k, ib = b >= 0 && b < k;
        if (ia) atomicAdd(&S.G[a * k + a], 1);
        if (ib) atomicAdd(&S.G[b * k + b], 1);
        if (ia && ib) { atomicAdd(&S.G[a * k + b], -1); atomicAdd(&S.G[b * k + a], -1); }
    }
    // incidence list of node a, built by lane a in entry order (deterministic sums below)
    int cnt = 0;
    if (lane < k)
        for (int t = 0; t < np; ++t) cnt += (S.la[t] == lane) + (S.lb[t] == lane);
    int incl = cnt;
    for (int o = 1; o < 32; o <<= 1) {
        int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane < k) {
        int c = incl - cnt;
        S.inc_ptr[lane] = c;
        for (int t = 0; t < np; ++t) {
            if (S.la[t] == lane) S.inc[c++] = (int16_t)((t << 1) | 1);
            if (S.lb[t] == lane) S.inc[c++] = (int16_t)(t << 1);
        }
        if (lane == k - 1) S.inc_ptr[k] = c;
    }
    __syncwarp();
    for (int q = lane; q < k * k; q += 32) S.L[q] = (float)S.G[q];
    __syncwarp();
    int ok = 1;
    for (int j = 0; j < k; ++j) {
        float d = S.L[j * k + j];
        if (!(d > 1e-6f)) ok = 0;          // a disconnected local graph leaves a zero pivot
        float inv = 1.0f / (d > 1e-6f ? d : 1.0f);
        int rem = k - j - 1;
        for (int q = lane; q < rem * rem; q += 32) {
            int r = j + 1 + q / rem, c = j + 1 + q % rem;
            if (c <= r) S.L[r * k + c] -= S.L[r * k + j] * S.L[c * k + j] * inv;
        }
        __syncwarp();
        for (int r = j + 1 + lane; r < k; r += 32) S.L[r * k + j] *= inv;
        if (lane == 0) S.dinv[j] = inv;
        __syncwarp();
    }
    if (k > np) ok = 0;
    return ok ? k : -1;
}

// x := (L D L^T)^-1 x in FP32 (one lane)
__device__ inline void ldl_solve32(const float* L, const float* dinv, int k, float* x) {
    for (int r = 0; r < k; ++r) {
        float s = x[r];
        for (int c = 0; c < r; ++c) s -= L[r * k + c] * x[c];
        x[r] = s;
    }
    for (int r = 0; r < k; ++r) x[r] *= dinv[r];
    for (int r = k - 1; r >= 0; --r) {
        float s = x[r];
        for (int c = r + 1; c < k; ++c) s -= L[c * k + r] * x[c];
        x[r] = s;
    }
}

// (G~ z)_t for pattern entry t
__device__ inline double gz(const LocalSys& S, int t, int k, const double* z) {
    double v = 0.0;
    int a = S.la[t], b = S.lb[t];
    if (a >= 0 && a < k) v -= z[a];
    if (b >= 0 && b < k) v += z[b];
    return v;
}

// (G~^T v)_a for node a < k (one lane per node)
__device__ inline double gtv(const LocalSys& S, int a, const double* v) {
    double s = 0.0;
    for (int q = S.inc_ptr[a]; q < S.inc_ptr[a + 1]; ++q) {
        int code = S.inc[q];
        double x = v[code >> 1];
        s += (code & 1) ? -x : x;
    }
    return s;
}

// S.z = (G~^T G~)^-1 S.rhs: FP32 solve, then two FP64-residual refinement steps.  An FP64
// instruction costs the whole warp's issue slot however many lanes are active, so every FP64
// step is spread over the lanes; only the FP32 triangular solves run on one lane.
__device__ void refine_solve(LocalSys& S, int k, int np) {
    int lane = threadIdx.x & 31;
    if (lane < k) S.xs[lane] = (float)S.rhs[lane];
    __syncwarp();
    if (lane == 0) ldl_solve32(S.L, S.dinv, k, S.xs);
    __syncwarp();
    if (lane < k) S.z[lane] = (double)S.xs[lane];
    __syncwarp();
    for (int step = 0; step < REFINE_STEPS; ++step) {
        for (int t = lane; t < np; t += 32) S.w[t] = gz(S, t, k, S.z);
        __syncwarp();
        if (lane < k) S.xs[lane] = (float)(S.rhs[lane] - gtv(S, lane, S.w));
        __syncwarp();
        if (lane == 0) ldl_solve32(S.L, S.dinv, k, S.xs);
        __syncwarp();
        if (lane < k) S.z[lane] += (double)S.xs[lane];
        __syncwarp();
    }
}

// least-norm initial guess P0_i = G~ (G~^T G~)^-1 r~_i
template <typename DT>
__global__ void __launch_bounds__(LOC_WARPS * 32)
k_p0(int64_t ne, const int32_t* rows, const int64_t* trp, const int32_t* tci, const double* tv, const int64_t* nrp,
     const int32_t* nci, const int64_t* hrp, const int32_t* hci, const double* hv, const DT* d, double* p0,
     int* fail) {
    extern __shared__ unsigned char smem_raw[];
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    LocalSys& S = ((LocalSys*)smem_raw)[w];
    int64_t i = (int64_t)blockIdx.x * LOC_WARPS + w;
    if (i >= ne) return;
    if (rows) i = rows[i];
    int m, np;
    int k = local_setup(S, i, trp, tci, tv, nrp, nci, hrp, hci, hv, &m, &np);
    if (np == 0) return;
    if (k < 0) { if (lane == 0) atomicAdd(fail, 1); return; }
    int64_t n0 = nrp[i];
    // p = d + G~ z with (G~^T G~) z = r~ - G~^T d: the point of {G~^T p = r~} nearest to d
    // (d = 0: the least-norm solution; d = the MLP correction: P0 + (I - G~ (G~^T G~)^-1 G~^T) d)
    double dt[MAX_NP / 32];
    for (int t = lane, q = 0; t < np; t += 32, ++q) {
        dt[q] = d ? (double)d[n0 + t] : 0.0;
        S.w[t] = dt[q];
    }
    __syncwarp();
    if (lane < k) S.rhs[lane] = d ? S.r[lane] - gtv(S, lane, S.w) : S.r[lane];
    __syncwarp();
    refine_solve(S, k, np);
    for (int t = lane, q = 0; t < np; t += 32, ++q) p0[n0 + t] = dt[q] + gz(S, t, k, S.z);
}

// one projected-Jacobi step (eq. (9)): dP = D^-1 (A P)|_N, projected row by row, P' = P - w dP
__global__ void __launch_bounds__(LOC_WARPS * 32)
k_emin(int64_t ne, const int32_t* rows, const int64_t* arp, const int32_t* aci, const double* av, const int64_t* trp,
       const int32_t* tci, const double* tv, const int64_t* nrp, const int32_t* nci, const int64_t* hrp,
       const int32_t* hci, const double* hv, const double* P, double* Pout, double omega, int* fail,
       int grad_only) {
    extern __shared__ unsigned char smem_raw[];
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    LocalSys& S = ((LocalSys*)smem_raw)[w];
    int64_t i = (int64_t)blockIdx.x * LOC_WARPS + w;
    if (i >= ne) return;
    if (rows) i = rows[i];
    int m, np;
    int k = local_setup(S, i, trp, tci, tv, nrp, nci, hrp, hci, hv, &m, &np);
    if (np == 0) return;
    if (k < 0) { if (lane == 0) atomicAdd(fail, 1); return; }
    // masked product (A P)_{i, N_i}: a group of L lanes owns a pattern entry (L as large as the
    // row allows, so the whole warp works on short rows); its lanes split A's row i and search
    // each P row f for the entry's column (one FMA per match, no atomics), then add up.
    int64_t a0 = arp[i], a1 = arp[i + 1];
    double aii = 1.0;
    for (int64_t ka = a0; ka < a1; ++ka)
        if (aci[ka] == i) aii = av[ka];
    double inv_aii = 1.0 / aii;
    int L = 1;
    while (L < 32 && np * (2 * L) <= 32) L *= 2;
    int G = 32 / L, grp = lane / L, sub = lane & (L - 1);
    int trips = (np + G - 1) / G;
    for (int it = 0; it < trips; ++it) {
        int t = grp + it * G;
        double acc = 0.0;
        if (t < np) {
            int32_t j = S.N[t];
            for (int64_t ka = a0 + sub; ka < a1; ka += L) {
                int32_t f = aci[ka];
                int64_t lo = nrp[f], hi = nrp[f + 1] - 1;
                while (lo < hi) {
                    int64_t mid = (lo + hi) >> 1;
                    if (nci[mid] < j) lo = mid + 1; else hi = mid;
                }
                if (lo <= hi && nci[lo] == j) acc += av[ka] * P[lo];
            }
        }
        for (int d = L >> 1; d > 0; d >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, d);
        if (t < np && sub == 0) S.w[t] = acc * inv_aii;
    }
    __syncwarp();
    // projection onto null(G~^T): dp = w - G~ (G~^T G~)^-1 G~^T w
    if (lane < k) S.rhs[lane] = gtv(S, lane, S.w);
    __syncwarp();
    double wt[MAX_NP / 32];
    for (int t = lane, q = 0; t < np; t += 32, ++q) wt[q] = S.w[t];
    __syncwarp();
    refine_solve(S, k, np);
    int64_t n0 = nrp[i];
    for (int t = lane, q = 0; t < np; t += 32, ++q) {
        double dp = wt[q] - gz(S, t, k, S.z);
        Pout[n0 + t] = grad_only ? dp : P[n0 + t] - omega * dp;
    }
}

// ------------------------------------------------------------------ thread-per-row local solves
// The local systems of a fine row are tiny: G~ has one column per kept coarse node of T_i and one
// row per pattern entry, with a -1 and a +1 (or a single +-1) per row.  Rows with at most TK
// coarse nodes and TNP pattern entries (every row of the fine levels of the Kuhn meshes) are
// solved by one thread each: G~ as two bitmasks per node (entries carrying +1 / -1 there), the
// integer G~^T G~ from popcounts, and an FP64 Cholesky factor in registers.  Larger rows go to
// the warp-per-row kernels above through a row list.
constexpr int TK = 8, TNP = 32;

struct RowSys {
    uint32_t pos[TK], neg[TK];
    double r[TK];
    double L[TK][TK];
    int k, np;
    int64_t n0;
};

// Coarse edge e of D_H as two codes 2 node + (value < 0), the second -1 for a single-node row:
// one 8-byte load per pattern entry instead of a row pointer and then its entries.
__global__ void k_edge_codes(const int64_t* __restrict__ hrp, const int32_t* __restrict__ hci,
                             const double* __restrict__ hv, int64_t nE, int2* __restrict__ E) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nE) return;
    int64_t b = hrp[e];
    int len = (int)(hrp[e + 1] - b);
    int2 c = make_int2(-1, -1);
    if (len >= 1) c.x = 2 * hci[b] + (hv[b] < 0 ? 1 : 0);
    if (len >= 2) c.y = 2 * hci[b + 1] + (hv[b + 1] < 0 ? 1 : 0);
    E[e] = c;
}

// 1: factored; 0: infeasible; -1: too large for one thread; 2: empty row.  The row's pattern
// entries are read four at a time (their edge ids, then their codes), so the loads overlap.
__device__ __forceinline__ int row_factor(int64_t i, const int64_t* __restrict__ trp, const int32_t* __restrict__ tci,
                                          const double* __restrict__ tv, const int64_t* __restrict__ nrp,
                                          const int32_t* __restrict__ nci, const int2* __restrict__ E, RowSys& S) {
    int64_t t0 = trp[i];
    int m = (int)(trp[i + 1] - t0);
    S.n0 = nrp[i];
    S.np = (int)(nrp[i + 1] - S.n0);
    if (S.np == 0) return 2;
    if (m > TK || S.np > TNP) return -1;
    int32_t T[TK];
#pragma unroll
    for (int a = 0; a < TK; ++a) {
        T[a] = a < m ? tci[t0 + a] : -1;
        S.r[a] = a < m ? tv[t0 + a] : 0.0;
        S.pos[a] = 0u;
        S.neg[a] = 0u;
    }
    bool single = false;
    for (int t0 = 0; t0 < S.np; t0 += 4) {
        int32_t e[4];
        int2 c[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) e[u] = t0 + u < S.np ? nci[S.n0 + t0 + u] : -1;
#pragma unroll
        for (int u = 0; u < 4; ++u) c[u] = e[u] >= 0 ? E[e[u]] : make_int2(-1, -1);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (e[u] < 0) continue;
            const int t = t0 + u;
            if (c[u].x >= 0 && c[u].y < 0) single = true;
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int32_t code = q == 0 ? c[u].x : c[u].y;
                if (code < 0) continue;
                const int32_t nd = code >> 1;
                const bool minus = code & 1;
#pragma unroll
                for (int a = 0; a < TK; ++a)
                    if (T[a] == nd) {
                        if (minus) S.neg[a] |= 1u << t;
                        else S.pos[a] |= 1u << t;
                    }
            }
        }
    }
    int k = single ? m : m - 1;     // Reduce_Dimension drops the largest coarse node
    if (k < 0) k = 0;
    S.k = k;
    if (k > S.np) return 0;
    // G~^T G~ (identity beyond k) and its Cholesky factor, left-looking
#pragma unroll
    for (int a = 0; a < TK; ++a)
#pragma unroll
        for (int b = 0; b <= a; ++b) {
            double g;
            if (a < k && b < k)
                g = a == b ? (double)__popc(S.pos[a] | S.neg[a])
                           : -(double)(__popc(S.pos[a] & S.neg[b]) + __popc(S.neg[a] & S.pos[b]));
            else
                g = a == b ? 1.0 : 0.0;
            S.L[a][b] = g;
        }
    // Columns and rows from k on are the identity padding of the unrolled loops (their entries of
    // L stay 1 on the diagonal and 0 elsewhere): they are skipped, which leaves every entry of the
    // k x k factor as it is and saves the FP64 work of the padding (k is mostly 4..6 of TK = 8).
    bool ok = true;
#pragma unroll
    for (int j = 0; j < TK; ++j) {
        if (j >= k) continue;
        double d = S.L[j][j];
#pragma unroll
        for (int c = 0; c < j; ++c) d -= S.L[j][c] * S.L[j][c];
        if (!(d > 1e-6)) { ok = false; d = 1.0; }   // a disconnected local graph leaves a zero pivot
        double inv = rsqrt(d);                         // the diagonal is kept as its inverse
        S.L[j][j] = inv;
#pragma unroll
        for (int r = j + 1; r < TK; ++r) {
            if (r >= k) continue;
            double v = S.L[r][j];
#pragma unroll
            for (int c = 0; c < j; ++c) v -= S.L[r][c] * S.L[j][c];
            S.L[r][j] = v * inv;
        }
    }
    return ok ? 1 : 0;
}
// x := (L L^T)^-1 x (L's diagonal holds 1 / L_aa)
// (only the k x k system: the padding rows of x are 0 and stay 0)
__device__ __forceinline__ void row_solve(const RowSys& S, double x[TK]) {
    const int k = S.k;
#pragma unroll
    for (int a = 0; a < TK; ++a) {
        if (a >= k) continue;
        double v = x[a];
#pragma unroll
        for (int c = 0; c < a; ++c) v -= S.L[a][c] * x[c];
        x[a] = v * S.L[a][a];
    }
#pragma unroll
    for (int a = TK - 1; a >= 0; --a) {
        if (a >= k) continue;
        double v = x[a];
#pragma unroll
        for (int r = a + 1; r < TK; ++r)
            if (r < k) v -= S.L[r][a] * x[r];
        x[a] = v * S.L[a][a];
    }
}
// (G~ z)_t.  Row t of G~ has at most one +1 and one -1 among the kept columns, so the two values
// are picked by integer selects and the FP64 pipe (thin on this GPU) does one subtraction.
__device__ __forceinline__ double row_gz(const RowSys& S, int t, const double z[TK]) {
    double zh = 0.0, zt = 0.0;
#pragma unroll
    for (int a = 0; a < TK; ++a) {
        const bool in = a < S.k;
        zh = in && ((S.pos[a] >> t) & 1u) ? z[a] : zh;
        zt = in && ((S.neg[a] >> t) & 1u) ? z[a] : zt;
    }
    return zh - zt;
}
// x -= G~^T v (v read from memory, one value per pattern entry): per kept column, the entries of
// its set bits only
template <typename V>
__device__ __forceinline__ void row_sub_gtv(const RowSys& S, const V* v, double x[TK]) {
#pragma unroll
    for (int a = 0; a < TK; ++a) {
        if (a >= S.k) continue;
        double acc = x[a];
        for (uint32_t m = S.pos[a]; m; m &= m - 1u) acc -= (double)v[S.n0 + __ffs(m) - 1];
        for (uint32_t m = S.neg[a]; m; m &= m - 1u) acc += (double)v[S.n0 + __ffs(m) - 1];
        x[a] = acc;
    }
}

// The factored local system of every thread-handled row, kept from the P0 solve for the
// energy-minimisation steps, which project onto the same constraints: the node bitmasks, the
// number of kept constraints k (-1: no system for the row) and the lower triangle of the Cholesky
// factor, stored structure of arrays (entry e of row i at e * ne + i).
constexpr int TL = TK * (TK + 1) / 2;
struct RowCache {
    uint32_t* pm;        // 2 * TK masks
    int8_t* k;
    double* L;           // TL entries
    int64_t ne;
};
__device__ __forceinline__ void cache_put(const RowCache& C, int64_t i, const RowSys& S) {
#pragma unroll
    for (int a = 0; a < TK; ++a) {
        C.pm[(2 * a) * C.ne + i] = S.pos[a];
        C.pm[(2 * a + 1) * C.ne + i] = S.neg[a];
    }
    int e = 0;
#pragma unroll
    for (int a = 0; a < TK; ++a)
#pragma unroll
        for (int b = 0; b <= a; ++b) C.L[(int64_t)(e++) * C.ne + i] = S.L[a][b];
    C.k[i] = (int8_t)S.k;
}
__device__ __forceinline__ void cache_get(const RowCache& C, int64_t i, RowSys& S) {
#pragma unroll
    for (int a = 0; a < TK; ++a) {
        S.pos[a] = C.pm[(2 * a) * C.ne + i];
        S.neg[a] = C.pm[(2 * a + 1) * C.ne + i];
    }
    int e = 0;
#pragma unroll
    for (int a = 0; a < TK; ++a)
#pragma unroll
        for (int b = 0; b <= a; ++b) S.L[a][b] = C.L[(int64_t)(e++) * C.ne + i];
}

// P0 of every small row: the point of {G~^T p = r~} nearest to d (d null: 0), p = d + G~ z with
// (G~^T G~) z = r~ - G~^T d.  Rows too large for a thread are appended to `big`.  Every row's
// factored system (or k = -1) goes to the cache.
template <typename DT>
__global__ void __launch_bounds__(128)
k_p0_rows(int64_t ne, const int64_t* __restrict__ trp, const int32_t* __restrict__ tci, const double* __restrict__ tv,
          const int64_t* __restrict__ nrp, const int32_t* __restrict__ nci, const int2* __restrict__ E,
          const DT* __restrict__ d, double* __restrict__ p0, int* fail, int32_t* big, int* nbig, RowCache cache) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ne) return;
    RowSys S;
    int code = row_factor(i, trp, tci, tv, nrp, nci, E, S);
    if (code != 1) cache.k[i] = -1;
    if (code == 2) return;
    if (code == -1) { big[warp_reserve(nbig)] = (int32_t)i; return; }
    if (code == 0) { atomicAdd(fail, 1); return; }
    cache_put(cache, i, S);
    double z[TK];
#pragma unroll
    for (int a = 0; a < TK; ++a) z[a] = a < S.k ? S.r[a] : 0.0;
    if (d) row_sub_gtv(S, d, z);
    row_solve(S, z);
    for (int t = 0; t < S.np; ++t) p0[S.n0 + t] = (d ? (double)d[S.n0 + t] : 0.0) + row_gz(S, t, z);
}

// Masked product of eq. (9) for every row that the thread-per-row projection handles:
// w_{i,t} = (A P)_{i, N_i(t)} / a_ii, one warp per row.  L lanes share pattern entry t (L the
// largest power of two with np L <= 32) and split A's row: each lane takes every L-th entry f and
// finds column N_i(t) in the sorted P row f by binary search.  A lane runs PP_ILP searches at
// once, branch-free with a fixed step count for rows of up to 32 entries, so their loads overlap
// instead of forming one long chain; a lane sums its matches in A's row order and the L lanes of
// an entry are added in a fixed pattern, so the result does not depend on scheduling.  Acc is
// double, or float for the FP32 accumulation of opts.emin_fp32 (the projection stays FP64).
constexpr int PP_WARPS = 4;
constexpr int PP_ILP = 4;
// P is read in the accumulation type: the FP32 mode gets an FP32 copy of P's values, converted once
// per step, because on this GPU a double-to-float conversion per pair would run on the same thin
// FP64 pipe as an FP64 FMA (ncu: 82 % FP64-pipe activity with per-pair conversions).
template <typename Acc>
__global__ void __launch_bounds__(PP_WARPS * 32)
k_emin_pp(int64_t ne, const int64_t* __restrict__ arp, const int32_t* __restrict__ aci, const Acc* __restrict__ av,
          const Acc* __restrict__ dinv, const int64_t* __restrict__ nrp, const int32_t* __restrict__ nci,
          const Acc* __restrict__ P, const int8_t* __restrict__ ck, Acc* __restrict__ w) {
    const int lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * PP_WARPS + (threadIdx.x >> 5);
    if (i >= ne || ck[i] < 0) return;                  // whole warp: no row, or a row k_emin handles
    const int64_t n0 = nrp[i];
    const int np = (int)(nrp[i + 1] - n0);
    if (np <= 0 || np > 32) return;
    int L = 1;
    while (L < 32 && np * (2 * L) <= 32) L *= 2;
    const int t = lane / L, sub = lane & (L - 1);
    const bool owner = t < np;
    const int32_t key = owner ? nci[n0 + t] : -1;
    const int64_t a0 = arp[i], a1 = arp[i + 1];
    Acc acc = Acc(0);
    for (int64_t kb = a0 + sub; kb < a1; kb += (int64_t)PP_ILP * L) {
        int64_t lo[PP_ILP];
        int len[PP_ILP];
        Acc a[PP_ILP];
#pragma unroll
        for (int j = 0; j < PP_ILP; ++j) {
            const int64_t ka = kb + (int64_t)j * L;
            lo[j] = 0;
            len[j] = 0;
            a[j] = Acc(0);
            if (ka < a1) {
                const int32_t f = aci[ka];
                a[j] = av[ka];
                lo[j] = nrp[f];
                len[j] = (int)(nrp[f + 1] - lo[j]);
            }
        }
        if (!owner) continue;
        int pos[PP_ILP];
#pragma unroll
        for (int j = 0; j < PP_ILP; ++j) pos[j] = 0;
        bool longrow = false;
#pragma unroll
        for (int j = 0; j < PP_ILP; ++j) longrow = longrow || len[j] > 32;
        if (!longrow) {
            // last position with column <= key, five halving steps (rows of at most 32 entries)
#pragma unroll
            for (int h = 16; h > 0; h >>= 1)
#pragma unroll
                for (int j = 0; j < PP_ILP; ++j)
                    if (pos[j] + h < len[j] && nci[lo[j] + pos[j] + h] <= key) pos[j] += h;
        } else {
#pragma unroll
            for (int j = 0; j < PP_ILP; ++j) {
                int lo2 = 0, hi2 = len[j];                 // first position with column >= key
                while (lo2 < hi2) {
                    const int mid = (lo2 + hi2) >> 1;
                    if (nci[lo[j] + mid] < key) lo2 = mid + 1; else hi2 = mid;
                }
                pos[j] = lo2 < len[j] ? lo2 : 0;
            }
        }
#pragma unroll
        for (int j = 0; j < PP_ILP; ++j)
            if (len[j] > 0 && nci[lo[j] + pos[j]] == key) acc += a[j] * P[lo[j] + pos[j]];
    }
    for (int d = L >> 1; d > 0; d >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, d);
    if (owner && sub == 0) w[n0 + t] = acc * dinv[i];
}

// 1 / a_ii of every row (1 where the row has no diagonal entry), in FP64 and rounded to FP32: the
// D^-1 of eq. (9), formed once per level for the masked product
__global__ void k_diag_inv(int64_t n, const int64_t* __restrict__ arp, const int32_t* __restrict__ aci,
                           const double* __restrict__ av, double* __restrict__ dinv, float* __restrict__ dinvf) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double aii = 1.0;
    for (int64_t k = arp[i]; k < arp[i + 1]; ++k)
        if (aci[k] == (int32_t)i) {
            aii = av[k];
            break;
        }
    const double d = 1.0 / aii;
    dinv[i] = d;
    if (dinvf) dinvf[i] = (float)d;
}

// projection and update of eq. (9) for every small row: dp = w - G~ (G~^T G~)^-1 G~^T w,
// P' = P - omega dp, with the system factored by k_p0_rows (rows too large for a thread are
// handled by k_emin through a row list)
template <typename V>
__global__ void __launch_bounds__(128)
k_emin_rows(int64_t ne, const int64_t* __restrict__ nrp, const V* __restrict__ w, const double* __restrict__ P,
            double* __restrict__ Pout, double omega, RowCache cache, int grad_only) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ne) return;
    const int k = cache.k[i];
    if (k < 0) return;                               // empty, large (k_emin) or infeasible row
    RowSys S;
    S.k = k;
    S.n0 = nrp[i];
    S.np = (int)(nrp[i + 1] - S.n0);
    cache_get(cache, i, S);
    double z[TK];
#pragma unroll
    for (int a = 0; a < TK; ++a) z[a] = 0.0;
    row_sub_gtv(S, w, z);
#pragma unroll
    for (int a = 0; a < TK; ++a) z[a] = -z[a];
    row_solve(S, z);
    for (int t = 0; t < S.np; ++t) {
        double dp = (double)w[S.n0 + t] - row_gz(S, t, z);
        Pout[S.n0 + t] = grad_only ? dp : P[S.n0 + t] - omega * dp;
    }
}

// ------------------------------------------------------------------ projected CG (Sec. 3, eq. (8))
// partial sums of sum_i a_ii x_i . y_i over the pattern rows (thread per row, block sums in a
// fixed order); the inner product of the D^-1-preconditioned projected CG
__global__ void __launch_bounds__(256)
k_wdot_rows(int64_t ne, const int64_t* __restrict__ nrp, const double* __restrict__ d, const double* __restrict__ x,
            const double* __restrict__ y, double* __restrict__ part) {
    __shared__ double sw[8];
    double sacc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ne; i += (int64_t)gridDim.x * blockDim.x) {
        double si = 0.0;
        for (int64_t q = nrp[i]; q < nrp[i + 1]; ++q) si += x[q] * y[q];
        sacc += d[i] * si;
    }
    for (int o = 16; o > 0; o >>= 1) sacc += __shfl_down_sync(0xffffffffu, sacc, o);
    if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = sacc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += sw[w];
        part[blockIdx.x] = t;
    }
}
__global__ void k_sum_parts(const double* part, int n, double* out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < n; ++q) t += part[q];
        *out = t;
    }
}
__global__ void k_neg_copy(const double* a, double* b, double* c, int64_t n) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < n) { b[q] = -a[q]; c[q] = -a[q]; }
}
// P += alpha p, z -= alpha w
__global__ void k_cg_update(double* P, const double* pd, double* z, const double* w, double alpha, int64_t n) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < n) { P[q] += alpha * pd[q]; z[q] -= alpha * w[q]; }
}
__global__ void k_cg_dir(double* pd, const double* z, double beta, int64_t n) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < n) pd[q] = z[q] + beta * pd[q];
}

// ------------------------------------------------------------------ learned warm start
// centroid of each aggregate (coordinates of the coarse nodes); members sorted, so the sums are
// taken in a fixed order
__global__ void k_centroids(const int64_t* mptr, const int32_t* members, int64_t nagg, const double* X, double* Xc) {
    int64_t U = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (U >= nagg) return;
    double c[3] = {0.0, 0.0, 0.0};
    int64_t b = mptr[U], e = mptr[U + 1];
    for (int64_t q = b; q < e; ++q)
        for (int a = 0; a < 3; ++a) c[a] += X[3 * (int64_t)members[q] + a];
    double inv = e > b ? 1.0 / (double)(e - b) : 0.0;
    for (int a = 0; a < 3; ++a) Xc[3 * U + a] = c[a] * inv;
}

// Per fine row: the quantities all its pattern entries share (features.cuh).
__global__ void k_row_feat(int64_t ne, const int64_t* __restrict__ drp, const int32_t* __restrict__ dci,
                           const double* __restrict__ dv, const int64_t* __restrict__ arp,
                           const int32_t* __restrict__ aci, const double* __restrict__ av,
                           const int64_t* __restrict__ nrp, const int64_t* __restrict__ trp,
                           const double* __restrict__ X, const double* __restrict__ sig, RowFeat* out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ne) return;
    RowFeat R;
    int32_t u = -1, v = -1;
    for (int64_t k = drp[i]; k < drp[i + 1]; ++k) { if (dv[k] < 0) u = dci[k]; else v = dci[k]; }
    R.u = u;
    R.v = v;
    bool two = u >= 0 && v >= 0;
    float xu[3] = {0, 0, 0}, xv[3] = {0, 0, 0}, t[3] = {0, 0, 0};
    if (u >= 0) for (int a = 0; a < 3; ++a) xu[a] = (float)X[3 * (int64_t)u + a];
    if (v >= 0) for (int a = 0; a < 3; ++a) xv[a] = (float)X[3 * (int64_t)v + a];
    float h = 1.f;
    if (two) {
        for (int a = 0; a < 3; ++a) t[a] = xv[a] - xu[a];
        h = sqrtf(t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
        if (!(h > 0.f)) h = 1.f;
    }
    R.ih = 1.f / h;
    for (int a = 0; a < 3; ++a) {
        R.t[a] = t[a] * R.ih;
        R.mid[a] = 0.5f * (xu[a] + xv[a]);
    }
    R.two = two ? 1.f : 0.f;
    R.nlen = (float)(nrp[i + 1] - nrp[i]) / 32.f;
    R.tlen = (float)(trp[i + 1] - trp[i]) / 16.f;
    float aii = 0.f, l1 = 0.f;
    for (int64_t k = arp[i]; k < arp[i + 1]; ++k) {
        float x = (float)av[k];
        l1 += fabsf(x);
        if (aci[k] == i) aii = x;
    }
    R.diag = l1 > 0.f ? aii / l1 : 0.f;
    R.lsig = sig ? log10f(fmaxf((float)sig[i], 1e-30f)) / 6.f : 0.f;
    out[i] = R;
}
__global__ void k_to_float(const double* a, int64_t n, float* b) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (float)a[i];
}

int feat_prepare(const Level& L, const DBuf<double>& Xc, int lev, FeatBufs& B, FeatArgs& g, cudaStream_t s) {
    if (!L.X.p || !Xc.p) {
        set_error("features need node coordinates (pass coords to sphc_setup)");
        return SPHC_EINVAL;
    }
    int64_t ne = L.A.nr;
    SPHC_TRY(B.tvf.alloc(L.T.nnz, s));
    SPHC_TRY(B.pvf.alloc(L.Pn.nnz, s));
    SPHC_TRY(B.Xcf.alloc(Xc.n, s));
    SPHC_TRY(B.rf.alloc(ne, s));
    if (L.T.nnz > 0) SPHC_LAUNCH(k_to_float<<<grid_for(L.T.nnz, 256), 256, 0, s>>>(L.T.v.p, L.T.nnz, B.tvf.p));
    if (L.Pn.nnz > 0) SPHC_LAUNCH(k_to_float<<<grid_for(L.Pn.nnz, 256), 256, 0, s>>>(L.Pn.v.p, L.Pn.nnz, B.pvf.p));
    if (Xc.n > 0) SPHC_LAUNCH(k_to_float<<<grid_for(Xc.n, 256), 256, 0, s>>>(Xc.p, Xc.n, B.Xcf.p));
    if (ne > 0)
        SPHC_LAUNCH(k_row_feat<<<grid_for(ne, 256), 256, 0, s>>>(ne, L.D.rp.p, L.D.ci.p, L.D.v.p, L.A.rp.p, L.A.ci.p,
                                                                L.A.v.p, L.P0.rp.p, L.T.rp.p, L.X.p, L.sig.p, B.rf.p));
    g = FeatArgs();
    g.ne = ne;
    g.nnzN = L.P0.nnz;
    g.lev = lev;
    g.trp = L.T.rp.p; g.tci = L.T.ci.p; g.tvf = B.tvf.p;
    g.nrp = L.P0.rp.p; g.nci = L.P0.ci.p;
    g.hrp = L.DH.rp.p; g.hci = L.DH.ci.p;
    g.prp = L.Pn.rp.p; g.pci = L.Pn.ci.p; g.pvf = B.pvf.p;
    g.Xcf = B.Xcf.p;
    g.rf = B.rf.p;
    SPHC_CK(cudaGetLastError());
    return SPHC_OK;
}

// Features of every pattern entry (i, j) of a level (SPHC_MLP_NFEAT floats each, see sphc.h).
// One thread per pattern entry; the row of an entry is found by binary search in the pattern's
// row pointers.  (The setup itself uses the fused feature + inference kernel of mlp.cu.)
__global__ void k_features(FeatArgs g, float* F) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= g.nnzN) return;
    int64_t lo = 0, hi = g.ne - 1;                 // row i: nrp[i] <= q < nrp[i+1]
    while (lo < hi) {
        int64_t mid = (lo + hi + 1) >> 1;
        if (g.nrp[mid] <= q) lo = mid; else hi = mid - 1;
    }
    float f[SPHC_MLP_NFEAT];
    entry_features(g, lo, q, f);
    float* out = F + q * SPHC_MLP_NFEAT;
    for (int c = 0; c < SPHC_MLP_NFEAT; ++c) out[c] = f[c];
}

// the fused tensor-core inference (features computed in the kernel) on every pattern entry
int level_prediction(const Level& L, const DBuf<double>& Xc, int lev, const float* params_dev, float* out,
                     cudaStream_t s) {
    FeatBufs B;
    FeatArgs g;
    SPHC_TRY(feat_prepare(L, Xc, lev, B, g, s));
    SPHC_TRY(mlp_predict_level(params_dev, g, out, s));
    SPHC_CK(cudaStreamSynchronize(s));          // B is released on return
    return SPHC_OK;
}
int level_features(const Level& L, const DBuf<double>& Xc, int lev, float* F, cudaStream_t s) {
    FeatBufs B;
    FeatArgs g;
    SPHC_TRY(feat_prepare(L, Xc, lev, B, g, s));
    if (g.nnzN > 0) SPHC_LAUNCH(k_features<<<grid_for(g.nnzN, 256), 256, 0, s>>>(g, F));
    SPHC_CK(cudaStreamSynchronize(s));          // B is released on return
    SPHC_CK(cudaGetLastError());
    return SPHC_OK;
}

// histogram of the local sub-problem sizes (|N_i|, |T_i|), clipped at 32: block-local counts
__global__ void k_ls_hist(const int64_t* nrp, const int64_t* trp, int64_t ne, unsigned long long* hist) {
    __shared__ unsigned int h[33 * 33];
    for (int q = threadIdx.x; q < 33 * 33; q += blockDim.x) h[q] = 0;
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ne; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t np = nrp[i + 1] - nrp[i], m = trp[i + 1] - trp[i];
        atomicAdd(&h[(np < 32 ? np : 32) * 33 + (m < 32 ? m : 32)], 1u);
    }
    __syncthreads();
    for (int q = threadIdx.x; q < 33 * 33; q += blockDim.x)
        if (h[q]) atomicAdd(&hist[q], (unsigned long long)h[q]);
}

// ------------------------------------------------------------------ dense coarsest factor
__global__ void k_dense_from_csr(const int64_t* rp, const int32_t* ci, const double* v, int64_t n, double* M) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int64_t c = 0; c < n; ++c) M[i * n + c] = 0.0;
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) M[i * n + ci[k]] = v[k];
}
// column j of the Cholesky factor (one block)
__global__ void k_chol_col(double* M, int n, int j, int* bad) {
    __shared__ double d;
    if (threadIdx.x == 0) {
        double a = M[(int64_t)j * n + j];
        if (!(a > 0.0)) { atomicExch(bad, 1); a = 1.0; }
        d = sqrt(a);
        M[(int64_t)j * n + j] = d;
    }
    __syncthreads();
    for (int r = j + 1 + threadIdx.x; r < n; r += blockDim.x) M[(int64_t)r * n + j] /= d;
}
// rank-1 update of the trailing lower triangle
__global__ void k_chol_update(double* M, int n, int j) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int rem = n - j - 1;
    if (q >= (int64_t)rem * rem) return;
    int r = j + 1 + (int)(q / rem), c = j + 1 + (int)(q % rem);
    if (c > r) return;
    M[(int64_t)r * n + c] -= M[(int64_t)r * n + j] * M[(int64_t)c * n + j];
}
// inverse column c: solve L L^T x = e_c (one block per column)
__global__ void k_chol_inverse(const double* L, int n, double* Ainv) {
    extern __shared__ double xs[];
    int c = blockIdx.x;
    for (int r = threadIdx.x; r < n; r += blockDim.x) xs[r] = (r == c) ? 1.0 : 0.0;
    __syncthreads();
    for (int j = 0; j < n; ++j) {          // forward: L y = e_c
        if (threadIdx.x == 0) xs[j] /= L[(int64_t)j * n + j];
        __syncthreads();
        double yj = xs[j];
        for (int r = j + 1 + threadIdx.x; r < n; r += blockDim.x) xs[r] -= L[(int64_t)r * n + j] * yj;
        __syncthreads();
    }
    for (int j = n - 1; j >= 0; --j) {     // backward: L^T x = y
        if (threadIdx.x == 0) xs[j] /= L[(int64_t)j * n + j];
        __syncthreads();
        double xj = xs[j];
        for (int r = threadIdx.x; r < j; r += blockDim.x) xs[r] -= L[(int64_t)j * n + r] * xj;
        __syncthreads();
    }
    for (int r = threadIdx.x; r < n; r += blockDim.x) Ainv[(int64_t)r * n + c] = xs[r];
}

__global__ void k_shift_diag(double* M, int64_t n, double rel) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) M[i * n + i] *= (1.0 + rel);
}

// Dense FP64 inverse of a small SPD operator.  With allow_shift, a singular operator (the
// nodal operator of a natural-boundary problem, whose constants are in its null space) is
// factored after scaling its diagonal by 1 + 1e-10.
int coarse_inverse(const DCSR& A, DBuf<double>& Ainv, bool allow_shift, cudaStream_t s) {
    int64_t n = A.nr;
    if (n > 8192) { set_error("coarsest level of %lld rows is too large for the dense solve", (long long)n); return SPHC_ELIMIT; }
    SPHC_TRY(Ainv.alloc(n * n, s));
    if (n == 0) return SPHC_OK;
    DBuf<double> M;
    SPHC_TRY(M.alloc(n * n, s));
    DBuf<int> bad;
    SPHC_TRY(bad.alloc(1, s));
    for (int attempt = 0; attempt < 2; ++attempt) {
        SPHC_TRY(bad.zero(s));
        SPHC_LAUNCH(k_dense_from_csr<<<grid_for(n, 128), 128, 0, s>>>(A.rp.p, A.ci.p, A.v.p, n, M.p));
        if (attempt == 1) SPHC_LAUNCH(k_shift_diag<<<grid_for(n, 128), 128, 0, s>>>(M.p, n, 1e-10));
        for (int j = 0; j < n; ++j) {
            SPHC_LAUNCH(k_chol_col<<<1, 256, 0, s>>>(M.p, (int)n, j, bad.p));
            int64_t rem = n - j - 1;
            if (rem > 0) SPHC_LAUNCH(k_chol_update<<<grid_for(rem * rem, 256), 256, 0, s>>>(M.p, (int)n, j));
        }
        int hb = 0;
        SPHC_CK(cudaMemcpyAsync(&hb, bad.p, sizeof(int), cudaMemcpyDeviceToHost, s));
        SPHC_CK(cudaStreamSynchronize(s));
        if (!hb) break;
        if (!allow_shift || attempt == 1) {
            set_error("coarsest operator is not numerically positive definite");
            return SPHC_ENUMERIC;
        }
    }
    size_t sm = sizeof(double) * n;
    if (sm > 48 * 1024) SPHC_CK(cudaFuncSetAttribute(k_chol_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    SPHC_LAUNCH(k_chol_inverse<<<(unsigned)n, 256, sm, s>>>(M.p, (int)n, Ainv.p));
    SPHC_CK(cudaGetLastError());
    return SPHC_OK;
}

// ------------------------------------------------------------------ one level of Alg. 3
// coordinates of the next level's nodes: centroids of the aggregates
static int coarse_coords(const Level& L, DBuf<double>& Xc, cudaStream_t s) {
    int64_t nv = L.An.nr, nagg = L.nagg;
    if (!L.X.p) return SPHC_OK;
    DBuf<int32_t> cnt, members;
    DBuf<int64_t> mptr;
    DBuf<unsigned long long> cur;
    SPHC_TRY(cnt.alloc(nagg + 1, s));
    SPHC_TRY(cnt.zero(s));
    SPHC_TRY(mptr.alloc(nagg + 1, s));
    SPHC_TRY(members.alloc(nv, s));
    SPHC_TRY(cur.alloc(nagg + 1, s));
    if (nv > 0) SPHC_LAUNCH(k_count_agg<<<grid_for(nv, 256), 256, 0, s>>>(L.agg.p, nv, cnt.p));
    SPHC_TRY(scan_i32_to_i64(cnt.p, mptr.p, nagg, s, nullptr));
    SPHC_LAUNCH(k_i64_to_u64b<<<grid_for(nagg + 1, 256), 256, 0, s>>>(mptr.p, cur.p, nagg + 1));
    if (nv > 0) SPHC_LAUNCH(k_scatter_agg<<<grid_for(nv, 256), 256, 0, s>>>(L.agg.p, nv, cur.p, members.p));
    int64_t mx = 0;
    SPHC_TRY(max_row_length(mptr.p, nagg, s, &mx));
    SPHC_TRY(segmented_sort(mptr.p, nagg, members.p, nullptr, mx, s));
    SPHC_TRY(Xc.alloc(nagg * 3, s));
    if (nagg > 0) SPHC_LAUNCH(k_centroids<<<grid_for(nagg, 256), 256, 0, s>>>(mptr.p, members.p, nagg, L.X.p, Xc.p));
    SPHC_CK(cudaGetLastError());
    return SPHC_OK;
}

// section name with the level index, e.g. "setup_P0_l1"
static std::string lev_name(const char* what, int lev) { return std::string(what) + "_l" + std::to_string(lev); }

// ------------------------------------------------------------------ strength of connection (theta > 0)
// Symmetric smoothed-aggregation criterion: an off-diagonal a_ij is strong when
// |a_ij| >= theta sqrt(a_ii a_jj).  The filtered matrix keeps the diagonal and the strong entries
// (columns stay sorted); every dropped entry is added to the diagonal in column order, so row
// sums (and with them the constants in the null space) are unchanged.
__global__ void k_strength_count(const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                 const double* __restrict__ v, const double* __restrict__ d, int64_t n, double theta,
                                 int64_t* __restrict__ cnt) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t c = 0;
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
        const int32_t j = ci[k];
        if (j == (int32_t)i || fabs(v[k]) >= theta * sqrt(d[i] * d[j])) ++c;
    }
    cnt[i] = c;
}
__global__ void k_strength_fill(const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                const double* __restrict__ v, const double* __restrict__ d, int64_t n, double theta,
                                const int64_t* __restrict__ frp, int32_t* __restrict__ fci, double* __restrict__ fv) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double diag = d[i];
    int64_t q = frp[i], qd = -1;
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
        const int32_t j = ci[k];
        if (j == (int32_t)i) {
            qd = q;
            fci[q] = j;
            fv[q++] = 0.0;
        } else if (fabs(v[k]) >= theta * sqrt(d[i] * d[j])) {
            fci[q] = j;
            fv[q++] = v[k];
        } else {
            diag += v[k];
        }
    }
    if (qd >= 0) fv[qd] = diag;
}
static int strength_filter(const DCSR& A, const double* d, double theta, DCSR& F, cudaStream_t s) {
    const int64_t n = A.nr;
    DBuf<int64_t> cnt;
    SPHC_TRY(cnt.alloc(n + 1, s));
    if (n > 0) SPHC_LAUNCH(k_strength_count<<<grid_for(n, 256), 256, 0, s>>>(A.rp.p, A.ci.p, A.v.p, d, n, theta, cnt.p));
    int64_t nnz = 0;
    SPHC_TRY(F.alloc(n, A.nc, 0, s));
    SPHC_TRY(exclusive_scan_i64(cnt.p, F.rp.p, n, s, &nnz));
    F.nnz = nnz;
    SPHC_TRY(F.ci.alloc(nnz, s));
    SPHC_TRY(F.v.alloc(nnz, s));
    if (n > 0)
        SPHC_LAUNCH(k_strength_fill<<<grid_for(n, 256), 256, 0, s>>>(A.rp.p, A.ci.p, A.v.p, d, n, theta, F.rp.p, F.ci.p,
                                                                    F.v.p));
    SPHC_CK(cudaGetLastError());
    return SPHC_OK;
}

// ------------------------------------------------------------------ Alg. 1 (Gen_Piecewise_Const)
// Each row of the smoothed P_n (m_h x m_H) is assigned to one column for the construction of D_H
// (Sec. 4.1).  The paper sweeps the columns one after another; here, as in the oracle, the
// columns of a pass choose simultaneously: column j proposes its ceil(target_j / passes) rows of
// largest |P_rj| that are unassigned when the pass starts (ties: lower row), target_j =
// ceil(nnz(P_:j) m_h / nnz(P)); a row proposed by several columns goes to the largest |P_rj|
// (ties: lower column).  Remaining rows go to their column of largest |P_rj| (ties: lower
// column); a column left empty takes back its largest row where that row's column keeps another
// (in column order).
__global__ void k_alg1_nass(const int64_t* __restrict__ tp, int64_t nc, int64_t m, int64_t nnz, int passes,
                            int32_t* __restrict__ nass) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nc) return;
    const int64_t cnt = tp[j + 1] - tp[j];
    const int64_t target = nnz > 0 ? (cnt * m + nnz - 1) / nnz : 0;
    nass[j] = (int32_t)((target + passes - 1) / passes);
}
// warp per column: mark its proposals and raise best[r] to the proposal's |P_rj| (as ordered bits)
__global__ void k_alg1_propose(const int64_t* __restrict__ tp, const int32_t* __restrict__ tr,
                               const double* __restrict__ tv, int64_t nc, const int32_t* __restrict__ nass,
                               const int32_t* __restrict__ assign, int8_t* __restrict__ prop,
                               unsigned long long* __restrict__ best) {
    const int lane = threadIdx.x & 31;
    const int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (j >= nc) return;
    const int64_t k0 = tp[j], k1 = tp[j + 1];
    for (int64_t k = k0 + lane; k < k1; k += 32) prop[k] = 0;
    __syncwarp();
    for (int t = 0; t < nass[j]; ++t) {
        double ba = -1.0;
        int32_t br = 0x7fffffff;
        int64_t bk = -1;
        for (int64_t k = k0 + lane; k < k1; k += 32) {
            const int32_t r = tr[k];
            if (prop[k] || assign[r] >= 0) continue;
            const double a = fabs(tv[k]);
            if (a > ba || (a == ba && r < br)) { ba = a; br = r; bk = k; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double oa = __shfl_xor_sync(0xffffffffu, ba, o);
            const int32_t orr = __shfl_xor_sync(0xffffffffu, br, o);
            const int64_t ok = __shfl_xor_sync(0xffffffffu, bk, o);
            if (oa > ba || (oa == ba && orr < br)) { ba = oa; br = orr; bk = ok; }
        }
        if (bk < 0) break;                          // no assignable row left in this column
        if (lane == 0) {
            prop[bk] = 1;
            atomicMax(&best[br], (unsigned long long)__double_as_longlong(ba));
        }
        __syncwarp();
    }
}
// proposals that reach best[r]: the lowest such column wins row r
__global__ void k_alg1_resolve(const int64_t* __restrict__ tp, const int32_t* __restrict__ tr,
                               const double* __restrict__ tv, int64_t nc, const int8_t* __restrict__ prop,
                               const unsigned long long* __restrict__ best, int32_t* __restrict__ bcol) {
    const int lane = threadIdx.x & 31;
    const int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (j >= nc) return;
    for (int64_t k = tp[j] + lane; k < tp[j + 1]; k += 32)
        if (prop[k] && (unsigned long long)__double_as_longlong(fabs(tv[k])) == best[tr[k]])
            atomicMin(&bcol[tr[k]], (int32_t)j);
}
constexpr int32_t ALG1_NONE = 0x7f7f7f7f;     // bcol before any proposal (a memset of 0x7f bytes)
__global__ void k_alg1_commit(int64_t m, int32_t* __restrict__ assign, const int32_t* __restrict__ bcol) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r < m && bcol[r] != ALG1_NONE) assign[r] = bcol[r];
}
__global__ void k_alg1_greedy(const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                              const double* __restrict__ v, int64_t m, int32_t* __restrict__ assign,
                              int32_t* __restrict__ count) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= m) return;
    if (assign[r] < 0) {
        double ba = -1.0;
        int32_t bj = -1;
        for (int64_t k = rp[r]; k < rp[r + 1]; ++k) {
            const double a = fabs(v[k]);
            if (a > ba || (a == ba && ci[k] < bj)) { ba = a; bj = ci[k]; }
        }
        assign[r] = bj;
    }
    if (assign[r] >= 0) atomicAdd(&count[assign[r]], 1);
}
__global__ void k_alg1_empty(const int64_t* __restrict__ tp, int64_t nc, const int32_t* __restrict__ count,
                             int64_t* __restrict__ flag) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < nc) flag[j] = (count[j] == 0 && tp[j + 1] > tp[j]) ? 1 : 0;
}
// one thread, in column order over the (normally empty) list of empty columns
__global__ void k_alg1_safeguard(const int64_t* __restrict__ tp, const int32_t* __restrict__ tr,
                                 const double* __restrict__ tv, const int64_t* __restrict__ flag,
                                 const int64_t* __restrict__ pos, int64_t nc, int32_t* __restrict__ assign,
                                 int32_t* __restrict__ count) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    for (int64_t j = 0; j < nc; ++j) {
        if (!flag[j] || count[j] > 0) continue;
        double ba = -1.0;
        int32_t br = -1;
        for (int64_t k = tp[j]; k < tp[j + 1]; ++k) {
            const double a = fabs(tv[k]);
            if (a > ba || (a == ba && tr[k] < br)) { ba = a; br = tr[k]; }
        }
        if (br >= 0 && assign[br] >= 0 && count[assign[br]] >= 2) {
            count[assign[br]]--;
            assign[br] = (int32_t)j;
            count[j]++;
        }
    }
    (void)pos;
}
static int gen_piecewise_const(const DCSR& Pn, int passes, DBuf<int32_t>& assign, cudaStream_t s) {
    const int64_t m = Pn.nr, nc = Pn.nc, nnz = Pn.nnz;
    DCSR Pt;
    SPHC_TRY(transpose(Pn, Pt, s));
    DBuf<int32_t> nass, bcol, count;
    DBuf<int8_t> prop;
    DBuf<unsigned long long> best;
    DBuf<int64_t> flag;
    SPHC_TRY(assign.alloc(m > 0 ? m : 1, s));
    SPHC_TRY(nass.alloc(nc > 0 ? nc : 1, s));
    SPHC_TRY(bcol.alloc(m > 0 ? m : 1, s));
    SPHC_TRY(count.alloc(nc > 0 ? nc : 1, s));
    SPHC_TRY(prop.alloc(nnz > 0 ? nnz : 1, s));
    SPHC_TRY(best.alloc(m > 0 ? m : 1, s));
    SPHC_TRY(flag.alloc(nc > 0 ? nc : 1, s));
    SPHC_CK(cudaMemsetAsync(assign.p, 0xff, sizeof(int32_t) * (m > 0 ? m : 1), s));     // -1
    if (nc > 0) SPHC_LAUNCH(k_alg1_nass<<<grid_for(nc, 256), 256, 0, s>>>(Pt.rp.p, nc, m, nnz, passes, nass.p));
    for (int pass = 0; pass < passes; ++pass) {
        SPHC_TRY(best.zero(s));
        SPHC_CK(cudaMemsetAsync(bcol.p, 0x7f, sizeof(int32_t) * (m > 0 ? m : 1), s));   // ALG1_NONE
        if (nc > 0) {
            SPHC_LAUNCH(k_alg1_propose<<<grid_for(nc * 32, 256), 256, 0, s>>>(Pt.rp.p, Pt.ci.p, Pt.v.p, nc, nass.p,
                                                                             assign.p, prop.p, best.p));
            SPHC_LAUNCH(k_alg1_resolve<<<grid_for(nc * 32, 256), 256, 0, s>>>(Pt.rp.p, Pt.ci.p, Pt.v.p, nc, prop.p,
                                                                             best.p, bcol.p));
        }
        if (m > 0) SPHC_LAUNCH(k_alg1_commit<<<grid_for(m, 256), 256, 0, s>>>(m, assign.p, bcol.p));
    }
    SPHC_TRY(count.zero(s));
    if (m > 0) SPHC_LAUNCH(k_alg1_greedy<<<grid_for(m, 256), 256, 0, s>>>(Pn.rp.p, Pn.ci.p, Pn.v.p, m, assign.p,
                                                                        count.p));
    if (nc > 0) {
        SPHC_LAUNCH(k_alg1_empty<<<grid_for(nc, 256), 256, 0, s>>>(Pt.rp.p, nc, count.p, flag.p));
        SPHC_LAUNCH(k_alg1_safeguard<<<1, 32, 0, s>>>(Pt.rp.p, Pt.ci.p, Pt.v.p, flag.p, nullptr, nc, assign.p,
                                                      count.p));
    }
    SPHC_CK(cudaGetLastError());
    return SPHC_OK;
}

int build_level(Level& L, int lev, const sphc_opts& o, DCSR& Anext, DCSR& Dnext, DCSR& Annext, DBuf<double>& Xnext,
                const float* mlp_params, Profiler* prof, cudaStream_t s, bool reuse) {
    uint64_t seed = o.seed + 1000ULL * (uint64_t)lev;
    int64_t nv = L.An.nr, ne = L.A.nr;
    // With reuse (a related system: new values of A on the same pattern, paper Sec. 3 warm-start
    // remark) the structural steps are kept: the aggregates, D_H and the pattern N depend only on
    // the patterns of A and D; P_n, T, P0 and everything after are recomputed, P0 starting from
    // the previous P_e projected onto the new constraints.
    DBuf<double> warm;
    if (reuse) warm = std::move(L.Pe.v);
    // drop tolerance theta > 0: aggregation and smoothing on the filtered nodal matrix
    DBuf<double> dn;
    SPHC_TRY(dn.alloc(nv, s));
    SPHC_TRY(csr_diag(L.An, dn.p, s));
    DCSR Af;
    if (o.sa_theta > 0.0) {
        SPHC_TRY(strength_filter(L.An, dn.p, o.sa_theta, Af, s));
        SPHC_TRY(csr_diag(Af, dn.p, s));
    }
    const DCSR& Ag = o.sa_theta > 0.0 ? Af : L.An;
    // aggregation on the nodal graph (drop tolerance 0: every structural entry is strong)
    if (!reuse) {
        Section sec(prof, lev_name("setup_aggregate", lev).c_str(), s);
        SPHC_TRY(aggregate(Ag, seed + 1, L.agg, &L.nagg, s));
    }
    Section* sec_pn = new Section(prof, lev_name("setup_Pn", lev).c_str(), s);
    // smoothed nodal prolongator
    SPHC_TRY(power_rho(Ag, dn.p, seed + 4, o.power_iters, &L.rho, s));
    L.omega_sa = 4.0 / (3.0 * L.rho);
    DCSR Pb;
    SPHC_TRY(Pb.alloc(nv, L.nagg, nv, s));
    SPHC_LAUNCH(k_pbar<<<grid_for(nv + 1, 256), 256, 0, s>>>(nv, L.agg.p, Pb.rp.p, Pb.ci.p, Pb.v.p));
    SPHC_TRY(spgemm(Ag, Pb, L.Pn, s));
    DBuf<int> fl;
    SPHC_TRY(fl.alloc(2, s));
    SPHC_TRY(fl.zero(s));
    if (nv > 0)
        SPHC_LAUNCH(k_pn_finish<<<grid_for(nv, 256), 256, 0, s>>>(L.Pn.rp.p, L.Pn.ci.p, L.Pn.v.p, nv, L.agg.p, dn.p, L.omega_sa, 1,
                                                     fl.p, fl.p + 1));
    int hf[2];
    SPHC_CK(cudaMemcpyAsync(hf, fl.p, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
    SPHC_CK(cudaStreamSynchronize(s));
    if (hf[1]) { set_error("non-finite nodal prolongator row sum on level %d", lev); return SPHC_ENUMERIC; }
    L.n_rows_unsmoothed = hf[0];
    delete sec_pn;
    // coarse gradient from the tentative aggregates, or from Alg. 1 applied to the smoothed P_n
    if (!reuse) {
        Section sec(prof, lev_name("setup_DH", lev).c_str(), s);
        if (o.pn_alg1) {
            DBuf<int32_t> pc;
            SPHC_TRY(gen_piecewise_const(L.Pn, o.alg1_passes, pc, s));
            SPHC_TRY(coarse_gradient(L.D, L.Dt, pc.p, L.nagg, L.DH, s));
            SPHC_CK(cudaStreamSynchronize(s));
        } else {
            SPHC_TRY(coarse_gradient(L.D, L.Dt, L.agg.p, L.nagg, L.DH, s));
        }
    }
    Section* sec_pat = new Section(prof, lev_name("setup_pattern", lev).c_str(), s);
    // T = D P_n (values r), N (Alg. 2), made irreducible
    SPHC_TRY(dmul(L.D, L.Pn, L.T, s));
    DCSR DHt, Mt;
    DBuf<int64_t> ncnt;
    DBuf<int> st, pctl;
    DBuf<int32_t> pbig, pbad;
    DBuf<uint64_t> pairs;
    DBuf<int2> E2;
    SPHC_TRY(ncnt.alloc(ne + 1, s));
    SPHC_TRY(st.alloc(8, s));
    SPHC_TRY(pbig.alloc(ne > 0 ? ne : 1, s));
    SPHC_TRY(pbad.alloc(ne > 0 ? ne : 1, s));
    SPHC_TRY(pctl.alloc(2, s));
    int hs[8] = {0};
    int npbig = 0;
    if (!reuse) L.n_added = 0;
    for (int pass = 0; !reuse; ++pass) {
        // counts of N_i and disconnected rows against the current D_H; rows with more than
        // PT_K coarse nodes go to the warp-per-row kernel through a list (st[6] counts them)
        SPHC_TRY(transpose(L.DH, DHt, s));
        SPHC_TRY(E2.alloc(L.DH.nr > 0 ? L.DH.nr : 1, s));
        if (L.DH.nr > 0) SPHC_LAUNCH(k_edge_pairs<<<grid_for(L.DH.nr, 256), 256, 0, s>>>(L.DH.rp.p, L.DH.ci.p, L.DH.nr, E2.p));
        SPHC_TRY(st.zero(s));
        if (ne > 0)
            SPHC_LAUNCH(k_pattern_rows<<<grid_for(ne, 128), 128, 0, s>>>(L.T.rp.p, L.T.ci.p, ne, DHt.rp.p, DHt.ci.p,
                                                                       E2.p, 0, ncnt.p, nullptr, nullptr, st.p,
                                                                       pbig.p, st.p + 6, pbad.p));
        SPHC_CK(cudaMemcpyAsync(hs, st.p, 8 * sizeof(int), cudaMemcpyDeviceToHost, s));
        SPHC_CK(cudaStreamSynchronize(s));
        npbig = hs[6];
        if (npbig > 0) {
            SPHC_LAUNCH(k_pattern<<<grid_for(npbig, PAT_WARPS), PAT_WARPS * 32, 0, s>>>(
                L.T.rp.p, L.T.ci.p, npbig, pbig.p, DHt.rp.p, DHt.ci.p, L.DH.rp.p, L.DH.ci.p, 0, ncnt.p, nullptr,
                nullptr, st.p, pbad.p));
            SPHC_CK(cudaMemcpyAsync(hs, st.p, 8 * sizeof(int), cudaMemcpyDeviceToHost, s));
            SPHC_CK(cudaStreamSynchronize(s));
        }
        if (hs[0]) { set_error("level %d: a row of T exceeds %d coarse nodes", lev, MAX_T); return SPHC_ELIMIT; }
        if (hs[1]) { set_error("level %d: a row of the pattern exceeds %d coarse edges", lev, MAX_NP); return SPHC_ELIMIT; }
        int nbad = hs[2];
        if (nbad == 0 || pass == 8) break;
        // make_irreducible: new coarse edges joining the components of the disconnected rows
        if (Mt.nr == 0) SPHC_TRY(transpose(L.T, Mt, s));
        SPHC_TRY(pairs.alloc(IRR_CAP, s));
        SPHC_TRY(pctl.zero(s));
        SPHC_LAUNCH(k_irreducible<<<grid_for(nbad, IRR_WARPS), IRR_WARPS * 32, 0, s>>>(
            pbad.p, nbad, L.T.rp.p, L.T.ci.p, DHt.rp.p, DHt.ci.p, L.DH.rp.p, L.DH.ci.p, Mt.rp.p, Mt.ci.p, Mt.v.p,
            pairs.p, pctl.p, pctl.p + 1));
        int hp[2];
        SPHC_CK(cudaMemcpyAsync(hp, pctl.p, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
        SPHC_CK(cudaStreamSynchronize(s));
        if (hp[1]) {
            set_error("level %d: make_irreducible would add more than %d coarse edges in one pass", lev, IRR_CAP);
            return SPHC_ELIMIT;
        }
        if (hp[0] == 0) break;
        int64_t n2 = L.DH.nnz - L.DH.nr;                 // two-node rows come first
        SPHC_LAUNCH(k_pairs_unique<<<1, 1024, 0, s>>>(pairs.p, hp[0], L.DH.rp.p, L.DH.ci.p, n2, pctl.p));
        int nu = 0;
        SPHC_CK(cudaMemcpyAsync(&nu, pctl.p, sizeof(int), cudaMemcpyDeviceToHost, s));
        SPHC_CK(cudaStreamSynchronize(s));
        if (nu == 0) break;
        DCSR H2;
        SPHC_TRY(H2.alloc(L.DH.nr + nu, L.DH.nc, L.DH.nnz + 2 * (int64_t)nu, s));
        SPHC_LAUNCH(k_dh_merge<<<grid_for(L.DH.nr + nu + 1, 256), 256, 0, s>>>(L.DH.rp.p, L.DH.ci.p, L.DH.v.p, L.DH.nr,
                                                                              n2, pairs.p, nu, H2.rp.p, H2.ci.p,
                                                                              H2.v.p));
        L.DH = std::move(H2);
        L.n_added += nu;
    }
    SPHC_TRY(max_row_length(L.T.rp.p, ne, s, &L.max_m));
    int64_t nnzN = reuse ? L.P0.nnz : 0;
    if (!reuse) {
    SPHC_TRY(L.P0.alloc(ne, L.DH.nr, 0, s));
    SPHC_TRY(exclusive_scan_i64(ncnt.p, L.P0.rp.p, ne, s, &nnzN));
    L.P0.nnz = nnzN;
    SPHC_TRY(L.P0.ci.alloc(nnzN, s));
    SPHC_TRY(L.P0.v.alloc(nnzN, s));
    SPHC_TRY(max_row_length(L.P0.rp.p, ne, s, &L.max_np));
    if (ne > 0)
        SPHC_LAUNCH(k_pattern_rows<<<grid_for(ne, 128), 128, 0, s>>>(L.T.rp.p, L.T.ci.p, ne, DHt.rp.p, DHt.ci.p, E2.p,
                                                                   1, nullptr, L.P0.rp.p, L.P0.ci.p, st.p, nullptr,
                                                                   nullptr, nullptr));
    if (npbig > 0)
        SPHC_LAUNCH(k_pattern<<<grid_for(npbig, PAT_WARPS), PAT_WARPS * 32, 0, s>>>(L.T.rp.p, L.T.ci.p, npbig, pbig.p,
                                                                      DHt.rp.p, DHt.ci.p, L.DH.rp.p, L.DH.ci.p, 1,
                                                                      nullptr, L.P0.rp.p, L.P0.ci.p, st.p, nullptr));
    }
    delete sec_pat;
    // learned warm start: the MLP correction of every pattern entry (its features do not depend
    // on P0), passed to the P0 kernel, which projects it onto the row constraints
    if (!reuse) {
        Section sec(prof, lev_name("setup_coords", lev).c_str(), s);
        SPHC_TRY(coarse_coords(L, Xnext, s));
    }
    int emin_iters = o.emin_iters;
    DBuf<float> corr;
    if (o.learned && !reuse) {
        Section sec(prof, lev_name("setup_learned", lev).c_str(), s);
        if (!mlp_params) { set_error("learned warm start without MLP parameters"); return SPHC_EINVAL; }
        if (!L.X.p || !Xnext.p) {
            set_error("the learned warm start needs node coordinates (pass coords to sphc_setup)");
            return SPHC_EINVAL;
        }
        SPHC_TRY(corr.alloc(nnzN, s));
        FeatBufs fb;
        FeatArgs fg;
        SPHC_TRY(feat_prepare(L, Xnext, lev, fb, fg, s));
        SPHC_TRY(mlp_predict_level(mlp_params, fg, corr.p, s, o.mlp_wait_polls));
        emin_iters = o.learned_emin_iters;
    }
    Section* sec_p0 = new Section(prof, lev_name("setup_P0", lev).c_str(), s);
    // initial guess and energy minimisation
    SPHC_TRY(L.hist.alloc(33 * 33, s));
    SPHC_TRY(L.hist.zero(s));
    if (ne > 0) SPHC_LAUNCH(k_ls_hist<<<1024, 256, 0, s>>>(L.P0.rp.p, L.T.rp.p, ne, L.hist.p));
    SPHC_TRY(st.zero(s));
    size_t sm = sizeof(LocalSys) * LOC_WARPS;
    SPHC_CK(cudaFuncSetAttribute(k_p0<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    SPHC_CK(cudaFuncSetAttribute(k_p0<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    SPHC_CK(cudaFuncSetAttribute(k_emin, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    // rows too large for the thread-per-row kernels (listed by k_p0_rows, reused by every step)
    DBuf<int32_t> big;
    DBuf<int> nbig;
    SPHC_TRY(big.alloc(ne > 0 ? ne : 1, s));
    SPHC_TRY(nbig.alloc(1, s));
    SPHC_TRY(nbig.zero(s));
    int hbig = 0;
    // factored local systems, kept for the energy-minimisation steps
    DBuf<uint32_t> cpm;
    DBuf<int8_t> ck;
    DBuf<double> cL;
    SPHC_TRY(cpm.alloc(2 * TK * (ne > 0 ? ne : 1), s));
    SPHC_TRY(ck.alloc(ne > 0 ? ne : 1, s));
    SPHC_TRY(cL.alloc(TL * (ne > 0 ? ne : 1), s));
    RowCache cache{cpm.p, ck.p, cL.p, ne};
    DBuf<int2> ecodes;
    SPHC_TRY(ecodes.alloc(L.DH.nr > 0 ? L.DH.nr : 1, s));
    if (L.DH.nr > 0)
        SPHC_LAUNCH(k_edge_codes<<<grid_for(L.DH.nr, 256), 256, 0, s>>>(L.DH.rp.p, L.DH.ci.p, L.DH.v.p, L.DH.nr, ecodes.p));
    if (ne > 0) {
        // P0: the point of each row's constraint set nearest to the warm start (0: least-norm; the
        // MLP correction; or, with reuse, the previous P_e)
        if (reuse)
            SPHC_LAUNCH(k_p0_rows<double><<<grid_for(ne, 128), 128, 0, s>>>(
                ne, L.T.rp.p, L.T.ci.p, L.T.v.p, L.P0.rp.p, L.P0.ci.p, ecodes.p, warm.p, L.P0.v.p, st.p, big.p,
                nbig.p, cache));
        else
            SPHC_LAUNCH(k_p0_rows<float><<<grid_for(ne, 128), 128, 0, s>>>(
                ne, L.T.rp.p, L.T.ci.p, L.T.v.p, L.P0.rp.p, L.P0.ci.p, ecodes.p, corr.p, L.P0.v.p, st.p, big.p,
                nbig.p, cache));
        SPHC_CK(cudaMemcpyAsync(&hbig, nbig.p, sizeof(int), cudaMemcpyDeviceToHost, s));
        SPHC_CK(cudaStreamSynchronize(s));
        if (hbig > 0) {
            if (reuse)
                SPHC_LAUNCH(k_p0<double><<<grid_for(hbig, LOC_WARPS), LOC_WARPS * 32, sm, s>>>(
                    hbig, big.p, L.T.rp.p, L.T.ci.p, L.T.v.p, L.P0.rp.p, L.P0.ci.p, L.DH.rp.p, L.DH.ci.p, L.DH.v.p,
                    warm.p, L.P0.v.p, st.p));
            else
                SPHC_LAUNCH(k_p0<float><<<grid_for(hbig, LOC_WARPS), LOC_WARPS * 32, sm, s>>>(
                    hbig, big.p, L.T.rp.p, L.T.ci.p, L.T.v.p, L.P0.rp.p, L.P0.ci.p, L.DH.rp.p, L.DH.ci.p, L.DH.v.p,
                    corr.p, L.P0.v.p, st.p));
        }
    }
    warm = DBuf<double>();
    delete sec_p0;
    corr = DBuf<float>();
    Section* sec_cp = new Section(prof, lev_name("setup_copy_P0", lev).c_str(), s);
    SPHC_TRY(csr_copy(L.P0, L.Pe, s));
    DBuf<double> Pnew;
    SPHC_TRY(Pnew.alloc(nnzN, s));
    delete sec_cp;
    // algorithmic bytes of one step: A (values in the product's precision, columns, row pointers)
    // once; P's pattern (row pointers, columns, values) once, however often its rows are gathered;
    // w written and read; per row the stored factor (masks, k, lower triangle); P read and P'
    // written by the update
    const size_t wsz = o.emin_fp32 ? sizeof(float) : sizeof(double);
    double emin_bytes = (double)L.A.nnz * (4.0 + (double)wsz) + (double)(ne + 1) * 8.0 * 2 + (double)nnzN * (4 + 8) +
                        (double)nnzN * 2.0 * (double)wsz + (double)ne * (2 * TK * 4 + 1 + TL * 8) +
                        (double)nnzN * 16.0;
    int tid = prof ? prof->find(lev_name("emin_level", lev).c_str(), emin_bytes) : -1;
    DBuf<double> W;
    DBuf<float> W32;
    if (emin_iters > 0) {
        if (o.emin_fp32) SPHC_TRY(W32.alloc(nnzN, s));
        else SPHC_TRY(W.alloc(nnzN, s));
    }
    // projected gradient g = Pi D^-1 (A V)|_N of values V on the pattern (small rows by the product
    // and thread-per-row projection kernels, large rows by k_emin)
    DBuf<float> P32;                            // FP32 copy of the values the product reads
    DBuf<float> A32, Dinv32;                    // FP32 copies of A's values and of 1 / a_ii
    DBuf<double> Dinv;
    if (emin_iters > 0 && ne > 0) {
        SPHC_TRY(Dinv.alloc(ne, s));
        if (o.emin_fp32) {
            SPHC_TRY(P32.alloc(nnzN, s));
            SPHC_TRY(A32.alloc(L.A.nnz, s));
            SPHC_TRY(Dinv32.alloc(ne, s));
            if (L.A.nnz > 0) SPHC_LAUNCH(k_to_float<<<grid_for(L.A.nnz, 256), 256, 0, s>>>(L.A.v.p, L.A.nnz, A32.p));
        }
        SPHC_LAUNCH(k_diag_inv<<<grid_for(ne, 256), 256, 0, s>>>(ne, L.A.rp.p, L.A.ci.p, L.A.v.p, Dinv.p,
                                                                  o.emin_fp32 ? Dinv32.p : nullptr));
    }
    auto to_f32 = [&](const double* V) {
        if (nnzN > 0) SPHC_LAUNCH(k_to_float<<<grid_for(nnzN, 256), 256, 0, s>>>(V, nnzN, P32.p));
    };
    auto proj_grad = [&](const double* V, double* g) -> int {
        const int gpp = grid_for(ne, PP_WARPS);
        if (o.emin_fp32) {
            to_f32(V);
            SPHC_LAUNCH(k_emin_pp<float><<<gpp, PP_WARPS * 32, 0, s>>>(ne, L.A.rp.p, L.A.ci.p, A32.p, Dinv32.p, L.Pe.rp.p,
                                                                      L.Pe.ci.p, P32.p, cache.k, W32.p));
            SPHC_LAUNCH(k_emin_rows<float><<<grid_for(ne, 128), 128, 0, s>>>(ne, L.Pe.rp.p, W32.p, V, g, 0.0, cache, 1));
        } else {
            SPHC_LAUNCH(k_emin_pp<double><<<gpp, PP_WARPS * 32, 0, s>>>(ne, L.A.rp.p, L.A.ci.p, L.A.v.p, Dinv.p, L.Pe.rp.p,
                                                                       L.Pe.ci.p, V, cache.k, W.p));
            SPHC_LAUNCH(k_emin_rows<double><<<grid_for(ne, 128), 128, 0, s>>>(ne, L.Pe.rp.p, W.p, V, g, 0.0, cache, 1));
        }
        if (hbig > 0)
            SPHC_LAUNCH(k_emin<<<grid_for(hbig, LOC_WARPS), LOC_WARPS * 32, sm, s>>>(
                hbig, big.p, L.A.rp.p, L.A.ci.p, L.A.v.p, L.T.rp.p, L.T.ci.p, L.T.v.p, L.Pe.rp.p, L.Pe.ci.p,
                L.DH.rp.p, L.DH.ci.p, L.DH.v.p, V, g, 0.0, st.p, 1));
        SPHC_CK(cudaGetLastError());
        return SPHC_OK;
    };
    if (o.emin_method == 1 && emin_iters > 0 && ne > 0) {
        // projected CG on eq. (8) from the feasible P0: z = -Pi D^-1 A P, p = z, and per step
        // w = Pi D^-1 A p, alpha = (z, z)_D / (p, w)_D, P += alpha p, z -= alpha w, beta, p = z + beta p,
        // with (x, y)_D = sum_i a_ii x_i . y_i (the preconditioner D^-1 commutes with Pi)
        if (tid >= 0) prof->begin(tid, s);
        DBuf<double> dg, Z, Pd, Gv, part, sc;
        SPHC_TRY(dg.alloc(ne, s));
        SPHC_TRY(csr_diag(L.A, dg.p, s));
        SPHC_TRY(Z.alloc(nnzN, s));
        SPHC_TRY(Pd.alloc(nnzN, s));
        SPHC_TRY(Gv.alloc(nnzN, s));
        constexpr int WD_BLOCKS = 512;
        SPHC_TRY(part.alloc(WD_BLOCKS, s));
        SPHC_TRY(sc.alloc(1, s));
        auto wdot = [&](const double* x, const double* y, double* out_host) -> int {
            SPHC_LAUNCH(k_wdot_rows<<<WD_BLOCKS, 256, 0, s>>>(ne, L.Pe.rp.p, dg.p, x, y, part.p));
            SPHC_LAUNCH(k_sum_parts<<<1, 32, 0, s>>>(part.p, WD_BLOCKS, sc.p));
            SPHC_CK(cudaMemcpyAsync(out_host, sc.p, sizeof(double), cudaMemcpyDeviceToHost, s));
            SPHC_CK(cudaStreamSynchronize(s));
            return SPHC_OK;
        };
        SPHC_TRY(proj_grad(L.Pe.v.p, Gv.p));
        SPHC_LAUNCH(k_neg_copy<<<grid_for(nnzN, 256), 256, 0, s>>>(Gv.p, Z.p, Pd.p, nnzN));
        double rz = 0.0;
        SPHC_TRY(wdot(Z.p, Z.p, &rz));
        for (int it = 0; it < emin_iters && rz > 0.0; ++it) {
            SPHC_TRY(proj_grad(Pd.p, Gv.p));
            double pq = 0.0;
            SPHC_TRY(wdot(Pd.p, Gv.p, &pq));
            if (!(pq > 0.0)) break;
            const double alpha = rz / pq;
            SPHC_LAUNCH(k_cg_update<<<grid_for(nnzN, 256), 256, 0, s>>>(L.Pe.v.p, Pd.p, Z.p, Gv.p, alpha, nnzN));
            double rz_new = 0.0;
            SPHC_TRY(wdot(Z.p, Z.p, &rz_new));
            const double beta = rz_new / rz;
            rz = rz_new;
            SPHC_LAUNCH(k_cg_dir<<<grid_for(nnzN, 256), 256, 0, s>>>(Pd.p, Z.p, beta, nnzN));
        }
        if (tid >= 0) prof->end(tid, s);
        emin_iters = 0;                          // done: skip the Jacobi loop below
    }
    for (int it = 0; it < emin_iters; ++it) {
        if (tid >= 0) prof->begin(tid, s);
        if (ne > 0) {
            const int gpp = grid_for(ne, PP_WARPS);
            {
                Section sp(prof, lev_name("emin_product", lev).c_str(), s);
                if (o.emin_fp32) {
                    to_f32(L.Pe.v.p);
                    SPHC_LAUNCH(k_emin_pp<float><<<gpp, PP_WARPS * 32, 0, s>>>(ne, L.A.rp.p, L.A.ci.p, A32.p, Dinv32.p, L.Pe.rp.p,
                                                                           L.Pe.ci.p, P32.p, cache.k, W32.p));
                }
                else
                    SPHC_LAUNCH(k_emin_pp<double><<<gpp, PP_WARPS * 32, 0, s>>>(ne, L.A.rp.p, L.A.ci.p, L.A.v.p, Dinv.p, L.Pe.rp.p,
                                                                            L.Pe.ci.p, L.Pe.v.p, cache.k, W.p));
            }
            {
                Section sr(prof, lev_name("emin_rows", lev).c_str(), s);
                if (o.emin_fp32)
                    SPHC_LAUNCH(k_emin_rows<float><<<grid_for(ne, 128), 128, 0, s>>>(ne, L.Pe.rp.p, W32.p, L.Pe.v.p,
                                                                                     Pnew.p, o.emin_omega, cache, 0));
                else
                    SPHC_LAUNCH(k_emin_rows<double><<<grid_for(ne, 128), 128, 0, s>>>(ne, L.Pe.rp.p, W.p, L.Pe.v.p,
                                                                                      Pnew.p, o.emin_omega, cache, 0));
            }
            if (hbig > 0)
                SPHC_LAUNCH(k_emin<<<grid_for(hbig, LOC_WARPS), LOC_WARPS * 32, sm, s>>>(
                    hbig, big.p, L.A.rp.p, L.A.ci.p, L.A.v.p, L.T.rp.p, L.T.ci.p, L.T.v.p, L.Pe.rp.p, L.Pe.ci.p,
                    L.DH.rp.p, L.DH.ci.p, L.DH.v.p, L.Pe.v.p, Pnew.p, o.emin_omega, st.p, 0));
        }
        if (tid >= 0) prof->end(tid, s);
        std::swap(L.Pe.v.p, Pnew.p);
    }
    SPHC_CK(cudaMemcpyAsync(hs, st.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    SPHC_CK(cudaStreamSynchronize(s));
    if (hs[0]) { set_error("level %d: %d local constraint systems are infeasible", lev, hs[0]); return SPHC_EINFEASIBLE; }
    // Galerkin operators of the next level
    {
        Section sec(prof, lev_name("setup_PeT", lev).c_str(), s);
        SPHC_TRY(transpose(L.Pe, L.PeT, s));
    }
    {
        int rid = prof ? prof->find(lev_name("rap_level", lev).c_str(), 0.0) : -1;
        if (rid >= 0) prof->begin(rid, s);
        DCSR AP;
        {
            Section sec(prof, lev_name("rap_AP", lev).c_str(), s);
            SPHC_TRY(spgemm(L.A, L.Pe, AP, s));
        }
        {
            Section sec(prof, lev_name("rap_PtAP", lev).c_str(), s);
            SPHC_TRY(spgemm_sym(L.PeT, AP, Anext, s));
        }
        if (rid >= 0) prof->end(rid, s);
        if (prof) {
            // algorithmic bytes: each operand read once (values, columns, row pointers), the
            // product written once
            auto csr_bytes = [](const DCSR& M) { return 12.0 * (double)M.nnz + 8.0 * (double)(M.nr + 1); };
            const double b_ap = csr_bytes(L.A) + csr_bytes(L.Pe) + csr_bytes(AP);
            const double b_ptap = csr_bytes(L.PeT) + csr_bytes(AP) + csr_bytes(Anext);
            prof->timers[prof->find(lev_name("rap_AP", lev).c_str(), 0.0)].bytes = b_ap;
            prof->timers[prof->find(lev_name("rap_PtAP", lev).c_str(), 0.0)].bytes = b_ptap;
            prof->timers[rid].bytes = b_ap + b_ptap;
        }
    }
    {
        Section sec(prof, lev_name("setup_nodal_rap", lev).c_str(), s);
        DCSR PnT, AnP;
        SPHC_TRY(transpose(L.Pn, PnT, s));
        SPHC_TRY(spgemm(L.An, L.Pn, AnP, s));
        SPHC_TRY(spgemm_sym(PnT, AnP, Annext, s));
    }
    SPHC_TRY(csr_copy(L.DH, Dnext, s));
    SPHC_CK(cudaGetLastError());
    return SPHC_OK;
}

}  // namespace sphc
