// Hierarchy data structures shared by the setup (setup.cu), the solve (solve.cu) and the C ABI.
#pragma once
#include <memory>

#include "sphc_internal.cuh"

namespace sphc {

// Limits of the warp-per-row local kernels (documented in include/sphc.h).
constexpr int MAX_T = 24;       // coarse nodes of one row of T (|J_i|)
constexpr int MAX_NP = 128;     // coarse edges of one row of the pattern (|I_i|)
constexpr int PAT_WARPS = 4;
constexpr int LOC_WARPS = 4;
// A smoothed nodal-prolongator row whose sum does not exceed this keeps its tentative values.
constexpr double SA_MIN_ROWSUM = 0.125;

// Sliced ELLPACK for one warp per slice.  A slice holds R = 32 / lpr consecutive rows (never
// across a colour boundary: srow[s] .. srow[s+1]) and lpr lanes share a row.  The slice is a
// dense block of width W (a multiple of lpr * ch): chunk k = j / ch of row q (ch consecutive
// entries j) belongs to lane q * lpr + k % lpr at step k / lpr and sits at
// soff[s] + ((k / lpr) * 32 + q * lpr + k % lpr) * ch + j % ch, so every step of the warp reads
// 32 * ch consecutive entries and every lane receives ch entries of its own row.  Rows shorter
// than W are padded with value 0 and a valid column index.
constexpr int SELL_C = 32;
template <typename T>
struct Sell {
    int64_t nr = 0, nc = 0, nnz = 0, nslice = 0, stored = 0;
    int ch = 4;                      // entries a lane loads at once (1, 2 or 4)
    int lpr = 1;                     // lanes per row (1, 2, 4, 8, 16 or 32)
    DBuf<int64_t> soff;              // nslice + 1
    DBuf<int32_t> srow;              // nslice + 1
    DBuf<int32_t> ci;
    DBuf<T> v;
};

// State of the grid barrier of the persistent sweep (device memory, zeroed when the V-cycle
// operators are built): arrivals at the current barrier, its generation, and an error word that a
// wait sets when it gives up.
struct GridBar {
    unsigned count;
    unsigned gen;
    int err;
    int pad;
};
// polls of a barrier wait before it gives up, unless sphc_opts.grid_wait_polls says otherwise
static constexpr unsigned GRID_BAR_POLLS = 1u << 22;

// Operator of one smoother in the level's V-cycle numbering (rows grouped by colour).
template <typename T>
struct SmoothOp {
    int64_t n = 0, nnz = 0;
    int ncolor = 0;
    std::vector<int64_t> cslice;     // colour c owns slices [cslice[c], cslice[c+1])
    DBuf<int64_t> cslice_dev;
    Sell<T> m;
    DBuf<T> dinv;
    int cluster = 0;                 // 1: whole sweeps on one thread-block cluster (x in shared memory)
    int grid = 0;                    // co-resident CTAs of the persistent grid sweep (0: not used)
    GridBar* bar = nullptr;          // its barrier state
    unsigned polls = 0;              // polls of a barrier wait before it gives up
    int64_t n_last = 0, nnz_last = 0; // rows and nonzeros of the last colour (swept once per sweep)
};
// smoothers of at most this many rows sweep in one thread block (colours separated by block
// barriers)
static constexpr int SGS_BLOCK_MAX_ROWS = 2048;
// how sgs() runs op: 0 a launch per colour, 1 the cluster sweep, 2 the one-block sweep, 3 the
// persistent grid sweep
template <typename T>
inline int sweep_kind(const SmoothOp<T>& op) {
    if (op.n == 0) return 0;
    if (op.cluster) return 1;
    if (op.grid) return 3;
    return op.n <= SGS_BLOCK_MAX_ROWS ? 2 : 0;
}

// Plain CSR in the V-cycle precision.
template <typename T>
struct VCSR {
    int64_t nr = 0, nc = 0, nnz = 0;
    DBuf<int32_t> rp, ci;
    DBuf<T> v;
    bool rows32 = false;  // products by the row-block kernel (short rows), else lanes per row
};

// Operator only multiplied (transfers, A D): SELL when its rows pad well, CSR otherwise.
template <typename T>
struct XOp {
    int64_t nr = 0, nc = 0, nnz = 0;
    bool sell = false;
    Sell<T> s;
    VCSR<T> c;
};

// Renumbering of one level's edges and nodes for the V-cycle: colour by colour, and inside a
// colour by row length (stable), so that a colour sweep reads its rows, right sides and iterates
// contiguously and a slice of 32 rows pads little.  p: new -> old, i: old -> new.  Empty on the
// coarsest level (identity).
struct LevelOrder {
    DBuf<int32_t> pe, ie, pn, in;
    std::vector<int64_t> ce, cn;     // colour starts in the new numbering
};

template <typename T>
struct VLevel {
    SmoothOp<T> A, An;
    DBuf<int2> D;                    // per edge: (node with -1, node with +1), -1 if absent
    DBuf<int32_t> Dt_rp, Dt_e;       // D^T: per node the incident edges, (edge << 1) | (coef < 0)
    XOp<T> Pe, PeT;
    // split iterate x = y + D c (FP32 V-cycle): A D formed in FP64 and P_n
    XOp<T> AD, Pn;
    DBuf<T> x, b, r, g, c, bp, dc;
};

struct Level {
    DCSR A, D, An, Dt;
    DCSR AD;                         // A D (FP64), kept from the nodal operator of level 0
    DBuf<double> X;                  // node coordinates [n_nodes x 3] (coarse levels: aggregate centroids)
    DBuf<double> sig;                // per-edge sigma (level 0 only)
    DBuf<int32_t> col_e, col_n;
    int ncol_e = 0, ncol_n = 0;
    int rounds_e = 0, rounds_n = 0;  // Jones-Plassmann rounds of the two colourings
    // transfer data (absent on the coarsest level)
    bool has_transfer = false;
    DBuf<int32_t> agg;
    int64_t nagg = 0;
    DCSR Pn, DH, T, Pe, P0, PeT;
    double rho = 0.0, omega_sa = 0.0;
    int64_t n_added = 0, n_rows_unsmoothed = 0, max_np = 0, max_m = 0;
    DBuf<unsigned long long> hist;   // 33 x 33 counts of (|N_i|, |T_i|)
};

// setup.cu
struct Profiler;
// prof (optional): sub-timers "colour_build_<tag>" (graph of the rounds built and instantiated) and
// "colour_rounds_<tag>" (the rounds and the colour count)
int color_graph(const DCSR& G, uint64_t seed, DBuf<int32_t>& color, int* ncolors, cudaStream_t s, int* rounds = nullptr,
                Profiler* prof = nullptr, const char* tag = nullptr);
int aggregate(const DCSR& G, uint64_t seed, DBuf<int32_t>& agg, int64_t* nagg, cudaStream_t s);
int power_rho(const DCSR& A, const double* diag, uint64_t seed, int iters, double* rho, cudaStream_t s);
int coarse_gradient(const DCSR& D, const DCSR& Dt, const int32_t* agg, int64_t nagg, DCSR& DH, cudaStream_t s);
int coarse_inverse(const DCSR& A, DBuf<double>& Ainv, bool allow_shift, cudaStream_t s);

// Section timers: CUDA events recorded on the work stream around a named section; resolved
// (cudaEventElapsedTime) when the profile is read.
struct Timer {
    std::string name;
    double ms = 0.0;
    int64_t calls = 0;
    double bytes = 0.0;                       // algorithmic bytes of one call
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;
};
struct Profiler {
    bool on = false;
    std::vector<Timer> timers;
    int find(const char* name, double bytes);
    void begin(int id, cudaStream_t s);
    void end(int id, cudaStream_t s);
    int resolve();
    ~Profiler();
};

// reuse: keep L's aggregates, D_H and pattern, recompute the values (warm start from L.Pe)
int build_level(Level& L, int lev, const sphc_opts& o, DCSR& Anext, DCSR& Dnext, DCSR& Annext, DBuf<double>& Xnext,
                const float* mlp_params, Profiler* prof, cudaStream_t s, bool reuse = false);
int level_features(const Level& L, const DBuf<double>& Xc, int lev, float* F, cudaStream_t s);
int level_prediction(const Level& L, const DBuf<double>& Xc, int lev, const float* params_dev, float* out,
                     cudaStream_t s);
// mlp.cu
int mlp_predict(const float* params_dev, const float* X, int64_t m, float* out, cudaStream_t s);
struct FeatArgs;
// features of every pattern entry of a level computed on the fly and fed to the MLP (no feature buffer)
// polls > 0: the per-tile completion waits give up after that many non-blocking checks (SPHC_ETIMEOUT)
int mlp_predict_level(const float* params_dev, const FeatArgs& g, float* out, cudaStream_t s, int polls = 0);

// Scoped section timer (no-op when prof is null).
struct Section {
    Profiler* p;
    int id = -1;
    cudaStream_t s;
    Section(Profiler* prof, const char* name, cudaStream_t stream, double bytes = 0.0) : p(prof), s(stream) {
        if (p) {
            id = p->find(name, bytes);
            p->begin(id, s);
        }
    }
    ~Section() {
        if (p) p->end(id, s);
    }
};

// Work vectors of the block right-hand-side solve (block.cu): NB interleaved columns per vector.
template <typename T>
struct BlockLevel {
    DBuf<T> x, b, r, g, c, bp, dc;
};
struct BlockWork {
    int nb = 0;
    std::vector<BlockLevel<float>> V32;
    std::vector<BlockLevel<double>> V64;
    DBuf<double> X, R, Z, P, Q, Rold, B;    // CG vectors (FP64, level-0 V-cycle numbering)
    DBuf<double> cb, cx, cgn, ccn;          // coarsest-level work (FP64)
    DBuf<double> part, sc;                  // dot-product partials; per-column scalars
    DBuf<int> st;                           // per-column iteration counts and status
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    long long body_launches = 0;
    ~BlockWork();
};

// solve.cu
struct Hierarchy {
    sphc_opts opts;
    int nlev = 0;
    std::vector<Level> L;
    DBuf<double> coarse_inv;         // dense inverse of the coarsest operator (FP64)
    DBuf<double> coarse_inv_n;       // dense inverse of the coarsest nodal operator (split V-cycle)
    int64_t n_coarse = 0, n_coarse_nodes = 0;
    DBuf<double> cgn, ccn;           // coarsest nodal work vectors (FP64)
    // V-cycle copies in the chosen precision
    std::vector<LevelOrder> ord;
    std::vector<VLevel<float>> V32;
    std::vector<VLevel<double>> V64;
    Sell<double> A0;                 // level-0 operator for CG in the V-cycle numbering (FP32 V-cycle)
    // CG work vectors (FP64)
    // (CG runs in the level-0 V-cycle numbering; bperm is b in that numbering, xo the batched
    // solution scattered back to the caller's numbering)
    DBuf<double> x, r, z, p, q, rold, scal, bin, bperm, xo;
    DBuf<double> cb, cx;             // coarsest right side / solution (FP64)
    // CG as one CUDA graph: a device-side while loop (conditional node) around one iteration
    DBuf<double> dpart;              // partial sums of the dot products
    DBuf<int> itc;                   // [0] iterations, [1] status (0 converged, 1 breakdown, 2 cap)
    DBuf<GridBar> gbar;              // barrier of the persistent grid sweeps (shared: they run in turn)
    cudaGraph_t cg_graph = nullptr;
    cudaGraphExec_t cg_exec = nullptr;
    cudaStream_t cap_stream = nullptr;
    bool capturing = false;          // section timers are off while a graph is being captured
    long long body_launches = 0;     // kernels in one CG graph iteration (for the launch count)
    long long branch_launches = 0;   // kernels of a captured CG outside its loop
    double setup_ms = 0.0, solve_ms = 0.0;
    Profiler prof;
    DBuf<float> mlp;                 // MLP parameters on the device (learned warm start)
    std::unique_ptr<BlockWork> blk;  // block right-hand-side work (allocated by the first block solve)
    ~Hierarchy() {
        blk.reset();
        if (cg_exec) cudaGraphExecDestroy(cg_exec);
        if (cg_graph) cudaGraphDestroy(cg_graph);
        if (cap_stream) cudaStreamDestroy(cap_stream);
    }
    int last_iters = 0;
    double last_relres = 0.0;
};

int build_vcycle_ops(Hierarchy& H, cudaStream_t s);
// layout.cu
int stable_partition(const int32_t* key, int64_t n, int nkeys, DBuf<int32_t>& perm, std::vector<int64_t>& kstart,
                     cudaStream_t s);
int level_order(const DCSR& A, const int32_t* color, int ncolor, DBuf<int32_t>& p, DBuf<int32_t>& ip,
                std::vector<int64_t>& cstart, cudaStream_t s);
template <typename T>
int build_sell(const DCSR& A, const int32_t* rmap, const int32_t* cmap, const std::vector<int64_t>& seg, int ch,
               int lpr, Sell<T>& S, T* dinv, std::vector<int64_t>* segslice, cudaStream_t s);
template <typename T>
int build_csr_perm(const DCSR& A, const int32_t* rmap, const int32_t* cmap, VCSR<T>& B, cudaStream_t s);
template <typename T>
int build_xop(const DCSR& A, const int32_t* rmap, const int32_t* cmap, XOp<T>& X, cudaStream_t s);
template <typename T>
int build_smooth(const DCSR& A, const int32_t* rmap, const int32_t* cmap, const std::vector<int64_t>& cstart, int ch,
                 int lpr, SmoothOp<T>& op, cudaStream_t s);
int sell_lpr_for(const DCSR& A, int ncolor);
int sell_pick_ch(const DCSR& A, const int32_t* rmap, const std::vector<int64_t>& seg, int lpr, cudaStream_t s, int* ch,
                 int64_t* stored = nullptr);
int build_d_pairs(const DCSR& D, const int32_t* pe, const int32_t* in, DBuf<int2>& out, cudaStream_t s);
int build_dt_enc(const DCSR& Dt, const int32_t* pn, const int32_t* ie, DBuf<int32_t>& rp, DBuf<int32_t>& enc,
                 cudaStream_t s);
int gather64(const double* src, const int32_t* p, int64_t n, double* dst, cudaStream_t s);
int scatter64(const double* src, const int32_t* p, int64_t n, double* dst, cudaStream_t s);
int apply_vcycle(Hierarchy& H, const double* r, double* z, cudaStream_t s);
int grid_barrier_check(int extra, unsigned max_polls, int* timed_out, cudaStream_t s);
int apply_vcycle_user(Hierarchy& H, const double* r, double* z, cudaStream_t s);
int pcg_solve(Hierarchy& H, const double* b, double* x, double tol, cudaStream_t s, int* iters, double* relres);
int capture_cg(Hierarchy& H, cudaStream_t s);
// block.cu: nrhs <= 16 right-hand sides (device arrays, caller layout nrhs x n_e) solved together
int pcg_block(Hierarchy& H, const double* b, double* x, int nrhs, double tol, cudaStream_t s, int* iters,
              double* relres);
int autotune_vcycle(Hierarchy& H, cudaStream_t s);

}  // namespace sphc

// The opaque handle of the C ABI.
struct sphc_handle {
    sphc::Hierarchy H;
    int device = 0;
    int64_t device_bytes = 0;        // growth of the library pool's used memory across setup
};
