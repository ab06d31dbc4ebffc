/*
 * sphc.h -- C ABI of the sm_103a (GB300) SpHcurlAMG library, libsphc.so.
 *
 * The library solves the lowest-order edge-element eddy-current system A_e u = f
 * (Tuminaro & Glusa, Sec. 1, eqs. (1)-(2)) with conjugate gradients preconditioned by one
 * V-cycle of the structure-preserving H(curl) AMG method (Sec. 6.1), whose edge prolongators
 * are built by constrained energy minimisation (Sec. 3 eq. (9), Sec. 4, Algs. 2-3).
 *
 * Conventions shared by every entry point:
 *   - Pointers may address host memory or device memory of the current CUDA device; the
 *     library detects which (cudaPointerGetAttributes) and copies host data itself.
 *   - All GPU work is enqueued on the caller's stream (`stream`, a cudaStream_t; NULL = the
 *     legacy default stream).  Entry points that return host-visible results synchronise that
 *     stream before returning.
 *   - The caller owns every buffer it passes.  sphc_setup copies what it keeps into memory the
 *     handle owns (stream-ordered cudaMallocAsync); sphc_destroy releases it.
 *   - Return value: SPHC_OK (0) or a negative error code below; sphc_last_error() gives a
 *     thread-local message.  No C++ exception crosses the ABI.
 *   - Handles are not thread-safe: one thread (or one stream) at a time per handle.
 */
#ifndef SPHC_H
#define SPHC_H

#include <stdint.h>

#if defined(__GNUC__)
#define SPHC_API __attribute__((visibility("default")))
#else
#define SPHC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

enum {
    SPHC_OK = 0,
    SPHC_EINVAL = -1,        /* malformed input: sizes, CSR structure, D_h entries not +-1, ... */
    SPHC_ENOMEM = -2,        /* device allocation failed */
    SPHC_ECUDA = -3,         /* a CUDA call failed */
    SPHC_ENOTCONV = -4,      /* CG reached max_iter before the tolerance */
    SPHC_EBREAKDOWN = -5,    /* CG breakdown: p^T A p <= 0 or not finite */
    SPHC_EINFEASIBLE = -6,   /* a local commuting-constraint system has no solution */
    SPHC_ETIMEOUT = -7,      /* a bounded device wait gave up */
    SPHC_ESTAGNATION = -8,   /* CG stagnated: two consecutive iterates are identical (Sec. 7) */
    SPHC_ENUMERIC = -9,      /* non-finite or non-positive quantity where a positive one is required */
    SPHC_ELIMIT = -10        /* a size exceeded a documented kernel limit */
};

/* Compressed sparse row matrix.  rowptr[nrows+1] (int64), col[nnz] (int32, sorted and unique
 * within each row), val[nnz] (FP64). */
typedef struct {
    int64_t nrows, ncols;
    const int64_t* rowptr;
    const int32_t* col;
    const double* val;
} sphc_csr;

typedef struct {
    int32_t max_levels;      /* hierarchy depth cap (default 8) */
    int32_t emin_iters;      /* projected-Jacobi energy-minimisation steps, eq. (9) (default 1, Sec. 6.1) */
    int64_t max_coarse;      /* a level with at most this many edges is solved directly (default 1000) */
    double emin_omega;       /* damping of eq. (9) (default 0.5, Sec. 6.1) */
    uint64_t seed;           /* seed of the aggregation / colouring priorities (default 0) */
    int32_t power_iters;     /* power-iteration steps for rho(D^-1 A_n) (default 15) */
    int32_t vcycle_fp32;     /* 1: V-cycle in FP32 inside FP64 CG; 0: all FP64 (default 1) */
    int32_t max_iter;        /* CG iteration cap (default 500) */
    int32_t flexible;        /* 1: flexible (Polak-Ribiere) CG beta; 0: Fletcher-Reeves (default: = vcycle_fp32) */
    int32_t profile;         /* 1: record CUDA-event section timers (sphc_get_profile); with cg_graph the
                                timers cover the first CG iteration, which runs outside the graph (default 0) */
    int32_t cg_graph;        /* 1: run the CG iterations as one CUDA graph with a device-side loop (default 1) */
    int32_t learned;         /* 1: learned warm start of P_e (needs mlp_params and coords) (default 0) */
    int32_t learned_emin_iters; /* energy-minimisation steps after the learned warm start (default 0) */
    const float* mlp_params; /* SPHC_MLP_NPARAM floats (host or device), see sphc_mlp_train */
    int32_t autotune;        /* 1: time the smoother kernels' lanes-per-row widths at setup (default 0) */
    int32_t sweep_form;      /* smoothers with more rows than one thread block sweeps: 0 a cost model
                                picks between one launch per colour and one launch per sweep on a
                                thread-block cluster (x in shared memory, where it fits); 1 always
                                a launch per colour; 2 the cluster wherever x fits; 3 one cooperative
                                launch per sweep over the whole GPU with a grid barrier between
                                colours (slower than form 0 on the meshes measured; default 0;
                                autotune overrides it with forms 1 and 2).  A grid sweep whose barrier
                                wait runs out of polls makes the solve or V-cycle call that ran it
                                return SPHC_ETIMEOUT; the batched solve's graph always uses
                                per-colour launches instead */
    int32_t mlp_wait_polls;  /* polls of the learned warm start's per-tile tensor-core completion waits
                                before the kernel gives up and setup returns SPHC_ETIMEOUT (0: the
                                default of 2^20 blocking polls; n > 0: n non-blocking checks).  The
                                wait that drains an MMA still in flight before the tensor memory is
                                freed always uses the default.  A small value exists to test the
                                timeout path without hanging anything. */
    int32_t sell_lpr0;       /* level-0 edge smoother: lanes per row of its SELL-32 copy (1, 2, 4, 8,
                                16 or 32; 0: chosen from the mean row length, default) */
    int32_t sell_ch0;        /* level-0 edge smoother: entries per lane load (1, 2 or 4; 0: the widest
                                that pads little, default).  These two fix the shape the 128^3
                                workload gets (1 and 2) on small meshes, for parity tests. */
    int32_t emin_fp32;       /* 1: the masked product (A P)|_N / a_ii of eq. (9) accumulates in FP32;
                                its projection onto the row constraints and the update of P_e stay
                                FP64, so P_e D_H = D_h P_n holds to FP64 rounding either way
                                (default 0: FP64 throughout) */
    int32_t block_rhs;       /* 1: sphc_solve with nrhs >= 2 solves the right-hand sides in blocks of up
                                to 16, one CG per column sharing every operator read (vectors
                                interleaved per row); 0: one right-hand side after another (default 1) */
    int32_t emin_method;     /* energy minimisation of P_e: 0 projected Jacobi, eq. (9), with emin_omega;
                                1 projected CG on the KKT system of eq. (8) (Sec. 3), D^-1
                                preconditioned, emin_iters steps (default 0) */
    int32_t pn_alg1;         /* 1: D_H from Alg. 1 (Gen_Piecewise_Const) applied to the smoothed P_n
                                instead of the tentative aggregates (Sec. 4.1; default 0) */
    double sa_theta;         /* smoothed-aggregation drop tolerance: an off-diagonal a_ij of A_n is
                                strong when |a_ij| >= theta sqrt(a_ii a_jj); aggregation runs on the
                                strong graph and P_n is smoothed with the filtered matrix, dropped
                                entries lumped into the diagonal (Sec. 7; default 0: every
                                structural entry is strong, Sec. 6.1) */
    int32_t alg1_passes;     /* passes of Alg. 1 (default 2) */
    int32_t grid_wait_polls; /* polls of a grid sweep's barrier wait before it gives up and the call
                                returns SPHC_ETIMEOUT (0: the default, 4194304, well over a second) */
} sphc_opts;

/* Learned warm start (not part of the paper).  For every pattern entry (i, j) of P_e a
 * multilayer perceptron maps SPHC_MLP_NFEAT local features (fine- and coarse-edge geometry
 * relative to the fine edge length, the constraint values r_i, the P_n entries of the fine
 * edge's ends, row sizes, A_e row scaling, log10 sigma, level; feature 19 is unused and 0) to a
 * correction c of the least-norm initial guess.  The initial guess is then the point of the
 * row's constraint set nearest to c, i.e. P0 + (I - G (G^T G)^-1 G^T) c, computed in the same
 * local solve as P0, so P_e D_H = D_h P_n holds exactly as without it.
 * Parameters (floats, in this order): feature means [32], feature scales [32],
 * W1 [32 x 128] (row = input), b1 [128], W2 [128 x 128], b2 [128], w3 [128], b3. */
#define SPHC_MLP_NFEAT 32
#define SPHC_MLP_HIDDEN 128
#define SPHC_MLP_NPARAM 20929

typedef struct {
    int32_t steps;           /* Adam steps (default 3000) */
    int32_t batch;           /* minibatch rows (default 4096) */
    float lr, beta1, beta2, eps, weight_decay;   /* Adam (1e-3, 0.9, 0.999, 1e-8, 0) */
    int32_t pad;
    uint64_t seed;           /* minibatch sampling seed (default 1) */
    int32_t reserved[4];
} sphc_train_opts;

typedef struct sphc_handle sphc_handle;

/* Per-level sizes of a built hierarchy. */
typedef struct {
    int64_t n_edges, n_nodes;        /* rows of A_l, columns of D_l */
    int64_t nnz_A, nnz_An;           /* nonzeros of A_l and of the nodal operator */
    int64_t n_aggregates;            /* coarse nodes (0 on the coarsest level) */
    int64_t n_coarse_edges;          /* rows of D_H */
    int64_t nnz_Pn, nnz_Pe, nnz_T;   /* nodal prolongator, edge prolongator, pattern T */
    int32_t n_colors_edge, n_colors_node;
    int64_t n_added_edges;           /* coarse edges added by make_irreducible */
    int64_t n_rows_unsmoothed;       /* P_n rows kept at their tentative values */
    double rho, omega_sa;            /* rho(D^-1 A_n) estimate and the prolongator damping */
    int64_t max_pattern_row;         /* largest |N_i| (pattern entries of one P_e row) */
    int64_t max_T_row;               /* largest |T_i| (coarse nodes of one row) */
    /* V-cycle copies of the smoothers (sliced ELLPACK, 32-lane slices; 0 where there is none):
     * lanes per row, entries per lane load and stored entries (nonzeros plus padding) */
    int32_t sell_lpr_edge, sell_ch_edge, sell_lpr_node, sell_ch_node;
    int64_t sell_stored_edge, sell_stored_node;
    /* Jones-Plassmann rounds run by the edge and node colourings (8 per device-loop iteration,
     * so up to 7 more than the rounds that coloured something) */
    int32_t colour_rounds_edge, colour_rounds_node;
    /* smoother sweep form: 0 one launch per colour, 1 one launch per sweep on one thread-block
     * cluster (x held in shared memory), 2 one launch per sweep on one thread block, 3 one
     * cooperative launch per sweep over the whole GPU (grid barrier between colours) */
    int32_t sweep_kind_edge, sweep_kind_node;
} sphc_level_info;

typedef struct {
    int32_t n_levels;
    double operator_complexity;      /* sum_l nnz(A_l) / nnz(A_0), Sec. 6.1 */
    double setup_ms;                 /* wall time of the last sphc_setup */
    double solve_ms;                 /* wall time of the last sphc_solve */
    int32_t last_iters;              /* CG iterations of the last solve (first RHS) */
    double last_relres;              /* true relative residual of the last solve (first RHS) */
    int64_t device_bytes;            /* bytes the handle holds: growth of the library pool's used
                                        memory across its sphc_setup */
} sphc_stats;

/* One section timer of the profile (opts.profile = 1): total device time of the section's
 * calls, measured with CUDA events on the work stream, and the algorithmic bytes one call moves
 * (0 where no byte count is defined). */
typedef struct {
    char name[32];
    double ms;
    int64_t calls;
    double bytes_per_call;
} sphc_timer;

/* Export ids for sphc_export_size / sphc_export (per level). */
enum {
    SPHC_X_A = 0,      /* A_l (CSR) */
    SPHC_X_D = 1,      /* D_l (CSR) */
    SPHC_X_AN = 2,     /* nodal operator (CSR) */
    SPHC_X_PN = 3,     /* nodal prolongator (CSR) */
    SPHC_X_DH = 4,     /* coarse gradient D_H (CSR) */
    SPHC_X_T = 5,      /* pattern T = |D_l||P_n| with the values D_l P_n (CSR) */
    SPHC_X_PE = 6,     /* edge prolongator P_e (CSR, pattern N) */
    SPHC_X_P0 = 7,     /* initial guess of the energy minimisation (CSR, pattern N) */
    SPHC_X_AGG = 16,   /* aggregate of each node (int32 vector) */
    SPHC_X_COLE = 17,  /* colour of each edge row (int32 vector) */
    SPHC_X_COLN = 18   /* colour of each node row (int32 vector) */
};

/* Fill *opts with the defaults listed above.  Returns SPHC_OK or SPHC_EINVAL (NULL). */
SPHC_API int sphc_default_opts(sphc_opts* opts);

/*
 * Build the AMG hierarchy (Alg. 3 on every level, Sec. 6.1 settings).
 *   A_e:   n_e x n_e SPD edge operator S_e + M_e (Sec. 1).
 *   D_h:   n_e x n_v discrete gradient, at most two entries per row, -1 at the tail and +1 at
 *          the head; rows with one entry are edges with one Dirichlet end (Sec. 1).
 *   coords: n_v x 3 node coordinates (row-major) or NULL; sigma_edge: n_e per-edge conductivity
 *          or NULL.  Both are only features of the learned warm start and may be NULL.
 *   opts:  NULL for the defaults.
 * On success *out receives a new handle.  Errors: SPHC_EINVAL (malformed input), SPHC_ENOMEM,
 * SPHC_ECUDA, SPHC_EINFEASIBLE (a local constraint system cannot be satisfied), SPHC_ELIMIT
 * (a row of the pattern exceeds the kernels' limits: 128 entries of N_i, 24 nodes of T_i),
 * SPHC_ENUMERIC.
 */
SPHC_API int sphc_setup(const sphc_csr* A_e, const sphc_csr* D_h, const double* coords, const double* sigma_edge,
               const sphc_opts* opts, void* stream, sphc_handle** out);

/*
 * Rebuild the hierarchy for a related system: new values A_values[nnz(A_e)] (host or device) on
 * the pattern given to sphc_setup, e.g. the next time step or nonlinear iterate.  Following the
 * warm-start remark of Sec. 3, the structural parts are kept (colourings, aggregates, D_H, the
 * pattern N of P_e), and the rest is recomputed from the new values: A_n, P_n, the constraint
 * values D_h P_n, the initial guess (the previous P_e projected onto the new row constraints, in
 * place of P0 or the learned correction), opts.emin_iters energy-minimisation steps, the Galerkin
 * operators, the coarsest factor and the V-cycle copies.  Synchronises the stream.  Errors:
 * SPHC_EINVAL (NULL, non-finite value, missing diagonal), SPHC_ENOMEM, SPHC_ECUDA, SPHC_ENUMERIC,
 * SPHC_EINFEASIBLE.
 */
SPHC_API int sphc_setup_update(sphc_handle* h, const double* A_values, void* stream);

/*
 * Solve A_e x = b for nrhs right-hand sides (b and x are nrhs x n_e, row-major, FP64) with
 * V-cycle preconditioned CG: x0 = 0, stop when ||r_k|| <= tol ||b|| (Sec. 6.1).
 * iters[nrhs] and relres[nrhs] (true residual ||b - A x|| / ||b||) may be NULL.
 * Returns SPHC_OK when every right-hand side converged, else the first failure:
 *   SPHC_ENOTCONV     opts.max_iter iterations without reaching the tolerance;
 *   SPHC_EBREAKDOWN   p^T A p <= 0 or a non-finite residual;
 *   SPHC_ESTAGNATION  an iteration left every entry of x unchanged (the stagnation criterion of
 *                     Sec. 7: two consecutive iterations with the same solution), which happens
 *                     when the tolerance lies below what FP64 rounding lets CG reach;
 *   SPHC_EINVAL, SPHC_ECUDA.
 * On every failure x holds the last iterate and relres its true residual.
 */
SPHC_API int sphc_solve(sphc_handle* h, const double* b, double* x, int nrhs, double tol, void* stream,
               int* iters, double* relres);

/* 1-norm condition estimate of D^-1 A_e (D = diag(A_e)), which Sec. 6.1 uses (through Matlab's
 * condest) to cap the CG tolerance at kappa / 1e16.  ||D^-1 A_e||_1 is computed exactly (A_e is
 * symmetric: column j sums |a_ji| / a_ii); ||(D^-1 A_e)^-1||_1 is Hager's estimate (a lower bound,
 * usually exact) from at most max_steps iterations, each two solves with the handle's CG to a
 * relative residual of 1e-10.  kappa, norm_b (= ||D^-1 A_e||_1) and norm_binv may be NULL.  Not a
 * hot-path call.  Errors: SPHC_EINVAL, SPHC_ENOMEM, SPHC_ECUDA, SPHC_EBREAKDOWN. */
SPHC_API int sphc_cond_estimate(sphc_handle* h, int max_steps, double* kappa, double* norm_b, double* norm_binv,
                                void* stream);

/* Convergence factor of the V-cycle as a stationary iteration: x <- x + M^-1 (b - A_e x) with
 * b = 0, from x uniform in [-1, 1] (splitmix64(seed, i)); *factor = geometric mean of the ratios
 * ||x_k||_A / ||x_{k-1}||_A over the last `tail` of `iters` iterations.  Not part of the paper; the
 * yardstick of the learned warm start.  Errors: SPHC_EINVAL, SPHC_ENOMEM, SPHC_ECUDA. */
SPHC_API int sphc_vcycle_factor(sphc_handle* h, int iters, int tail, uint64_t seed, double* factor, void* stream);

/* A-energy trace(P_e^T A_l P_e) = sum_j P_:j^T A_l P_:j of level `level`'s edge prolongator, the
 * objective of the energy minimisation (Sec. 3, eq. (7)).  Synchronises the stream.  Errors:
 * SPHC_EINVAL (no prolongator on that level), SPHC_ENOMEM, SPHC_ECUDA. */
SPHC_API int sphc_prolongator_energy(const sphc_handle* h, int level, double* energy, void* stream);

/* Apply one V-cycle z = M^-1 r (FP64 in and out, n_e entries) with the handle's precision.
 * Errors: SPHC_EINVAL, SPHC_ECUDA, SPHC_ETIMEOUT (a grid sweep's barrier wait gave up). */
SPHC_API int sphc_vcycle(sphc_handle* h, const double* r, double* z, void* stream);

/* Diagnostic of the grid barrier that separates the colours of the persistent smoother sweep
 * (sphc_opts.sweep_form): one cooperative grid (all SMs) passes three barriers that count
 * `extra_arrivals` more arrivals than it has thread blocks, each wait limited to `polls` polls
 * (0: the sweep's default).  With extra_arrivals > 0 no barrier can complete, every wait gives up
 * and *timed_out = 1; with 0 the barriers complete and *timed_out = 0.  Either way the kernel
 * returns and the device stays usable.  Synchronises the stream.  Errors: SPHC_EINVAL (negative
 * argument, or the device has no cooperative launch), SPHC_ENOMEM, SPHC_ECUDA. */
SPHC_API int sphc_grid_barrier_check(int extra_arrivals, int polls, int* timed_out, void* stream);

SPHC_API int sphc_get_stats(const sphc_handle* h, sphc_stats* stats);
SPHC_API int sphc_get_level_info(const sphc_handle* h, int level, sphc_level_info* info);

/* Sizes of an exported array: CSR ids give nrows/ncols/nnz, vector ids give nrows = length. */
SPHC_API int sphc_export_size(const sphc_handle* h, int level, int what, int64_t* nrows, int64_t* ncols, int64_t* nnz);
/* Copy an exported array into caller buffers (host or device).  CSR ids fill rowptr/col/val
 * (any may be NULL); vector ids fill ivec.  Synchronises the stream. */
SPHC_API int sphc_export(const sphc_handle* h, int level, int what, int64_t* rowptr, int32_t* col, double* val,
                int32_t* ivec, void* stream);

/* Release the handle and every device buffer it owns (NULL is ignored).  The memory goes back to
 * the library's memory pool of that device, which keeps it mapped for the next setup. */
SPHC_API void sphc_destroy(sphc_handle* h);

/* Return the memory the library's pool of `device` holds beyond keep_bytes to the driver
 * (cudaMemPoolTrimTo).  Memory still owned by live handles is not affected.  Not part of the
 * paper: the library caches device memory across setups the way a caching allocator does, and
 * this is how a caller that needs the memory for something else gets it back.  Returns
 * SPHC_EINVAL for a device without a pool, SPHC_ECUDA if the runtime call fails. */
SPHC_API int sphc_trim_memory(int device, uint64_t keep_bytes);

/* Copy up to max timers of the handle's profile into out (host memory); *n receives the number
 * of timers.  Synchronises on the recorded events.  Timers accumulate over the handle's life. */
SPHC_API int sphc_get_profile(sphc_handle* h, sphc_timer* out, int max, int* n);

/* Device memory of the library's pool on `device`: *used = bytes currently allocated from it
 * (live handles and temporaries in flight), *reserved = bytes the pool holds mapped (used plus
 * the cache that sphc_trim_memory returns).  Either pointer may be NULL.  Not part of the paper.
 * Returns SPHC_EINVAL for a device without a pool, SPHC_ECUDA if a runtime call fails. */
SPHC_API int sphc_memory_usage(int device, int64_t* used, int64_t* reserved);

/* Number of kernels the library has launched in this process so far. */
SPHC_API int64_t sphc_launch_count(void);

/* Many independent systems of uneven size (not part of the paper).  sphc_setup_batched builds
 * one hierarchy per system (arrays of nsys descriptors; coords / sigma_edge may be NULL or hold
 * NULL entries) and captures every system's whole CG (a device-side while loop per system) as
 * parallel branches of one CUDA graph.  sphc_solve_batched launches that graph once per
 * right-hand side: b[k] and x[k] are nrhs x n_e(k) FP64 arrays (host or device) of system k;
 * iters and relres (nsys x nrhs, may be NULL) receive the CG iterations and true relative
 * residuals.  Returns SPHC_OK if every system converged, else the first failure code. */
typedef struct sphc_batch sphc_batch;
SPHC_API int sphc_setup_batched(int nsys, const sphc_csr* A_e, const sphc_csr* D_h, const double* const* coords,
                                const double* const* sigma_edge, const sphc_opts* opts, void* stream, sphc_batch** out);
SPHC_API int sphc_solve_batched(sphc_batch* batch, const double* const* b, double* const* x, int nrhs, double tol,
                                void* stream, int* iters, double* relres);
SPHC_API void sphc_batch_destroy(sphc_batch* batch);

/* Fill *opts with the training defaults. */
SPHC_API int sphc_default_train_opts(sphc_train_opts* opts);

/* Train the MLP on m samples: X [m x SPHC_MLP_NFEAT] (row-major FP32) and targets y [m] (host
 * or device).  params [SPHC_MLP_NPARAM] holds the initial parameters (including the feature
 * means and scales, which are not trained) and receives the trained ones.  loss_history
 * [steps] (may be NULL) receives the minibatch mean squared errors.  Synchronises the stream. */
SPHC_API int sphc_mlp_train(const float* X, const float* y, int64_t m, const sphc_train_opts* opts, float* params,
                            float* loss_history, void* stream);

/* Apply the MLP (BF16 tensor-core inference, FP32 accumulate) to m feature rows. */
SPHC_API int sphc_mlp_predict(const float* params, const float* X, int64_t m, float* out, void* stream);

/* Gradient of the mean squared error over the B rows (X, y) with respect to params (the
 * normalisation entries of grad are left 0), and the loss; the training kernels' backward pass. */
SPHC_API int sphc_mlp_gradient(const float* params, const float* X, const float* y, int B, float* grad, float* loss,
                               void* stream);

/* Features [nnz(P_e) x SPHC_MLP_NFEAT] of level `level`'s pattern entries and the training
 * target P_e - P0 [nnz(P_e)] (either pointer may be NULL; host or device).  Needs coords at
 * setup.  Synchronises the stream. */
SPHC_API int sphc_export_features(const sphc_handle* h, int level, float* X, float* y, void* stream);

/* The learned warm start's inference as setup runs it (features computed inside the
 * tensor-core kernel, no feature matrix in memory), applied with `params` (SPHC_MLP_NPARAM
 * floats, host or device) to every pattern entry of level `level`: out[nnz(P_e)] (host or
 * device) receives the raw network outputs, before the constraint projection.  For parity tests
 * against the network's definition on the features of sphc_export_features.  Needs coords at
 * setup.  Synchronises the stream.  Errors: SPHC_EINVAL, SPHC_ENOMEM, SPHC_ECUDA, SPHC_ETIMEOUT. */
SPHC_API int sphc_mlp_predict_level(const sphc_handle* h, int level, const float* params, float* out, void* stream);

/* Largest nrhs that sphc_relres_noalloc accepts (its fixed scratch holds this many). */
#define SPHC_NOALLOC_MAX_RHS 64

/*
 * The paper has no counterpart to this entry point; it serves callers that cannot allocate
 * device memory (an allocator callback, a framework that has reserved all device memory, a
 * real-time loop that forbids allocation after start-up).
 *
 * Computes relres[k] = ||b_k - A_e x_k|| / ||b_k|| (0 when b_k = 0) for k < nrhs, the same
 * quantity sphc_solve reports, with A_e the handle's finest operator.  b and x are nrhs x n_e
 * FP64 arrays (row-major) in device memory; relres[nrhs] may be host or device memory.
 * It allocates nothing: its partial sums live in one file-scope device array of
 * SPHC_NOALLOC_MAX_RHS x 513 doubles (about 257 KB) that every GPU loading the library keeps
 * until the process exits.  The first call on a device looks up that array's device address
 * (cudaGetSymbolAddress), so make it before any stream capture.  All calls share the array:
 * calls that overlap on the GPU (other streams, other threads) race and must be serialised by
 * the caller.  Synchronises the stream.  Errors: SPHC_EINVAL (NULL pointer, nrhs outside
 * 1..SPHC_NOALLOC_MAX_RHS, host b or x, current device not the handle's), SPHC_ECUDA.
 */
SPHC_API int sphc_relres_noalloc(const sphc_handle* h, const double* b, const double* x, int nrhs, double* relres,
                                 void* stream);

/* Thread-local message of the last error ("" if none). */
SPHC_API const char* sphc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
