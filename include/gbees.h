/*
 * gbees.h -- C ABI of the GB300 (sm_103a) GBEES propagation library.
 *
 * GBEES (Grid-based Bayesian Estimation Exploiting Sparsity; Hanson, Rubio,
 * Garcia-Gutierrez, Bewley, "GBEES-GPU", arXiv 2508.13986) propagates a
 * probability density p(x, t) of a state x in R^n by a finite-volume solution
 * of the advection form of the Fokker-Planck equation (Eq. 3), on a sparse
 * Cartesian grid that holds only the cells where p is non-negligible, and
 * folds in measurements by Bayes' rule (Eq. 4).
 *
 * One call sequence (the estimation loop of Sec. 2):
 *   gbees_workspace_bytes -> caller allocates device memory and a stream
 *   gbees_create -> gbees_init_gaussian | gbees_init_cells
 *   { gbees_propagate(t_m) -> gbees_correct_gaussian(y_m) }* -> gbees_propagate(t_end)
 *   gbees_read_cells / gbees_moments -> gbees_destroy
 *
 * Conventions for every entry point:
 *   - Return value: a gbees_status (0 = success, negative = error). No entry
 *     point throws or aborts; gbees_last_error() returns a message.
 *   - After GBEES_ECAPACITY, GBEES_EKEYRANGE, GBEES_ETABLE or GBEES_EDEGENERATE
 *     the context is poisoned: every later call except gbees_last_error /
 *     gbees_status / gbees_destroy returns the same status until
 *     gbees_init_gaussian or gbees_init_cells starts a new grid. GBEES_ECUDA
 *     poisons the context for good (destroy it).
 *   - Device memory: the caller owns the workspace (one allocation of
 *     gbees_workspace_bytes bytes, 256-byte aligned) and the CUDA stream; the
 *     library owns only its small host-side context. All work is issued on the
 *     caller's stream. Every call returns after its work has completed on that
 *     stream (the host buffers it writes are valid on return).
 *   - Host pointers (mean, cov, idx, p, y, R, ...) belong to the caller and are
 *     read or written only during the call.
 *   - Device: a context belongs to the CUDA device that was current at
 *     gbees_create (its workspace must be on that device). A call made while
 *     another device is current returns GBEES_EINVAL (the context stays
 *     usable).
 *   - Cell indices are signed integers; cell i has centre x0 + i * h (Eq. 5).
 *     Keys pack the indices with floor(63 / n) bits per dimension (32 for n = 1),
 *     i.e. -2^(bits-1) <= i_j < 2^(bits-1). An active cell must lie one layer
 *     inside that range (-2^(bits-1) < i_j < 2^(bits-1) - 1), so that its face
 *     neighbours have keys; an active cell outside is GBEES_EKEYRANGE.
 *   - Capacity: the pool holds the active cells and their halo (every face
 *     neighbour of an active cell that is not active, kept with p = 0 so that
 *     the update reaches all its stencil cells through links). max_cells
 *     bounds both together; gbees_stats.n_pool reports the current total.
 */
#ifndef GBEES_H
#define GBEES_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GBEES_OK = 0,
    GBEES_EINVAL = -1,      /* bad argument or configuration */
    GBEES_ECAPACITY = -2,   /* more active and halo cells than max_cells (fixed capacity, Sec. 4.1) */
    GBEES_EKEYRANGE = -3,   /* a cell index does not fit the packed key */
    GBEES_EDEGENERATE = -4, /* total probability is zero or not finite (e.g. C = 0 in Eq. 4) */
    GBEES_ECUDA = -5,       /* a CUDA runtime call failed */
    GBEES_ETIMEOUT = -6,    /* a bounded device wait gave up */
    GBEES_ETABLE = -7       /* the hashtable probe sequence found no free slot (Algorithm 2) */
} gbees_status;

/* Drift models f(x) (Sec. 5.1). Parameter layout in gbees_config.params:
 *   GBEES_DYN_CONSTANT          f = (c_1..c_n)                        params[0..n)
 *   GBEES_DYN_LINEAR            f = A x + b, A row-major n x n, then b params[0..n*n+n)
 *   GBEES_DYN_LORENZ63          n = 3, (sigma (y-x), x (rho - z) - y, x y - beta z)
 *                               params = sigma, rho, beta
 *   GBEES_DYN_LORENZ63_SHIFTED  n = 3, the form printed in Sec. 5.1.1:
 *                               (sigma (x2-x1), -x2 - x1 x3, -b x3 + x1 x2 - b r)
 *                               params = sigma, b, r
 *   GBEES_DYN_LORENZ96          n >= 4, f_j = (x_{j+1} - x_{j-2}) x_{j-1} - x_j + F
 *                               (cyclic, Sec. 5.1.2), params = F */
enum {
    GBEES_DYN_CONSTANT = 0,
    GBEES_DYN_LINEAR = 1,
    GBEES_DYN_LORENZ63 = 2,
    GBEES_DYN_LORENZ63_SHIFTED = 3,
    GBEES_DYN_LORENZ96 = 4
};

/* Limiter of the high-resolution correction term (Sec. 2.1). MC is the
 * default; NONE (first order: DCU + CTU only) and LW (phi = 1, Lax-Wendroff)
 * exist for testing. */
enum { GBEES_LIM_MC = 0, GBEES_LIM_NONE = 1, GBEES_LIM_LW = 2 };

/* Storage and flux precision. FP64: everything in double. FP32: probabilities
 * stored and fluxes computed in float; the normalisation sum, the maximum, the
 * CFL reduction, the grow/prune decisions and the likelihood stay in double. */
enum { GBEES_FP64 = 0, GBEES_FP32 = 1 };

typedef struct {
    int32_t n;              /* state dimension, 1..6 */
    int32_t dynamics;       /* GBEES_DYN_* */
    double params[64];      /* model parameters, see above */
    double h[6];            /* cell width per dimension, > 0 */
    double x0[6];           /* centre of cell 0 (grid origin) */
    double thr_rel;         /* a cell is significant when p > thr_rel * max p */
    double cfl;             /* CFL number (dt = cfl / max rate, Eq. 8) */
    int32_t prune_interval; /* prune every K steps (and after every measurement); 0 = only after measurements */
    int32_t precision;      /* GBEES_FP64 | GBEES_FP32 */
    int32_t limiter;        /* GBEES_LIM_* */
    int32_t probe_width;    /* lanes that probe the hashtable together: 1, 2, 4, 8, 16 or 32 (0 = 1) */
    int64_t max_cells;      /* fixed capacity of active plus halo cells (Sec. 4.1) */
    double table_factor;    /* hashtable slots per cell of capacity, >= 1.25 (0 = 2.0, Sec. 4.2) */
    int32_t launch_mode;    /* GBEES_LAUNCH_*: how propagate drives the time steps */
    int32_t storage_order;  /* GBEES_ORDER_*: order of the pool after a prune of a large grid */
    int32_t block_threads;  /* threads per block of the step kernels of the graph and direct launch
                               modes: 64, 128 or 256 (0 = 256) */
    int64_t persist_max_entries; /* AUTO runs the persistent kernel while the pool holds at most this
                                    many entries, the CUDA graph beyond (0 = 2^18) */
} gbees_config;

/* Storage order of the pool entries after a prune of a grid of more than
 * 2^18 entries (smaller grids keep their order; the results never depend on
 * it, only the speed of the neighbour gathers does):
 *   KEY        active cells first, then the halo cells, each in lexicographic
 *              order of the cell indices (dimension 0 slowest), so that the
 *              neighbours of a warp's consecutive cells in any dimension are
 *              consecutive too
 *   MORTON     the same split, each part in Morton (Z-curve) order
 *   NONE       the survivors keep their order (active cells first, then halo)
 *   KEY_MIXED  active and halo cells interleaved in lexicographic order
 *   ROW_MORTON the KEY split, each part with the rows along the last
 *              dimension kept whole (in key order) and the rows in Morton
 *              order of the other indices */
enum {
    GBEES_ORDER_KEY = 0,
    GBEES_ORDER_MORTON = 1,
    GBEES_ORDER_NONE = 2,
    GBEES_ORDER_KEY_MIXED = 3,
    GBEES_ORDER_ROW_MORTON = 4
};

/* Launch modes of gbees_propagate (all give bit-identical results):
 *   AUTO        persistent kernel while the grid is small, CUDA graph beyond
 *   PERSISTENT  one cooperative launch runs many steps, phases separated by
 *               grid barriers (one block per SM)
 *   GRAPH       one CUDA-graph launch runs many steps: a device-side WHILE loop
 *               over the step's kernels, an IF node around the prune
 *   DIRECT      one host launch per kernel (used whenever profiling is on) */
enum { GBEES_LAUNCH_AUTO = 0, GBEES_LAUNCH_PERSISTENT = 1, GBEES_LAUNCH_GRAPH = 2, GBEES_LAUNCH_DIRECT = 3 };

typedef struct {
    int64_t steps;        /* time steps taken by the call */
    int64_t cell_updates; /* sum over those steps of the active cells advanced */
    double t;             /* time reached */
    double last_dt;       /* size of the last step */
    int64_t total_steps;  /* steps since the last init */
    int64_t n_cells;      /* active cells on return */
    double norm;          /* (prod h) * sum of the stored values before the last normalisation */
    int64_t n_pool;       /* active cells plus halo cells on return (what max_cells bounds) */
} gbees_stats;

typedef struct gbees_ctx gbees_ctx;

/* Bytes of device workspace that gbees_create needs for this configuration
 * (cell pools, double buffers, hashtable and scalars). Returns 0 for an
 * invalid configuration. */
size_t gbees_workspace_bytes(const gbees_config* cfg);

/* Create a context on the current CUDA device. d_workspace: device pointer to
 * at least gbees_workspace_bytes(cfg) bytes, 256-byte aligned, owned by the
 * caller and not touched by anyone else until gbees_destroy. cuda_stream: a
 * cudaStream_t (NULL = legacy default stream). On success *out receives the
 * context. The configuration is copied. */
int gbees_create(const gbees_config* cfg, void* d_workspace, size_t workspace_bytes, void* cuda_stream,
                 gbees_ctx** out);

/* Start a new grid from a Gaussian N(mean, cov) sampled at cell centres
 * (the initial PDFs of Sec. 5.1): every cell with p > thr_rel * max p is
 * active, and p is normalised so that (prod h) sum p = 1. mean: n doubles;
 * cov: n x n row-major, symmetric positive definite. t0: initial time. */
int gbees_init_gaussian(gbees_ctx* ctx, const double* mean, const double* cov, double t0);

/* Start a new grid from explicit cells (a checkpoint, or any test set).
 * idx: N x n int32 row-major cell indices, all distinct; p: N densities,
 * taken as given (not renormalised); t0: time; step0: steps already taken
 * (the prune schedule counts from it; 0 for a new run). N may be 0. */
int gbees_init_cells(gbees_ctx* ctx, const int32_t* idx, const double* p, int64_t N, double t0, int64_t step0);

/* Propagate until t == t_end (the grow / step / prune loop of Sec. 3): each
 * step grows the downwind neighbours of the significant cells (Sec. 3.3),
 * takes dt = min(cfl / max_i sum_j |f_j(x_{i-e_j/2})| / h_j, t_end - t) over
 * the active cells (Eq. 8), applies the DCU flux (Eq. 7), the corner-transport
 * corrections (Algorithm 1) and the limited high-resolution correction,
 * prunes every prune_interval steps (Algorithm 3) and normalises. stats may be
 * NULL. t_end <= t takes no step. */
int gbees_propagate(gbees_ctx* ctx, double t_end, gbees_stats* stats);

/* Many independent grids in one launch (batched propagation). ctxs: count
 * contexts with a grid each, all with the dimension, dynamics and precision of
 * ctxs[0] and on the same device; t_end: count target times. One kernel runs
 * on ctxs[0]'s stream with the same phases and arithmetic as gbees_propagate,
 * so every grid ends bit-identical to its own gbees_propagate. When all grids
 * fit on the GPU at once, each grid gets a team of thread blocks in proportion
 * to its work (active cells x remaining time / h, or active cells alone when
 * max_steps > 0; cooperative launch, a barrier per team); otherwise each block takes the next grid from a queue
 * and runs its whole step loop alone. max_steps = 0 runs every grid to its
 * t_end; max_steps > 0 makes one launch in which every grid takes at most
 * max_steps steps (a round of a serving loop: stats[i].t < t_end[i] tells
 * that grid i is not there yet, and the next call continues). d_scratch:
 * device memory of gbees_batch_workspace_bytes(count) bytes, 256-byte
 * aligned, owned by the caller. stats: NULL or count entries. Returns the
 * first error of any grid (that grid's context is poisoned as by
 * gbees_propagate), GBEES_EINVAL for mismatched contexts or a context listed
 * more than once. The contexts must have no work in flight. */
size_t gbees_batch_workspace_bytes(int32_t count);
int gbees_batch_propagate(gbees_ctx* const* ctxs, int32_t count, const double* t_end, int64_t max_steps,
                          void* d_scratch, size_t scratch_bytes, gbees_stats* stats);

/* Blocks of a batched launch whose first context is ctx, at most (0, the
 * default: as many as the GPU holds resident). Batches issued concurrently on
 * different streams (one per model family of a serving loop) share the GPU
 * when each is capped to its part: a team launch is cooperative and waits
 * until all its blocks fit. A batch with more grids than blocks runs in the
 * queue form. max_blocks >= 0. */
int gbees_set_batch_blocks(gbees_ctx* ctx, int32_t max_blocks);

/* Blocks of the persistent step-loop kernel of ctx, at most (0, the default:
 * one per SM). A grid of 10^4 cells has a few cells per block at one block per
 * SM; fewer blocks make each grid barrier cheaper (fewer arrivals) at the cost
 * of more cells per block. The result does not depend on it (sums are exact).
 * max_blocks >= 0. */
int gbees_set_persist_blocks(gbees_ctx* ctx, int32_t max_blocks);

/* Bayesian measurement update (Eq. 4) with the Gaussian likelihood
 * exp(-1/2 (y - x_H)^T R^{-1} (y - x_H)) of m measured components
 * x_H = (x[H_idx[0]], ..., x[H_idx[m-1]]) at the cell centres, followed by a
 * prune and the normalisation (C of Eq. 4). y: m doubles; R: m x m row-major
 * symmetric positive definite; 1 <= m <= n. */
int gbees_correct_gaussian(gbees_ctx* ctx, const double* y, const double* R, const int32_t* H_idx, int32_t m);

/* Number of active cells. */
int gbees_count(gbees_ctx* ctx, int64_t* n_cells);

/* Copy the active cells to host memory: idx (cap x n int32) and p (cap
 * doubles, normalised densities). *n_cells receives the count; when it
 * exceeds cap only cap cells are written and GBEES_EINVAL is returned.
 * sorted != 0 returns the cells in lexicographic index order (dimension 0
 * slowest); otherwise in storage order. */
int gbees_read_cells(gbees_ctx* ctx, int32_t* idx, double* p, int64_t cap, int64_t* n_cells, int32_t sorted);

/* Mean (n doubles) and covariance (n x n row-major) of the grid density:
 * mean = (prod h) sum_i x_i p_i, cov = (prod h) sum_i (x_i - mean)(x_i - mean)^T p_i,
 * both summed exactly. */
int gbees_moments(gbees_ctx* ctx, double* mean, double* cov);

/* Time, step count, cell count and last normaliser without a propagation. */
int gbees_get_stats(gbees_ctx* ctx, gbees_stats* stats);

/* Per-phase timing of the library's own kernels (diagnostics). While enabled,
 * every launch of a phase is bracketed by CUDA events on the context's stream
 * and its duration is added up; launches counts every kernel the library
 * issues, enabled or not. Phases: */
enum {
    GBEES_PHASE_GROW = 0,    /* directional grow (Sec. 3.3) with the waves of the existing entries */
    GBEES_PHASE_HALO = 1,    /* halo cells around the newly active cells */
    GBEES_PHASE_LINK = 2,    /* neighbour links of the new entries, CFL step (Sec. 4.1, Eq. 8) */
    GBEES_PHASE_FACES = 3,   /* face fluxes: DCU + CTU + high-resolution term (Eq. 7, Algorithm 1) */
    GBEES_PHASE_APPLY = 4,   /* conservative update, normalisation partials */
    GBEES_PHASE_PRUNE = 5,   /* mark, status, Morton-order sort (graph and direct launch modes),
                                compaction, relink and rehash (Algorithm 3) */
    GBEES_PHASE_CORRECT = 6, /* Bayesian update (Eq. 4) */
    GBEES_PHASE_OTHER = 7,   /* init, read-out, moments */
    GBEES_NPHASES = 8
};
typedef struct {
    int64_t launches[GBEES_NPHASES]; /* kernel launches per phase since the last reset */
    double ms[GBEES_NPHASES];        /* summed event time per phase (while enabled) */
    int64_t timed[GBEES_NPHASES];    /* launches that were timed */
    int64_t total_launches;          /* all kernel launches since the last reset */
    int64_t fallback_lookups;        /* hashtable lookups of the flux update (0: every stencil cell is linked) */
    /* persistent kernel (GBEES_LAUNCH_PERSISTENT / AUTO): microseconds that its
     * block 0 spent per phase, measured with the SM clock between grid
     * barriers -- grow, halo, link, faces, apply, prune, step scalars, unused --
     * and the steps covered (accumulated since the last init, not reset by
     * reset) */
    double persist_us[8];
    int64_t persist_steps;
    /* every persistent launch (and every batch launch, counted on the batch's
     * first context) bracketed by CUDA events (always, not only while
     * enabled): summed device time, launches, and the cell updates they made */
    double persist_ms;
    int64_t persist_launches;
    int64_t persist_updates;
} gbees_profile;

/* enable != 0 turns event timing on; reset != 0 zeroes the counters. */
int gbees_profile_control(gbees_ctx* ctx, int32_t enable, int32_t reset);
int gbees_profile_read(gbees_ctx* ctx, gbees_profile* out);

/* Bound of the device-side waits of the context's multi-block launches (the
 * grid barriers of the persistent kernel and of a batch's teams): a barrier
 * gives up after `spins` polls of its generation word (2^26 by default, about
 * two seconds), records GBEES_ETIMEOUT in the device scalars and every block
 * leaves the launch; the call then returns GBEES_ETIMEOUT with the context
 * poisoned until the next init, and the device stays usable.
 * extra_arrivals (0 in normal use) makes every grid barrier wait for that
 * many blocks beyond those launched, so that no barrier can complete: a way
 * to exercise the bounded wait and its error path. spins >= 1. */
int gbees_set_wait_limit(gbees_ctx* ctx, int64_t spins, int32_t extra_arrivals);

/* Last error status and message of the context (never NULL). */
int gbees_get_status(gbees_ctx* ctx);
const char* gbees_last_error(gbees_ctx* ctx);

/* Free the host context. The workspace stays the caller's. */
void gbees_destroy(gbees_ctx* ctx);

/* Size of the library's built-in device scratch used by
 * gbees_propagate_cells_noalloc (16 MiB). */
#define GBEES_NOALLOC_SCRATCH_BYTES ((size_t)16 << 20)

/* Propagation without any device allocation by the caller or the library.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot call cudaMalloc -- real-time loops that cannot afford the implicit
 * synchronisation and latency of an allocation, and host applications that
 * own all device memory through their own allocator and forbid side
 * allocations.
 *
 * It does what gbees_create + gbees_init_cells + gbees_propagate +
 * gbees_read_cells(sorted = 0) do, but its workspace is a file-scope device
 * array of GBEES_NOALLOC_SCRATCH_BYTES inside the library, which every GPU
 * that loads the library holds until the process exits. Inputs and outputs
 * are the caller's host buffers, as in those calls: idx (N x n int32), p (N
 * densities, taken as given), t0 and step0 as in gbees_init_cells; t_end as in
 * gbees_propagate; the active cells at t_end are written in storage order to
 * idx_out (cap_out x n) and p_out (cap_out, normalised densities), their count
 * to *n_out; stats may be NULL. cuda_stream: the stream to work on (NULL =
 * legacy default stream).
 *
 * Synchronisation: like the calls it mirrors, it synchronises cuda_stream
 * (it reads the device scalars back between its phases and before it
 * returns), so it must not be called while cuda_stream is being captured
 * into a CUDA graph, nor while any stream is captured in global capture
 * mode. It returns after its work has completed.
 *
 * Errors: GBEES_ECAPACITY when gbees_workspace_bytes(cfg) exceeds
 * GBEES_NOALLOC_SCRATCH_BYTES (use the regular entry points with your own
 * workspace instead), GBEES_EINVAL for bad arguments or more than cap_out
 * result cells (the first cap_out are written), and any status of the
 * calls it mirrors. No context outlives the call, so no error message is kept.
 *
 * The first call on a device looks up the device address of the array on
 * that device (once per device, while it is current) and keeps it for the
 * rest of the process. A device reset (cudaDeviceReset, or any other
 * teardown of the device's primary context) invalidates that address: after
 * one, do not call this entry point again in the same process. Every call
 * on a device uses the same array and the array keeps the last call's
 * contents; each call clears what has to start empty (the scalars and the
 * hashtable) before using it. Calls whose work overlaps on one GPU (other
 * host threads, other streams) race on the array and corrupt each other:
 * serialise them. */
int gbees_propagate_cells_noalloc(const gbees_config* cfg, const int32_t* idx, const double* p, int64_t N,
                                  double t0, int64_t step0, double t_end, void* cuda_stream, int32_t* idx_out,
                                  double* p_out, int64_t cap_out, int64_t* n_out, gbees_stats* stats);

#ifdef __cplusplus
}
#endif

#endif /* GBEES_H */
