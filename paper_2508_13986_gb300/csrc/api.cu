// Host side of the GBEES C ABI (include/gbees.h): configuration checks,
// workspace layout, the per-step launch sequence and the host<->device
// transfers of the public calls. All arithmetic of the method runs in the
// kernels of gbees_kernels.cuh, gbees_phases.cuh and gbees_persistent.cuh.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <numeric>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/gbees.h"
#include "gbees_misc_kernels.cuh"

namespace gbees {
// update_inst.cu, one object per precision and model family
#define GBEES_DECL(p, fam) bool update_kernels_p##p##_f##fam(int n, int dyn, Kernels* k);
GBEES_DECL(64, 0) GBEES_DECL(64, 1) GBEES_DECL(64, 2) GBEES_DECL(64, 3) GBEES_DECL(64, 4) GBEES_DECL(64, 5)
GBEES_DECL(32, 0) GBEES_DECL(32, 1) GBEES_DECL(32, 2) GBEES_DECL(32, 3) GBEES_DECL(32, 4) GBEES_DECL(32, 5)
#undef GBEES_DECL

// The kernels of one time step of a model (before and after the link phase)
// and its persistent step-loop kernel.
bool update_kernels(const Model& m, bool f32, Kernels* k) {
    int fam;
    switch (m.dyn) {
        case DYN_LORENZ63:
        case DYN_LORENZ63_SHIFTED: fam = 0; break;
        case DYN_LORENZ96: fam = 1; break;
        case DYN_LINEAR: fam = m.n <= 3 ? 2 : 3; break;
        default: fam = m.n <= 3 ? 4 : 5; break;
    }
    typedef bool (*Entry)(int, int, Kernels*);
    static const Entry e64[6] = {update_kernels_p64_f0, update_kernels_p64_f1, update_kernels_p64_f2,
                                 update_kernels_p64_f3, update_kernels_p64_f4, update_kernels_p64_f5};
    static const Entry e32[6] = {update_kernels_p32_f0, update_kernels_p32_f1, update_kernels_p32_f2,
                                 update_kernels_p32_f3, update_kernels_p32_f4, update_kernels_p32_f5};
    return (f32 ? e32 : e64)[fam](m.n, m.dyn, k);
}
}  // namespace gbees

using namespace gbees;

struct gbees_ctx {
    gbees_config cfg;
    Model m;
    Bufs b;
    cudaStream_t stream;
    int dev = -1;      // CUDA device of the workspace (-1: not recorded)
    int grid;          // blocks of the fixed launch grid
    int status;        // sticky status
    bool has_grid;     // an init succeeded
    std::string err;
    DevScalars hs;     // host copy of the device scalars
    // diagnostics: per-phase launch counts and event timings
    bool prof_on = false;
    gbees_profile prof{};
    std::vector<cudaEvent_t> ev_pool;
    struct Pending {
        int phase;
        cudaEvent_t a, b;
    };
    std::vector<Pending> pending;
    // the propagate loop as one CUDA graph: a WHILE node over one step, an IF
    // node around the prune (built on first use; direct launches if it fails)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    bool graph_tried = false;
    long long graph_launches = 0;
    // update kernels of the configured model (graph and direct paths) and the
    // persistent step-loop kernel with its cooperative grid size (0: unusable)
    Kernels kern{};
    bool kern_ok = false;
    int persist_grid = 0;
    long long persist_max_cells = 1ll << 18;  // AUTO: persistent kernel up to this many pool entries
    int step_threads = THREADS;                // threads per block of the graph/direct step kernels
    int batch_blocks = 0;  // blocks of a batched launch led by this context at most (0: all resident)
    int persist_blocks = 0;  // blocks of the persistent kernel at most (0: one per SM)
    // blocks of the step kernels of the graph and direct paths: as many as the
    // GPU holds resident for each (SMs x blocks per SM by occupancy), so that one
    // wave covers the grid-stride loops: pre[0..npre), link, post[0..npost)
    int pre_grid[3] = {0, 0, 0}, link_grid = 0, post_grid[3] = {0, 0, 0};
    // device time of every persistent launch (always measured: few launches)
    cudaEvent_t pev[2] = {nullptr, nullptr};
    ~gbees_ctx() {
        for (auto e : pev)
            if (e) cudaEventDestroy(e);
        if (gexec) cudaGraphExecDestroy(gexec);
        if (graph) cudaGraphDestroy(graph);
        for (auto& p : pending) {
            cudaEventDestroy(p.a);
            cudaEventDestroy(p.b);
        }
        for (auto e : ev_pool) cudaEventDestroy(e);
    }
};

namespace {

constexpr size_t ALIGN = 256;

size_t align_up(size_t x) { return (x + ALIGN - 1) / ALIGN * ALIGN; }

struct Layout {
    size_t sc, blk, part, sorthist, key[2], q[2], link[2], om[2], slot[2], u[2], rate[2], keep, map, table, wl, wg,
        tg, fl, total;
    unsigned long long slots;
};

int key_bits_for(int n) { return n == 1 ? 32 : 63 / n; }

bool config_ok(const gbees_config* c, std::string* why) {
    auto fail = [&](const char* s) {
        if (why) *why = s;
        return false;
    };
    if (!c) return fail("null configuration");
    if (c->n < 1 || c->n > 6) return fail("n must be 1..6");
    for (int j = 0; j < c->n; ++j) {
        if (!(c->h[j] > 0.0) || !std::isfinite(c->h[j])) return fail("cell widths must be positive");
        if (!std::isfinite(c->x0[j])) return fail("grid origin must be finite");
    }
    switch (c->dynamics) {
        case GBEES_DYN_CONSTANT:
        case GBEES_DYN_LINEAR:
            break;
        case GBEES_DYN_LORENZ63:
        case GBEES_DYN_LORENZ63_SHIFTED:
            if (c->n != 3) return fail("Lorenz '63 needs n = 3");
            break;
        case GBEES_DYN_LORENZ96:
            if (c->n < 4) return fail("Lorenz '96 needs n >= 4");
            break;
        default:
            return fail("unknown dynamics");
    }
    if (!(c->cfl > 0.0) || !std::isfinite(c->cfl)) return fail("cfl must be positive");
    if (!(c->thr_rel >= 0.0) || !(c->thr_rel < 1.0)) return fail("thr_rel must be in [0, 1)");
    if (c->prune_interval < 0) return fail("prune_interval must be >= 0");
    if (c->precision != GBEES_FP64 && c->precision != GBEES_FP32) return fail("unknown precision");
    if (c->limiter < 0 || c->limiter > 2) return fail("unknown limiter");
    int pw = c->probe_width;
    if (!(pw == 0 || pw == 1 || pw == 2 || pw == 4 || pw == 8 || pw == 16 || pw == 32))
        return fail("probe_width must be 1, 2, 4, 8, 16 or 32");
    if (c->max_cells < 1 || c->max_cells > 0x7fffffffll) return fail("max_cells must be in 1..2^31-1");
    if (!(c->table_factor == 0.0 || c->table_factor >= 1.25)) return fail("table_factor must be 0 or >= 1.25");
    if (c->launch_mode < GBEES_LAUNCH_AUTO || c->launch_mode > GBEES_LAUNCH_DIRECT) return fail("unknown launch_mode");
    if (c->storage_order < GBEES_ORDER_KEY || c->storage_order > GBEES_ORDER_ROW_MORTON)
        return fail("unknown storage_order");
    if (!(c->block_threads == 0 || c->block_threads == 64 || c->block_threads == 128 || c->block_threads == 256))
        return fail("block_threads must be 0, 64, 128 or 256");
    if (c->persist_max_entries < 0) return fail("persist_max_entries must be >= 0");
    return true;
}

bool make_layout(const gbees_config* c, Layout* L) {
    if (!config_ok(c, nullptr)) return false;
    const size_t cap = (size_t)c->max_cells;
    const size_t S = c->precision == GBEES_FP32 ? 4 : 8;
    const double tf = c->table_factor > 0.0 ? c->table_factor : 2.0;
    unsigned long long want = (unsigned long long)std::ceil(tf * (double)cap);
    unsigned long long slots = 64;
    while (slots < want) slots <<= 1;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t at = off;
        off = align_up(off + bytes);
        return at;
    };
    L->sc = take(sizeof(DevScalars));
    L->blk = take(sizeof(long long) * 2 * (GRID_MAX + 1));
    L->part = take(sizeof(Partial) * GRID_MAX);
    L->sorthist = take(sizeof(unsigned int) * 256 * SORT_BLOCKS);
    for (int g = 0; g < 2; ++g) L->key[g] = take(8 * cap);
    for (int g = 0; g < 2; ++g) L->q[g] = take(S * cap);
    for (int g = 0; g < 2; ++g) L->link[g] = take((size_t)4 * 2 * c->n * std::max<size_t>(cap, 1));
    for (int g = 0; g < 2; ++g) L->om[g] = take(2 * cap);
    for (int g = 0; g < 2; ++g) L->slot[g] = take(4 * cap);
    L->keep = take(cap);
    L->map = take(4 * cap);
    L->table = take(sizeof(Slot) * slots);
    // face velocities (two generations) and the scratch of the three-pass
    // update, storage type, n values per entry (one for tg)
    const size_t rows = S * (size_t)c->n * cap;
    for (int g = 0; g < 2; ++g) L->u[g] = take(rows);
    for (int g = 0; g < 2; ++g) L->rate[g] = take(8 * cap);
    L->wl = take(rows);
    L->wg = take(rows);
    L->tg = take(S * cap);
    L->fl = take(rows);
    L->total = off;
    L->slots = slots;
    return true;
}

// The model constants and the buffer pointers of a context over a workspace
// laid out by make_layout.
void bind_context(gbees_ctx* ctx, const gbees_config* cfg, const Layout& L, void* workspace, cudaStream_t stream) {
    ctx->cfg = *cfg;
    ctx->stream = stream;
    ctx->status = GBEES_OK;
    ctx->has_grid = false;
    Model& m = ctx->m;
    std::memset(&m, 0, sizeof m);
    m.n = cfg->n;
    m.dyn = cfg->dynamics;
    m.limiter = cfg->limiter;
    m.key_bits = key_bits_for(cfg->n);
    m.prune_interval = cfg->prune_interval;
    m.probe_width = cfg->probe_width ? cfg->probe_width : 1;
    m.sort_order = cfg->storage_order;
    m.bar_extra = 0;
    m.spin_limit = BARRIER_SPIN_LIMIT;
    m.cap = cfg->max_cells;
    m.tmask = L.slots - 1;
    std::memcpy(m.a, cfg->params, sizeof m.a);
    m.prod_h = 1.0;
    for (int j = 0; j < cfg->n; ++j) {
        m.h[j] = cfg->h[j];
        m.x0[j] = cfg->x0[j];
        m.prod_h *= cfg->h[j];
    }
    m.thr_rel = cfg->thr_rel;
    m.cfl = cfg->cfl;
    m.h_pow2 = 0;
    for (int j = 0; j < cfg->n; ++j) {
        m.inv_h[j] = 1.0 / cfg->h[j];
        m.inv_2h[j] = 1.0 / (2.0 * cfg->h[j]);
        int ex = 0;
        if (std::frexp(cfg->h[j], &ex) == 0.5 && std::isnormal(m.inv_h[j])) m.h_pow2 |= 1 << j;
        m.hf[j] = (float)cfg->h[j];
        m.x0f[j] = (float)cfg->x0[j];
    }
    for (int i = 0; i < 48; ++i) m.af[i] = (float)cfg->params[i];
    char* base = (char*)workspace;
    Bufs& b = ctx->b;
    b.sc = (DevScalars*)(base + L.sc);
    b.blk = (long long*)(base + L.blk);
    b.blk2 = b.blk + (GRID_MAX + 1);
    b.part = (Partial*)(base + L.part);
    b.sorthist = (unsigned int*)(base + L.sorthist);
    for (int g = 0; g < 2; ++g) {
        b.key[g] = (unsigned long long*)(base + L.key[g]);
        b.q[g] = (void*)(base + L.q[g]);
        b.link[g] = (int*)(base + L.link[g]);
        b.om[g] = (unsigned short*)(base + L.om[g]);
        b.slot[g] = (unsigned int*)(base + L.slot[g]);
    }
    b.keep = (unsigned char*)(base + L.keep);
    b.map = (int*)(base + L.map);
    b.table = (Slot*)(base + L.table);
    for (int g = 0; g < 2; ++g) b.u[g] = (void*)(base + L.u[g]);
    for (int g = 0; g < 2; ++g) b.rate[g] = (double*)(base + L.rate[g]);
    b.wl = (void*)(base + L.wl);
    b.wg = (void*)(base + L.wg);
    b.tg = (void*)(base + L.tg);
    b.fl = (void*)(base + L.fl);
    ctx->step_threads = cfg->block_threads > 0 ? cfg->block_threads : THREADS;
    ctx->persist_max_cells = cfg->persist_max_entries > 0 ? cfg->persist_max_entries : (1ll << 18);
}

void set_err(gbees_ctx* ctx, int st, const std::string& msg) {
    if (ctx->status == GBEES_OK || st == GBEES_OK) ctx->status = st;
    ctx->err = msg;
}

const char* status_text(int st) {
    switch (st) {
        case GBEES_OK: return "ok";
        case GBEES_EINVAL: return "invalid argument";
        case GBEES_ECAPACITY: return "cell capacity exceeded (max_cells)";
        case GBEES_EKEYRANGE: return "cell index outside the packed-key range";
        case GBEES_EDEGENERATE: return "total probability is zero or not finite";
        case GBEES_ECUDA: return "CUDA error";
        case GBEES_ETIMEOUT: return "device wait timed out";
        case GBEES_ETABLE: return "hashtable full";
    }
    return "unknown status";
}

bool cuda_ok(gbees_ctx* ctx, cudaError_t e, const char* where) {
    if (e == cudaSuccess) return true;
    set_err(ctx, GBEES_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
    return false;
}

cudaEvent_t take_event(gbees_ctx* ctx) {
    if (!ctx->ev_pool.empty()) {
        cudaEvent_t e = ctx->ev_pool.back();
        ctx->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

// Brackets the kernels of one phase: counts them and, when profiling is on,
// times them with a pair of events on the context's stream.
struct Phase {
    gbees_ctx* ctx;
    int phase;
    int kernels;
    cudaEvent_t a = nullptr;
    Phase(gbees_ctx* c, int ph, int nk) : ctx(c), phase(ph), kernels(nk) {
        if (ctx->prof_on && (a = take_event(ctx))) cudaEventRecord(a, ctx->stream);
    }
    ~Phase() {
        ctx->prof.launches[phase] += kernels;
        ctx->prof.total_launches += kernels;
        if (a) {
            cudaEvent_t b = take_event(ctx);
            if (b) {
                cudaEventRecord(b, ctx->stream);
                ctx->pending.push_back({phase, a, b});
            } else {
                ctx->ev_pool.push_back(a);
            }
        }
    }
};

// Add up the timed phases whose events have completed (after a stream sync).
void drain_events(gbees_ctx* ctx) {
    for (auto& p : ctx->pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            ctx->prof.ms[p.phase] += ms;
            ctx->prof.timed[p.phase] += 1;
        }
        ctx->ev_pool.push_back(p.a);
        ctx->ev_pool.push_back(p.b);
    }
    ctx->pending.clear();
}

// Copy the device scalars back and fold a device error into the status.
bool sync_scalars(gbees_ctx* ctx, const char* where) {
    if (!cuda_ok(ctx, cudaGetLastError(), where)) return false;
    if (!cuda_ok(ctx, cudaMemcpyAsync(&ctx->hs, ctx->b.sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, ctx->stream),
                 where))
        return false;
    if (!cuda_ok(ctx, cudaStreamSynchronize(ctx->stream), where)) return false;
    drain_events(ctx);
    ctx->prof.fallback_lookups = ctx->hs.lookups_fallback;
    if (ctx->hs.error) {
        set_err(ctx, ctx->hs.error, std::string(where) + ": " + status_text(ctx->hs.error));
        return false;
    }
    return true;
}

// Kernels of a context must run on the device of its workspace: a call made
// while another device is current is refused (the context stays usable).
bool on_ctx_device(gbees_ctx* ctx) {
    if (ctx->dev < 0) return true;
    int cur = -1;
    if (cudaGetDevice(&cur) == cudaSuccess && cur == ctx->dev) return true;
    ctx->err = "the current CUDA device is not the device of the context's workspace";
    return false;
}

int guard(gbees_ctx* ctx, bool need_grid) {
    if (!ctx) return GBEES_EINVAL;
    if (ctx->status != GBEES_OK) return ctx->status;
    if (!on_ctx_device(ctx)) return GBEES_EINVAL;
    if (need_grid && !ctx->has_grid) {
        ctx->err = "no grid: call gbees_init_gaussian or gbees_init_cells first";
        return GBEES_EINVAL;
    }
    return GBEES_OK;
}

// Run f(N, T) for the configured dimension and precision.
template <typename F>
void with_nt(const gbees_ctx* ctx, F&& f) {
    const bool f32 = ctx->cfg.precision == GBEES_FP32;
    switch (ctx->cfg.n) {
#define GBEES_CASE(NN)                                                  \
    case NN:                                                            \
        if (f32) f(std::integral_constant<int, NN>{}, float{});        \
        else f(std::integral_constant<int, NN>{}, double{});           \
        break;
        GBEES_CASE(1)
        GBEES_CASE(2)
        GBEES_CASE(3)
        GBEES_CASE(4)
        GBEES_CASE(5)
        GBEES_CASE(6)
#undef GBEES_CASE
    }
}

template <int N, typename T>
void* link_kernel(int probe_width) {
    switch (probe_width) {
        case 2: return (void*)k_link<N, 2, T>;
        case 4: return (void*)k_link<N, 4, T>;
        case 8: return (void*)k_link<N, 8, T>;
        case 16: return (void*)k_link<N, 16, T>;
        case 32: return (void*)k_link<N, 32, T>;
        default: return (void*)k_link<N, 1, T>;
    }
}

// step != 0: the link of a time step (its last block also fixes dt).
template <int N, typename T>
void launch_link(gbees_ctx* ctx, int step) {
    void* args[] = {&ctx->m, &ctx->b, &step};
    const int G = ctx->link_grid > 0 ? ctx->link_grid : ctx->grid;
    cudaLaunchKernel(link_kernel<N, T>(ctx->m.probe_width), dim3(G), dim3(ctx->step_threads), args, 0, ctx->stream);
}

// Blocks of a step kernel f: one resident wave (SMs x blocks per SM); with
// at_least_fixed, at least the context's fixed grid (the hashtable probes of
// the link phase, latency-bound with few resident blocks, gain from a second
// wave that overlaps the first one's tail; measured on the 6-D grid).
int resident_grid(gbees_ctx* ctx, const void* f, int sms, bool at_least_fixed = false) {
    int per_sm = 0;
    const int bt = ctx->step_threads;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, bt, 0) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        return ctx->grid * (THREADS / bt);
    }
    const int wave = sms * per_sm;
    // the fixed grid holds the same threads whatever the block size
    return std::min(GRID_MAX, at_least_fixed ? std::max(ctx->grid * (THREADS / bt), wave) : wave);
}

void resolve_update_kernels(gbees_ctx* ctx) {
    if (ctx->kern_ok) return;
    ctx->kern_ok = update_kernels(ctx->m, ctx->cfg.precision == GBEES_FP32, &ctx->kern);
    int dev = 0, sms = 0, per_sm = 0;
    if (ctx->kern_ok && cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ctx->kern.persist, THREADS, 0) == cudaSuccess &&
            per_sm >= 1)
            ctx->persist_grid = std::min(GRID_MAX, sms);
        for (int i = 0; i < ctx->kern.npre; ++i) ctx->pre_grid[i] = resident_grid(ctx, ctx->kern.pre[i], sms);
        for (int i = 0; i < ctx->kern.npost; ++i) ctx->post_grid[i] = resident_grid(ctx, ctx->kern.post[i], sms);
        with_nt(ctx, [&](auto NN, auto TT) {
            constexpr int N = decltype(NN)::value;
            ctx->link_grid = resident_grid(ctx, link_kernel<N, decltype(TT)>(ctx->m.probe_width), sms, true);
        });
    }
    cudaGetLastError();
}

void launch_list(gbees_ctx* ctx, void* const* f, const int* grids, int nf) {
    void* args[] = {&ctx->m, &ctx->b};
    for (int i = 0; i < nf; ++i) {
        const int G = grids[i] > 0 ? grids[i] : ctx->grid;
        cudaLaunchKernel(f[i], dim3(G), dim3(ctx->step_threads), args, 0, ctx->stream);
    }
}

// The prune of Algorithm 3 (directional marking, status, compaction, relink,
// rehash). It runs only when the device flag prune_now is set. A large grid's
// survivors are sorted into the configured storage order (key or Morton order
// of the cell indices), which keeps the neighbour gathers of a sweep close
// together; a grid that fits in L2 keeps its order (stream compaction).
constexpr int kSortPasses = 8;                          // 8-bit digits of the 64-bit sort key
constexpr int kPruneKernelsSorted = 3 + 1 + 3 * kSortPasses + 1 + 2;
constexpr int kPruneKernelsPlain = 3 + 1 + 1;
constexpr long long kSortMinEntries = 1ll << 18;        // smaller pools are not sorted

bool sorts(const gbees_ctx* ctx) { return ctx->cfg.storage_order != GBEES_ORDER_NONE; }

// Blocks of the sort kernels for a pool of N entries: about 16 tiles of
// THREADS entries per block, at most SORT_BLOCKS.
int sort_blocks(long long N) {
    const long long per = (long long)THREADS * 16;
    return (int)std::max(1ll, std::min<long long>(SORT_BLOCKS, (N + per - 1) / per));
}

void launch_prune(gbees_ctx* ctx) {
    const int G = ctx->grid;
    cudaStream_t s = ctx->stream;
    // the host's copy of the pool size (possibly a few steps old: it only
    // decides the storage order, which no result depends on)
    const long long N = ctx->hs.N;
    const bool sorted = sorts(ctx) && N > kSortMinEntries;
    const int Gs = sort_blocks(N);
    Phase ph(ctx, GBEES_PHASE_PRUNE, sorted ? kPruneKernelsSorted : kPruneKernelsPlain);
    with_nt(ctx, [&](auto NN, auto TT) {
        constexpr int N = decltype(NN)::value;
        using T = decltype(TT);
        k_prune_mark<T><<<G, THREADS, 0, s>>>(ctx->m, ctx->b);
        k_prune_scatter<N, T><<<G, THREADS, 0, s>>>(ctx->m, ctx->b);
        k_prune_count<N><<<G, THREADS, 0, s>>>(ctx->m, ctx->b);
        if (sorted) {
            k_sort_init<<<G, THREADS, 0, s>>>(ctx->m, ctx->b);
            for (int pass = 0; pass < kSortPasses; ++pass) {
                k_sort_hist<<<Gs, THREADS, 0, s>>>(ctx->m, ctx->b, pass & 1, 8 * pass);
                k_sort_scan<<<1, SCAN_THREADS, 0, s>>>(ctx->m, ctx->b, Gs);
                k_sort_scatter<<<Gs, THREADS, 0, s>>>(ctx->m, ctx->b, pass & 1, 8 * pass);
            }
            k_sort_map<<<G, THREADS, 0, s>>>(ctx->m, ctx->b);
            k_prune_compact_sorted<N, T><<<G, THREADS, 0, s>>>(ctx->m, ctx->b);
        } else {
            k_prune_compact<N, T><<<G, THREADS, 0, s>>>(ctx->m, ctx->b);
        }
        k_prune_relink<N><<<G, THREADS, 0, s>>>(ctx->m, ctx->b, G);
    });
}

// The active cells (indices, densities) into d_idx / d_p in storage order.
void launch_readout(gbees_ctx* ctx, int* d_idx, double* d_p) {
    const int G = ctx->grid;
    cudaStream_t s = ctx->stream;
    k_readout_count<<<G, THREADS, 0, s>>>(ctx->m, ctx->b);
    k_scan_blocks<<<1, THREADS, 0, s>>>(ctx->b, G, ctx->m.cap);
    with_nt(ctx, [&](auto NN, auto TT) {
        constexpr int NC = decltype(NN)::value;
        using T = decltype(TT);
        k_readout<NC, T><<<G, THREADS, 0, s>>>(ctx->m, ctx->b, d_idx, d_p);
    });
}

// One time step: grow, halo, link the new entries, flux update (the last block of the
// update advances t and decides whether a prune is due).
void launch_step(gbees_ctx* ctx) {
    resolve_update_kernels(ctx);
    {
        Phase ph(ctx, GBEES_PHASE_GROW, 2);
        launch_list(ctx, ctx->kern.pre, ctx->pre_grid, 2);
    }
    {
        Phase ph(ctx, GBEES_PHASE_HALO, 1);
        launch_list(ctx, ctx->kern.pre + 2, ctx->pre_grid + 2, 1);
    }
    {
        Phase ph(ctx, GBEES_PHASE_LINK, 1);
        with_nt(ctx, [&](auto NN, auto TT) {
            constexpr int N = decltype(NN)::value;
            launch_link<N, decltype(TT)>(ctx, 1);
        });
    }
    {
        Phase ph(ctx, GBEES_PHASE_FACES, 1);
        launch_list(ctx, ctx->kern.post, ctx->post_grid, 1);
    }
    Phase ph(ctx, GBEES_PHASE_APPLY, 1);
    launch_list(ctx, ctx->kern.post + 1, ctx->post_grid + 1, 1);
}

// ---- the step loop as a CUDA graph

constexpr long long kGraphMaxIter = 1ll << 16;  // steps per graph launch at most
constexpr long long kPersistSteps = 1ll << 13;  // steps per persistent launch at most

struct GraphBuilder {
    cudaGraph_t g;
    cudaError_t err = cudaSuccess;
    cudaGraphNode_t add(cudaGraph_t into, cudaGraphNode_t prev, void* func, int grid, int block, void** args) {
        cudaKernelNodeParams p{};
        p.func = func;
        p.gridDim = dim3(grid);
        p.blockDim = dim3(block);
        p.sharedMemBytes = 0;
        p.kernelParams = args;
        p.extra = nullptr;
        cudaGraphNode_t node = nullptr;
        if (err == cudaSuccess) err = cudaGraphAddKernelNode(&node, into, prev ? &prev : nullptr, prev ? 1 : 0, &p);
        return node;
    }
    cudaGraphNode_t cond(cudaGraph_t into, cudaGraphNode_t prev, cudaGraphConditionalHandle h,
                         cudaGraphConditionalNodeType type, cudaGraph_t* body) {
        cudaGraphNodeParams p{};
        p.type = cudaGraphNodeTypeConditional;
        p.conditional.handle = h;
        p.conditional.type = type;
        p.conditional.size = 1;
        cudaGraphNode_t node = nullptr;
        if (err == cudaSuccess) err = cudaGraphAddNode(&node, into, prev ? &prev : nullptr, nullptr, prev ? 1 : 0, &p);
        if (err == cudaSuccess) *body = p.conditional.phGraph_out[0];
        return node;
    }
};

template <int N, typename T>
void graph_nodes(gbees_ctx* ctx, GraphBuilder& gb, cudaGraph_t body, cudaGraphConditionalHandle hw,
                 cudaGraphConditionalHandle hp) {
    const int G = ctx->grid;
    Model* m = &ctx->m;
    Bufs* b = &ctx->b;
    void* mb[] = {m, b};
    int one = 1;
    void* link_args[] = {m, b, &one};
    resolve_update_kernels(ctx);
    cudaGraphNode_t n = nullptr;
    auto grid_or = [&](int g) { return g > 0 ? g : G; };
    const int bt = ctx->step_threads;
    for (int i = 0; i < ctx->kern.npre; ++i) n = gb.add(body, n, ctx->kern.pre[i], grid_or(ctx->pre_grid[i]), bt, mb);
    n = gb.add(body, n, link_kernel<N, T>(ctx->m.probe_width), grid_or(ctx->link_grid), bt, link_args);
    for (int i = 0; i < ctx->kern.npost; ++i)
        n = gb.add(body, n, ctx->kern.post[i], grid_or(ctx->post_grid[i]), bt, mb);
    DevScalars* sc = ctx->b.sc;
    long long maxit = kGraphMaxIter;
    int step_kernels = ctx->kern.npre + 1 + ctx->kern.npost + 1;
    int prune_kernels = sorts(ctx) ? kPruneKernelsSorted : kPruneKernelsPlain;
    void* ctl_args[] = {&sc, &hw, &hp, &maxit, &step_kernels, &prune_kernels};
    n = gb.add(body, n, (void*)k_loop_ctl, 1, 1, ctl_args);
    cudaGraph_t pb = nullptr;
    gb.cond(body, n, hp, cudaGraphCondTypeIf, &pb);
    if (gb.err != cudaSuccess) return;
    int nblk = G;
    void* relink_args[] = {m, b, &nblk};
    const int Gs = std::min(G, SORT_BLOCKS);
    static int srcs[2] = {0, 1};
    static int shifts[kSortPasses] = {0, 8, 16, 24, 32, 40, 48, 56};
    static int nsort = 0;
    nsort = Gs;
    cudaGraphNode_t q = gb.add(pb, nullptr, (void*)k_prune_mark<T>, G, THREADS, mb);
    q = gb.add(pb, q, (void*)k_prune_scatter<N, T>, G, THREADS, mb);
    q = gb.add(pb, q, (void*)k_prune_count<N>, G, THREADS, mb);
    if (sorts(ctx)) {
        q = gb.add(pb, q, (void*)k_sort_init, G, THREADS, mb);
        for (int pass = 0; pass < kSortPasses; ++pass) {
            void* pass_args[] = {m, b, &srcs[pass & 1], &shifts[pass]};
            void* scan_args[] = {m, b, &nsort};
            q = gb.add(pb, q, (void*)k_sort_hist, Gs, THREADS, pass_args);
            q = gb.add(pb, q, (void*)k_sort_scan, 1, SCAN_THREADS, scan_args);
            q = gb.add(pb, q, (void*)k_sort_scatter, Gs, THREADS, pass_args);
        }
        q = gb.add(pb, q, (void*)k_sort_map, G, THREADS, mb);
        q = gb.add(pb, q, (void*)k_prune_compact_sorted<N, T>, G, THREADS, mb);
    } else {
        q = gb.add(pb, q, (void*)k_prune_compact<N, T>, G, THREADS, mb);
    }
    gb.add(pb, q, (void*)k_prune_relink<N>, G, THREADS, relink_args);
}

// Build and instantiate the step-loop graph of this context. False if the
// runtime cannot (the caller then launches kernel by kernel).
bool build_step_graph(gbees_ctx* ctx) {
    ctx->graph_tried = true;
    GraphBuilder gb;
    if (cudaGraphCreate(&gb.g, 0) != cudaSuccess) return false;
    cudaGraphConditionalHandle hw = 0, hp = 0;
    if (cudaGraphConditionalHandleCreate(&hw, gb.g, 1, cudaGraphCondAssignDefault) != cudaSuccess ||
        cudaGraphConditionalHandleCreate(&hp, gb.g, 0, cudaGraphCondAssignDefault) != cudaSuccess) {
        cudaGraphDestroy(gb.g);
        cudaGetLastError();
        return false;
    }
    DevScalars* sc = ctx->b.sc;
    void* reset_args[] = {&sc};
    cudaGraphNode_t r = gb.add(gb.g, nullptr, (void*)k_loop_reset, 1, 1, reset_args);
    cudaGraph_t body = nullptr;
    gb.cond(gb.g, r, hw, cudaGraphCondTypeWhile, &body);
    if (gb.err == cudaSuccess) {
        with_nt(ctx, [&](auto NN, auto TT) {
            constexpr int N = decltype(NN)::value;
            using T = decltype(TT);
            graph_nodes<N, T>(ctx, gb, body, hw, hp);
        });
    }
    cudaGraphExec_t exec = nullptr;
    if (gb.err == cudaSuccess) gb.err = cudaGraphInstantiate(&exec, gb.g, 0);
    if (gb.err != cudaSuccess) {
        cudaGraphDestroy(gb.g);
        cudaGetLastError();
        return false;
    }
    ctx->graph = gb.g;
    ctx->gexec = exec;
    return true;
}

// Inverse of a small symmetric positive definite matrix (Cholesky factor,
// then the inverse of the factor). Returns false if not positive definite.
bool spd_inverse(int m, const double* A, double* Ainv) {
    double L[36] = {0}, Li[36] = {0};
    for (int i = 0; i < m; ++i) {
        for (int j = 0; j <= i; ++j) {
            double s = A[i * m + j];
            for (int k = 0; k < j; ++k) s -= L[i * m + k] * L[j * m + k];
            if (i == j) {
                if (!(s > 0.0)) return false;
                L[i * m + i] = std::sqrt(s);
            } else {
                L[i * m + j] = s / L[j * m + j];
            }
        }
    }
    for (int i = 0; i < m; ++i) {
        Li[i * m + i] = 1.0 / L[i * m + i];
        for (int j = 0; j < i; ++j) {
            double s = 0.0;
            for (int k = j; k < i; ++k) s -= L[i * m + k] * Li[k * m + j];
            Li[i * m + j] = s / L[i * m + i];
        }
    }
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) {
            double s = 0.0;
            for (int k = std::max(i, j); k < m; ++k) s += Li[k * m + i] * Li[k * m + j];
            Ainv[i * m + j] = s;
        }
    return true;
}

bool box_for(const gbees_ctx* ctx, const double* mean, const double* cov, double r2, InitBox* bx) {
    const int n = ctx->cfg.n;
    long long total = 1;
    for (int k = 0; k < n; ++k) {
        double ctr = std::round((mean[k] - ctx->cfg.x0[k]) / ctx->cfg.h[k]);
        double hw = std::ceil(std::sqrt(r2 * cov[k * n + k]) / ctx->cfg.h[k]) + 1.0;
        if (!std::isfinite(ctr) || !std::isfinite(hw) || std::fabs(ctr) + hw > 2.0e9) return false;
        bx->lo[k] = (int)(ctr - hw);
        bx->dims[k] = (long long)(2.0 * hw + 1.0);
        if (total > (1ll << 42) / bx->dims[k]) return false;
        total *= bx->dims[k];
    }
    bx->total = total;
    return true;
}

}  // namespace

extern "C" {

size_t gbees_workspace_bytes(const gbees_config* cfg) {
    Layout L;
    if (!make_layout(cfg, &L)) return 0;
    return L.total;
}

int gbees_create(const gbees_config* cfg, void* d_workspace, size_t workspace_bytes, void* cuda_stream,
                 gbees_ctx** out) {
    if (!out) return GBEES_EINVAL;
    *out = nullptr;
    std::string why;
    if (!config_ok(cfg, &why)) return GBEES_EINVAL;
    Layout L;
    make_layout(cfg, &L);
    if (!d_workspace || workspace_bytes < L.total || ((uintptr_t)d_workspace % ALIGN) != 0) return GBEES_EINVAL;
    gbees_ctx* ctx = new gbees_ctx();
    bind_context(ctx, cfg, L, d_workspace, (cudaStream_t)cuda_stream);
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        delete ctx;
        return GBEES_ECUDA;
    }
    ctx->dev = dev;
    ctx->grid = std::min(GRID_MAX, std::max(1, sms * 4));
    k_reset<<<1, 1, 0, ctx->stream>>>(ctx->b.sc, 0.0);
    if (!sync_scalars(ctx, "create")) {
        int st = ctx->status;
        delete ctx;
        return st;
    }
    *out = ctx;
    return GBEES_OK;
}

void gbees_destroy(gbees_ctx* ctx) { delete ctx; }

int gbees_profile_control(gbees_ctx* ctx, int32_t enable, int32_t reset) {
    if (!ctx) return GBEES_EINVAL;
    if (ctx->prof_on && !enable) {
        cudaStreamSynchronize(ctx->stream);
        drain_events(ctx);
    }
    ctx->prof_on = enable != 0;
    if (reset) {
        cudaStreamSynchronize(ctx->stream);
        drain_events(ctx);
        ctx->prof = gbees_profile{};
    }
    return GBEES_OK;
}

int gbees_profile_read(gbees_ctx* ctx, gbees_profile* out) {
    if (!ctx || !out) return GBEES_EINVAL;
    cudaStreamSynchronize(ctx->stream);
    drain_events(ctx);
    *out = ctx->prof;
    DevScalars hs;
    if (cudaMemcpy(&hs, ctx->b.sc, sizeof(DevScalars), cudaMemcpyDeviceToHost) == cudaSuccess) {
        int dev = 0, khz = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev);
        const double per_us = khz > 0 ? khz / 1e3 : 1.0;
        for (int q = 0; q < 8; ++q) out->persist_us[q] = hs.phase_cycles[q] / per_us;
        out->persist_steps = hs.phase_steps;
    }
    cudaGetLastError();
    return GBEES_OK;
}

int gbees_set_batch_blocks(gbees_ctx* ctx, int32_t max_blocks) {
    if (!ctx || max_blocks < 0) return GBEES_EINVAL;
    ctx->batch_blocks = max_blocks;
    return GBEES_OK;
}

int gbees_set_persist_blocks(gbees_ctx* ctx, int32_t max_blocks) {
    if (!ctx || max_blocks < 0) return GBEES_EINVAL;
    ctx->persist_blocks = max_blocks;
    return GBEES_OK;
}

int gbees_set_wait_limit(gbees_ctx* ctx, int64_t spins, int32_t extra_arrivals) {
    if (!ctx || spins < 1 || extra_arrivals < 0 || extra_arrivals > GRID_MAX) return GBEES_EINVAL;
    ctx->m.spin_limit = spins;
    ctx->m.bar_extra = extra_arrivals;
    return GBEES_OK;
}

int gbees_get_status(gbees_ctx* ctx) { return ctx ? ctx->status : GBEES_EINVAL; }

const char* gbees_last_error(gbees_ctx* ctx) {
    if (!ctx) return "null context";
    return ctx->err.c_str();
}

int gbees_init_gaussian(gbees_ctx* ctx, const double* mean, const double* cov, double t0) {
    if (!ctx) return GBEES_EINVAL;
    if (!on_ctx_device(ctx)) return GBEES_EINVAL;
    if (ctx->status != GBEES_OK && ctx->status != GBEES_ECUDA) {  // a new grid clears a poisoned state
        ctx->status = GBEES_OK;
        ctx->err.clear();
    }
    if (ctx->status != GBEES_OK) return ctx->status;
    ctx->has_grid = false;
    const int n = ctx->cfg.n;
    if (!mean || !cov || !std::isfinite(t0)) {
        ctx->err = "null mean or covariance";
        return GBEES_EINVAL;
    }
    InitBox bx;
    std::memset(&bx, 0, sizeof bx);
    for (int k = 0; k < n; ++k) bx.mean[k] = mean[k];
    if (!spd_inverse(n, cov, bx.icov)) {
        ctx->err = "covariance is not symmetric positive definite";
        return GBEES_EINVAL;
    }
    const double thr = ctx->cfg.thr_rel > 0.0 ? ctx->cfg.thr_rel : 1e-300;
    if (!box_for(ctx, mean, cov, -2.0 * std::log(thr), &bx)) {
        ctx->err = "initial box too large";
        return GBEES_EINVAL;
    }
    const int G = ctx->grid;
    cudaStream_t s = ctx->stream;
    {
        Phase ph(ctx, GBEES_PHASE_OTHER, 3);
        k_reset<<<1, 1, 0, s>>>(ctx->b.sc, t0);
        k_table_clear<<<G, THREADS, 0, s>>>(ctx->m, ctx->b);
        with_nt(ctx, [&](auto NN, auto) {
            constexpr int N = decltype(NN)::value;
            k_init_max<N><<<G, THREADS, 0, s>>>(ctx->m, ctx->b, bx);
        });
    }
    if (!sync_scalars(ctx, "init_gaussian")) return ctx->status;
    unsigned long long ordk = ctx->hs.tmp_ord;
    double gmax = 0.0;
    if (ordk) {
        unsigned long long bits = (ordk >> 63) ? (ordk & 0x7FFFFFFFFFFFFFFFull) : ~ordk;
        std::memcpy(&gmax, &bits, 8);
    }
    if (!(gmax > 0.0)) {
        set_err(ctx, GBEES_EDEGENERATE, "initial density underflows on the grid");
        return ctx->status;
    }
    bx.pstar = ctx->cfg.thr_rel * gmax;
    if (!box_for(ctx, mean, cov, -2.0 * std::log(thr * gmax), &bx)) {
        ctx->err = "initial box too large";
        return GBEES_EINVAL;
    }
    {
        Phase ph(ctx, GBEES_PHASE_OTHER, 7);
        with_nt(ctx, [&](auto NN, auto TT) {
            constexpr int N = decltype(NN)::value;
            using T = decltype(TT);
            k_init_count<N><<<G, THREADS, 0, s>>>(ctx->m, ctx->b, bx);
            k_scan_blocks<<<1, THREADS, 0, s>>>(ctx->b, G, ctx->m.cap);
            k_init_write<N, T><<<G, THREADS, 0, s>>>(ctx->m, ctx->b, bx);
        });
        k_set_count_from_new<<<1, 1, 0, s>>>(ctx->b.sc);
        with_nt(ctx, [&](auto NN, auto TT) {
            constexpr int N = decltype(NN)::value;
            using T = decltype(TT);
            k_halo<N, T, 0><<<G, THREADS, 0, s>>>(ctx->m, ctx->b);
            launch_link<N, T>(ctx, 0);
        });
        k_finalise<<<1, 1, 0, s>>>(ctx->m, ctx->b.sc, 0);
    }
    if (!sync_scalars(ctx, "init_gaussian")) return ctx->status;
    ctx->has_grid = true;
    return GBEES_OK;
}

int gbees_init_cells(gbees_ctx* ctx, const int32_t* idx, const double* p, int64_t N, double t0, int64_t step0) {
    if (!ctx) return GBEES_EINVAL;
    if (!on_ctx_device(ctx)) return GBEES_EINVAL;
    if (ctx->status != GBEES_OK && ctx->status != GBEES_ECUDA) {
        ctx->status = GBEES_OK;
        ctx->err.clear();
    }
    if (ctx->status != GBEES_OK) return ctx->status;
    ctx->has_grid = false;
    const int n = ctx->cfg.n;
    if (N < 0 || N > ctx->m.cap || (N > 0 && (!idx || !p)) || !std::isfinite(t0) || step0 < 0) {
        ctx->err = "bad cell list (count above max_cells or null pointers)";
        return GBEES_EINVAL;
    }
    cudaStream_t s = ctx->stream;
    const int G = ctx->grid;
    Phase ph(ctx, GBEES_PHASE_OTHER, N > 0 ? 7 : 6);
    k_reset<<<1, 1, 0, s>>>(ctx->b.sc, t0);
    k_table_clear<<<G, THREADS, 0, s>>>(ctx->m, ctx->b);
    // stage the inputs in the second buffer set (unused outside a prune)
    int* d_idx = ctx->b.link[1];
    double* d_p = reinterpret_cast<double*>(ctx->b.key[1]);
    if (N > 0) {
        if (!cuda_ok(ctx, cudaMemcpyAsync(d_idx, idx, sizeof(int32_t) * n * N, cudaMemcpyHostToDevice, s), "init_cells"))
            return ctx->status;
        if (!cuda_ok(ctx, cudaMemcpyAsync(d_p, p, sizeof(double) * N, cudaMemcpyHostToDevice, s), "init_cells"))
            return ctx->status;
    }
    with_nt(ctx, [&](auto NN, auto TT) {
        constexpr int NC = decltype(NN)::value;
        using T = decltype(TT);
        if (N > 0) k_init_cells<NC, T><<<G, THREADS, 0, s>>>(ctx->m, ctx->b, d_idx, d_p, N);
    });
    k_set_count<<<1, 1, 0, s>>>(ctx->b.sc, N, step0);
    with_nt(ctx, [&](auto NN, auto TT) {
        constexpr int NC = decltype(NN)::value;
        using T = decltype(TT);
        k_halo<NC, T, 0><<<G, THREADS, 0, s>>>(ctx->m, ctx->b);
        launch_link<NC, T>(ctx, 0);
    });
    k_finalise<<<1, 1, 0, s>>>(ctx->m, ctx->b.sc, 2);
    if (!sync_scalars(ctx, "init_cells")) return ctx->status;
    ctx->has_grid = true;
    return GBEES_OK;
}

static void fill_stats(const gbees_ctx* ctx, gbees_stats* st) {
    if (!st) return;
    st->steps = ctx->hs.steps_call;
    st->cell_updates = ctx->hs.updates_call;
    st->t = ctx->hs.t;
    st->last_dt = ctx->hs.dt;
    st->total_steps = ctx->hs.step;
    st->n_cells = ctx->hs.NA;
    st->norm = ctx->hs.w;
    st->n_pool = ctx->hs.N;
}

int gbees_propagate(gbees_ctx* ctx, double t_end, gbees_stats* stats) {
    int st = guard(ctx, true);
    if (st) return st;
    if (!std::isfinite(t_end)) {
        ctx->err = "t_end must be finite";
        return GBEES_EINVAL;
    }
    cudaStream_t s = ctx->stream;
    {
        Phase ph(ctx, GBEES_PHASE_OTHER, 1);
        k_begin<<<1, 1, 0, s>>>(ctx->b.sc, t_end);
    }
    if (!sync_scalars(ctx, "propagate")) return ctx->status;
    // Persistent path: one cooperative launch runs up to kPersistSteps steps
    // with grid barriers between the phases (small grids).
    resolve_update_kernels(ctx);
    const int mode = ctx->cfg.launch_mode;
    if (mode == GBEES_LAUNCH_PERSISTENT && ctx->persist_grid == 0) {
        set_err(ctx, GBEES_ECUDA, "propagate: the persistent kernel cannot be made resident");
        return ctx->status;
    }
    const bool persist_ok = !ctx->prof_on && ctx->persist_grid > 0 &&
                            (mode == GBEES_LAUNCH_PERSISTENT || mode == GBEES_LAUNCH_AUTO);
    if (persist_ok) {
        bool used = false;
        const long long limit = mode == GBEES_LAUNCH_PERSISTENT ? (1ll << 62) : ctx->persist_max_cells;
        for (auto& e : ctx->pev)
            if (!e && !cuda_ok(ctx, cudaEventCreate(&e), "propagate")) return ctx->status;
        while (!ctx->hs.done && ctx->hs.N <= limit) {
            used = true;
            const long long before = ctx->hs.steps_call;
            const long long upd_before = ctx->hs.updates_call;
            long long max_steps = kPersistSteps;
            long long max_pool = limit;
            void* args[] = {&ctx->m, &ctx->b, &max_steps, &max_pool};
            cudaEventRecord(ctx->pev[0], s);
            const int pg = ctx->persist_blocks > 0 ? std::min(ctx->persist_blocks, ctx->persist_grid) : ctx->persist_grid;
            // the kernel's barriers count arrivals from zero
            if (!cuda_ok(ctx, cudaMemsetAsync(&ctx->b.sc->bar_seq, 0, sizeof(unsigned long long), s), "propagate"))
                return ctx->status;
            if (!cuda_ok(ctx, cudaLaunchCooperativeKernel(ctx->kern.persist, dim3(pg), dim3(THREADS), args, 0, s),
                         "propagate"))
                return ctx->status;
            cudaEventRecord(ctx->pev[1], s);
            ctx->prof.total_launches += 1;
            if (!sync_scalars(ctx, "propagate")) return ctx->status;
            float ms = 0.0f;
            if (cudaEventElapsedTime(&ms, ctx->pev[0], ctx->pev[1]) == cudaSuccess) {
                ctx->prof.persist_ms += ms;
                ctx->prof.persist_launches += 1;
                ctx->prof.persist_updates += ctx->hs.updates_call - upd_before;
            }
            if (!ctx->hs.done && ctx->hs.steps_call == before && ctx->hs.N <= limit) {
                set_err(ctx, GBEES_ETIMEOUT, "propagate: a persistent launch made no progress");
                return ctx->status;
            }
        }
        if (used && ctx->hs.done) {
            fill_stats(ctx, stats);
            return GBEES_OK;
        }
    }
    // Graph path: one launch runs the whole loop on the device (up to
    // kGraphMaxIter steps); the per-phase event timing needs the direct path.
    const bool graph_ok = !ctx->prof_on && mode != GBEES_LAUNCH_DIRECT;
    if (graph_ok && !ctx->graph_tried) build_step_graph(ctx);
    if (graph_ok && ctx->gexec) {
        const long long k0 = ctx->hs.graph_kernels;
        while (!ctx->hs.done) {
            const long long before = ctx->hs.steps_call;
            if (!cuda_ok(ctx, cudaGraphLaunch(ctx->gexec, s), "propagate")) return ctx->status;
            ctx->graph_launches += 1;
            if (!sync_scalars(ctx, "propagate")) return ctx->status;
            if (!ctx->hs.done && ctx->hs.steps_call == before) {
                set_err(ctx, GBEES_ETIMEOUT, "propagate: a graph launch made no progress");
                return ctx->status;
            }
        }
        ctx->prof.total_launches += ctx->hs.graph_kernels - k0;
        fill_stats(ctx, stats);
        return GBEES_OK;
    }
    const int K = ctx->cfg.prune_interval;
    long long host_step = ctx->hs.step;
    long long batch = 4;
    while (!ctx->hs.done) {
        for (long long i = 0; i < batch; ++i) {
            ++host_step;
            launch_step(ctx);
            if (K > 0 && host_step % K == 0) launch_prune(ctx);
        }
        if (!sync_scalars(ctx, "propagate")) return ctx->status;
        host_step = ctx->hs.step;
        if (ctx->hs.done) break;
        const double rem = ctx->hs.t_target - ctx->hs.t;
        const double est = ctx->hs.dt > 0.0 ? rem / ctx->hs.dt : 1.0;
        batch = (long long)std::min(256.0, std::max(1.0, std::ceil(est * 1.02) + 1.0));
    }
    fill_stats(ctx, stats);
    return GBEES_OK;
}

// ---- many grids in one launch

namespace {
struct BatchLayout {
    size_t next, slots, items, collect, total;
};
BatchLayout batch_layout(int32_t count) {
    BatchLayout L;
    L.next = 0;
    L.slots = align_up(sizeof(unsigned int));
    L.items = align_up(L.slots + sizeof(TeamSlot) * GRID_MAX);
    L.collect = align_up(L.items + sizeof(BatchItem) * (size_t)count);
    L.total = align_up(L.collect + sizeof(DevScalars) * (size_t)count);
    return L;
}
constexpr long long kBatchSteps = 1ll << 20;  // steps per grid and launch at most
constexpr int kMaxTeam = 256;                 // blocks per grid in a team launch at most

// Team sizes of a team launch over G resident blocks: one block per grid plus
// the rest in proportion to each grid's work, at most kMaxTeam. Without a step
// cap the work is the whole run (active cells x remaining time / smallest
// cell width, the step count scaling as 1/h); with one (every grid takes the
// same number of steps) it is the work of a step (active cells).
std::vector<int> team_sizes(gbees_ctx* const* ctxs, int32_t count, const double* t_end, int G, bool per_step) {
    std::vector<double> w((size_t)count, 0.0);
    double W = 0.0;
    for (int32_t i = 0; i < count; ++i) {
        const gbees_ctx* c = ctxs[i];
        double hmin = c->cfg.h[0];
        for (int j = 1; j < c->cfg.n; ++j) hmin = std::min(hmin, c->cfg.h[j]);
        const double rem = t_end[i] - c->hs.t;
        const double cells = (double)std::max(1ll, c->hs.NA);
        w[i] = rem > 0.0 ? (per_step ? cells : cells * rem / hmin) : 0.0;
        W += w[i];
    }
    std::vector<int> k((size_t)count, 1);
    if (W <= 0.0) return k;
    int used = 0;
    std::vector<double> rest((size_t)count, 0.0);
    for (int32_t i = 0; i < count; ++i) {
        const double ideal = w[i] / W * G;
        k[i] = std::max(1, std::min(kMaxTeam, (int)std::floor(ideal)));
        rest[i] = ideal - k[i];
        used += k[i];
    }
    while (used > G) {  // the floor of 1 per grid overshot: shrink the largest teams
        int j = (int)(std::max_element(k.begin(), k.end()) - k.begin());
        if (k[j] <= 1) break;
        --k[j];
        --used;
    }
    while (used < G) {  // hand out the remainder by largest shortfall
        int j = -1;
        for (int32_t i = 0; i < count; ++i)
            if (k[i] < kMaxTeam && (j < 0 || rest[i] > rest[j])) j = i;
        if (j < 0 || rest[j] <= 0.0) break;
        ++k[j];
        rest[j] -= 1.0;
        ++used;
    }
    return k;
}
}  // namespace

size_t gbees_batch_workspace_bytes(int32_t count) { return count < 1 ? 0 : batch_layout(count).total; }

int gbees_batch_propagate(gbees_ctx* const* ctxs, int32_t count, const double* t_end, int64_t max_steps,
                          void* d_scratch, size_t scratch_bytes, gbees_stats* stats) {
    if (!ctxs || count < 1 || !t_end || !d_scratch || max_steps < 0) return GBEES_EINVAL;
    const BatchLayout L = batch_layout(count);
    if (scratch_bytes < L.total || ((uintptr_t)d_scratch % ALIGN) != 0) return GBEES_EINVAL;
    gbees_ctx* c0 = ctxs[0];
    {  // one block (or team) per grid: a context listed twice would be stepped twice at once
        std::vector<gbees_ctx*> sorted_ctxs(ctxs, ctxs + count);
        std::sort(sorted_ctxs.begin(), sorted_ctxs.end());
        if (std::adjacent_find(sorted_ctxs.begin(), sorted_ctxs.end()) != sorted_ctxs.end()) {
            if (c0) c0->err = "batch: a context appears more than once";
            return GBEES_EINVAL;
        }
    }
    for (int32_t i = 0; i < count; ++i) {
        gbees_ctx* c = ctxs[i];
        if (!c) return GBEES_EINVAL;
        int st = guard(c, true);
        if (st) return st;
        if (!std::isfinite(t_end[i])) {
            c->err = "t_end must be finite";
            return GBEES_EINVAL;
        }
        if (c->cfg.n != c0->cfg.n || c->cfg.dynamics != c0->cfg.dynamics || c->cfg.precision != c0->cfg.precision) {
            c->err = "batch: every grid needs the dimension, dynamics and precision of the first";
            return GBEES_EINVAL;
        }
    }
    resolve_update_kernels(c0);
    if (!c0->kern_ok || !c0->kern.batch) {
        set_err(c0, GBEES_EINVAL, "batch: no kernels for this model");
        return c0->status;
    }
    cudaStream_t s = c0->stream;
    char* base = (char*)d_scratch;
    unsigned int* next = (unsigned int*)(base + L.next);
    TeamSlot* slots = (TeamSlot*)(base + L.slots);
    BatchItem* items = (BatchItem*)(base + L.items);
    DevScalars* collect = (DevScalars*)(base + L.collect);
    std::vector<BatchItem> h_items((size_t)count);
    for (int32_t i = 0; i < count; ++i) {
        std::memset(&h_items[i], 0, sizeof(BatchItem));
        h_items[i].m = ctxs[i]->m;
        h_items[i].b = ctxs[i]->b;
        h_items[i].t_end = t_end[i];
    }
    if (!cuda_ok(c0, cudaMemcpyAsync(items, h_items.data(), sizeof(BatchItem) * count, cudaMemcpyHostToDevice, s),
                 "batch_propagate"))
        return c0->status;
    k_batch_begin<<<(count + THREADS - 1) / THREADS, THREADS, 0, s>>>(items, count);
    int dev = 0, sms = 0, per_sm = 0;
    if (!cuda_ok(c0, cudaGetDevice(&dev), "batch_propagate") ||
        !cuda_ok(c0, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "batch_propagate") ||
        !cuda_ok(c0, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, c0->kern.batch, THREADS, 0),
                 "batch_propagate"))
        return c0->status;
    const int cap_blocks = c0->batch_blocks > 0 ? c0->batch_blocks : GRID_MAX;
    int G = std::max(1, std::min({count, sms * std::max(per_sm, 1), cap_blocks}));
    // teams: every grid resident at once with blocks in proportion to its work
    int per_sm_team = 0;
    bool teams = c0->kern.batch_teams &&
                 cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_team, c0->kern.batch_teams, THREADS, 0) ==
                     cudaSuccess &&
                 per_sm_team >= 1 && count <= std::min({GRID_MAX, sms * per_sm_team, cap_blocks});
    cudaGetLastError();
    if (teams) {
        const int Gt = std::min({GRID_MAX, sms * per_sm_team, cap_blocks});
        const std::vector<int> k = team_sizes(ctxs, count, t_end, Gt, max_steps > 0);
        std::vector<TeamSlot> h_slots;
        for (int32_t i = 0; i < count; ++i)
            for (int j = 0; j < k[i]; ++j) h_slots.push_back(TeamSlot{(int)i, k[i], j});
        G = (int)h_slots.size();
        if (!cuda_ok(c0, cudaMemcpyAsync(slots, h_slots.data(), sizeof(TeamSlot) * G, cudaMemcpyHostToDevice, s),
                     "batch_propagate"))
            return c0->status;
    }
    std::vector<DevScalars> hs((size_t)count);
    std::vector<long long> steps_before((size_t)count, -1), upd_before((size_t)count, 0);
    const bool one_launch = max_steps > 0;
    long long launch_steps = one_launch ? max_steps : kBatchSteps;
    for (auto& e : c0->pev)
        if (!e && !cuda_ok(c0, cudaEventCreate(&e), "batch_propagate")) return c0->status;
    for (int round = 0;; ++round) {
        if (!cuda_ok(c0, cudaMemsetAsync(next, 0, sizeof(unsigned int), s), "batch_propagate")) return c0->status;
        void* args[] = {&items, &count, &next, &launch_steps};
        void* targs[] = {&items, &slots, &launch_steps};
        cudaEventRecord(c0->pev[0], s);
        const cudaError_t le = teams ? cudaLaunchCooperativeKernel(c0->kern.batch_teams, dim3(G), dim3(THREADS), targs, 0, s)
                                     : cudaLaunchKernel(c0->kern.batch, dim3(G), dim3(THREADS), args, 0, s);
        if (!cuda_ok(c0, le, "batch_propagate")) return c0->status;
        cudaEventRecord(c0->pev[1], s);
        k_batch_collect<<<std::min(1024, (count * (int)(sizeof(DevScalars) / 8) + THREADS - 1) / THREADS), THREADS, 0,
                          s>>>(items, count, collect);
        if (!cuda_ok(c0, cudaMemcpyAsync(hs.data(), collect, sizeof(DevScalars) * count, cudaMemcpyDeviceToHost, s),
                     "batch_propagate") ||
            !cuda_ok(c0, cudaStreamSynchronize(s), "batch_propagate"))
            return c0->status;
        c0->prof.total_launches += 3;
        float ms = 0.0f;
        long long upd = 0;
        bool all_done = true, progress = false;
        for (int32_t i = 0; i < count; ++i) {
            if (!hs[i].done && !hs[i].error) all_done = false;
            if (hs[i].steps_call != steps_before[i]) progress = true;
            steps_before[i] = hs[i].steps_call;
            upd += hs[i].updates_call - upd_before[i];
            upd_before[i] = hs[i].updates_call;
        }
        if (cudaEventElapsedTime(&ms, c0->pev[0], c0->pev[1]) == cudaSuccess) {
            c0->prof.persist_ms += ms;
            c0->prof.persist_launches += 1;
            c0->prof.persist_updates += upd;
        }
        if (all_done || one_launch) break;
        if (!progress) {
            set_err(c0, GBEES_ETIMEOUT, "batch_propagate: a launch made no progress");
            return c0->status;
        }
    }
    int first_err = GBEES_OK;
    for (int32_t i = 0; i < count; ++i) {
        gbees_ctx* c = ctxs[i];
        c->hs = hs[i];
        if (c->hs.error) {
            set_err(c, c->hs.error, std::string("batch_propagate: ") + status_text(c->hs.error));
            if (first_err == GBEES_OK) first_err = c->status;
        }
        if (stats) fill_stats(c, stats + i);
    }
    return first_err;
}

int gbees_correct_gaussian(gbees_ctx* ctx, const double* y, const double* R, const int32_t* H_idx, int32_t m) {
    int st = guard(ctx, true);
    if (st) return st;
    const int n = ctx->cfg.n;
    if (!y || !R || !H_idx || m < 1 || m > n) {
        ctx->err = "bad measurement";
        return GBEES_EINVAL;
    }
    Meas ms;
    std::memset(&ms, 0, sizeof ms);
    ms.m = m;
    for (int a = 0; a < m; ++a) {
        if (H_idx[a] < 0 || H_idx[a] >= n || !std::isfinite(y[a])) {
            ctx->err = "bad measurement index or value";
            return GBEES_EINVAL;
        }
        ms.H[a] = H_idx[a];
        ms.y[a] = y[a];
    }
    if (!spd_inverse(m, R, ms.Rinv)) {
        ctx->err = "measurement covariance is not symmetric positive definite";
        return GBEES_EINVAL;
    }
    const int G = ctx->grid;
    cudaStream_t s = ctx->stream;
    {
        Phase ph(ctx, GBEES_PHASE_CORRECT, 1);
        with_nt(ctx, [&](auto NN, auto TT) {
            constexpr int N = decltype(NN)::value;
            using T = decltype(TT);
            k_correct<N, T><<<G, THREADS, 0, s>>>(ctx->m, ctx->b, ms);
        });
    }
    launch_prune(ctx);
    if (!sync_scalars(ctx, "correct")) return ctx->status;
    return GBEES_OK;
}

int gbees_count(gbees_ctx* ctx, int64_t* n_cells) {
    int st = guard(ctx, true);
    if (st) return st;
    if (!n_cells) return GBEES_EINVAL;
    if (!sync_scalars(ctx, "count")) return ctx->status;
    *n_cells = ctx->hs.NA;
    return GBEES_OK;
}

int gbees_get_stats(gbees_ctx* ctx, gbees_stats* stats) {
    int st = guard(ctx, true);
    if (st) return st;
    if (!sync_scalars(ctx, "get_stats")) return ctx->status;
    fill_stats(ctx, stats);
    return GBEES_OK;
}

int gbees_read_cells(gbees_ctx* ctx, int32_t* idx, double* p, int64_t cap, int64_t* n_cells, int32_t sorted) {
    int st = guard(ctx, true);
    if (st) return st;
    if (!sync_scalars(ctx, "read_cells")) return ctx->status;
    const long long N = ctx->hs.NA;
    if (n_cells) *n_cells = N;
    if (N == 0) return GBEES_OK;
    if ((!idx || !p) && cap > 0) return GBEES_EINVAL;
    const int n = ctx->cfg.n;
    const int g = ctx->hs.gen;
    int* d_idx = ctx->b.link[g ^ 1];
    double* d_p = reinterpret_cast<double*>(ctx->b.key[g ^ 1]);
    cudaStream_t s = ctx->stream;
    {
        Phase ph(ctx, GBEES_PHASE_OTHER, 3);
        launch_readout(ctx, d_idx, d_p);
    }
    std::vector<int32_t> hidx((size_t)N * n);
    std::vector<double> hp((size_t)N);
    if (!cuda_ok(ctx, cudaMemcpyAsync(hidx.data(), d_idx, sizeof(int32_t) * n * N, cudaMemcpyDeviceToHost, s), "read_cells"))
        return ctx->status;
    if (!cuda_ok(ctx, cudaMemcpyAsync(hp.data(), d_p, sizeof(double) * N, cudaMemcpyDeviceToHost, s), "read_cells"))
        return ctx->status;
    if (!cuda_ok(ctx, cudaStreamSynchronize(s), "read_cells")) return ctx->status;
    std::vector<long long> order((size_t)N);
    std::iota(order.begin(), order.end(), 0ll);
    if (sorted) {
        std::sort(order.begin(), order.end(), [&](long long a, long long c) {
            return std::lexicographical_compare(&hidx[a * n], &hidx[a * n] + n, &hidx[c * n], &hidx[c * n] + n);
        });
    }
    const long long w = std::min<long long>(N, cap);
    for (long long r = 0; r < w; ++r) {
        std::memcpy(idx + r * n, &hidx[order[r] * n], sizeof(int32_t) * n);
        p[r] = hp[order[r]];
    }
    return N > cap ? GBEES_EINVAL : GBEES_OK;
}

int gbees_moments(gbees_ctx* ctx, double* mean, double* cov) {
    int st = guard(ctx, true);
    if (st) return st;
    if (!mean || !cov) return GBEES_EINVAL;
    const int n = ctx->cfg.n;
    const int G = ctx->grid;
    cudaStream_t s = ctx->stream;
    DevScalars* sc = ctx->b.sc;
    Phase ph(ctx, GBEES_PHASE_OTHER, 6);
    k_moments_clear<<<1, THREADS, 0, s>>>(sc);
    with_nt(ctx, [&](auto NN, auto TT) {
        constexpr int NC = decltype(NN)::value;
        using T = decltype(TT);
        k_moments<NC, T><<<G, THREADS, 0, s>>>(ctx->m, ctx->b, 0, sc->mom_mean);
    });
    k_moments_final<<<1, 32, 0, s>>>(ctx->m, sc, sc->mom_mean, n);
    k_moments_clear<<<1, THREADS, 0, s>>>(sc);
    with_nt(ctx, [&](auto NN, auto TT) {
        constexpr int NC = decltype(NN)::value;
        using T = decltype(TT);
        k_moments<NC, T><<<G, THREADS, 0, s>>>(ctx->m, ctx->b, 1, sc->mom_mean);
    });
    k_moments_final<<<1, 32, 0, s>>>(ctx->m, sc, sc->mom_out, n * (n + 1) / 2);
    if (!sync_scalars(ctx, "moments")) return ctx->status;
    for (int a = 0; a < n; ++a) mean[a] = ctx->hs.mom_mean[a];
    int slot = 0;
    for (int a = 0; a < n; ++a)
        for (int e = a; e < n; ++e, ++slot) cov[a * n + e] = cov[e * n + a] = ctx->hs.mom_out[slot];
    return GBEES_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ no-allocation entry point
//
// The workspace of gbees_propagate_cells_noalloc lives in this file-scope device
// array. Host code must not pass the array's name to a kernel: on the host it is
// only a stand-in symbol. Its device address is looked up once per device with
// cudaGetSymbolAddress while that device is current, and kept for the life of
// the process (a device reset would invalidate it; the header says so).

namespace {

__device__ __align__(256) unsigned char g_noalloc_scratch[GBEES_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
void* g_noalloc_addr[kMaxDevices] = {};

// Device address of the scratch on the current device (set up on first use).
cudaError_t noalloc_scratch(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return cudaSuccess;
}

// A context over a given workspace, on the stack (the set-up of gbees_create).
bool noalloc_setup(gbees_ctx* ctx, const gbees_config* cfg, void* base_ptr, cudaStream_t stream) {
    Layout L;
    if (!make_layout(cfg, &L)) return false;
    bind_context(ctx, cfg, L, base_ptr, stream);
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return false;
    ctx->grid = std::min(GRID_MAX, std::max(1, sms * 4));
    return true;
}

}  // namespace

extern "C" int gbees_propagate_cells_noalloc(const gbees_config* cfg, const int32_t* idx, const double* p, int64_t N,
                                             double t0, int64_t step0, double t_end, void* cuda_stream,
                                             int32_t* idx_out, double* p_out, int64_t cap_out, int64_t* n_out,
                                             gbees_stats* stats) {
    if (!config_ok(cfg, nullptr) || !n_out || cap_out < 0 || (cap_out > 0 && (!idx_out || !p_out)))
        return GBEES_EINVAL;
    if (gbees_workspace_bytes(cfg) > GBEES_NOALLOC_SCRATCH_BYTES) return GBEES_ECAPACITY;
    void* base = nullptr;
    if (noalloc_scratch(&base) != cudaSuccess) return GBEES_ECUDA;
    gbees_ctx ctx;
    if (!noalloc_setup(&ctx, cfg, base, (cudaStream_t)cuda_stream)) return GBEES_ECUDA;
    int st = gbees_init_cells(&ctx, idx, p, N, t0, step0);
    if (st) return st;
    st = gbees_propagate(&ctx, t_end, stats);
    if (st) return st;
    const long long Nc = ctx.hs.NA;
    *n_out = Nc;
    if (Nc == 0) return GBEES_OK;
    const int n = cfg->n;
    const int g = ctx.hs.gen;
    int* d_idx = ctx.b.link[g ^ 1];
    double* d_p = reinterpret_cast<double*>(ctx.b.key[g ^ 1]);
    launch_readout(&ctx, d_idx, d_p);
    const long long w = std::min<long long>(Nc, cap_out);
    if (w > 0) {
        if (cudaMemcpyAsync(idx_out, d_idx, sizeof(int32_t) * n * w, cudaMemcpyDeviceToHost, ctx.stream) != cudaSuccess ||
            cudaMemcpyAsync(p_out, d_p, sizeof(double) * w, cudaMemcpyDeviceToHost, ctx.stream) != cudaSuccess)
            return GBEES_ECUDA;
    }
    if (cudaStreamSynchronize(ctx.stream) != cudaSuccess || cudaGetLastError() != cudaSuccess) return GBEES_ECUDA;
    return Nc > cap_out ? GBEES_EINVAL : GBEES_OK;
}
