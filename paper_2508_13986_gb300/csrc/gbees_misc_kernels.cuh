// Untemplated helper kernels of the host-side call sequences (begin, reset,
// finalisation, graph-loop control, scans, counts, moments). Included by one
// translation unit only.
#pragma once

#include "gbees_kernels.cuh"

namespace gbees {

// Start a propagate call: record the target and whether any step is due.
__global__ void k_begin(DevScalars* sc, double t_target) {
    sc->t_target = t_target;
    sc->done = !(sc->t < t_target) || sc->error != 0;
    sc->steps_call = 0;
    sc->updates_call = 0;
}

// Normalisation scalars of a new grid (one thread).
__global__ void k_finalise(const Model m, DevScalars* sc, int mode) { finalise_norm(m, sc, mode); }

// Start a batched propagate call: k_begin for every grid of the batch.
__global__ void k_batch_begin(const BatchItem* items, int count) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        DevScalars* sc = items[i].b.sc;
        const double tt = items[i].t_end;
        sc->t_target = tt;
        sc->done = !(sc->t < tt) || sc->error != 0;
        sc->steps_call = 0;
        sc->updates_call = 0;
    }
}

// Copy the scalars of every grid of a batch into one array (one read-back).
__global__ void k_batch_collect(const BatchItem* items, int count, DevScalars* out) {
    constexpr int W = sizeof(DevScalars) / 8;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < (long long)count * W;
         k += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(k / W), q = (int)(k % W);
        reinterpret_cast<long long*>(out + i)[q] = __ldcg(reinterpret_cast<const long long*>(items[i].b.sc) + q);
    }
}

// Control of the device-side step loop of a graph launch (a WHILE node whose
// body is one step and an IF node around the prune): after the flux update of
// a step, decide whether the prune runs and whether another step follows.
// The loop ends when the target time is reached, on any error, or after
// max_iter iterations of this launch (the host then launches again).
__global__ void k_loop_reset(DevScalars* sc) {
    sc->loop_iter = 0;
    sc->graph_kernels += 1;
}

// step_kernels: kernels of one step up to and including this one; a prune adds
// prune_kernels.
__global__ void k_loop_ctl(DevScalars* sc, cudaGraphConditionalHandle h_while, cudaGraphConditionalHandle h_prune,
                           long long max_iter, int step_kernels, int prune_kernels) {
    const long long it = ++sc->loop_iter;
    const int err = sc->error;
    const bool prune = sc->prune_now && !err;
    sc->graph_kernels += step_kernels + (prune ? prune_kernels : 0);
    cudaGraphSetConditional(h_prune, prune ? 1u : 0u);
    cudaGraphSetConditional(h_while, (!sc->done && !err && it < max_iter) ? 1u : 0u);
}

// Empty every hashtable slot.
__global__ void k_table_clear(const Model m, Bufs b) {
    const unsigned long long T = m.tmask + 1;
    for (unsigned long long s = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; s < T;
         s += (unsigned long long)gridDim.x * blockDim.x) {
        reinterpret_cast<ulonglong2*>(b.table)[s] = make_ulonglong2(EMPTY_KEY, ~0ull);
    }
}

// Exclusive scan of blk[0..nblk) by one block; the total goes to sc->N_new.
__global__ void k_scan_blocks(Bufs b, int nblk, long long cap) {
    __shared__ long long s_part[THREADS];
    const int per = (nblk + THREADS - 1) / THREADS;
    const int i0 = threadIdx.x * per;
    long long sum = 0;
    for (int i = i0; i < i0 + per && i < nblk; ++i) sum += b.blk[i];
    s_part[threadIdx.x] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long run = 0;
        for (int t = 0; t < THREADS; ++t) {
            long long v = s_part[t];
            s_part[t] = run;
            run += v;
        }
        b.sc->N_new = run;
        if (run > cap) set_error(b.sc, ST_ECAPACITY);
    }
    __syncthreads();
    long long run = s_part[threadIdx.x];
    for (int i = i0; i < i0 + per && i < nblk; ++i) {
        long long v = b.blk[i];
        b.blk[i] = run;
        run += v;
    }
}

// Reset the grid scalars before an init.
__global__ void k_reset(DevScalars* sc, double t0) {
    sc->N = 0;
    sc->N_prev = 0;
    sc->N_new = 0;
    sc->NA = 0;
    sc->NA_new = 0;
    sc->n_halo = 0;
    sc->n_act = 0;
    sc->n_glist = 0;
    sc->t = t0;
    sc->t_target = t0;
    sc->dt = 0.0;
    sc->maxrate_bits = 0;
    sc->maxq_ord = 0;
    sc->maxq = 0.0;
    sc->w = 1.0;
    sc->scale = 1.0;
    for (int q = 0; q < NDIG; ++q) sc->acc[q] = 0;
    sc->step = 0;
    sc->steps_call = 0;
    sc->updates_call = 0;
    sc->lookups_fallback = 0;
    sc->pbuf = 0;
    sc->gen = 0;
    sc->done = 1;
    sc->error = 0;
    sc->prune_now = 0;
    sc->ticket = 0;
    sc->tmp_ord = 0;
    sc->loop_iter = 0;
    sc->graph_kernels = 0;
    sc->bar_word = 0;
    sc->bar_seq = 0;
    for (int e = 0; e < 2; ++e) {
        sc->loop_rate[e] = 0;
        sc->loop_maxq[e] = 0;
        for (int q = 0; q < NDIG; ++q) sc->loop_acc[e][q] = 0;
    }
    for (int q = 0; q < 8; ++q) sc->phase_cycles[q] = 0;
    sc->phase_steps = 0;
}

// Initial grid: the active cells written so far are the whole pool; the halo
// kernel adds their halo next.
__global__ void k_set_count_from_new(DevScalars* sc) {
    sc->N = sc->N_new;
    sc->NA = sc->N_new;
    sc->N_prev = 0;
    sc->n_act = 0;
}

// Counts and step number of a grid loaded from explicit cells.
__global__ void k_set_count(DevScalars* sc, long long count, long long step0) {
    sc->N = count;
    sc->NA = count;
    sc->N_prev = 0;
    sc->n_act = 0;
    sc->step = step0;
}

// ------------------------------------------------------------------ storage order at a prune
// The prune of a large grid gives the survivors a new storage order with a
// stable LSD radix sort of (order key, old index), 8 bits per pass: the
// lexicographic order of the cell indices (the packed key itself, dimension 0
// most significant), so that the face neighbours of a warp's consecutive cells
// in any dimension are consecutive too and the neighbour gathers coalesce, or
// the Morton order of the indices. Scratch: the other generation's key/slot
// arrays (A) and its link/value arrays (B), free until the compaction writes
// them.

constexpr int SORT_BLOCKS = 1024;  // blocks of the sort kernels at most (histogram rows)
constexpr int SCAN_THREADS = 1024; // threads of the histogram scan

struct SortBufs {
    unsigned long long* key[2];
    unsigned int* val[2];
};

__device__ __forceinline__ SortBufs sort_bufs(const Bufs& b, const StepView& v) {
    SortBufs s;
    s.key[0] = b.key[v.g ^ 1];
    s.key[1] = reinterpret_cast<unsigned long long*>(b.link[v.g ^ 1]);
    s.val[0] = b.slot[v.g ^ 1];
    s.val[1] = static_cast<unsigned int*>(b.q[v.pb ^ 1]);
    return s;
}

// keep[c] = status (0 drop, 1 active, 2 halo, from the status pass in map);
// A = (order key, c): active cells first, then the halo (each in the order of
// the configured code), or both interleaved in key order; dropped entries
// last (every result is independent of the storage order; only the speed
// depends on it). A live entry's order key
// is below 2^63: keys use at most 63 bits, and only an all-ones key has an
// all-ones Morton code, a key no cell that survives a prune has.
__global__ void __launch_bounds__(THREADS) k_sort_init(const Model m, Bufs b) {
    if (!prune_due(b.sc)) return;
    const StepView v = view_of(m, b.sc);
    const SortBufs sb = sort_bufs(b, v);
    const unsigned long long* key = b.key[v.g];
    long long c0, c1;
    block_chunk(v.N, c0, c1);
    const int order = m.sort_order;        // GBEES_ORDER_*
    const bool mixed = order == 3;          // halo cells among the active ones
    for (long long c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
        const int st = b.map[c];
        b.keep[c] = (unsigned char)st;
        const unsigned long long region = (st == 2 && !mixed) ? (1ull << 63) : 0ull;
        const unsigned long long code = order == 1   ? morton_code(key[c], m.n, m.key_bits)
                                        : order == 4 ? row_morton_code(key[c], m.n, m.key_bits)
                                                     : key[c];
        sb.key[0][c] = st == 0 ? ~0ull : (region | code);
        sb.val[0][c] = (unsigned int)c;
    }
}

// Pass histogram: sorthist[d * nblk + block] = entries of this block's chunk
// whose digit (key >> shift) & 255 is d.
__global__ void __launch_bounds__(THREADS) k_sort_hist(const Model m, Bufs b, int src, int shift) {
    if (!prune_due(b.sc)) return;
    __shared__ unsigned int cnt[256];
    const StepView v = view_of(m, b.sc);
    const SortBufs sb = sort_bufs(b, v);
    for (int d = threadIdx.x; d < 256; d += blockDim.x) cnt[d] = 0;
    __syncthreads();
    long long c0, c1;
    block_chunk(v.N, c0, c1);
    for (long long c = c0 + threadIdx.x; c < c1; c += blockDim.x)
        atomicAdd(&cnt[(unsigned)(sb.key[src][c] >> shift) & 255u], 1u);
    __syncthreads();
    for (int d = threadIdx.x; d < 256; d += blockDim.x) b.sorthist[(long long)d * gridDim.x + blockIdx.x] = cnt[d];
}

// Exclusive scan of the 256 x nblk histogram in place (one block of
// SCAN_THREADS threads: each sums a run of counters, a block-wide scan of the
// run totals, then each writes its run's offsets).
__global__ void __launch_bounds__(SCAN_THREADS) k_sort_scan(const Model m, Bufs b, int nblk) {
    if (!prune_due(b.sc)) return;
    __shared__ unsigned long long s_warp[SCAN_THREADS / 32];
    unsigned int* hist = b.sorthist;
    const long long total = 256ll * nblk;
    const long long per = (total + blockDim.x - 1) / blockDim.x;
    const long long i0 = min(total, threadIdx.x * per), i1 = min(total, i0 + per);
    unsigned long long sum = 0;
    for (long long i = i0; i < i1; ++i) sum += hist[i];
    // inclusive scan of the run totals: within the warp, then over the warps
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned long long x = sum;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, x, off);
        if (lane >= off) x += y;
    }
    if (lane == 31) s_warp[wid] = x;
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        unsigned long long w = lane < nw ? s_warp[lane] : 0ull;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, w, off);
            if (lane >= off) w += y;
        }
        if (lane < nw) s_warp[lane] = w;
    }
    __syncthreads();
    unsigned long long run = x - sum + (wid > 0 ? s_warp[wid - 1] : 0ull);
    for (long long i = i0; i < i1; ++i) {
        const unsigned int c = hist[i];
        hist[i] = (unsigned int)run;
        run += c;
    }
}

// Stable scatter of a pass: every block walks its chunk in tiles of one
// element per thread; an element's place is its digit's offset for the block,
// plus the elements of that digit in earlier tiles, earlier warps of the tile
// and earlier lanes of its warp.
__global__ void __launch_bounds__(THREADS) k_sort_scatter(const Model m, Bufs b, int src, int shift) {
    if (!prune_due(b.sc)) return;
    __shared__ unsigned int base[256];
    __shared__ unsigned int wcnt[WARPS][256];
    const StepView v = view_of(m, b.sc);
    const SortBufs sb = sort_bufs(b, v);
    for (int d = threadIdx.x; d < 256; d += blockDim.x) base[d] = b.sorthist[(long long)d * gridDim.x + blockIdx.x];
    long long c0, c1;
    block_chunk(v.N, c0, c1);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (long long t0 = c0; t0 < c1; t0 += blockDim.x) {
        for (int i = threadIdx.x; i < WARPS * 256; i += blockDim.x) (&wcnt[0][0])[i] = 0;
        __syncthreads();
        const long long c = t0 + threadIdx.x;
        const bool ok = c < c1;
        unsigned long long k = 0;
        unsigned int val = 0;
        int d = 256 + lane;  // distinct dummies for lanes past the end
        if (ok) {
            k = sb.key[src][c];
            val = sb.val[src][c];
            d = (int)((k >> shift) & 255u);
        }
        const unsigned same = __match_any_sync(0xffffffffu, d);
        const int rank = __popc(same & ((1u << lane) - 1u));
        if (ok && rank == 0) wcnt[wid][d] = __popc(same);
        __syncthreads();
        if (ok) {
            unsigned int off = base[d] + rank;
            for (int w = 0; w < wid; ++w) off += wcnt[w][d];
            sb.key[src ^ 1][off] = k;
            sb.val[src ^ 1][off] = val;
        }
        __syncthreads();
        for (int dd = threadIdx.x; dd < 256; dd += blockDim.x) {
            unsigned int tot = 0;
            for (int w = 0; w < WARPS; ++w) tot += wcnt[w][dd];
            base[dd] += tot;
        }
        __syncthreads();
    }
}

// New index of every survivor: its rank in the sorted order (survivors sort
// before the dropped entries); -1 for the dropped.
__global__ void __launch_bounds__(THREADS) k_sort_map(const Model m, Bufs b) {
    if (!prune_due(b.sc)) return;
    const StepView v = view_of(m, b.sc);
    const SortBufs sb = sort_bufs(b, v);
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < v.N; r += (long long)gridDim.x * blockDim.x) {
        const unsigned int c = sb.val[0][r];
        b.map[c] = b.keep[c] ? (int)r : -1;
    }
}

// Per-block counts of the active cells (read-out, first pass).
__global__ void __launch_bounds__(THREADS) k_readout_count(const Model m, Bufs b) {
    DevScalars* sc = b.sc;
    const long long ncell = min(*(volatile long long*)&sc->N, m.cap);
    const unsigned short* om = b.om[*(volatile int*)&sc->gen];
    long long c0, c1;
    block_chunk(ncell, c0, c1);
    int cnt = 0;
    for (long long c = c0 + threadIdx.x; c < c1; c += blockDim.x) cnt += !is_halo(om, c);
    const long long t = block_count(cnt);
    if (threadIdx.x == 0) b.blk[blockIdx.x] = t;
}

// Zero the exact accumulators of the moments.
__global__ void k_moments_clear(DevScalars* sc) {
    for (int i = threadIdx.x; i < 28 * NDIG; i += blockDim.x) (&sc->mom[0][0])[i] = 0;
}

// Convert the moment sums to doubles times prod h: out[slot].
__global__ void k_moments_final(const Model m, DevScalars* sc, double* out, int nslots) {
    int s = threadIdx.x;
    if (s < nslots) out[s] = __dmul_rn(m.prod_h, acc_to_double(sc->mom[s]));
}

}  // namespace gbees
