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

// step_kernels: kernels of one step up to and including this one; a prune adds 5.
__global__ void k_loop_ctl(DevScalars* sc, cudaGraphConditionalHandle h_while, cudaGraphConditionalHandle h_prune,
                           long long max_iter, int step_kernels) {
    const long long it = ++sc->loop_iter;
    const int err = sc->error;
    const bool prune = sc->prune_now && !err;
    sc->graph_kernels += step_kernels + (prune ? 5 : 0);
    cudaGraphSetConditional(h_prune, prune ? 1u : 0u);
    cudaGraphSetConditional(h_while, (!sc->done && !err && it < max_iter) ? 1u : 0u);
}

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
    sc->t = t0;
    sc->t_target = t0;
    sc->dt = 0.0;
    sc->maxrate_bits = 0;
    sc->maxrate_new_bits = 0;
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
    sc->bar_count = 0;
    sc->bar_gen = 0;
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

__global__ void k_set_count(DevScalars* sc, long long count, long long step0) {
    sc->N = count;
    sc->NA = count;
    sc->N_prev = 0;
    sc->n_act = 0;
    sc->step = step0;
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

__global__ void k_moments_clear(DevScalars* sc) {
    for (int i = threadIdx.x; i < 28 * NDIG; i += blockDim.x) (&sc->mom[0][0])[i] = 0;
}

// Convert the moment sums to doubles times prod h: out[slot].
__global__ void k_moments_final(const Model m, DevScalars* sc, double* out, int nslots) {
    int s = threadIdx.x;
    if (s < nslots) out[s] = __dmul_rn(m.prod_h, acc_to_double(sc->mom[s]));
}

}  // namespace gbees
