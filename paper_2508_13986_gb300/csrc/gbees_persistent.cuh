// The whole step loop of a propagate call in one launch.
//
// k_persistent: for the grids of 10^4-10^5 cells of the Lorenz '63 workloads a
// time step is a few microseconds of work split into dependent phases; kernel
// launches and their drain would dominate. This cooperative kernel keeps one
// block per SM resident and separates the phases by a bounded grid barrier
// (the cooperative-kernel structure of Sec. 4, with GB300's block count).
//
// k_batch: many independent grids in one launch. Each block takes a grid from
// a queue and runs its whole step loop alone, the phases separated by block
// barriers; blocks never wait on each other, so the launch needs no
// co-residency and ragged grids balance over the SMs.
//
// Every block computes the step's scalars (dt, normalisation, maximum) itself
// from the same per-block partials, so the scalars need no extra barrier;
// block 0 of the grid writes them back.
//
// Barriers per step: grow + waves | halo | link | faces | apply (halo and link
// are skipped in a step whose grow added and activated nothing); a prune adds
// mark | scatter | status | compact | relink.
#pragma once

#include "gbees_kernels.cuh"

namespace gbees {

// The step's scalars, computed by one thread of each block (FP64 divisions are
// expensive on this chip) and read by the others from shared memory.
struct StepShared {
    double dt, t_new, scale, maxq, w;
    double dth[MAXN], ch[MAXN];
    unsigned long long maxrate;
    int last, bad;
};

// w = (prod h) sum, 1 / w and the maximum from combined partials (one thread).
__device__ __forceinline__ void normalisation(const Model& m, const Combined& c, StepShared& ss) {
    const double w = m.prod_h * acc_to_double(c.acc);
    ss.w = w;
    ss.bad = !(w > 0.0) || !isfinite(w);
    ss.scale = ss.bad ? 0.0 : 1.0 / w;
    ss.maxq = c.maxq_ord ? ord_val(c.maxq_ord) : 0.0;
}

// Up to max_steps steps of the grid (m, b) by the nb blocks of index bi that
// share it (the whole launch, a team of a batched launch, or one block): grid
// barriers between the phases, block barriers when the block is alone.
// max_pool: the loop also stops after a step that leaves more pool entries
// than that (the persistent kernel hands a grown grid to the graph path; every
// block sees the same count, so all leave together).
// seq: the nb blocks are the whole launch and sc->bar_seq was zero when it
// began (the persistent kernel), so the barriers count arrivals without reset.
template <int N, int DYN, typename T>
__device__ __forceinline__ void step_loop(const Model& m, const Bufs& b, long long max_steps, int nb, int bi,
                                          long long max_pool = 0x7fffffffffffffffll, bool seq = false) {
    __shared__ StepShared ss;
    DevScalars* sc = b.sc;
    // The result is the same for every thread of the block: a warp that read
    // the error flag after another warp of the block had already raised it in
    // the next phase must not return while the others go on (their block
    // barriers would then pair with the wrong ones).
    unsigned long long n_bar = 0;
    auto barrier = [&]() -> bool {
        if (nb == 1) return __syncthreads_and(!*(volatile int*)&sc->error) != 0;
        if (seq) return grid_barrier_seq(sc, nb + m.bar_extra, n_bar, m.spin_limit);
        return grid_barrier(sc, nb + m.bar_extra, m.spin_limit);
    };
    StepView v = view_of(m, sc);
    v.nb = nb;
    v.bi = bi;
    double t = *(volatile double*)&sc->t;
    const double tt = *(volatile double*)&sc->t_target;
    int done = *(volatile int*)&sc->done;
    long long step = *(volatile long long*)&sc->step;
    unsigned long long maxrate = *(volatile unsigned long long*)&sc->maxrate_bits;
    double w = *(volatile double*)&sc->w;
    double last_dt = *(volatile double*)&sc->dt;
    long long nsteps = 0, nupd = 0;
    // the running reductions start from the state (before the first barrier,
    // which orders these writes before every use)
    int ep = 0;  // parity of the prune epoch in loop_rate
    if (bi == 0 && threadIdx.x == 0 && !done) {
        sc->loop_rate[0] = maxrate;
        for (int e = 0; e < 2; ++e) {
            sc->loop_maxq[e] = 0;
            for (int q = 0; q < NDIG; ++q) sc->loop_acc[e][q] = 0;
        }
    }
    // every block has read the state before anyone changes it
    if (done || *(volatile int*)&sc->error || !barrier()) return;
    // phase timing by block 0 (cycles between the barriers it passes)
    long long pc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    long long t_mark = clock64();
    auto mark = [&](int ph) {
        if (bi == 0 && threadIdx.x == 0) {
            const long long now = clock64();
            pc[ph] += now - t_mark;
            t_mark = now;
        }
    };

    for (long long it = 0; it < max_steps && !done; ++it) {
        // grow (appends active cells to sc->N, activates halo cells) and the
        // waves of the existing entries alongside
        const double rg = grow_body<N, T>(m, b, v);
        waves_body<N, DYN, T>(m, b, v, v.N_prev);
        if (!barrier()) return;
        mark(0);
        // every block read the other apply slot in the previous step: clear it
        // for the next one
        if (bi == 0 && threadIdx.x == 0) {
            sc->loop_maxq[(it + 1) & 1] = 0;
            for (int q = 0; q < NDIG; ++q) sc->loop_acc[(it + 1) & 1][q] = 0;
        }
        // halo cells around the newly active cells (appended after sc->N, which
        // stays put until the link phase)
        const long long n_ins = min(*(volatile long long*)&sc->N, m.cap);
        const long long n_active = *(volatile long long*)&sc->NA;
        const long long n_act = *(volatile long long*)&sc->n_act;
        if (n_ins == v.N_prev && n_act == 0) {
            // the grow added and activated nothing (every block reads the same
            // counts): no halo to make, no entry to link, no new CFL rate
            v.N = n_ins;
            mark(1);
            mark(2);
        } else {
            halo_body<N, T>(m, b, v, v.N_prev, n_ins, n_act);
            if (!barrier()) return;
            mark(1);
            v.N = min(n_ins + *(volatile long long*)&sc->n_halo, m.cap);
            // link the new entries; CFL rates of the new active cells
            {
                const double r = fmax(rg, link_body<N, T>(m, b, v.N_prev, v.N, v.g, nb, bi));
                long long zero[NDIG] = {0, 0, 0, 0, 0, 0};
                block_atomics(nullptr, nullptr, &sc->loop_rate[ep], zero, -INFINITY, r);
            }
            if (bi == 0 && threadIdx.x == 0) sc->N = v.N;  // read again only after the next grow
            if (!barrier()) return;
            mark(2);
            // everyone has read the halo and activation counts: reset them
            if (bi == 0 && threadIdx.x == 0) {
                sc->n_halo = 0;
                sc->n_act = 0;
            }
            // the epoch's largest rate, every block's included (thread 0 uses it)
            if (threadIdx.x == 0) maxrate = max(maxrate, *(volatile unsigned long long*)&sc->loop_rate[ep]);
        }
        if (threadIdx.x == 0) {
            const StepTime st0 = step_time(m, __longlong_as_double((long long)maxrate), t, tt, ss.dth, ss.ch);
            ss.dt = st0.dt;
            ss.t_new = st0.t_new;
            ss.last = st0.last;
        }
        __syncthreads();
        StepTime st;
        st.dt = ss.dt;
        st.t_new = ss.t_new;
        st.last = ss.last;
        v.dt = ss.dt;
#pragma unroll
        for (int k = 0; k < MAXN; ++k) {
            v.dth[k] = ss.dth[k];
            v.ch[k] = ss.ch[k];
        }
        __syncthreads();
        if (!(st.dt > 0.0)) {
            set_error(sc, ST_EDEGENERATE);
            return;
        }
        mark(6);
        // flux update
        long long d[NDIG] = {0, 0, 0, 0, 0, 0};
        double mx = -INFINITY;
        int err = 0;
        faces_body<N, DYN, T, true>(m, b, v);
        if (!barrier()) return;
        mark(3);
        apply_body<N, T, true>(m, b, v, d, mx, err);
        if (err) set_error(sc, ST_EDEGENERATE);
        block_atomics(sc->loop_acc[it & 1], &sc->loop_maxq[it & 1], nullptr, d, mx, 0.0);
        if (!barrier()) return;
        mark(4);
        {
            if (threadIdx.x == 0) {
                Combined cs;
#pragma unroll
                for (int q = 0; q < NDIG; ++q) cs.acc[q] = *(volatile long long*)&sc->loop_acc[it & 1][q];
                cs.maxq_ord = *(volatile unsigned long long*)&sc->loop_maxq[it & 1];
                cs.rate_bits = 0;
                normalisation(m, cs, ss);
            }
            __syncthreads();
            w = ss.w;
            v.scale = ss.scale;
            v.maxq = ss.maxq;
            const int bad = ss.bad;
            __syncthreads();
            if (bad) {
                set_error(sc, ST_EDEGENERATE);
                return;
            }
        }
        t = st.t_new;
        last_dt = st.dt;
        done = st.last;
        step += 1;
        nsteps += 1;
        nupd += n_active;
        v.pb ^= 1;
        v.N_prev = v.N;
        mark(6);
        // prune (Algorithm 3) every prune_interval steps
        if (m.prune_interval > 0 && step % m.prune_interval == 0) {
            prune_mark_body<T>(m, b, v);
            if (!barrier()) return;
            prune_scatter_body<N, T>(m, b, v);
            if (!barrier()) return;
            prune_count_body<N>(m, b, v);
            if (!barrier()) return;
            const Survivors sv = block_offsets(b, v.nb, v.bi);
            const long long total = sv.total_a + sv.total_g;
            if (bi == 0 && threadIdx.x == 0) {  // before the next grow appends
                sc->N = total;
                sc->NA = sv.total_a;
            }
            {
                long long dp[NDIG] = {0, 0, 0, 0, 0, 0};
                double mxp = -INFINITY, rmax = 0.0;
                int errp = 0;
                prune_compact_body<N, T>(m, b, v, sv, dp, mxp, rmax, errp);
                if (errp) set_error(sc, ST_EDEGENERATE);
                block_partial(b.part, dp, mxp, rmax, bi);
            }
            if (!barrier()) return;
            prune_relink_body<N>(m, b, v);
            if (!barrier()) return;
            Combined cp = combine_partials(b.part, nb);
            if (threadIdx.x == 0) normalisation(m, cp, ss);
            __syncthreads();
            w = ss.w;
            v.scale = ss.scale;
            v.maxq = ss.maxq;
            const int bad = ss.bad || sv.total_a == 0;
            __syncthreads();
            if (bad) {
                set_error(sc, ST_EDEGENERATE);
                return;
            }
            maxrate = cp.rate_bits;
            // a new epoch of the running rate starts from the survivors' largest
            ep ^= 1;
            if (bi == 0 && threadIdx.x == 0) sc->loop_rate[ep] = maxrate;
            mark(5);
            v.N = total;
            v.N_prev = total;
            v.g ^= 1;
            v.pb ^= 1;
        }
        if (v.N > max_pool) break;
    }
    if (bi == 0 && threadIdx.x == 0) {
        sc->N = v.N;
        sc->N_prev = v.N_prev;
        sc->pbuf = v.pb;
        sc->gen = v.g;
        sc->maxq = v.maxq;
        sc->scale = v.scale;
        sc->w = w;
        sc->t = t;
        sc->dt = last_dt;
        sc->step = step;
        sc->done = done;
        sc->maxrate_bits = maxrate;
        sc->steps_call += nsteps;
        sc->updates_call += nupd;
        sc->prune_now = 0;
    }
    if (bi == 0 && threadIdx.x == 0) {
        for (int q = 0; q < 8; ++q) sc->phase_cycles[q] += pc[q];
        sc->phase_steps += nsteps;
    }
}


template <int N, int DYN, typename T>
__global__ void __launch_bounds__(THREADS, 1) k_persistent(const Model m, Bufs b, long long max_steps,
                                                           long long max_pool) {
    step_loop<N, DYN, T>(m, b, max_steps, gridDim.x, blockIdx.x, max_pool, true);
}

// Resident blocks per SM of the batch kernels: the register cap (64) spills a
// little, but four blocks keep four times the loads of one in flight, and the
// phases are bound by dependent global loads (measured: 2.1x the throughput of
// two blocks per SM on 256 Lorenz '63 grids).
constexpr int BATCH_BLOCKS_PER_SM = 4;

// k_batch: block after block takes the next grid of the queue (next counts the
// grids handed out) and runs up to max_steps of its steps. A grid that is done
// or in error returns at once, so a launch can be repeated until all are done.
template <int N, int DYN, typename T>
__global__ void __launch_bounds__(THREADS, BATCH_BLOCKS_PER_SM) k_batch(const BatchItem* items, int count, unsigned int* next,
                                                  long long max_steps) {
    __shared__ int s_item;
    for (;;) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(next, 1u);
        __syncthreads();
        const int i = s_item;
        __syncthreads();
        if (i >= count) return;
        const Bufs b = items[i].b;
        step_loop<N, DYN, T>(items[i].m, b, max_steps, 1, 0);
        __syncthreads();
    }
}

// k_batch_teams: a cooperative launch in which every grid has a team of
// blocks (slots[blockIdx.x]) sized to its work, the team's phases separated by
// a barrier on the grid's own scalars.
template <int N, int DYN, typename T>
__global__ void __launch_bounds__(THREADS, BATCH_BLOCKS_PER_SM) k_batch_teams(const BatchItem* items, const TeamSlot* slots,
                                                        long long max_steps) {
    const TeamSlot ts = slots[blockIdx.x];
    if (ts.item < 0) return;
    const Bufs b = items[ts.item].b;
    step_loop<N, DYN, T>(items[ts.item].m, b, max_steps, ts.nb, ts.bi);
}

}  // namespace gbees
