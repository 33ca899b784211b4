// Kernels of the GBEES step other than the flux update: initial grid, directional
// grow (Sec. 3.3, Algorithm 2), neighbour links (Sec. 4.1), Bayesian update
// (Eq. 4), directional prune with stream compaction and rehash (Algorithm 3),
// read-out and moments. All kernels use a fixed grid and loop over the cells,
// whose count they read from device memory, so that no step needs the host.
#pragma once

#include "gbees_phases.cuh"

namespace gbees {

// ------------------------------------------------------------------ begin / finalise

// ------------------------------------------------------------------ hashtable helpers

// ------------------------------------------------------------------ links

// Finish a step's time after the link phase: the maximum CFL rate over all
// cells (old maximum and the new cells' partials) and dt with its coefficients.
__device__ __forceinline__ void finish_link(const Model& m, DevScalars* sc, const Combined& cr, int step) {
    unsigned long long r = max(sc->maxrate_bits, cr.rate_bits);
    sc->maxrate_bits = r;
    if (step) {
        StepTime st = step_time(m, __longlong_as_double((long long)r), sc->t, sc->t_target, sc->coef_dth, sc->coef_ch);
        if (!(st.dt > 0.0)) set_error(sc, ST_EDEGENERATE);  // no progress possible
        sc->step_dt = st.dt;
        sc->step_t_new = st.t_new;
        sc->step_last = st.last;
    }
    sc->ticket = 0;
}

// Link entries [N_prev, N) (neighbour references of Sec. 4.1), set their outward
// masks and rates; with step != 0 the last block also fixes dt (Eq. 8).
// W lanes probe the hashtable together (warp-cooperative probing).
template <int N, int W, typename T>
__global__ void __launch_bounds__(THREADS) k_link(const Model m, Bufs b, int step) {
    DevScalars* sc = b.sc;
    if (*(volatile int*)&sc->error) return;
    if (step && *(volatile int*)&sc->done) return;
    const StepView v = view_of(m, sc);
    const double r = (W == 1) ? link_body<N, T>(m, b, v.N_prev, v.N, v.g, v.nb, v.bi)
                              : link_body_tile<N, W, T>(m, b, v.N_prev, v.N, v.g, v.nb, v.bi);
    long long zero[NDIG] = {0, 0, 0, 0, 0, 0};
    block_partial(b.part, zero, -INFINITY, r);
    if (last_block(sc)) {
        Combined cr = combine_partials(b.part, gridDim.x);
        if (threadIdx.x == 0) finish_link(m, sc, cr, step);
    }
}

// ------------------------------------------------------------------ initial Gaussian

struct InitBox {
    int lo[MAXN];
    long long dims[MAXN];
    long long total;
    double mean[MAXN];
    double icov[MAXN * MAXN];
    double pstar;
};

template <int N>
__device__ __forceinline__ void box_index(const InitBox& bx, long long lin, int* I) {
#pragma unroll
    for (int k = N - 1; k >= 0; --k) {
        I[k] = bx.lo[k] + (int)(lin % bx.dims[k]);
        lin /= bx.dims[k];
    }
}

// exp(-1/2 (x - mean)^T icov (x - mean)) at the centre of cell I.
template <int N>
__device__ __forceinline__ double gauss_at(const Model& m, const InitBox& bx, const int* I) {
    double dx[N];
#pragma unroll
    for (int k = 0; k < N; ++k) dx[k] = __dsub_rn(centre64(m, k, I[k]), bx.mean[k]);
    double q = 0.0;
#pragma unroll
    for (int a = 0; a < N; ++a)
#pragma unroll
        for (int c = 0; c < N; ++c) q = __dadd_rn(q, __dmul_rn(__dmul_rn(dx[a], bx.icov[a * N + c]), dx[c]));
    return exp(__dmul_rn(-0.5, q));
}

// Initial Gaussian (Sec. 5.1), pass 1: the largest density over the box of
// candidate cells, which fixes the threshold p* = thr_rel * max p.
template <int N>
__global__ void __launch_bounds__(THREADS) k_init_max(const Model m, Bufs b, const InitBox bx) {
    double mx = 0.0;
    for (long long lin = blockIdx.x * (long long)blockDim.x + threadIdx.x; lin < bx.total;
         lin += (long long)gridDim.x * blockDim.x) {
        int I[N];
        box_index<N>(bx, lin, I);
        mx = fmax(mx, gauss_at<N>(m, bx, I));
    }
    mx = block_max(mx);
    if (threadIdx.x == 0 && mx > 0.0) atomicMax(&b.sc->tmp_ord, ord_key(mx));
}

// Initial Gaussian, pass 2: per-block counts of the box cells above p*, the
// offsets of the write pass.
template <int N>
__global__ void __launch_bounds__(THREADS) k_init_count(const Model m, Bufs b, const InitBox bx) {
    long long c0, c1;
    block_chunk(bx.total, c0, c1);
    int cnt = 0;
    for (long long lin = c0 + threadIdx.x; lin < c1; lin += blockDim.x) {
        int I[N];
        box_index<N>(bx, lin, I);
        cnt += gauss_at<N>(m, bx, I) > bx.pstar;
    }
    for (int off = 16; off > 0; off >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, off);
    __shared__ int s[WARPS];
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s[w];
        b.blk[blockIdx.x] = t;
    }
}

// Write the kept cells of the box in lexicographic order, insert them in the
// table, and reduce their sum, maximum and CFL rates.
template <int N, typename T>
__global__ void __launch_bounds__(THREADS) k_init_write(const Model m, Bufs b, const InitBox bx) {
    DevScalars* sc = b.sc;
    if (*(volatile int*)&sc->error) return;
    long long c0, c1;
    block_chunk(bx.total, c0, c1);
    long long base = b.blk[blockIdx.x];
    long long d[NDIG] = {0, 0, 0, 0, 0, 0};
    double mx = -INFINITY, rmax = 0.0;
    int err = 0;
    for (long long t0 = c0; t0 < c1; t0 += blockDim.x) {
        long long lin = t0 + threadIdx.x;
        int I[N];
        double g = 0.0;
        int f = 0;
        if (lin < c1) {
            box_index<N>(bx, lin, I);
            g = gauss_at<N>(m, bx, I);
            f = g > bx.pstar;
        }
        int total;
        int pos = block_exclusive_scan(f, total);
        if (f) {
            long long c = base + pos;
            unsigned long long k;
            if (c >= m.cap) {
                set_error(sc, ST_ECAPACITY);
            } else if (!interior<N>(m, I) || !pack_key<N>(m, I, k)) {
                set_error(sc, ST_EKEYRANGE);
            } else {
                T v = (T)g;
                b.key[0][c] = k;
                static_cast<T*>(b.q[0])[c] = v;
                b.om[0][c] = (unsigned short)outward_mask<N>(m, I);
                table_insert_new(m, b, k, c, b.slot[0]);
                acc_add(d, (double)v, err);
                mx = fmax(mx, (double)v);
                rmax = fmax(rmax, cfl_rate64<N>(m, I));
            }
        }
        base += total;
    }
    if (err) set_error(sc, ST_EDEGENERATE);
    block_reduce_acc_max(d, mx, sc->acc, &sc->maxq_ord);
    double r = block_max(rmax);
    if (threadIdx.x == 0 && r > 0.0) atomicMax(&sc->maxrate_bits, (unsigned long long)__double_as_longlong(r));
}

// ------------------------------------------------------------------ explicit cells

// Load N cells given as int32 indices (staged in device memory) and doubles.
template <int N, typename T>
__global__ void __launch_bounds__(THREADS) k_init_cells(const Model m, Bufs b, const int* __restrict__ idx,
                                                        const double* __restrict__ p, long long count) {
    DevScalars* sc = b.sc;
    double mx = -INFINITY, rmax = 0.0;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < count;
         c += (long long)gridDim.x * blockDim.x) {
        int I[N];
#pragma unroll
        for (int k = 0; k < N; ++k) I[k] = idx[c * N + k];
        unsigned long long k;
        if (!interior<N>(m, I) || !pack_key<N>(m, I, k)) {
            set_error(sc, ST_EKEYRANGE);
            continue;
        }
        T v = (T)p[c];
        b.key[0][c] = k;
        static_cast<T*>(b.q[0])[c] = v;
        b.om[0][c] = (unsigned short)outward_mask<N>(m, I);
        table_insert_new(m, b, k, c, b.slot[0]);
        mx = fmax(mx, (double)v);
        rmax = fmax(rmax, cfl_rate64<N>(m, I));
    }
    mx = block_max(mx);
    double r = block_max(rmax);
    if (threadIdx.x == 0) {
        if (mx > -INFINITY) atomicMax(&sc->maxq_ord, ord_key(mx));
        if (r > 0.0) atomicMax(&sc->maxrate_bits, (unsigned long long)__double_as_longlong(r));
    }
}

// ------------------------------------------------------------------ grow

// The CFL rates of the halo cells that grow made active join the running maximum.
__device__ __forceinline__ void grow_rates(DevScalars* sc, double r) {
    r = block_max(r);
    if (threadIdx.x == 0 && r > 0.0) atomicMax(&sc->maxrate_bits, (unsigned long long)__double_as_longlong(r));
}

// Halo cells around the cells that grow made active (inserted ones: [N_prev, N)
// at entry; activated ones: the n_act entries listed in map). With STEP == 0
// (initial grid) it runs whatever the done flag says. The last block appends
// the new halo cells to the count.
template <int N, typename T, int STEP>
__global__ void __launch_bounds__(THREADS) k_halo(const Model m, Bufs b) {
    DevScalars* sc = b.sc;
    if (*(volatile int*)&sc->error) return;
    if (STEP && *(volatile int*)&sc->done) return;
    const StepView v = view_of(m, sc);
    halo_body<N, T>(m, b, v, v.N_prev, v.N, *(volatile long long*)&sc->n_act);
    if (last_block(sc)) {
        if (threadIdx.x == 0) {
            sc->N = min(sc->N + sc->n_halo, m.cap);
            sc->n_halo = 0;
            sc->n_act = 0;
            sc->n_glist = 0;
            sc->ticket = 0;
        }
    }
}

// ------------------------------------------------------------------ step completion

// Time, step count, buffers, prune schedule and normalisation after the flux
// update of a step, from the combined partials of the update's blocks.
__device__ __forceinline__ void finish_step(const Model& m, DevScalars* sc, const Combined& cs, int pb) {
    sc->dt = sc->step_dt;
    sc->t = sc->step_t_new;
    sc->step += 1;
    sc->steps_call += 1;
    sc->updates_call += sc->NA;
    sc->done = sc->step_last;
    sc->pbuf = pb ^ 1;
    sc->prune_now = (m.prune_interval > 0 && (sc->step % m.prune_interval) == 0);
    sc->N_prev = sc->N;
    const double w = m.prod_h * acc_to_double(cs.acc);
    sc->w = w;
    if (!(w > 0.0) || !isfinite(w)) {
        set_error(sc, ST_EDEGENERATE);
        sc->scale = 0.0;
    } else {
        sc->scale = 1.0 / w;
    }
    sc->maxq = cs.maxq_ord ? ord_val(cs.maxq_ord) : 0.0;
    sc->ticket = 0;
}

// The first phase of a step of a large grid in two kernels: the waves of the
// existing entries, listing the cells that grow (no block-wide rounds over the
// whole pool), then every (listed cell, candidate) pair over the grid.
template <int N, int DYN, typename T>
__global__ void __launch_bounds__(THREADS) k_waves_list(const Model m, Bufs b) {
    DevScalars* sc = b.sc;
    if (*(volatile int*)&sc->done | *(volatile int*)&sc->error) return;
    const StepView v = view_of(m, sc);
    waves_body<N, DYN, T, true>(m, b, v, v.N_prev);
}

template <int N, typename T>
__global__ void __launch_bounds__(THREADS) k_grow_list(const Model m, Bufs b) {
    DevScalars* sc = b.sc;
    if (*(volatile int*)&sc->done | *(volatile int*)&sc->error) return;
    const StepView v = view_of(m, sc);
    grow_rates(sc, grow_list_body<N, T>(m, b, v));
}

// Flux update, pass 2: the flux through every face that touches an active
// cell: donor cell (Eq. 7), the transverse terms of Algorithm 1 read from the
// upwind cell's wave row, and the limited high-resolution term.
template <int N, int DYN, typename T>
__global__ void __launch_bounds__(THREADS) k_faces(const Model m, Bufs b) {
    DevScalars* sc = b.sc;
    if (*(volatile int*)&sc->done | *(volatile int*)&sc->error) return;
    faces_body<N, DYN, T>(m, b, view_of(m, sc));
}

// Flux update, pass 3: the conservative update of every active cell from the
// fluxes of its 2n faces, divided by the last normaliser; exact per-block
// partial sums and maximum for the next one; the last block ends the step.
template <int N, typename T>
__global__ void __launch_bounds__(THREADS) k_apply(const Model m, Bufs b) {
    DevScalars* sc = b.sc;
    if (*(volatile int*)&sc->done | *(volatile int*)&sc->error) return;
    const StepView v = view_of(m, sc);
    long long d[NDIG] = {0, 0, 0, 0, 0, 0};
    double mx = -INFINITY;
    int err = 0;
    apply_body<N, T>(m, b, v, d, mx, err);
    if (err) set_error(sc, ST_EDEGENERATE);
    block_partial(b.part, d, mx, 0.0);
    if (last_block(sc)) {
        Combined cs = combine_partials(b.part, gridDim.x);
        if (threadIdx.x == 0) finish_step(m, sc, cs, v.pb);
    }
}

// ------------------------------------------------------------------ measurement update

struct Meas {
    int m;
    int H[MAXN];
    double y[MAXN];
    double Rinv[MAXN * MAXN];
};

// p <- exp(-1/2 (y - x_H)^T R^-1 (y - x_H)) p at the cell centres (Eq. 4); the
// maximum is reduced for the prune that follows.
template <int N, typename T>
__global__ void __launch_bounds__(THREADS) k_correct(const Model m, Bufs b, const Meas ms) {
    DevScalars* sc = b.sc;
    if (*(volatile int*)&sc->error) return;
    const long long ncell = min(*(volatile long long*)&sc->N, m.cap);
    const int g = *(volatile int*)&sc->gen, pb = *(volatile int*)&sc->pbuf;
    T* Q = static_cast<T*>(b.q[pb]);
    const unsigned long long* key = b.key[g];
    double mx = -INFINITY;
    for (WarpRuns wr(ncell); wr.next();) {
        const long long c = wr.c;
        if (c >= ncell) continue;
        int I[N];
        unpack_key<N>(m, key[c], I);
        double r[MAXN];
        for (int a = 0; a < ms.m; ++a) r[a] = __dsub_rn(ms.y[a], centre64(m, ms.H[a], I[ms.H[a]]));
        double qf = 0.0;
        for (int a = 0; a < ms.m; ++a)
            for (int e = 0; e < ms.m; ++e) qf = __dadd_rn(qf, __dmul_rn(__dmul_rn(r[a], ms.Rinv[a * ms.m + e]), r[e]));
        double L = exp(__dmul_rn(-0.5, qf));
        T v = (T)__dmul_rn(L, (double)Q[c]);
        Q[c] = v;
        mx = fmax(mx, (double)v);
    }
    long long zero[NDIG] = {0, 0, 0, 0, 0, 0};
    block_partial(b.part, zero, mx, 0.0);
    if (last_block(sc)) {
        Combined c = combine_partials(b.part, gridDim.x);
        if (threadIdx.x == 0) {
            sc->maxq = c.maxq_ord ? ord_val(c.maxq_ord) : 0.0;
            sc->ticket = 0;
            sc->prune_now = 1;
        }
    }
}

// ------------------------------------------------------------------ prune

__device__ __forceinline__ bool prune_due(const DevScalars* sc) {
    return *(volatile int*)&sc->prune_now && !*(volatile int*)&sc->error;
}

// Prune (Algorithm 3), pass 1: mark the significant cells S.
template <typename T>
__global__ void __launch_bounds__(THREADS) k_prune_mark(const Model m, Bufs b) {
    if (!prune_due(b.sc)) return;
    prune_mark_body<T>(m, b, view_of(m, b.sc));
}

// Prune, pass 2: mark the downwind set D(S) of every significant cell (the
// directional rule of Sec. 3.3).
template <int N, typename T>
__global__ void __launch_bounds__(THREADS) k_prune_scatter(const Model m, Bufs b) {
    if (!prune_due(b.sc)) return;
    prune_scatter_body<N, T>(m, b, view_of(m, b.sc));
}

// Prune, pass 3: the status of every entry (active, halo or dropped) and the
// per-block counts of the survivors.
template <int N>
__global__ void __launch_bounds__(THREADS) k_prune_count(const Model m, Bufs b) {
    if (!prune_due(b.sc)) return;
    prune_count_body<N>(m, b, view_of(m, b.sc));
}

// Prune, pass 4: write the survivors into the other buffer set in the order
// of the radix sort (Morton order of the cell indices), active cells first, with exact partial
// sums, maximum and CFL rates for the step scalars.
template <int N, typename T>
__global__ void __launch_bounds__(THREADS) k_prune_compact_sorted(const Model m, Bufs b) {
    DevScalars* sc = b.sc;
    if (!prune_due(sc)) return;
    const StepView v = view_of(m, sc);
    const Survivors sv = block_offsets(b, v.nb, v.bi);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        sc->N_new = sv.total_a + sv.total_g;
        sc->NA_new = sv.total_a;
    }
    long long d[NDIG] = {0, 0, 0, 0, 0, 0};
    double mx = -INFINITY, rmax = 0.0;
    int err = 0;
    prune_compact_sorted_body<N, T>(m, b, v, d, mx, rmax, err);
    if (err) set_error(sc, ST_EDEGENERATE);
    block_partial(b.part, d, mx, rmax);
}

// Prune, pass 4 without a sort: write the survivors into the other buffer set
// in storage order, active cells first, then the halo (stream compaction), with
// the same partials as the sorted form.
template <int N, typename T>
__global__ void __launch_bounds__(THREADS) k_prune_compact(const Model m, Bufs b) {
    DevScalars* sc = b.sc;
    if (!prune_due(sc)) return;
    const StepView v = view_of(m, sc);
    const Survivors sv = block_offsets(b, v.nb, v.bi);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        sc->N_new = sv.total_a + sv.total_g;
        sc->NA_new = sv.total_a;
    }
    long long d[NDIG] = {0, 0, 0, 0, 0, 0};
    double mx = -INFINITY, rmax = 0.0;
    int err = 0;
    prune_compact_body<N, T>(m, b, v, sv, d, mx, rmax, err);
    if (err) set_error(sc, ST_EDEGENERATE);
    block_partial(b.part, d, mx, rmax);
}

// The end of a prune: swap the buffer sets, new count, normalisation scalars
// and CFL maximum of the survivors.
__device__ __forceinline__ void finish_prune(const Model& m, DevScalars* sc, const Combined& cp, long long n_new) {
    sc->N = n_new;
    sc->N_prev = n_new;
    sc->NA = sc->NA_new;
    sc->gen ^= 1;
    sc->pbuf ^= 1;
    sc->maxrate_bits = cp.rate_bits;
    sc->prune_now = 0;
    const double w = m.prod_h * acc_to_double(cp.acc);
    sc->w = w;
    if (!(w > 0.0) || !isfinite(w)) {
        set_error(sc, ST_EDEGENERATE);
        sc->scale = 0.0;
    } else {
        sc->scale = 1.0 / w;
    }
    sc->maxq = cp.maxq_ord ? ord_val(cp.maxq_ord) : 0.0;
    sc->ticket = 0;
}

// Prune, pass 5: rehash the survivors and rebuild their links (Sec. 4.4.2);
// the last block swaps the buffer sets and sets the step scalars.
template <int N>
__global__ void __launch_bounds__(THREADS) k_prune_relink(const Model m, Bufs b, int nblk_compact) {
    DevScalars* sc = b.sc;
    if (!prune_due(sc)) return;
    prune_relink_body<N>(m, b, view_of(m, sc));
    if (last_block(sc)) {
        Combined cp = combine_partials(b.part, nblk_compact);
        if (threadIdx.x == 0) finish_prune(m, sc, cp, *(volatile long long*)&sc->N_new);
    }
}

// ------------------------------------------------------------------ read-out

// Read-out of the active cells in storage order: per-block counts
// (k_readout_count), an exclusive scan of them (k_scan_blocks), then every
// block writes its active cells at its offset.
template <int N, typename T>
__global__ void __launch_bounds__(THREADS) k_readout(const Model m, Bufs b, int* __restrict__ idx,
                                                     double* __restrict__ p) {
    DevScalars* sc = b.sc;
    const long long ncell = min(*(volatile long long*)&sc->N, m.cap);
    const int g = *(volatile int*)&sc->gen, pb = *(volatile int*)&sc->pbuf;
    const T* Q = static_cast<const T*>(b.q[pb]);
    const unsigned short* om = b.om[g];
    const double w = *(volatile double*)&sc->w;
    long long c0, c1;
    block_chunk(ncell, c0, c1);
    long long base = b.blk[blockIdx.x];
    for (long long t0 = c0; t0 < c1; t0 += blockDim.x) {
        const long long c = t0 + threadIdx.x;
        const int f = c < c1 && !is_halo(om, c);
        int total;
        const int pos = block_exclusive_scan(f, total);
        if (f) {
            const long long r = base + pos;
            int I[N];
            unpack_key<N>(m, b.key[g][c], I);
#pragma unroll
            for (int k = 0; k < N; ++k) idx[r * N + k] = I[k];
            p[r] = __ddiv_rn((double)Q[c], w);
        }
        base += total;
    }
}

// Moments: pass 0 sums x_a p (a < n) into mom[a]; pass 1 sums
// (x_a - mean_a)(x_b - mean_b) p (a <= b) into mom[n + pair].
template <int N, typename T>
__global__ void __launch_bounds__(THREADS) k_moments(const Model m, Bufs b, int pass, const double* __restrict__ mean) {
    DevScalars* sc = b.sc;
    const long long ncell = min(*(volatile long long*)&sc->N, m.cap);
    const int g = *(volatile int*)&sc->gen, pb = *(volatile int*)&sc->pbuf;
    const T* Q = static_cast<const T*>(b.q[pb]);
    const double w = *(volatile double*)&sc->w;
    __shared__ unsigned long long s_acc[28][NDIG];
    for (int i = threadIdx.x; i < 28 * NDIG; i += blockDim.x) (&s_acc[0][0])[i] = 0;
    __syncthreads();
    int err = 0;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell;
         c += (long long)gridDim.x * blockDim.x) {
        int I[N];
        unpack_key<N>(m, b.key[g][c], I);
        const double p = __ddiv_rn((double)Q[c], w);
        double x[N];
#pragma unroll
        for (int k = 0; k < N; ++k) x[k] = centre64(m, k, I[k]);
        int slot = 0;
        if (pass == 0) {
            for (int a = 0; a < N; ++a, ++slot) {
                long long dd[NDIG] = {0, 0, 0, 0, 0, 0};
                acc_add(dd, __dmul_rn(x[a], p), err);
                for (int q = 0; q < NDIG; ++q)
                    if (dd[q]) atomicAdd(&s_acc[slot][q], (unsigned long long)dd[q]);
            }
        } else {
            for (int a = 0; a < N; ++a)
                for (int e = a; e < N; ++e, ++slot) {
                    long long dd[NDIG] = {0, 0, 0, 0, 0, 0};
                    double v = __dmul_rn(__dmul_rn(__dsub_rn(x[a], mean[a]), __dsub_rn(x[e], mean[e])), p);
                    acc_add(dd, v, err);
                    for (int q = 0; q < NDIG; ++q)
                        if (dd[q]) atomicAdd(&s_acc[slot][q], (unsigned long long)dd[q]);
                }
        }
    }
    if (err) set_error(sc, ST_EDEGENERATE);
    __syncthreads();
    for (int i = threadIdx.x; i < 28 * NDIG; i += blockDim.x) {
        unsigned long long v = (&s_acc[0][0])[i];
        if (v) atomicAdd((unsigned long long*)&sc->mom[0][0] + i, v);
    }
}

}  // namespace gbees
