// Kernels of the GBEES step other than the flux update: initial grid, directional
// grow (Sec. 3.3, Algorithm 2), neighbour links (Sec. 4.1), Bayesian update
// (Eq. 4), directional prune with stream compaction and rehash (Algorithm 3),
// read-out and moments. All kernels use a fixed grid and loop over the cells,
// whose count they read from device memory, so that no step needs the host.
#pragma once

#include "gbees_device.cuh"

namespace gbees {

template <typename T>
__device__ __forceinline__ double q_at(const void* q, long long c) {
    return (double)static_cast<const T*>(q)[c];
}

// Significant-cell threshold p* = thr_rel * max p (Sec. 3.3), on the stored scale.
__device__ __forceinline__ double pstar_of(const Model& m, const DevScalars* sc) { return m.thr_rel * sc->maxq; }

// The outward directions of cell I: bit 2j+1 when the flow leaves through the
// upper j-face (f_j at the upper face > 0), bit 2j when it leaves through the
// lower j-face (f_j at the lower face < 0). FP64, as in Eq. 7.
template <int N>
__device__ __forceinline__ unsigned outward_mask(const Model& m, const int* I) {
    unsigned msk = 0;
#pragma unroll
    for (int j = 0; j < N; ++j) {
        int J[N];
#pragma unroll
        for (int k = 0; k < N; ++k) J[k] = I[k] + (k == j ? 1 : 0);
        if (face_velocity64<N>(m, J, j) > 0.0) msk |= 1u << (2 * j + 1);
        if (face_velocity64<N>(m, I, j) < 0.0) msk |= 1u << (2 * j);
    }
    return msk;
}

// Index of cell c + s1 e_j + s2 e_d (j != d) through the links, -2 when both
// intermediate cells are missing (the links cannot tell).
__device__ __forceinline__ int edge_by_links(const int* __restrict__ link, long long cap, const int* L, int j, int s1,
                                             int d, int s2) {
    int a = L[2 * j + s1];
    if (a >= 0) return __ldcg(link + (long long)(2 * d + s2) * cap + a);
    int b = L[2 * d + s2];
    if (b >= 0) return __ldcg(link + (long long)(2 * j + s1) * cap + b);
    return -2;
}

// ------------------------------------------------------------------ begin / finalise

// Start a propagate call: record the target and whether any step is due.
__global__ void k_begin(DevScalars* sc, double t_target) {
    sc->t_target = t_target;
    sc->done = !(sc->t < t_target) || sc->error != 0;
    sc->steps_call = 0;
    sc->updates_call = 0;
}

__global__ void k_finalise(const Model m, DevScalars* sc, int mode) { finalise_norm(m, sc, mode); }

// ------------------------------------------------------------------ hashtable helpers

__global__ void k_table_clear(const Model m, Bufs b) {
    const unsigned long long T = m.tmask + 1;
    for (unsigned long long s = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; s < T;
         s += (unsigned long long)gridDim.x * blockDim.x) {
        reinterpret_cast<ulonglong2*>(b.table)[s] = make_ulonglong2(EMPTY_KEY, 0ull);
    }
}

// Insert cell c (key k) into the table; the key must be new.
__device__ __forceinline__ void table_insert_new(const Model& m, Bufs& b, unsigned long long k, long long c) {
    unsigned long long slot;
    int r = table_claim(m, b.table, k, &slot);
    if (r == 1) {
        b.table[slot].val = c;
    } else if (r == 0) {
        set_error(b.sc, ST_EINVAL);  // duplicate cell
    } else {
        set_error(b.sc, ST_ETABLE);
    }
}

// ------------------------------------------------------------------ links

// Link cells [N_prev, N) to their 2n face neighbours and write the reverse
// links into those neighbours (the neighbour references of Sec. 4.1). W lanes
// look up one key together (warp-cooperative probing).
template <int N, int W>
__global__ void __launch_bounds__(THREADS) k_link(const Model m, Bufs b) {
    DevScalars* sc = b.sc;
    if (*(volatile int*)&sc->error) return;
    const long long lo = *(volatile long long*)&sc->N_prev;
    const long long hi = min(*(volatile long long*)&sc->N, m.cap);
    const int g = *(volatile int*)&sc->gen;
    const unsigned long long* key = b.key[g];
    int* link = b.link[g];
    const long long cap = m.cap;
    auto tile = cg::tiled_partition<W>(cg::this_thread_block());
    const long long tiles_per_grid = (long long)gridDim.x * (blockDim.x / W);
    const long long tile_id = (long long)blockIdx.x * (blockDim.x / W) + threadIdx.x / W;
    const long long work = (hi - lo) * 2 * N;  // one lookup per (cell, direction)
    for (long long wi = tile_id; wi < work; wi += tiles_per_grid) {
        const long long c = lo + wi / (2 * N);
        const int dir = (int)(wi % (2 * N));
        const int j = dir >> 1, s = dir & 1;
        int I[N];
        unpack_key<N>(m, key[c], I);
        I[j] += s ? 1 : -1;
        unsigned long long k;
        int nb = -1;
        if (pack_key<N>(m, I, k)) {
            if (W == 1) nb = table_find(m, b.table, k);
            else nb = table_find_tile<W>(m, b.table, k, tile);
        }
        if (tile.thread_rank() == 0) {
            link[(long long)dir * cap + c] = nb;
            if (nb >= 0) link[(long long)(2 * j + (1 - s)) * cap + nb] = (int)c;
        }
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

// chunk [c0, c1) of a range of `total` items handled by this block
__device__ __forceinline__ void block_chunk(long long total, long long& c0, long long& c1) {
    long long per = (total + gridDim.x - 1) / gridDim.x;
    per = (per + THREADS - 1) / THREADS * THREADS;
    c0 = min(total, per * blockIdx.x);
    c1 = min(total, c0 + per);
}

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
        for (int w = 0; w < WARPS; ++w) t += s[w];
        b.blk[blockIdx.x] = t;
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
            } else if (!pack_key<N>(m, I, k)) {
                set_error(sc, ST_EKEYRANGE);
            } else {
                T v = (T)g;
                b.key[0][c] = k;
                static_cast<T*>(b.q[0])[c] = v;
                table_insert_new(m, b, k, c);
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

// Reset the grid scalars before an init.
__global__ void k_reset(DevScalars* sc, double t0) {
    sc->N = 0;
    sc->N_prev = 0;
    sc->N_new = 0;
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
        if (!pack_key<N>(m, I, k)) {
            set_error(sc, ST_EKEYRANGE);
            continue;
        }
        T v = (T)p[c];
        b.key[0][c] = k;
        static_cast<T*>(b.q[0])[c] = v;
        table_insert_new(m, b, k, c);
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

__global__ void k_set_count_from_new(DevScalars* sc) {
    sc->N = sc->N_new;
    sc->N_prev = 0;
}

__global__ void k_set_count(DevScalars* sc, long long count, long long step0) {
    sc->N = count;
    sc->N_prev = 0;
    sc->step = step0;
}

// ------------------------------------------------------------------ grow

template <int N, typename T>
__device__ __forceinline__ void grow_insert(const Model& m, Bufs& b, int g, int pb, const int* I) {
    DevScalars* sc = b.sc;
    unsigned long long k;
    if (!pack_key<N>(m, I, k)) {
        set_error(sc, ST_EKEYRANGE);
        return;
    }
    unsigned long long slot;
    int r = table_claim(m, b.table, k, &slot);
    if (r < 0) {
        set_error(sc, ST_ETABLE);
        return;
    }
    if (r == 0) return;
    long long c = warp_aggregated_add(&sc->N);
    if (c >= m.cap) {
        set_error(sc, ST_ECAPACITY);
        return;
    }
    b.table[slot].val = c;
    b.key[g][c] = k;
    static_cast<T*>(b.q[pb])[c] = (T)0;
    double r64 = cfl_rate64<N>(m, I);
    if (r64 > 0.0) atomicMax(&sc->maxrate_bits, (unsigned long long)__double_as_longlong(r64));
}

// Directional grow (Sec. 3.3): every significant cell inserts the missing
// cells of its downwind set with p = 0 (Algorithm 2 with an atomicCAS claim of
// the key instead of the staged insertion).
template <int N, typename T>
__global__ void __launch_bounds__(THREADS) k_grow(const Model m, Bufs b) {
    DevScalars* sc = b.sc;
    if (*(volatile int*)&sc->done | *(volatile int*)&sc->error) return;
    const long long ncell = min(*(volatile long long*)&sc->N_prev, m.cap);
    const int g = *(volatile int*)&sc->gen, pb = *(volatile int*)&sc->pbuf;
    const double pstar = m.thr_rel * *(volatile double*)&sc->maxq;
    const T* Q = static_cast<const T*>(b.q[pb]);
    const unsigned long long* key = b.key[g];
    const int* link = b.link[g];
    const long long cap = m.cap;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell;
         c += (long long)gridDim.x * blockDim.x) {
        if (!((double)Q[c] > pstar)) continue;
        int I[N];
        unpack_key<N>(m, key[c], I);
        const unsigned out = outward_mask<N>(m, I);
        if (!out) continue;
        int L[2 * N];
#pragma unroll
        for (int d = 0; d < 2 * N; ++d) L[d] = link[(long long)d * cap + c];
#pragma unroll
        for (int d = 0; d < 2 * N; ++d) {
            if (!((out >> d) & 1u) || L[d] >= 0) continue;
            int J[N];
#pragma unroll
            for (int k = 0; k < N; ++k) J[k] = I[k];
            J[d >> 1] += (d & 1) ? 1 : -1;
            grow_insert<N, T>(m, b, g, pb, J);
        }
#pragma unroll
        for (int d1 = 0; d1 < 2 * N; ++d1) {
            if (!((out >> d1) & 1u)) continue;
#pragma unroll
            for (int d2 = 0; d2 < 2 * N; ++d2) {
                if ((d2 >> 1) <= (d1 >> 1) || !((out >> d2) & 1u)) continue;
                int e = edge_by_links(link, cap, L, d1 >> 1, d1 & 1, d2 >> 1, d2 & 1);
                if (e >= 0) continue;
                int J[N];
#pragma unroll
                for (int k = 0; k < N; ++k) J[k] = I[k];
                J[d1 >> 1] += (d1 & 1) ? 1 : -1;
                J[d2 >> 1] += (d2 & 1) ? 1 : -1;
                grow_insert<N, T>(m, b, g, pb, J);
            }
        }
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
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell;
         c += (long long)gridDim.x * blockDim.x) {
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
    mx = block_max(mx);
    if (threadIdx.x == 0 && mx > -INFINITY) atomicMax(&sc->maxq_ord, ord_key(mx));
    if (last_block(sc) && threadIdx.x == 0) {
        sc->maxq = sc->maxq_ord ? ord_val(sc->maxq_ord) : 0.0;
        sc->maxq_ord = 0;
        sc->ticket = 0;
        sc->prune_now = 1;
    }
}

// ------------------------------------------------------------------ prune

// keep[c] = (p_c > p*): the significant cells S.
template <typename T>
__global__ void __launch_bounds__(THREADS) k_prune_mark(const Model m, Bufs b) {
    DevScalars* sc = b.sc;
    if (!*(volatile int*)&sc->prune_now || *(volatile int*)&sc->error) return;
    const long long ncell = min(*(volatile long long*)&sc->N, m.cap);
    const int pb = *(volatile int*)&sc->pbuf;
    const double pstar = m.thr_rel * *(volatile double*)&sc->maxq;
    const T* Q = static_cast<const T*>(b.q[pb]);
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell;
         c += (long long)gridDim.x * blockDim.x)
        b.keep[c] = (double)Q[c] > pstar;
}

// keep[D(S)] = 1: each significant cell marks the existing cells of its
// downwind set, so that a cell below threshold survives only when an upwind
// significant neighbour points at it (Sec. 3.3, Fig. 3).
template <int N, typename T>
__global__ void __launch_bounds__(THREADS) k_prune_scatter(const Model m, Bufs b) {
    DevScalars* sc = b.sc;
    if (!*(volatile int*)&sc->prune_now || *(volatile int*)&sc->error) return;
    const long long ncell = min(*(volatile long long*)&sc->N, m.cap);
    const int g = *(volatile int*)&sc->gen, pb = *(volatile int*)&sc->pbuf;
    const double pstar = m.thr_rel * *(volatile double*)&sc->maxq;
    const T* Q = static_cast<const T*>(b.q[pb]);
    const unsigned long long* key = b.key[g];
    const int* link = b.link[g];
    const long long cap = m.cap;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell;
         c += (long long)gridDim.x * blockDim.x) {
        if (!((double)Q[c] > pstar)) continue;
        int I[N];
        unpack_key<N>(m, key[c], I);
        const unsigned out = outward_mask<N>(m, I);
        if (!out) continue;
        int L[2 * N];
#pragma unroll
        for (int d = 0; d < 2 * N; ++d) L[d] = link[(long long)d * cap + c];
#pragma unroll
        for (int d = 0; d < 2 * N; ++d)
            if (((out >> d) & 1u) && L[d] >= 0) b.keep[L[d]] = 1;
#pragma unroll
        for (int d1 = 0; d1 < 2 * N; ++d1) {
            if (!((out >> d1) & 1u)) continue;
#pragma unroll
            for (int d2 = 0; d2 < 2 * N; ++d2) {
                if ((d2 >> 1) <= (d1 >> 1) || !((out >> d2) & 1u)) continue;
                int e = edge_by_links(link, cap, L, d1 >> 1, d1 & 1, d2 >> 1, d2 & 1);
                if (e == -2) {
                    int J[N];
#pragma unroll
                    for (int k = 0; k < N; ++k) J[k] = I[k];
                    J[d1 >> 1] += (d1 & 1) ? 1 : -1;
                    J[d2 >> 1] += (d2 & 1) ? 1 : -1;
                    unsigned long long kk;
                    e = pack_key<N>(m, J, kk) ? table_find(m, b.table, kk) : -1;
                }
                if (e >= 0) b.keep[e] = 1;
            }
        }
    }
}

// Per-block count of kept cells; the table is cleared here for the rehash.
__global__ void __launch_bounds__(THREADS) k_prune_count(const Model m, Bufs b) {
    DevScalars* sc = b.sc;
    if (!*(volatile int*)&sc->prune_now || *(volatile int*)&sc->error) return;
    const long long ncell = min(*(volatile long long*)&sc->N, m.cap);
    long long c0, c1;
    block_chunk(ncell, c0, c1);
    int cnt = 0;
    for (long long c = c0 + threadIdx.x; c < c1; c += blockDim.x) cnt += b.keep[c] != 0;
    for (int off = 16; off > 0; off >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, off);
    __shared__ int s[WARPS];
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long t = 0;
        for (int w = 0; w < WARPS; ++w) t += s[w];
        b.blk[blockIdx.x] = t;
    }
    const unsigned long long T = m.tmask + 1;
    for (unsigned long long s2 = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; s2 < T;
         s2 += (unsigned long long)gridDim.x * blockDim.x)
        reinterpret_cast<ulonglong2*>(b.table)[s2] = make_ulonglong2(EMPTY_KEY, 0ull);
}

__global__ void k_scan_prune(Bufs b, int nblk, long long cap) {
    if (!*(volatile int*)&b.sc->prune_now || *(volatile int*)&b.sc->error) return;
    // same as k_scan_blocks, guarded
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
    }
    __syncthreads();
    long long run = s_part[threadIdx.x];
    for (int i = i0; i < i0 + per && i < nblk; ++i) {
        long long v = b.blk[i];
        b.blk[i] = run;
        run += v;
    }
}

// Stream compaction of the kept cells in storage order into the other buffer
// set; map[c] = new index or -1. Reduces the sum, maximum and CFL rates of
// the survivors.
template <int N, typename T>
__global__ void __launch_bounds__(THREADS) k_prune_compact(const Model m, Bufs b) {
    DevScalars* sc = b.sc;
    if (!*(volatile int*)&sc->prune_now || *(volatile int*)&sc->error) return;
    const long long ncell = min(*(volatile long long*)&sc->N, m.cap);
    const int g = *(volatile int*)&sc->gen, pb = *(volatile int*)&sc->pbuf;
    const T* Q = static_cast<const T*>(b.q[pb]);
    T* Qo = static_cast<T*>(b.q[pb ^ 1]);
    const unsigned long long* key = b.key[g];
    unsigned long long* keyo = b.key[g ^ 1];
    // Exact power-of-two rescale that brings the maximum into [1, 2): the values
    // keep their ratios bit for bit and the exact sum stays inside its window
    // even after a very unlikely measurement.
    const double mq = *(volatile double*)&sc->maxq;
    const double s2 = (mq > 0.0 && isfinite(mq)) ? ldexp(1.0, -ilogb(mq)) : 1.0;
    long long c0, c1;
    block_chunk(ncell, c0, c1);
    long long base = b.blk[blockIdx.x];
    long long d[NDIG] = {0, 0, 0, 0, 0, 0};
    double mx = -INFINITY, rmax = 0.0;
    int err = 0;
    for (long long t0 = c0; t0 < c1; t0 += blockDim.x) {
        long long c = t0 + threadIdx.x;
        int f = (c < c1) ? (b.keep[c] != 0) : 0;
        int total;
        int pos = block_exclusive_scan(f, total);
        if (c < c1) {
            if (f) {
                long long nc = base + pos;
                unsigned long long k = key[c];
                T v = (T)((double)Q[c] * s2);
                keyo[nc] = k;
                Qo[nc] = v;
                b.map[c] = (int)nc;
                acc_add(d, (double)v, err);
                mx = fmax(mx, (double)v);
                int I[N];
                unpack_key<N>(m, k, I);
                rmax = fmax(rmax, cfl_rate64<N>(m, I));
            } else {
                b.map[c] = -1;
            }
        }
        base += total;
    }
    if (err) set_error(sc, ST_EDEGENERATE);
    block_reduce_acc_max(d, mx, sc->acc, &sc->maxq_ord);
    double r = block_max(rmax);
    if (threadIdx.x == 0 && r > 0.0) atomicMax(&sc->maxrate_new_bits, (unsigned long long)__double_as_longlong(r));
}

// New links through the map and the rehash of the survivors (Algorithm 3's
// final steps); the last block swaps the buffers and normalises.
template <int N>
__global__ void __launch_bounds__(THREADS) k_prune_relink(const Model m, Bufs b) {
    DevScalars* sc = b.sc;
    if (!*(volatile int*)&sc->prune_now || *(volatile int*)&sc->error) return;
    const long long ncell = min(*(volatile long long*)&sc->N, m.cap);
    const int g = *(volatile int*)&sc->gen;
    const int* link = b.link[g];
    int* linko = b.link[g ^ 1];
    const unsigned long long* keyo = b.key[g ^ 1];
    const long long cap = m.cap;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell;
         c += (long long)gridDim.x * blockDim.x) {
        const int nc = b.map[c];
        if (nc < 0) continue;
#pragma unroll
        for (int d = 0; d < 2 * N; ++d) {
            int l = link[(long long)d * cap + c];
            linko[(long long)d * cap + nc] = l >= 0 ? b.map[l] : -1;
        }
        table_insert_new(m, b, keyo[nc], nc);
    }
    if (last_block(sc) && threadIdx.x == 0) finalise_norm(m, sc, 1);
}

// ------------------------------------------------------------------ read-out

template <int N, typename T>
__global__ void __launch_bounds__(THREADS) k_readout(const Model m, Bufs b, int* __restrict__ idx,
                                                     double* __restrict__ p) {
    DevScalars* sc = b.sc;
    const long long ncell = min(*(volatile long long*)&sc->N, m.cap);
    const int g = *(volatile int*)&sc->gen, pb = *(volatile int*)&sc->pbuf;
    const T* Q = static_cast<const T*>(b.q[pb]);
    const double w = *(volatile double*)&sc->w;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell;
         c += (long long)gridDim.x * blockDim.x) {
        int I[N];
        unpack_key<N>(m, b.key[g][c], I);
#pragma unroll
        for (int k = 0; k < N; ++k) idx[c * N + k] = I[k];
        p[c] = __ddiv_rn((double)Q[c], w);
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

__global__ void k_moments_clear(DevScalars* sc) {
    for (int i = threadIdx.x; i < 28 * NDIG; i += blockDim.x) (&sc->mom[0][0])[i] = 0;
}

// Convert the moment sums to doubles times prod h: out[slot].
__global__ void k_moments_final(const Model m, DevScalars* sc, double* out, int nslots) {
    int s = threadIdx.x;
    if (s < nslots) out[s] = __dmul_rn(m.prod_h, acc_to_double(sc->mom[s]));
}

}  // namespace gbees
