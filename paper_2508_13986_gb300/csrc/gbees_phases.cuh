// The phases of one GBEES time step as device functions over "all threads of
// the grid", shared by the one-kernel-per-phase path (gbees_kernels.cuh, run as
// a CUDA graph) and the persistent cooperative kernel (gbees_persistent.cuh).
// Data that a phase writes is read by later phases of the same persistent
// launch, so no pointer here is marked read-only (no non-coherent loads): the
// grid barrier's fences make plain loads see the other blocks' writes.
//
//   grow       directional grow of the significant cells (Sec. 3.3, Algorithm 2)
//   link       neighbour links, outward mask and CFL rate of the new cells (Sec. 4.1)
//   waves      FP64: per-cell velocities u_d and entering waves G_d
//   faces      FP64: one flux per face (Eq. 7 + Algorithm 1 gathered + HR term)
//   apply      FP64: P -= sum_j dt/h_j (F_hi - F_lo), normalised, reduced
//   gather     single-pass update (any precision), normalised, reduced
//   prune      mark S, mark D(S), count, compact, relink and rehash (Algorithm 3)
#pragma once

#include "gbees_device.cuh"

namespace gbees {

// What a phase needs to know about the step in progress.
struct StepView {
    long long N;       // active cells (clamped to the capacity)
    long long N_prev;  // cells before this step's grow
    int pb, g;         // current value buffer and key/link buffer
    double maxq;       // max stored value (threshold p* = thr_rel * maxq)
    double scale;      // 1 / w of the previous normalisation
    double dth[MAXN];  // dt / h_j of this step
    double ch[MAXN];   // dt / (2 h_j)
    double dt;         // dt of this step
};

__device__ __forceinline__ StepView view_of(const Model& m, DevScalars* sc) {
    StepView v;
    v.N = min(*(volatile long long*)&sc->N, m.cap);
    v.N_prev = min(*(volatile long long*)&sc->N_prev, m.cap);
    v.pb = *(volatile int*)&sc->pbuf;
    v.g = *(volatile int*)&sc->gen;
    v.maxq = *(volatile double*)&sc->maxq;
    v.scale = *(volatile double*)&sc->scale;
    for (int j = 0; j < MAXN; ++j) {
        v.dth[j] = *(volatile double*)&sc->coef_dth[j];
        v.ch[j] = *(volatile double*)&sc->coef_ch[j];
    }
    v.dt = *(volatile double*)&sc->step_dt;
    return v;
}

// dt of Eq. 8 (CFL over the maximum rate, clipped to land on the target) and
// its coefficients; the same IEEE operations wherever it is evaluated.
struct StepTime {
    double dt, t_new;
    int last;
};
__device__ __forceinline__ StepTime step_time(const Model& m, double rate, double t, double tt, double* dth,
                                              double* ch) {
    double dt = rate > 0.0 ? __ddiv_rn(m.cfl, rate) : (double)INFINITY;
    const double rem = __dsub_rn(tt, t);
    const bool last = dt >= rem;
    if (last) dt = rem;
    for (int j = 0; j < MAXN; ++j) {
        dth[j] = j < m.n ? dt * m.inv_h[j] : 0.0;
        ch[j] = j < m.n ? dt * m.inv_2h[j] : 0.0;
    }
    StepTime s;
    s.dt = dt;
    s.last = last;
    s.t_new = last ? tt : __dadd_rn(t, dt);
    return s;
}

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
__device__ __forceinline__ int edge_by_links(const int* link, long long cap, const int* L, int j, int s1,
                                             int d, int s2) {
    int a = L[2 * j + s1];
    if (a >= 0) return __ldcg(link + (long long)(2 * d + s2) * cap + a);
    int b = L[2 * d + s2];
    if (b >= 0) return __ldcg(link + (long long)(2 * j + s1) * cap + b);
    return -2;
}

// Insert cell c (key k) into the table; the key must be new. slots[c]
// records the table slot, so that a prune can empty exactly the used slots.
__device__ __forceinline__ void table_insert_new(const Model& m, const Bufs& b, unsigned long long k, long long c,
                                                 unsigned int* slots) {
    unsigned long long slot;
    int r = table_claim(m, b.table, k, &slot);
    if (r == 1) {
        b.table[slot].val = c;
        slots[c] = (unsigned int)slot;
    } else if (r == 0) {
        set_error(b.sc, ST_EINVAL);  // duplicate cell
    } else {
        set_error(b.sc, ST_ETABLE);
    }
}

// ------------------------------------------------------------------ grow

// Claim cell I if absent and append it with p = 0 (its links, outward mask and
// rate are set by the link phase).
template <int N, typename T>
__device__ __forceinline__ void grow_insert(const Model& m, const Bufs& b, int g, int pb, const int* I) {
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
    b.slot[g][c] = (unsigned int)slot;
    b.key[g][c] = k;
    static_cast<T*>(b.q[pb])[c] = (T)0;
}

// Directional grow (Sec. 3.3): every significant cell inserts the missing cells
// of its downwind set. A cell whose downwind set was found complete since the
// last prune is skipped.
template <int N, typename T>
__device__ __forceinline__ void grow_body(const Model& m, const Bufs& b, const StepView& v) {
    const long long ncell = v.N_prev;
    const double pstar = m.thr_rel * v.maxq;
    const T* Q = static_cast<const T*>(b.q[v.pb]);
    const unsigned long long* key = b.key[v.g];
    const int* link = b.link[v.g];
    unsigned short* om = b.om[v.g];
    const long long cap = m.cap;
    for (WarpRuns r(ncell); r.next();) {
        const long long c = r.c;
        if (c >= ncell) continue;
        if (!((double)Q[c] > pstar)) continue;
        const unsigned f = om[c];
        if (f & OM_COMPLETE) continue;
        const unsigned out = f & 0xfffu;
        if (out) {
            int I[N];
            unpack_key<N>(m, key[c], I);
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
                grow_insert<N, T>(m, b, v.g, v.pb, J);
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
                    grow_insert<N, T>(m, b, v.g, v.pb, J);
                }
            }
        }
        om[c] = (unsigned short)(f | OM_COMPLETE);
    }
}

// ------------------------------------------------------------------ link

// Cells [lo, hi) are new: look up their 2n face neighbours (one probe per
// thread and direction), write the reverse links into the neighbours, and set
// their outward masks; returns this thread's largest CFL rate among them.
template <int N>
__device__ __forceinline__ double link_body(const Model& m, const Bufs& b, long long lo, long long hi, int g) {
    const unsigned long long* key = b.key[g];
    int* link = b.link[g];
    const long long cap = m.cap;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nth = (long long)gridDim.x * blockDim.x;
    const long long work = (hi - lo) * 2 * N;
    for (long long wi = tid; wi < work; wi += nth) {
        const long long c = lo + wi / (2 * N);
        const int dir = (int)(wi % (2 * N));
        const int j = dir >> 1, s = dir & 1;
        int I[N];
        unpack_key<N>(m, key[c], I);
        I[j] += s ? 1 : -1;
        unsigned long long k;
        int nb = pack_key<N>(m, I, k) ? table_find(m, b.table, k) : -1;
        link[(long long)dir * cap + c] = nb;
        if (nb >= 0) link[(long long)(2 * j + (1 - s)) * cap + nb] = (int)c;
    }
    double rmax = 0.0;
    for (long long c = lo + tid; c < hi; c += nth) {
        int I[N];
        unpack_key<N>(m, key[c], I);
        b.om[g][c] = (unsigned short)outward_mask<N>(m, I);
        rmax = fmax(rmax, cfl_rate64<N>(m, I));
    }
    return rmax;
}

// Cooperative variant: W lanes probe W consecutive slots together.
template <int N, int W>
__device__ __forceinline__ double link_body_tile(const Model& m, const Bufs& b, long long lo, long long hi, int g) {
    const unsigned long long* key = b.key[g];
    int* link = b.link[g];
    const long long cap = m.cap;
    auto tile = cg::tiled_partition<W>(cg::this_thread_block());
    const long long tiles = (long long)gridDim.x * (blockDim.x / W);
    const long long tile_id = (long long)blockIdx.x * (blockDim.x / W) + threadIdx.x / W;
    const long long work = (hi - lo) * 2 * N;
    for (long long wi = tile_id; wi < work; wi += tiles) {
        const long long c = lo + wi / (2 * N);
        const int dir = (int)(wi % (2 * N));
        const int j = dir >> 1, s = dir & 1;
        int I[N];
        unpack_key<N>(m, key[c], I);
        I[j] += s ? 1 : -1;
        unsigned long long k;
        int nb = pack_key<N>(m, I, k) ? table_find_tile<W>(m, b.table, k, tile) : -1;
        if (tile.thread_rank() == 0) {
            link[(long long)dir * cap + c] = nb;
            if (nb >= 0) link[(long long)(2 * j + (1 - s)) * cap + nb] = (int)c;
        }
    }
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nth = (long long)gridDim.x * blockDim.x;
    double rmax = 0.0;
    for (long long c = lo + tid; c < hi; c += nth) {
        int I[N];
        unpack_key<N>(m, key[c], I);
        b.om[g][c] = (unsigned short)outward_mask<N>(m, I);
        rmax = fmax(rmax, cfl_rate64<N>(m, I));
    }
    return rmax;
}

// ------------------------------------------------------------------ FP64 three-pass update

// Index of c + s1 e_j + s2 e_d (j != d, s = 0 down, 1 up) through the links,
// falling back to the hashtable when both intermediate cells are missing.
template <int N>
__device__ __forceinline__ int edge_index(const Model& m, const Bufs& b, const int* link, long long cap,
                                          const int* L, const int* I, int j, int s1, int d, int s2, long long& fb) {
    int a = L[2 * j + s1];
    if (a >= 0) return __ldcg(link + (long long)(2 * d + s2) * cap + a);
    int c2 = L[2 * d + s2];
    if (c2 >= 0) return __ldcg(link + (long long)(2 * j + s1) * cap + c2);
    int J[N];
#pragma unroll
    for (int k = 0; k < N; ++k) J[k] = I[k];
    J[j] += s1 ? 1 : -1;
    J[d] += s2 ? 1 : -1;
    unsigned long long kk;
    ++fb;
    return pack_key<N>(m, J, kk) ? table_find(m, b.table, kk) : -1;
}

// Index of c + 2 s e_j.
template <int N>
__device__ __forceinline__ int second_index(const Model& m, const Bufs& b, const int* link,
                                            long long cap, const int* L, const int* I, int j, int s, long long& fb) {
    int a = L[2 * j + s];
    if (a >= 0) return __ldcg(link + (long long)(2 * j + s) * cap + a);
    int J[N];
#pragma unroll
    for (int k = 0; k < N; ++k) J[k] = I[k];
    J[j] += s ? 2 : -2;
    unsigned long long kk;
    ++fb;
    return pack_key<N>(m, J, kk) ? table_find(m, b.table, kk) : -1;
}

template <typename T>
__device__ __forceinline__ T q_or_zero(const T* Q, int i) {
    return i >= 0 ? Q[i] : (T)0;
}

// sum_{d != j} dt/(2 h_d) G_d(Y) for the missing cell Y = c + s e_j (P_Y = 0).
template <int N, int DYN, typename T>
__device__ __forceinline__ T waves_of_missing(const Model& m, const Bufs& b, const T* Q,
                                              const int* link, long long cap, const int* L, const int* I,
                                              const T* xc, const T* h, const T* ch, int j, int s, long long& fb) {
    T S = (T)0;
#pragma unroll
    for (int d = 0; d < N; ++d) {
        if (d == j) continue;
        const T Pm = q_or_zero<T>(Q, edge_index<N>(m, b, link, cap, L, I, j, s, d, 0, fb));
        const T Pp = q_or_zero<T>(Q, edge_index<N>(m, b, link, cap, L, I, j, s, d, 1, fb));
        const T ul = vel_at<N, DYN, T>(m, xc, h, j, s ? 1 : -1, d, -1);
        const T uh = vel_at<N, DYN, T>(m, xc, h, j, s ? 1 : -1, d, +1);
        S += ch[d] * (fmax(ul, (T)0) * ((T)0 - Pm) + fmin(uh, (T)0) * Pp);
    }
    return S;
}

// Pass 1, one work item per (cell, dimension d) of the cells [0, ncell): the
// lower-face velocity u_d and the entering wave G_d of the cell. New cells (of
// this step's grow) are left out: with P = 0 their waves are formed on the spot.
template <int N, int DYN>
__device__ __forceinline__ void waves_body(const Model& m, const Bufs& b, const StepView& v, long long ncell) {
    const double* Q = static_cast<const double*>(b.q[v.pb]);
    const unsigned long long* key = b.key[v.g];
    const int* link = b.link[v.g];
    const long long cap = m.cap;
    const long long items = ncell * N;
    double h[N];
#pragma unroll
    for (int k = 0; k < N; ++k) h[k] = m.h[k];
    for (WarpRuns wr(items); wr.next();) {
        const long long it = wr.c;
        if (it >= items) continue;
        const long long c = it / N;
        const int d = (int)(it - c * N);
        int I[N];
        unpack_key<N>(m, key[c], I);
        const double P0 = Q[c];
        const double Pm = q_or_zero<double>(Q, link[(long long)(2 * d) * cap + c]);
        const double Pp = q_or_zero<double>(Q, link[(long long)(2 * d + 1) * cap + c]);
        double xc[N];
#pragma unroll
        for (int k = 0; k < N; ++k) xc[k] = m.x0[k] + (double)I[k] * h[k];
        double ul = 0.0, uh = 0.0;
#pragma unroll
        for (int dd = 0; dd < N; ++dd)
            if (dd == d) {
                ul = vel_at<N, DYN, double>(m, xc, h, -1, 0, dd, -1);
                uh = vel_at<N, DYN, double>(m, xc, h, -1, 0, dd, +1);
            }
        b.wv_u[(long long)d * cap + c] = ul;
        b.wv_g[(long long)d * cap + c] = fmax(ul, 0.0) * (P0 - Pm) + fmin(uh, 0.0) * (Pp - P0);
    }
}

// sum_{d != j} dt/(2 h_d) G_d(Y) for Y = c + s e_j (s = -1, 0, +1) formed on the
// spot: y is Y's index (-1 when Y is missing, then P_Y = 0 and its transverse
// neighbours are found through c's links). Used for missing and new cells.
template <int N, int DYN>
__device__ __forceinline__ double waves_here(const Model& m, const Bufs& b, const double* Q, const int* link,
                                             long long cap, const int* L, const int* I, const double* xc,
                                             const double* h, const double* ch, int j, int s, long long y,
                                             long long& fb) {
    const double PY = y >= 0 ? Q[y] : 0.0;
    double S = 0.0;
#pragma unroll
    for (int d = 0; d < N; ++d) {
        if (d == j) continue;
        double Pm, Pp;
        if (y >= 0) {
            Pm = q_or_zero<double>(Q, link[(long long)(2 * d) * cap + y]);
            Pp = q_or_zero<double>(Q, link[(long long)(2 * d + 1) * cap + y]);
        } else {
            Pm = q_or_zero<double>(Q, edge_index<N>(m, b, link, cap, L, I, j, s > 0, d, 0, fb));
            Pp = q_or_zero<double>(Q, edge_index<N>(m, b, link, cap, L, I, j, s > 0, d, 1, fb));
        }
        const double ul = vel_at<N, DYN, double>(m, xc, h, s ? j : -1, s, d, -1);
        const double uh = vel_at<N, DYN, double>(m, xc, h, s ? j : -1, s, d, +1);
        S += ch[d] * (fmax(ul, 0.0) * (PY - Pm) + fmin(uh, 0.0) * (Pp - PY));
    }
    return S;
}

// Boundary faces, one item per (cell c, face f = 2j + s) of the cells [0, ncell)
// whose neighbour across f is missing; run before grow (with it), so that a
// neighbour that grow creates (P = 0, like a missing cell) has the same waves.
// Writes bu (face velocity) and, when the missing neighbour is upwind of the
// face, bt (its transverse waves over 2 h_d) and bp (the value two cells away).
template <int N, int DYN, typename T>
__device__ __forceinline__ void boundary_body(const Model& m, const Bufs& b, const StepView& v, long long ncell) {
    const T* Q = static_cast<const T*>(b.q[v.pb]);
    const unsigned long long* key = b.key[v.g];
    const int* link = b.link[v.g];
    const long long cap = m.cap;
    T* bu = static_cast<T*>(b.bu);
    T* bt = static_cast<T*>(b.bt);
    T* bp = static_cast<T*>(b.bp);
    T h[N], x0[N], i2h[N];
#pragma unroll
    for (int k = 0; k < N; ++k) {
        h[k] = sizeof(T) == 4 ? (T)m.hf[k] : (T)m.h[k];
        x0[k] = sizeof(T) == 4 ? (T)m.x0f[k] : (T)m.x0[k];
        i2h[k] = (T)m.inv_2h[k];
    }
    long long fb = 0;
    const long long items = ncell * 2 * N;
    // grow runs concurrently: only cells below ncell count, anything it creates
    // (or a slot it has claimed but not yet filled, value -1) is P = 0
    auto qold = [&](int i) -> T { return (i >= 0 && i < ncell) ? Q[i] : (T)0; };
    for (WarpRuns wr(items); wr.next();) {
        const long long it = wr.c;
        if (it >= items) continue;
        const long long c = it / (2 * N);
        const int f = (int)(it - c * 2 * N);
        if (link[(long long)f * cap + c] >= 0) continue;
        const int j = f >> 1, s = f & 1;
        int I[N];
        unpack_key<N>(m, key[c], I);
        T xc[N];
#pragma unroll
        for (int k = 0; k < N; ++k) xc[k] = x0[k] + (T)I[k] * h[k];
        T u = (T)0;
#pragma unroll
        for (int d = 0; d < N; ++d)
            if (d == j) u = vel_at<N, DYN, T>(m, xc, h, -1, 0, d, s ? +1 : -1);
        bu[(long long)f * cap + c] = u;
        if (s ? !(u < (T)0) : !(u > (T)0)) continue;  // the missing neighbour is not upwind
        int L[2 * N];
#pragma unroll
        for (int d = 0; d < 2 * N; ++d) L[d] = link[(long long)d * cap + c];
        const int sgn = s ? 1 : -1;
        T S = (T)0;
#pragma unroll
        for (int d = 0; d < N; ++d) {
            if (d == j) continue;
            const T Pm = qold(edge_index<N>(m, b, link, cap, L, I, j, s, d, 0, fb));
            const T Pp = qold(edge_index<N>(m, b, link, cap, L, I, j, s, d, 1, fb));
            const T ul = vel_at<N, DYN, T>(m, xc, h, j, sgn, d, -1);
            const T uh = vel_at<N, DYN, T>(m, xc, h, j, sgn, d, +1);
            S += i2h[d] * (fmax(ul, (T)0) * ((T)0 - Pm) + fmin(uh, (T)0) * Pp);
        }
        bt[(long long)f * cap + c] = S;
        bp[(long long)f * cap + c] = qold(second_index<N>(m, b, link, cap, L, I, j, s, fb));
    }
    if (fb) atomicAdd((unsigned long long*)&b.sc->lookups_fallback, (unsigned long long)fb);
}

// Pass 2, one work item per (cell c, dimension j): the flux through the lower
// j-face of c, and through its upper j-face when the upper neighbour is missing
// (Eq. 7, the gathered corrections of Algorithm 1, the limited HR term).
// Returns the fallback lookups.
template <int N, int DYN>
__device__ __forceinline__ long long faces_body(const Model& m, const Bufs& b, const StepView& v) {
    const long long ncell = v.N;
    const long long nold = v.N_prev;
    const double* Q = static_cast<const double*>(b.q[v.pb]);
    const unsigned long long* key = b.key[v.g];
    const int* link = b.link[v.g];
    const double* wu = b.wv_u;
    const double* wg = b.wv_g;
    const long long cap = m.cap;
    const int lim = m.limiter;
    double h[N];
#pragma unroll
    for (int k = 0; k < N; ++k) h[k] = m.h[k];
    long long fb = 0;
    const long long items = ncell * N;
    for (WarpRuns wr(items); wr.next();) {
        const long long it = wr.c;
        if (it >= items) continue;
        const long long c = it / N;
        const int j = (int)(it - c * N);
        const int Llo = link[(long long)(2 * j) * cap + c];
        const int Lhi = link[(long long)(2 * j + 1) * cap + c];
        const double P0 = Q[c];
        const double PL = q_or_zero<double>(Q, Llo);
        const double dthj = v.dth[j];
        int L[2 * N];
        int I[N];
        double xc[N];
        bool have_pos = false;
        auto pos = [&]() {
            if (!have_pos) {
#pragma unroll
                for (int d = 0; d < 2 * N; ++d) L[d] = link[(long long)d * cap + c];
                unpack_key<N>(m, key[c], I);
#pragma unroll
                for (int k = 0; k < N; ++k) xc[k] = m.x0[k] + (double)I[k] * h[k];
                have_pos = true;
            }
        };
        auto face_u = [&](int side) -> double {  // velocity at the lower (0) or upper (1) j-face of c
            pos();
            double u = 0.0;
#pragma unroll
            for (int dd = 0; dd < N; ++dd)
                if (dd == j) u = vel_at<N, DYN, double>(m, xc, h, -1, 0, dd, side ? +1 : -1);
            return u;
        };
        const bool old_cell = c < nold;
        const double* bt = static_cast<const double*>(b.bt);
        const double* bp = static_cast<const double*>(b.bp);
        const double* bu = static_cast<const double*>(b.bu);
        // transverse sum of the upwind cell Y = c + s e_j with index y; a missing or
        // new neighbour of an old cell has its sum precomputed (boundary_body)
        auto trans = [&](int s, long long y) -> double {
            if (y >= 0 && y < nold) {
                double S = 0.0;
#pragma unroll
                for (int d = 0; d < N; ++d)
                    if (d != j) S += v.ch[d] * wg[(long long)d * cap + y];
                return S;
            }
            if (old_cell && s != 0) {
                const int f = 2 * j + (s > 0);
                return v.dt * bt[(long long)f * cap + c];
            }
            pos();
            return waves_here<N, DYN>(m, b, Q, link, cap, L, I, xc, h, v.ch, j, s, y, fb);
        };
        // value at c + 2 s e_j (limiter)
        auto second = [&](int s) -> double {
            const int Lm = s > 0 ? Lhi : Llo;
            if (Lm >= 0) return q_or_zero<double>(Q, link[(long long)(2 * j + (s > 0)) * cap + Lm]);
            if (old_cell) return bp[(long long)(2 * j + (s > 0)) * cap + c];
            pos();
            return q_or_zero<double>(Q, second_index<N>(m, b, link, cap, L, I, j, s > 0, fb));
        };
        {  // lower face (c, j)
            const double u = old_cell ? wu[(long long)j * cap + c] : face_u(0);
            double f = 0.0;
            if (u != 0.0) {
                f = fmax(u, 0.0) * PL + fmin(u, 0.0) * P0;  // Eq. 7
                const double S = u > 0.0 ? trans(-1, (long long)Llo) : trans(0, c);
                f -= u * S;  // Algorithm 1, gathered
                const double W = P0 - PL;
                if (lim != LIM_NONE && W != 0.0) {
                    double Wup;
                    if (u > 0.0) {
                        Wup = PL - second(-1);
                    } else {
                        Wup = q_or_zero<double>(Q, Lhi) - P0;
                    }
                    const double au = fabs(u);
                    f += 0.5 * au * (1.0 - dthj * au) * limited_wave<double>(lim, W, Wup);
                }
            }
            b.fl[(long long)j * cap + c] = f;
        }
        if (Lhi < 0) {  // upper face (c + e_j, j): nobody else owns it
            const double u = old_cell ? bu[(long long)(2 * j + 1) * cap + c] : face_u(1);
            double f = 0.0;
            if (u != 0.0) {
                f = fmax(u, 0.0) * P0;  // PR = 0
                const double S = u > 0.0 ? trans(0, c) : trans(+1, -1);
                f -= u * S;
                const double W = 0.0 - P0;
                if (lim != LIM_NONE && W != 0.0) {
                    double Wup;
                    if (u > 0.0) {
                        Wup = P0 - PL;
                    } else {
                        Wup = second(+1) - 0.0;
                    }
                    const double au = fabs(u);
                    f += 0.5 * au * (1.0 - dthj * au) * limited_wave<double>(lim, W, Wup);
                }
            }
            b.fu[(long long)j * cap + c] = f;
        }
    }
    return fb;
}

// Pass 3: the conservative update with the previous normalisation applied;
// adds this thread's new values to its digits and maximum.
template <int N>
__device__ __forceinline__ void apply_body(const Model& m, const Bufs& b, const StepView& v, long long (&dacc)[NDIG],
                                           double& mx, int& err) {
    const long long ncell = v.N;
    const double* Q = static_cast<const double*>(b.q[v.pb]);
    double* Qn = static_cast<double*>(b.q[v.pb ^ 1]);
    const int* link = b.link[v.g];
    const double* fl = b.fl;
    const double* fu = b.fu;
    const long long cap = m.cap;
    const double scale = v.scale;
    for (WarpRuns wr(ncell); wr.next();) {
        const long long c = wr.c;
        if (c >= ncell) continue;
        double upd = 0.0;
#pragma unroll
        for (int j = 0; j < N; ++j) {
            const int up = link[(long long)(2 * j + 1) * cap + c];
            const double Fhi = up >= 0 ? fl[(long long)j * cap + up] : fu[(long long)j * cap + c];
            upd += v.dth[j] * (Fhi - fl[(long long)j * cap + c]);
        }
        const double qn = (Q[c] - upd) * scale;
        Qn[c] = qn;
        acc_add(dacc, qn, err);
        mx = fmax(mx, qn);
    }
}

// ------------------------------------------------------------------ single-pass gather update

// Every cell computes its 2n face fluxes from its own neighbourhood. The
// corrections that Algorithm 1 scatters onto face (X, j) add up to
//   -u_j(X) sum_{d != j} dt/(2 h_d) G_d(Y),  Y the cell upwind of the face,
//   G_d(Y) = max(u_d(Y), 0) (P_Y - P_{Y-e_d}) + min(u_d(Y+e_d), 0) (P_{Y+e_d} - P_Y),
// so each cell needs its face neighbours, the transverse neighbours of each
// upwind face neighbour, and one cell two steps away per dimension (limiter).
template <int N, int DYN, typename T>
__device__ __forceinline__ long long gather_body(const Model& m, const Bufs& b, const StepView& v,
                                                 long long (&dacc)[NDIG], double& mx, int& err) {
    const long long ncell = v.N;
    const T* Q = static_cast<const T*>(b.q[v.pb]);
    T* Qn = static_cast<T*>(b.q[v.pb ^ 1]);
    const unsigned long long* key = b.key[v.g];
    const int* link = b.link[v.g];
    const long long cap = m.cap;
    const int lim = m.limiter;
    const T scale = (T)v.scale;
    T h[N], dth[N], ch[N];
#pragma unroll
    for (int j = 0; j < N; ++j) {
        h[j] = (T)m.h[j];
        dth[j] = (T)v.dth[j];
        ch[j] = (T)v.ch[j];
    }
    long long fb = 0;
    for (WarpRuns wr(ncell); wr.next();) {
        const long long c = wr.c;
        if (c >= ncell) continue;
        int I[N];
        unpack_key<N>(m, key[c], I);
        int L[2 * N];
#pragma unroll
        for (int d = 0; d < 2 * N; ++d) L[d] = link[(long long)d * cap + c];
        const T P0 = Q[c];
        T Pn[2 * N];
#pragma unroll
        for (int d = 0; d < 2 * N; ++d) Pn[d] = q_or_zero<T>(Q, L[d]);
        T xc[N];
#pragma unroll
        for (int k = 0; k < N; ++k) xc[k] = (T)m.x0[k] + (T)I[k] * h[k];
        T ulo[N], uhi[N];
#pragma unroll
        for (int j = 0; j < N; ++j) {
            ulo[j] = vel_at<N, DYN, T>(m, xc, h, -1, 0, j, -1);
            uhi[j] = vel_at<N, DYN, T>(m, xc, h, -1, 0, j, +1);
        }
        T Gc[N];
#pragma unroll
        for (int d = 0; d < N; ++d)
            Gc[d] = fmax(ulo[d], (T)0) * (P0 - Pn[2 * d]) + fmin(uhi[d], (T)0) * (Pn[2 * d + 1] - P0);
        // sum_{d != j} dt/(2 h_d) G_d(c + s e_j), the neighbour possibly missing
        auto trans_nb = [&](int j, int sj) -> T {
            const T PY = Pn[2 * j + sj];
            const int sgn = sj ? 1 : -1;
            T S = (T)0;
#pragma unroll
            for (int d = 0; d < N; ++d) {
                if (d == j) continue;
                const T Pm = q_or_zero<T>(Q, edge_index<N>(m, b, link, cap, L, I, j, sj, d, 0, fb));
                const T Pp = q_or_zero<T>(Q, edge_index<N>(m, b, link, cap, L, I, j, sj, d, 1, fb));
                const T ul = vel_at<N, DYN, T>(m, xc, h, j, sgn, d, -1);
                const T uh = vel_at<N, DYN, T>(m, xc, h, j, sgn, d, +1);
                S += ch[d] * (fmax(ul, (T)0) * (PY - Pm) + fmin(uh, (T)0) * (Pp - PY));
            }
            return S;
        };
        T upd = (T)0;
#pragma unroll
        for (int j = 0; j < N; ++j) {
            T F[2];
#pragma unroll
            for (int side = 0; side < 2; ++side) {
                const T u = side ? uhi[j] : ulo[j];
                const T PL = side ? P0 : Pn[2 * j];
                const T PR = side ? Pn[2 * j + 1] : P0;
                T f = (T)0;
                if (u != (T)0) {
                    f = fmax(u, (T)0) * PL + fmin(u, (T)0) * PR;  // Eq. 7
                    const bool upwind_is_c = side ? (u > (T)0) : (u < (T)0);
                    T S;
                    if (upwind_is_c) {
                        S = (T)0;
#pragma unroll
                        for (int d = 0; d < N; ++d)
                            if (d != j) S += ch[d] * Gc[d];
                    } else {
                        S = trans_nb(j, side);
                    }
                    f -= u * S;  // Algorithm 1
                    const T W = PR - PL;
                    if (lim != LIM_NONE && W != (T)0) {
                        T Wup;
                        if (u > (T)0)
                            Wup = side ? (P0 - Pn[2 * j])
                                       : (Pn[2 * j] - q_or_zero<T>(Q, second_index<N>(m, b, link, cap, L, I, j, 0, fb)));
                        else
                            Wup = side ? (q_or_zero<T>(Q, second_index<N>(m, b, link, cap, L, I, j, 1, fb)) - Pn[2 * j + 1])
                                       : (Pn[2 * j + 1] - P0);
                        const T au = fabs(u);
                        f += (T)0.5 * au * ((T)1 - dth[j] * au) * limited_wave<T>(lim, W, Wup);
                    }
                }
                F[side] = f;
            }
            upd += dth[j] * (F[1] - F[0]);
        }
        const T qn = (P0 - upd) * scale;
        Qn[c] = qn;
        acc_add(dacc, (double)qn, err);
        mx = fmax(mx, (double)qn);
    }
    return fb;
}

// ------------------------------------------------------------------ single-pass update, one lane per face

// The same update as gather_body with the 2n faces of a cell spread over a
// group of G lanes (G = 8 for n <= 4, 16 for n = 5, 6; lane 2j + s owns the
// lower (s = 0) or upper (s = 1) j-face). The cell's own waves and the update
// are combined with shuffles inside the group, so each lane walks one face's
// neighbourhood: 2n times more independent work than one lane per cell.
template <int N, int DYN, typename T>
__device__ __forceinline__ long long gather_faces_body(const Model& m, const Bufs& b, const StepView& v,
                                                       long long (&dacc)[NDIG], double& mx, int& err) {
    constexpr int G = (2 * N <= 8) ? 8 : 16;
    const long long ncell = v.N;
    const T* Q = static_cast<const T*>(b.q[v.pb]);
    T* Qn = static_cast<T*>(b.q[v.pb ^ 1]);
    const unsigned long long* key = b.key[v.g];
    const int* link = b.link[v.g];
    const long long cap = m.cap;
    const int lim = m.limiter;
    const T scale = (T)v.scale;
    T h[N], x0[N], chT[N], dthT[N];
#pragma unroll
    for (int k = 0; k < N; ++k) {
        h[k] = sizeof(T) == 4 ? (T)m.hf[k] : (T)m.h[k];
        x0[k] = sizeof(T) == 4 ? (T)m.x0f[k] : (T)m.x0[k];
        chT[k] = (T)v.ch[k];
        dthT[k] = (T)v.dth[k];
    }
    T tmax = -INFINITY;
    long long fb = 0;
    const long long items = ncell * G;
    const unsigned full = 0xffffffffu;
    for (WarpRuns wr(items); wr.next();) {
        // every lane of the warp takes part in the shuffles below
        const long long it = wr.c;
        const long long c = it / G;
        const int l = (int)(it % G);
        const bool cell_ok = c < ncell;
        const bool face_ok = cell_ok && l < 2 * N;
        const int j = face_ok ? (l >> 1) : 0;
        const int side = l & 1;
        T P0 = (T)0, Pn = (T)0, u = (T)0;
        int Ls = -1;
        int I[N];
        T xc[N];
        if (cell_ok) {
            P0 = Q[c];
            unpack_key<N>(m, key[c], I);
#pragma unroll
            for (int k = 0; k < N; ++k) xc[k] = x0[k] + (T)I[k] * h[k];
        }
        if (face_ok) {
            Ls = link[(long long)(2 * j + side) * cap + c];
            Pn = q_or_zero<T>(Q, Ls);
#pragma unroll
            for (int d = 0; d < N; ++d)
                if (d == j) u = vel_at<N, DYN, T>(m, xc, h, -1, 0, d, side ? +1 : -1);
        }
        // the partner lane holds the other face of the same dimension
        const T u_o = __shfl_xor_sync(full, u, 1, G);
        const T Pn_o = __shfl_xor_sync(full, Pn, 1, G);
        const T ulo = side ? u_o : u, uhi = side ? u : u_o;
        const T Plo = side ? Pn_o : Pn, Phi = side ? Pn : Pn_o;
        // G_j(c), the j-waves entering c; and sum over d of dt/(2 h_d) G_d(c)
        const T Gj = face_ok ? fmax(ulo, (T)0) * (P0 - Plo) + fmin(uhi, (T)0) * (Phi - P0) : (T)0;
        T chj = (T)0, dthj = (T)0;
#pragma unroll
        for (int k = 0; k < N; ++k)
            if (k == j && face_ok) {
                chj = chT[k];
                dthj = dthT[k];
            }
        T tot = (side == 0) ? chj * Gj : (T)0;
#pragma unroll
        for (int off = G / 2; off > 0; off >>= 1) tot += __shfl_xor_sync(full, tot, off, G);
        T contrib = (T)0;
        if (face_ok) {
            const T PL = side ? P0 : Pn;
            const T PR = side ? Pn : P0;
            T f = (T)0;
            if (u != (T)0) {
                f = fmax(u, (T)0) * PL + fmin(u, (T)0) * PR;  // Eq. 7
                const bool upwind_is_c = side ? (u > (T)0) : (u < (T)0);
                T S;
                if (upwind_is_c) {
                    S = tot - chj * Gj;
                } else if (Ls < 0 && c < v.N_prev) {  // missing neighbour: precomputed waves
                    S = (T)v.dt * static_cast<const T*>(b.bt)[(long long)(2 * j + side) * cap + c];
                } else {  // the neighbour across this face (possibly new or missing)
                    int L[2 * N];
#pragma unroll
                    for (int d = 0; d < 2 * N; ++d) L[d] = link[(long long)d * cap + c];
                    const int sgn = side ? 1 : -1;
                    S = (T)0;
#pragma unroll
                    for (int d = 0; d < N; ++d) {
                        if (d == j) continue;
                        T Pm, Pp;
                        if (Ls >= 0) {
                            Pm = q_or_zero<T>(Q, link[(long long)(2 * d) * cap + Ls]);
                            Pp = q_or_zero<T>(Q, link[(long long)(2 * d + 1) * cap + Ls]);
                        } else {
                            Pm = q_or_zero<T>(Q, edge_index<N>(m, b, link, cap, L, I, j, side, d, 0, fb));
                            Pp = q_or_zero<T>(Q, edge_index<N>(m, b, link, cap, L, I, j, side, d, 1, fb));
                        }
                        const T ul = vel_at<N, DYN, T>(m, xc, h, j, sgn, d, -1);
                        const T uh = vel_at<N, DYN, T>(m, xc, h, j, sgn, d, +1);
                        S += chT[d] * (fmax(ul, (T)0) * (Pn - Pm) + fmin(uh, (T)0) * (Pp - Pn));
                    }
                }
                f -= u * S;  // Algorithm 1
                const T W = PR - PL;
                if (lim != LIM_NONE && W != (T)0) {
                    T Wup;
                    // value two cells away across this face
                    auto second = [&]() -> T {
                        if (Ls >= 0) return q_or_zero<T>(Q, link[(long long)(2 * j + side) * cap + Ls]);
                        if (c < v.N_prev) return static_cast<const T*>(b.bp)[(long long)(2 * j + side) * cap + c];
                        int L[2 * N];
#pragma unroll
                        for (int d = 0; d < 2 * N; ++d) L[d] = link[(long long)d * cap + c];
                        return q_or_zero<T>(Q, second_index<N>(m, b, link, cap, L, I, j, side, fb));
                    };
                    if (u > (T)0) Wup = side ? (P0 - Plo) : (Plo - second());
                    else Wup = side ? (second() - Phi) : (Phi - P0);
                    const T au = fabs(u);
                    f += (T)0.5 * au * ((T)1 - dthj * au) * limited_wave<T>(lim, W, Wup);
                }
            }
            contrib = (side ? (T)1 : (T)-1) * dthj * f;
        }
#pragma unroll
        for (int off = G / 2; off > 0; off >>= 1) contrib += __shfl_xor_sync(full, contrib, off, G);
        if (cell_ok && l == 0) {
            const T qn = (P0 - contrib) * scale;
            Qn[c] = qn;
            acc_add(dacc, qn, err);
            tmax = fmax(tmax, qn);
        }
    }
    if (tmax > -INFINITY) mx = fmax(mx, (double)tmax);
    return fb;
}

// ------------------------------------------------------------------ prune

// keep[c] = (p_c > p*): the significant cells S.
template <typename T>
__device__ __forceinline__ void prune_mark_body(const Model& m, const Bufs& b, const StepView& v) {
    const double pstar = m.thr_rel * v.maxq;
    const T* Q = static_cast<const T*>(b.q[v.pb]);
    for (WarpRuns r(v.N); r.next();) {
        const long long c = r.c;
        if (c < v.N) b.keep[c] = (double)Q[c] > pstar;
    }
}

// keep[D(S)] = 1: each significant cell marks the existing cells of its
// downwind set (Sec. 3.3, Fig. 3).
template <int N, typename T>
__device__ __forceinline__ void prune_scatter_body(const Model& m, const Bufs& b, const StepView& v) {
    const double pstar = m.thr_rel * v.maxq;
    const T* Q = static_cast<const T*>(b.q[v.pb]);
    const unsigned long long* key = b.key[v.g];
    const int* link = b.link[v.g];
    const unsigned short* om = b.om[v.g];
    const long long cap = m.cap;
    for (WarpRuns r(v.N); r.next();) {
        const long long c = r.c;
        if (c >= v.N) continue;
        if (!((double)Q[c] > pstar)) continue;
        const unsigned out = om[c] & 0xfffu;
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
                    int I[N];
                    unpack_key<N>(m, key[c], I);
                    I[d1 >> 1] += (d1 & 1) ? 1 : -1;
                    I[d2 >> 1] += (d2 & 1) ? 1 : -1;
                    unsigned long long kk;
                    e = pack_key<N>(m, I, kk) ? table_find(m, b.table, kk) : -1;
                }
                if (e >= 0) b.keep[e] = 1;
            }
        }
    }
}

// chunk [c0, c1) of a range of `total` items handled by this block
__device__ __forceinline__ void block_chunk(long long total, long long& c0, long long& c1) {
    long long per = (total + gridDim.x - 1) / gridDim.x;
    per = (per + THREADS - 1) / THREADS * THREADS;
    c0 = min(total, per * blockIdx.x);
    c1 = min(total, c0 + per);
}

// This block's count of kept cells into blk[blockIdx.x]; the table slots of
// the current cells are emptied for the rehash (the table holds nothing else).
__device__ __forceinline__ void prune_count_body(const Model& m, const Bufs& b, const StepView& v) {
    long long c0, c1;
    block_chunk(v.N, c0, c1);
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
    __syncthreads();
    const unsigned int* slots = b.slot[v.g];
    for (long long c = c0 + threadIdx.x; c < c1; c += blockDim.x)
        reinterpret_cast<ulonglong2*>(b.table)[slots[c]] = make_ulonglong2(EMPTY_KEY, ~0ull);
}

// Offset of this block's survivors (sum of the counts of the blocks before it)
// and the total, read by every block from blk (same values everywhere).
__device__ __forceinline__ void block_offset_total(const Bufs& b, long long& offset, long long& total) {
    __shared__ long long s_off[WARPS], s_tot[WARPS];
    long long o = 0, t = 0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
        long long v = __ldcg(&b.blk[i]);
        t += v;
        if (i < (int)blockIdx.x) o += v;
    }
    for (int off = 16; off > 0; off >>= 1) {
        o += __shfl_down_sync(0xffffffffu, o, off);
        t += __shfl_down_sync(0xffffffffu, t, off);
    }
    if ((threadIdx.x & 31) == 0) {
        s_off[threadIdx.x >> 5] = o;
        s_tot[threadIdx.x >> 5] = t;
    }
    __syncthreads();
    o = 0;
    t = 0;
    for (int w = 0; w < WARPS; ++w) {
        o += s_off[w];
        t += s_tot[w];
    }
    __syncthreads();
    offset = o;
    total = t;
}

// Stream compaction of the kept cells in storage order into the other buffer
// set, starting at `base`; map[c] = new index or -1. The values are rescaled by
// an exact power of two that brings the maximum into [1, 2) (their ratios do
// not change, and the exact sum stays in its window even after a very unlikely
// measurement). Adds the survivors' digits, maximum and CFL rates.
template <int N, typename T>
__device__ __forceinline__ void prune_compact_body(const Model& m, const Bufs& b, const StepView& v, long long base,
                                                   long long (&d)[NDIG], double& mx, double& rmax, int& err) {
    const T* Q = static_cast<const T*>(b.q[v.pb]);
    T* Qo = static_cast<T*>(b.q[v.pb ^ 1]);
    const unsigned long long* key = b.key[v.g];
    unsigned long long* keyo = b.key[v.g ^ 1];
    const unsigned short* om = b.om[v.g];
    unsigned short* omo = b.om[v.g ^ 1];
    const double mq = v.maxq;
    const double s2 = (mq > 0.0 && isfinite(mq)) ? ldexp(1.0, -ilogb(mq)) : 1.0;
    long long c0, c1;
    block_chunk(v.N, c0, c1);
    for (long long t0 = c0; t0 < c1; t0 += blockDim.x) {
        long long c = t0 + threadIdx.x;
        int f = (c < c1) ? (b.keep[c] != 0) : 0;
        int total;
        int pos = block_exclusive_scan(f, total);
        if (c < c1) {
            if (f) {
                long long nc = base + pos;
                unsigned long long k = key[c];
                T val = (T)((double)Q[c] * s2);
                keyo[nc] = k;
                Qo[nc] = val;
                omo[nc] = (unsigned short)(om[c] & ~OM_COMPLETE);
                b.map[c] = (int)nc;
                acc_add(d, (double)val, err);
                mx = fmax(mx, (double)val);
                int I[N];
                unpack_key<N>(m, k, I);
                rmax = fmax(rmax, cfl_rate64<N>(m, I));
            } else {
                b.map[c] = -1;
            }
        }
        base += total;
    }
}

// New links through the map, and the rehash of the survivors.
template <int N>
__device__ __forceinline__ void prune_relink_body(const Model& m, const Bufs& b, const StepView& v) {
    const int* link = b.link[v.g];
    int* linko = b.link[v.g ^ 1];
    const unsigned long long* keyo = b.key[v.g ^ 1];
    const long long cap = m.cap;
    for (WarpRuns r(v.N); r.next();) {
        const long long c = r.c;
        if (c >= v.N) continue;
        const int nc = b.map[c];
        if (nc < 0) continue;
#pragma unroll
        for (int d = 0; d < 2 * N; ++d) {
            int l = link[(long long)d * cap + c];
            linko[(long long)d * cap + nc] = l >= 0 ? b.map[l] : -1;
        }
        table_insert_new(m, b, keyo[nc], nc, b.slot[v.g ^ 1]);
    }
}

}  // namespace gbees
