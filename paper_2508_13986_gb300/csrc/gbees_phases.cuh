// The phases of one GBEES time step as device functions over "all threads of
// the grid", shared by the one-kernel-per-phase path (gbees_kernels.cuh, run as
// a CUDA graph) and the persistent cooperative kernel (gbees_persistent.cuh).
// Data that a phase writes is read by later phases of the same persistent
// launch, so no pointer here is marked read-only (no non-coherent loads): the
// grid barrier's fences make plain loads see the other blocks' writes.
//
//   grow       directional grow of the significant cells (Sec. 3.3, Algorithm 2)
//   halo       the missing face neighbours of the newly active cells, as halo cells
//   link       neighbour links, outward mask and CFL rate of the new entries (Sec. 4.1)
//   waves      per-entry velocities u_d and entering waves G_d
//   faces      one flux per face (Eq. 7 + Algorithm 1 gathered + HR term)
//   apply      P -= sum_j dt/h_j (F_hi - F_lo), normalised, reduced
//   prune      mark S, mark D(S), status, compact, relink and rehash (Algorithm 3)
//
// The pool holds the active cells and, as halo cells with p = 0, every face
// neighbour of an active cell that is not active (a missing cell of the method:
// p = 0, not updated). With links between all pool entries, every cell of the
// update stencil is reached through links and the update needs no hashtable.
#pragma once

#include "gbees_device.cuh"

namespace gbees {

// What a phase needs to know about the step in progress.
struct StepView {
    long long N;       // pool entries (clamped to the capacity)
    long long N_prev;  // pool entries before this step's grow
    int pb, g;         // current value buffer and key/link buffer
    double maxq;       // max stored value (threshold p* = thr_rel * maxq)
    double scale;      // 1 / w of the previous normalisation
    double dth[MAXN];  // dt / h_j of this step
    double ch[MAXN];   // dt / (2 h_j)
    double dt;         // dt of this step
    int nb, bi;        // the blocks that share this grid's work, and this block's index among them
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
    v.nb = gridDim.x;
    v.bi = blockIdx.x;
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
    // t + dt can round onto the target although dt < tt - t: that step ends
    // the call too (as the loop 'while t < t_target' of the method does)
    if (!last && !(s.t_new < tt)) {
        s.last = 1;
        s.t_new = tt;
    }
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

// Index of cell c + s1 e_j + s2 e_d (j != d) through the links (L: the links
// of c), -1 when it is not in the pool. For an active cell c the face
// neighbour c + s1 e_j is in the pool, so its link decides; -2 only when both
// intermediate cells are missing.
template <int N>
__device__ __forceinline__ int edge_by_links(const int* link, long long cap, const int* L, int j, int s1, int d,
                                             int s2) {
    int a = L[2 * j + s1];
    if (a >= 0) return __ldcg(link + (long long)(2 * d + s2) * cap + a);
    int b = L[2 * d + s2];
    if (b >= 0) return __ldcg(link + (long long)(2 * j + s1) * cap + b);
    return -2;
}

// The 2n links of entry c (direction-major arrays: one coalesced load per
// direction across a warp of consecutive entries).
template <int N>
__device__ __forceinline__ void load_links(const int* link, long long cap, long long c, int* L) {
#pragma unroll
    for (int d = 0; d < 2 * N; ++d) L[d] = link[(long long)d * cap + c];
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

// Entry e is a halo cell: make it active. True for the one thread that does.
__device__ __forceinline__ bool activate(unsigned short* om, long long e) {
    unsigned short old = *(volatile unsigned short*)&om[e];
    while (old & OM_GHOST) {
        const unsigned short prev = atomicCAS(&om[e], old, (unsigned short)(old & ~OM_GHOST));
        if (prev == old) return true;
        old = prev;
    }
    return false;
}

// Active cells keep one layer away from the edge of the key range, so that
// their face neighbours (halo cells) have keys.
template <int N>
__device__ __forceinline__ bool interior(const Model& m, const int* I) {
    const long long bias = 1ll << (m.key_bits - 1);
    const long long top = (1ll << m.key_bits) - 2;
#pragma unroll
    for (int k = 0; k < N; ++k) {
        const long long u = (long long)I[k] + bias;
        if (u < 1 || u > top) return false;
    }
    return true;
}

// Claim the key of cell I and append it to the pool at base + (*counter)++
// with p = 0 and the given flags. Returns the new index, or -1 when the key is
// present already (or on an error, which is recorded).
template <int N, typename T>
__device__ __forceinline__ long long insert_cell(const Model& m, const Bufs& b, const StepView& v, const int* I,
                                                 unsigned short flags, long long* counter, long long base) {
    DevScalars* sc = b.sc;
    unsigned long long k;
    if (!pack_key<N>(m, I, k)) {
        set_error(sc, ST_EKEYRANGE);
        return -1;
    }
    unsigned long long slot;
    const int r = table_claim(m, b.table, k, &slot);
    if (r < 0) {
        set_error(sc, ST_ETABLE);
        return -1;
    }
    if (r == 0) return -1;
    const long long c = base + warp_aggregated_add(counter);
    if (c >= m.cap) {
        set_error(sc, ST_ECAPACITY);
        return -1;
    }
    b.table[slot].val = c;
    b.slot[v.g][c] = (unsigned int)slot;
    b.key[v.g][c] = k;
    static_cast<T*>(b.q[v.pb])[c] = (T)0;
    b.om[v.g][c] = flags;
    return c;
}

// Directional grow (Sec. 3.3): every significant cell makes its downwind set
// active. A face neighbour of an active cell is always in the pool; an edge
// neighbour c + s1 e_j + s2 e_l is found through the link of the face
// neighbour c + s1 e_j. A halo cell found there becomes active (listed in map
// for the halo phase); a missing one is inserted as active. A cell whose
// downwind set was made active since the last prune is skipped.
//
// The candidates of a cell (2n faces, 4 C(n,2) edges, those that are not
// downwind skipped at once) are independent chains of dependent loads and
// atomics, spread over many threads: grow_body gathers a block's qualifying
// cells in shared memory (the persistent and batch step loops); for large
// grids the wave pass lists them (grow_list_mark) and a kernel of its own
// spreads every (cell, candidate) pair of the list over the grid
// (grow_list_body).
struct GrowWork {
    double rmax = 0.0;  // largest CFL rate of the halo cells this thread activated
};

// Candidate k of cell cc with downwind directions out.
template <int N, typename T>
__device__ __forceinline__ void grow_candidate(const Model& m, const Bufs& b, const StepView& v, long long cc,
                                               unsigned out, int k, GrowWork& gw) {
    DevScalars* sc = b.sc;
    const long long cap = m.cap;
    const int* link = b.link[v.g];
    unsigned short* om = b.om[v.g];
    int d1, d2 = -1;
    if (k < 2 * N) {
        d1 = k;
    } else {
        const int e = k - 2 * N;
        int rem = e >> 2, j = 0;
        while (rem >= N - 1 - j) {
            rem -= N - 1 - j;
            ++j;
        }
        d1 = 2 * j + (e & 1);
        d2 = 2 * (j + 1 + rem) + ((e >> 1) & 1);
    }
    if (!((out >> d1) & 1u) || (d2 >= 0 && !((out >> d2) & 1u))) return;
    const int a = link[(long long)d1 * cap + cc];
    long long e;
    if (d2 < 0) {
        e = a;
    } else if (a >= 0) {
        e = link[(long long)d2 * cap + a];
    } else {
        const int a2 = link[(long long)d2 * cap + cc];
        e = a2 >= 0 ? link[(long long)d1 * cap + a2] : -1;
    }
    if (e >= 0) {  // in the pool: a halo cell becomes active
        if (!(om[e] & OM_GHOST) || !activate(om, e)) return;
        warp_aggregated_add(&sc->NA);
        b.map[warp_aggregated_add(&sc->n_act)] = (int)e;
        gw.rmax = fmax(gw.rmax, b.rate[v.g][e]);  // fixed when the halo cell was linked
        return;
    }
    int J[N];
    unpack_key<N>(m, b.key[v.g][cc], J);
    J[d1 >> 1] += (d1 & 1) ? 1 : -1;
    if (d2 >= 0) J[d2 >> 1] += (d2 & 1) ? 1 : -1;
    if (!interior<N>(m, J)) {
        set_error(sc, ST_EKEYRANGE);
        return;
    }
    if (insert_cell<N, T>(m, b, v, J, 0, &sc->N, 0) >= 0) warp_aggregated_add(&sc->NA);
}

template <int N>
constexpr int GROW_K = 2 * N + 2 * N * (N - 1);  // candidates per cell

// Whether cell c takes part in this step's grow: significant, active, with
// outward directions, its downwind set not yet known to be active.
template <typename T>
__device__ __forceinline__ bool grows(const unsigned short* om, const T* Q, const Above<T>& above, long long c,
                                      unsigned& out) {
    if (!above(Q[c])) return false;
    const unsigned f = om[c];
    out = f & 0xfffu;
    return !(f & (OM_COMPLETE | OM_GHOST)) && out;
}

// The block-gathered form (all threads of the block must call it).
template <int N, typename T>
__device__ __forceinline__ double grow_body(const Model& m, const Bufs& b, const StepView& v) {
    constexpr int K = GROW_K<N>;
    const long long ncell = v.N_prev;
    const Above<T> above(m.thr_rel * v.maxq);
    const T* Q = static_cast<const T*>(b.q[v.pb]);
    unsigned short* om = b.om[v.g];
    __shared__ long long s_cell[THREADS];
    __shared__ unsigned s_out[THREADS];
    GrowWork gw;
    // rounds of one run of 32 cells per warp; the block's first warp has the most
    const long long runs = (ncell + 31) / 32;
    const long long stride = (long long)v.nb * (blockDim.x >> 5);
    const long long rounds = runs > v.bi ? (runs - v.bi + stride - 1) / stride : 0;
    const int wid = threadIdx.x >> 5;
    for (long long rd = 0; rd < rounds; ++rd) {
        const long long k = v.bi + (long long)v.nb * wid + stride * rd;
        const long long c = k * 32 + (threadIdx.x & 31);
        unsigned out = 0;
        const bool q = k < runs && c < ncell && grows<T>(om, Q, above, c, out);
        int nq;
        const int pos = block_exclusive_scan(q, nq);
        if (nq == 0) continue;
        if (q) {
            s_cell[pos] = c;
            s_out[pos] = out;
        }
        __syncthreads();
        const int pairs = nq * K;
        for (int t = threadIdx.x; t < pairs; t += blockDim.x) {
            const int rank = t / K;
            grow_candidate<N, T>(m, b, v, s_cell[rank], s_out[rank], t - rank * K, gw);
        }
        __syncthreads();
        if (q) om[c] = (unsigned short)(om[c] | OM_COMPLETE);
    }
    return gw.rmax;
}

// The listed form, first half: cell c (of the wave pass's sweep) joins the
// step's grow list (in the flux scratch, free until the flux pass) when it
// grows.
template <typename T>
__device__ __forceinline__ void grow_list_mark(const Bufs& b, const StepView& v, const Above<T>& above, long long c) {
    const T* Q = static_cast<const T*>(b.q[v.pb]);
    unsigned out;
    if (grows<T>(b.om[v.g], Q, above, c, out)) {
        int* glist = static_cast<int*>(b.fl);
        glist[warp_aggregated_add(&b.sc->n_glist)] = (int)c;
    }
}

// The listed form, second half: every (listed cell, candidate) pair, over all
// threads of the grid; the thread of a cell's first candidate marks it
// complete (only its own flag bit, and nothing else writes that word now).
template <int N, typename T>
__device__ __forceinline__ double grow_list_body(const Model& m, const Bufs& b, const StepView& v) {
    constexpr int K = GROW_K<N>;
    const int* glist = static_cast<const int*>(b.fl);
    unsigned short* om = b.om[v.g];
    const long long nl = *(volatile long long*)&b.sc->n_glist;
    GrowWork gw;
    const long long items = nl * K;
    const long long tid = (long long)v.bi * blockDim.x + threadIdx.x;
    const long long nth = (long long)v.nb * blockDim.x;
    for (long long it = tid; it < items; it += nth) {
        const long long rank = it / K;
        const int k = (int)(it - rank * K);
        const long long c = glist[rank];
        const unsigned out = om[c] & 0xfffu;
        grow_candidate<N, T>(m, b, v, c, out, k, gw);
        if (k == 0) om[c] = (unsigned short)(om[c] | OM_COMPLETE);
    }
    return gw.rmax;
}

// ------------------------------------------------------------------ halo

// The face neighbours of the cells made active by this step's grow that are
// not in the pool are appended as halo cells at base + n_halo. Work items
// (cell, face) over the inserted cells [lo, hi), which have no links yet (each
// neighbour is claimed, the claim finds the present ones), and over the nact
// activated halo cells listed in map (only their neighbours without a link).
template <int N, typename T>
__device__ __forceinline__ void halo_body(const Model& m, const Bufs& b, const StepView& v, long long lo, long long hi,
                                          long long nact) {
    const unsigned long long* key = b.key[v.g];
    const int* link = b.link[v.g];
    const long long cap = m.cap;
    const long long ni = hi - lo;
    const long long items = (ni + nact) * 2 * N;
    // runs of 32 items, one per warp, the warps of consecutive runs on
    // different SMs: a few hundred items of a small grid spread over the GPU
    for (WarpRuns wr(items, v.nb, v.bi); wr.next();) {
        const long long it = wr.c;
        if (it >= items) continue;
        const long long q = it / (2 * N);
        const int d = (int)(it - q * 2 * N);
        long long x;
        if (q < ni) {
            x = lo + q;
        } else {
            x = b.map[q - ni];
            if (link[(long long)d * cap + x] >= 0) continue;
        }
        int I[N];
        unpack_key<N>(m, key[x], I);
        I[d >> 1] += (d & 1) ? 1 : -1;
        insert_cell<N, T>(m, b, v, I, OM_GHOST, &b.sc->n_halo, hi);
    }
}

// ------------------------------------------------------------------ link

// Face velocities and outward masks of the new entries [lo, hi) (the mask is
// added to the flags their inserter wrote), and the largest CFL rate among the
// active ones (Eq. 8: the same IEEE operations as cfl_rate64).
template <int N, typename T>
__device__ __forceinline__ double link_masks(const Model& m, const Bufs& b, long long lo, long long hi, int g,
                                              int nb, int bi) {
    const unsigned long long* key = b.key[g];
    T* U = static_cast<T*>(b.u[g]);
    const long long cap = m.cap;
    double rmax = 0.0;
    // runs of 32 entries, one per warp, consecutive runs on different SMs (the
    // FP64 drift evaluations of a few hundred new entries spread over the GPU)
    for (WarpRuns wr(hi - lo, nb, bi); wr.next();) {
        const long long c = lo + wr.c;
        if (c >= hi) continue;
        int I[N];
        unpack_key<N>(m, key[c], I);
        const unsigned short f = b.om[g][c];
        unsigned msk = 0;
        double r = 0.0;
#pragma unroll
        for (int j = 0; j < N; ++j) {
            int J[N];
#pragma unroll
            for (int k = 0; k < N; ++k) J[k] = I[k] + (k == j ? 1 : 0);
            const double ul = face_velocity64<N>(m, I, j);
            if (face_velocity64<N>(m, J, j) > 0.0) msk |= 1u << (2 * j + 1);
            if (ul < 0.0) msk |= 1u << (2 * j);
            U[j * cap + c] = (T)ul;
            r = __dadd_rn(r, div_h(m, fabs(ul), j));
        }
        b.om[g][c] = (unsigned short)(f | msk);
        b.rate[g][c] = r;
        if (!(f & OM_GHOST)) rmax = fmax(rmax, r);
    }
    return rmax;
}

// Entries [lo, hi) are new: look up their 2n face neighbours (one probe per
// thread and direction), write the reverse links into the neighbours, and set
// their outward masks; returns this thread's largest CFL rate among the active
// ones.
template <int N, typename T>
__device__ __forceinline__ double link_body(const Model& m, const Bufs& b, long long lo, long long hi, int g, int nb,
                                             int bi) {
    const unsigned long long* key = b.key[g];
    int* link = b.link[g];
    const long long cap = m.cap;
    const long long work = (hi - lo) * 2 * N;
    for (WarpRuns wr(work, nb, bi); wr.next();) {
        const long long wi = wr.c;
        if (wi >= work) continue;
        const long long c = lo + wi / (2 * N);
        const int dir = (int)(wi % (2 * N));
        const int j = dir >> 1, s = dir & 1;
        int I[N];
        unpack_key<N>(m, key[c], I);
        I[j] += s ? 1 : -1;
        unsigned long long k;
        const int nbr = pack_key<N>(m, I, k) ? table_find(m, b.table, k) : -1;
        link[(long long)dir * cap + c] = nbr;
        if (nbr >= 0) link[(long long)(2 * j + (1 - s)) * cap + nbr] = (int)c;
    }
    return link_masks<N, T>(m, b, lo, hi, g, nb, bi);
}

// Cooperative variant: W lanes probe W consecutive slots together.
template <int N, int W, typename T>
__device__ __forceinline__ double link_body_tile(const Model& m, const Bufs& b, long long lo, long long hi, int g,
                                                  int nb, int bi) {
    const unsigned long long* key = b.key[g];
    int* link = b.link[g];
    const long long cap = m.cap;
    auto tile = cg::tiled_partition<W>(cg::this_thread_block());
    const long long tiles = (long long)nb * (blockDim.x / W);
    const long long tile_id = (long long)bi * (blockDim.x / W) + threadIdx.x / W;
    const long long work = (hi - lo) * 2 * N;
    for (long long wi = tile_id; wi < work; wi += tiles) {
        const long long c = lo + wi / (2 * N);
        const int dir = (int)(wi % (2 * N));
        const int j = dir >> 1, s = dir & 1;
        int I[N];
        unpack_key<N>(m, key[c], I);
        I[j] += s ? 1 : -1;
        unsigned long long k;
        const int nbr = pack_key<N>(m, I, k) ? table_find_tile<W>(m, b.table, k, tile) : -1;
        if (tile.thread_rank() == 0) {
            link[(long long)dir * cap + c] = nbr;
            if (nbr >= 0) link[(long long)(2 * j + (1 - s)) * cap + nbr] = (int)c;
        }
    }
    return link_masks<N, T>(m, b, lo, hi, g, nb, bi);
}

// ------------------------------------------------------------------ three-pass update

template <typename T>
__device__ __forceinline__ T q_or_zero(const T* Q, int i) {
    return i >= 0 ? Q[i] : (T)0;
}

__device__ __forceinline__ bool is_halo(const unsigned short* om, long long i) { return (om[i] & OM_GHOST) != 0; }

// 0 - x as IEEE subtraction gives it, without FP64 arithmetic for doubles:
// the sign flips, except that both zeros give +0.
__device__ __forceinline__ double zero_minus(double x) {
    const long long b = __double_as_longlong(x);
    return __longlong_as_double((b << 1) == 0 ? 0ll : (b ^ (long long)0x8000000000000000ull));
}
__device__ __forceinline__ float zero_minus(float x) { return 0.0f - x; }

// The entering wave of entry y in dimension d,
//   G_d(y) = max(u_lo, 0) (P_y - P_{y-e_d}) + min(u_hi, 0) (P_{y+e_d} - P_y),
// u_lo, u_hi the velocities at its lower and upper d-face (the upper one is the
// lower one of the neighbour above; a missing neighbour above of a halo cell
// leaves both P at 0), with the jump across the lower face in wlo. VOTE: the
// warp's lanes run this together (the wave pass), so terms that no lane needs
// are skipped by a warp vote.
template <int N, typename T, bool VOTE = false>
__device__ __forceinline__ T wave_of(const T* Q, const T* U, long long cap, const int* L, long long y, T Py, int d,
                                     T& wlo) {
    const int dn = L[2 * d], up = L[2 * d + 1];
    const T Pm = q_or_zero<T>(Q, dn);
    const T Pp = q_or_zero<T>(Q, up);
    const T ul = U[d * cap + y];
    const T uh = up >= 0 ? U[d * cap + up] : (T)0;
    wlo = Py - Pm;
    // one product in the usual case (flow through the cell, or out of it on one
    // side only); a cell that both faces flow into takes the second term too.
    // The flow direction varies slowly: when no lane of the warp takes flow in
    // through the upper face, the upper jump and the second term are skipped.
    const bool in_lo = gt0(ul), in_hi = lt0(uh);
    if constexpr (VOTE) {
        const unsigned act = __activemask();
        if (!__any_sync(act, in_hi)) return (in_lo ? ul : (T)0) * wlo;
        const T G = (in_lo ? ul : (in_hi ? uh : (T)0)) * (in_lo ? wlo : Pp - Py);
        if (!__any_sync(act, in_lo && in_hi)) return G;
        return (in_lo && in_hi) ? fmadd(uh, Pp - Py, G) : G;
    } else {
        const T G = (in_lo ? ul : (in_hi ? uh : (T)0)) * (in_lo ? wlo : Pp - Py);
        return (in_lo && in_hi) ? fmadd(uh, Pp - Py, G) : G;
    }
}

// wave_of for a halo entry, whose value is +0: the same results (0 - P_m and
// P_p - 0 are exact) without the two subtractions.
template <int N, typename T>
__device__ __forceinline__ T wave_of_halo(const T* Q, const T* U, long long cap, const int* L, long long y, int d,
                                          T& wlo) {
    const int dn = L[2 * d], up = L[2 * d + 1];
    const T Pm = q_or_zero<T>(Q, dn);
    const T Pp = q_or_zero<T>(Q, up);
    const T ul = U[d * cap + y];
    const T uh = up >= 0 ? U[d * cap + up] : (T)0;
    wlo = zero_minus(Pm);
    const bool in_lo = gt0(ul), in_hi = lt0(uh);
    const T G = (in_lo ? ul : (in_hi ? uh : (T)0)) * (in_lo ? wlo : Pp);
    if (!__any_sync(__activemask(), in_lo && in_hi)) return G;
    return (in_lo && in_hi) ? fmadd(uh, Pp, G) : G;
}

// Pass 1, one thread per entry c of [0, ncell) (active and halo), all
// dimensions d: the jump wl[d] = P - P_{-e_d}, the entering wave wg[d] and
// tg = sum_d wg[d] / (2 h_d). Entries added by this step's grow and halo phases
// are left out: they have p = 0, and their waves are formed on the spot. Runs
// beside grow: a cell that grow or halo adds has p = 0 like the missing cell it
// replaces, so these waves do not change.
template <int N, int DYN, typename T, bool LIST_GROW = false>
__device__ __forceinline__ void waves_body(const Model& m, const Bufs& b, const StepView& v, long long ncell) {
    const T* Q = static_cast<const T*>(b.q[v.pb]);
    const int* link = b.link[v.g];
    const T* U = static_cast<const T*>(b.u[v.g]);
    // the outputs alias no input (restrict: loads may be scheduled ahead of the
    // stores; no read-only cache path is implied)
    T* __restrict__ wl = static_cast<T*>(b.wl);
    T* __restrict__ wg = static_cast<T*>(b.wg);
    T* __restrict__ tg = static_cast<T*>(b.tg);
    const long long cap = m.cap;
    T i2h[N];  // 1 / (2 h_d) in the arithmetic type, converted once
#pragma unroll
    for (int d = 0; d < N; ++d) i2h[d] = (T)m.inv_2h[d];
    const Above<T> above(m.thr_rel * v.maxq);
    for (WarpRuns wr(ncell, v.nb, v.bi); wr.next();) {
        const long long c = wr.c;
        if (c >= ncell) continue;
        if (LIST_GROW) grow_list_mark<T>(b, v, above, c);
        int L[2 * N];
        load_links<N>(link, cap, c, L);
        const T P0 = Q[c];
        T t = (T)0;
        // a warp of halo entries (the pool keeps them together after a
        // prune) takes the form without the subtractions
        if (__all_sync(__activemask(), is_halo(b.om[v.g], c))) {
#pragma unroll
            for (int d = 0; d < N; ++d) {
                T wlo;
                const T G = wave_of_halo<N, T>(Q, U, cap, L, c, d, wlo);
                wl[d * cap + c] = wlo;
                wg[d * cap + c] = G;
                t = fmadd(G, i2h[d], t);
            }
        } else {
#pragma unroll
            for (int d = 0; d < N; ++d) {
                T wlo;
                const T G = wave_of<N, T, true>(Q, U, cap, L, c, P0, d, wlo);
                wl[d * cap + c] = wlo;
                wg[d * cap + c] = G;
                t = fmadd(G, i2h[d], t);
            }
        }
        tg[c] = t;
    }
}

// sum_{d != j} G_d(y) / (2 h_d) of a new pool entry y (p = 0, no pass-1 values),
// formed on the spot from its links.
template <int N, typename T>
__device__ __forceinline__ T waves_new(const Model& m, const T* Q, const T* U, const int* link, long long y, int j) {
    const long long cap = m.cap;
    int L[2 * N];
    load_links<N>(link, cap, y, L);
    T S = (T)0;
#pragma unroll
    for (int d = 0; d < N; ++d) {
        if (d == j) continue;
        T wlo;
        S = fmadd(wave_of<N, T>(Q, U, cap, L, y, (T)0, d, wlo), (T)m.inv_2h[d], S);
    }
    return S;
}

// The flux pass's view of the step (pointers and constants in the arithmetic type).
template <int N, typename T>
struct FaceCtx {
    const T* Q;
    const int* link;
    const T* U;
    const T* wl;
    const T* wg;
    const T* tg;
    long long cap, nold;
    int lim;
    T dt, i2h[N], dth[N];
};

// The flux through the lower j-face of pool entry X (Eq. 7, the corrections of
// Algorithm 1 gathered onto the face, the limited HR term), X's value P0. The
// corrections that Algorithm 1 scatters onto face (X, j) add up to
//   -u_j(X) dt sum_{d != j} G_d(Y) / (2 h_d),  Y the cell upwind of the face,
// with sum_{d != j} = tg(Y) - G_j(Y) / (2 h_j). Entries added by this step's
// grow and halo phases (index >= nold) have no pass-1 values; theirs are formed
// on the spot.
template <int N, typename T>
__device__ __forceinline__ T face_flux(const Model& m, const FaceCtx<N, T>& fc, long long X, T P0, int j) {
    const long long cap = fc.cap;
    const T u = fc.U[j * cap + X];
    if (!(gt0(u) || lt0(u))) return (T)0;
    const int Llo = fc.link[(long long)(2 * j) * cap + X];
    const bool up = gt0(u);  // the flow crosses the face upwards: the upwind cell is Llo
    const bool old_x = X < fc.nold;
    const T PL = (up || !old_x) ? q_or_zero<T>(fc.Q, Llo) : (T)0;
    const T W = old_x ? fc.wl[j * cap + X] : P0 - PL;
    // transverse sum of the cell upwind of the face
    const long long y = up ? (long long)Llo : X;
    T S;
    if (y < fc.nold) {
        S = fmadd(-fc.i2h[j], fc.wg[j * cap + y], fc.tg[y]);
    } else {
        S = waves_new<N, T>(m, fc.Q, fc.U, fc.link, y, j);
    }
    // Eq. 7 (donor cell) and the corrections of Algorithm 1, gathered
    T f = u * fmadd(-fc.dt, S, up ? PL : P0);
    if (fc.lim != LIM_NONE && (gt0(W) || lt0(W))) {
        T Wup;
        if (up) {  // jump across the lower face of Llo
            Wup = Llo < fc.nold ? fc.wl[j * cap + Llo]
                                : PL - q_or_zero<T>(fc.Q, fc.link[(long long)(2 * j) * cap + Llo]);
        } else {  // jump across the upper face of X
            const int Lup = fc.link[(long long)(2 * j + 1) * cap + X];
            Wup = (Lup >= 0 && Lup < fc.nold) ? fc.wl[j * cap + Lup]
                  : (Lup >= 0 ? fc.Q[Lup] - P0 : zero_minus(P0));
        }
        // the limited high-resolution term 1/2 |u| (1 - dt |u| / h_j) phi W
        const T au = abs_bits(u);
        f = fmadd(half_nonneg(au) * fmadd(-fc.dth[j], au, (T)1), limited_wave<T>(fc.lim, W, Wup), f);
    }
    return f;
}

// face_flux for the faces whose values all come from pass 1: X and the cell
// upwind of the face were in the pool before this step's grow, and so was the
// upper neighbour whose jump the limiter reads. The same operations on the
// same values as face_flux gives those faces; returns false, with nothing
// evaluated, for any other face (new entries are few, and their waves are
// formed on the spot by face_flux later, with all lanes of a warp).
template <int N, typename T>
__device__ __forceinline__ bool face_flux_old(const FaceCtx<N, T>& fc, long long X, T P0, int j, T& f) {
    const long long cap = fc.cap;
    const T u = fc.U[j * cap + X];
    if (!(gt0(u) || lt0(u))) {
        f = (T)0;
        return true;
    }
    const int Llo = fc.link[(long long)(2 * j) * cap + X];
    const bool up = gt0(u);
    const int Lup = up ? -1 : fc.link[(long long)(2 * j + 1) * cap + X];
    const long long y = up ? (long long)Llo : X;
    if (X >= fc.nold || y >= fc.nold || Lup >= fc.nold) return false;
    const T PL = up ? q_or_zero<T>(fc.Q, Llo) : (T)0;
    const T W = fc.wl[j * cap + X];
    const T S = fmadd(-fc.i2h[j], fc.wg[j * cap + y], fc.tg[y]);
    f = u * fmadd(-fc.dt, S, up ? PL : P0);
    if (fc.lim != LIM_NONE && (gt0(W) || lt0(W))) {
        const T Wup = up ? fc.wl[j * cap + Llo] : (Lup >= 0 ? fc.wl[j * cap + Lup] : zero_minus(P0));
        const T au = abs_bits(u);
        f = fmadd(half_nonneg(au) * fmadd(-fc.dth[j], au, (T)1), limited_wave<T>(fc.lim, W, Wup), f);
    }
    return true;
}

// Pass 2: the flux through every face with an active cell on at least one
// side, stored as the lower face of the entry above it: all n lower faces of
// an active cell, and the lower faces of a halo cell whose neighbour below is
// active. Each warp takes runs of 32 consecutive entries, queues their needed
// faces (entry, j) in shared memory, dimension by dimension, and evaluates
// them 32 at a time, so that the lanes of a warp all work although a halo cell
// needs only the few faces it shares with active cells. The upper face of an active cell
// is the lower face of its upper neighbour, which is in the pool (active or
// halo).
// LATENCY: the step loop of a small grid, bound by dependent loads, not by the
// FP64 pipe: faces that touch a new entry are evaluated where they stand (a
// second queue would add a flush to the critical path of every warp).
template <int N, int DYN, typename T, bool LATENCY = false>
__device__ __forceinline__ void faces_body(const Model& m, const Bufs& b, const StepView& v) {
    const long long ncell = v.N;
    const long long cap = m.cap;
    const unsigned short* om = b.om[v.g];
    T* __restrict__ fl = static_cast<T*>(b.fl);  // aliases no input
    FaceCtx<N, T> fc;
    fc.Q = static_cast<const T*>(b.q[v.pb]);
    fc.link = b.link[v.g];
    fc.U = static_cast<const T*>(b.u[v.g]);
    fc.wl = static_cast<const T*>(b.wl);
    fc.wg = static_cast<const T*>(b.wg);
    fc.tg = static_cast<const T*>(b.tg);
    fc.cap = cap;
    fc.nold = v.N_prev;
    fc.lim = m.limiter;
    fc.dt = (T)v.dt;
#pragma unroll
    for (int j = 0; j < N; ++j) {  // converted once
        fc.i2h[j] = (T)m.inv_2h[j];
        fc.dth[j] = (T)v.dth[j];
    }
    // The warp's needed faces wait in a queue in shared memory (entry, j) and
    // are evaluated 32 at a time once that many are queued, whatever runs
    // they come from; the rest at the end.
    constexpr int QCAP = 32 * N + 32;
    __shared__ int s_qx[WARPS][QCAP];
    __shared__ unsigned char s_qj[WARPS][QCAP];
    // FP64 (the pipe bounds it): faces that touch a new entry wait in a second
    // queue, so that face_flux's longer path runs with all lanes too
    constexpr bool DEFER = sizeof(T) == 8 && !LATENCY;
    __shared__ int s_lx[WARPS][DEFER ? 64 : 1];
    __shared__ unsigned char s_lj[WARPS][DEFER ? 64 : 1];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    int n_q = 0, n_later = 0;  // the same in every lane
    auto later_flush = [&](int k) {  // the top k deferred faces, one per lane
        n_later -= k;
        if (lane < k) {
            const long long X = s_lx[wid][n_later + lane];
            const int jj = s_lj[wid][n_later + lane];
            fl[jj * cap + X] = face_flux<N, T>(m, fc, X, fc.Q[X], jj);
        }
        __syncwarp();
    };
    auto eval = [&](int k) {  // the top k queued faces, one per lane
        n_q -= k;
        bool later = false;
        long long X = 0;
        int jj = 0;
        if (lane < k) {
            X = s_qx[wid][n_q + lane];
            jj = s_qj[wid][n_q + lane];
            if constexpr (DEFER) {
                T f;
                if (face_flux_old<N, T>(fc, X, fc.Q[X], jj, f)) fl[jj * cap + X] = f;
                else later = true;
            } else {
                fl[jj * cap + X] = face_flux<N, T>(m, fc, X, fc.Q[X], jj);
            }
        }
        if constexpr (DEFER) {
            const unsigned bal = __ballot_sync(0xffffffffu, later);
            if (later) {
                const int at = n_later + __popc(bal & lt);
                s_lx[wid][at] = (int)X;
                s_lj[wid][at] = (unsigned char)jj;
            }
            n_later += __popc(bal);
        }
        __syncwarp();
        if constexpr (DEFER) {
            if (n_later >= 32) later_flush(32);
        }
    };
    for (WarpRuns wr(ncell, v.nb, v.bi); wr.next();) {
        const long long c = wr.c;
        unsigned need = 0;
        if (c < ncell) {
            if (!is_halo(om, c)) {
                need = (1u << N) - 1u;
            } else {
#pragma unroll
                for (int j = 0; j < N; ++j) {
                    const int Llo = fc.link[(long long)(2 * j) * cap + c];
                    if (Llo >= 0 && !is_halo(om, Llo)) need |= 1u << j;
                }
            }
        }
#pragma unroll
        for (int j = 0; j < N; ++j) {
            const unsigned bal = __ballot_sync(0xffffffffu, (need >> j) & 1u);
            if ((need >> j) & 1u) {
                const int at = n_q + __popc(bal & lt);
                s_qx[wid][at] = (int)c;
                s_qj[wid][at] = (unsigned char)j;
            }
            n_q += __popc(bal);
        }
        __syncwarp();
        while (n_q >= 32) eval(32);
    }
    if (n_q > 0) eval(n_q);
    if constexpr (DEFER) {
        if (n_later > 0) later_flush(n_later);
    }
}

// Pass 3: the conservative update of the active cells with the previous
// normalisation applied (halo cells stay 0); adds this thread's new values to
// its digits and maximum. Large FP64 grids (not LATENCY): each warp queues the
// active cells of its runs in shared memory and updates them 32 at a time, so
// the FP64 lanes all work where halo and active entries mix (after growth);
// FP32 and small grids are bound by load latency and update in place.
template <int N, typename T, bool LATENCY = false>
__device__ __forceinline__ void apply_body(const Model& m, const Bufs& b, const StepView& v, long long (&dacc)[NDIG],
                                           double& mx, int& err) {
    const long long ncell = v.N;
    const long long cap = m.cap;
    const T* Q = static_cast<const T*>(b.q[v.pb]);
    T* __restrict__ Qn = static_cast<T*>(b.q[v.pb ^ 1]);  // aliases no input
    const int* link = b.link[v.g];
    const unsigned short* om = b.om[v.g];
    const T* fl = static_cast<const T*>(b.fl);
    const T scale = (T)v.scale;
    T dth[N];
#pragma unroll
    for (int k = 0; k < N; ++k) dth[k] = (T)v.dth[k];
    T tmax = -INFINITY;
    auto update = [&](long long c) {
        int L[2 * N];
        load_links<N>(link, cap, c, L);
        T upd = (T)0;
#pragma unroll
        for (int j = 0; j < N; ++j) {
            const int up = L[2 * j + 1];
            const T Fhi = up >= 0 ? fl[j * cap + up] : (T)0;
            upd = fmadd(dth[j], Fhi - fl[j * cap + c], upd);
        }
        const T qn = (Q[c] - upd) * scale;
        Qn[c] = qn;
        acc_add(dacc, qn, err);
        tmax = vmax(tmax, qn);
    };
    if constexpr (LATENCY || sizeof(T) == 4) {
        for (WarpRuns wr(ncell, v.nb, v.bi); wr.next();) {
            const long long c = wr.c;
            if (c >= ncell) continue;
            if (is_halo(om, c)) {
                Qn[c] = (T)0;
                continue;
            }
            update(c);
        }
    } else {
        __shared__ int s_ac[WARPS][64];
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        const unsigned lt = (1u << lane) - 1u;
        int n_a = 0;  // the same in every lane
        for (WarpRuns wr(ncell, v.nb, v.bi); wr.next();) {
            const long long c = wr.c;
            bool act = false;
            if (c < ncell) {
                if (is_halo(om, c)) Qn[c] = (T)0;
                else act = true;
            }
            const unsigned bal = __ballot_sync(0xffffffffu, act);
            if (act) s_ac[wid][n_a + __popc(bal & lt)] = (int)c;
            n_a += __popc(bal);
            __syncwarp();
            if (n_a >= 32) {
                n_a -= 32;
                update(s_ac[wid][n_a + lane]);
                __syncwarp();
            }
        }
        if (lane < n_a) update(s_ac[wid][lane]);
    }
    if (tmax > -INFINITY) mx = fmax(mx, (double)tmax);
}

// ------------------------------------------------------------------ prune

// keep[c] = (p_c > p*) for the active cells: the significant cells S.
template <typename T>
__device__ __forceinline__ void prune_mark_body(const Model& m, const Bufs& b, const StepView& v) {
    const double pstar = m.thr_rel * v.maxq;
    const Above<T> above(pstar);
    const T* Q = static_cast<const T*>(b.q[v.pb]);
    const unsigned short* om = b.om[v.g];
    for (WarpRuns r(v.N, v.nb, v.bi); r.next();) {
        const long long c = r.c;
        if (c < v.N) b.keep[c] = !is_halo(om, c) && above(Q[c]);
    }
}

// keep[D(S)] = 1: each significant cell marks the pool entries of its
// downwind set (Sec. 3.3, Fig. 3); only the active ones among them are kept.
template <int N, typename T>
__device__ __forceinline__ void prune_scatter_body(const Model& m, const Bufs& b, const StepView& v) {
    const double pstar = m.thr_rel * v.maxq;
    const Above<T> above(pstar);
    const T* Q = static_cast<const T*>(b.q[v.pb]);
    const int* link = b.link[v.g];
    const unsigned short* om = b.om[v.g];
    const long long cap = m.cap;
    for (WarpRuns r(v.N, v.nb, v.bi); r.next();) {
        const long long c = r.c;
        if (c >= v.N) continue;
        const unsigned f = om[c];
        if ((f & OM_GHOST) || !above(Q[c])) continue;
        const unsigned out = f & 0xfffu;
        if (!out) continue;
        int L[2 * N];
        load_links<N>(link, cap, c, L);
#pragma unroll
        for (int d = 0; d < 2 * N; ++d)
            if (((out >> d) & 1u) && L[d] >= 0) b.keep[L[d]] = 1;
#pragma unroll
        for (int d1 = 0; d1 < 2 * N; ++d1) {
            if (!((out >> d1) & 1u)) continue;
#pragma unroll
            for (int d2 = 0; d2 < 2 * N; ++d2) {
                if ((d2 >> 1) <= (d1 >> 1) || !((out >> d2) & 1u)) continue;
                const int e = edge_by_links<N>(link, cap, L, d1 >> 1, d1 & 1, d2 >> 1, d2 & 1);
                if (e >= 0) b.keep[e] = 1;
            }
        }
    }
}

// chunk [c0, c1) of a range of `total` items handled by block bi of nb
__device__ __forceinline__ void block_chunk(long long total, long long& c0, long long& c1, int nb, int bi) {
    long long per = (total + nb - 1) / nb;
    per = (per + THREADS - 1) / THREADS * THREADS;
    c0 = min(total, per * bi);
    c1 = min(total, c0 + per);
}
__device__ __forceinline__ void block_chunk(long long total, long long& c0, long long& c1) {
    block_chunk(total, c0, c1, gridDim.x, blockIdx.x);
}

// Sum of a per-thread count over the block (every thread gets it).
__device__ __forceinline__ long long block_count(int cnt) {
    __shared__ long long s[WARPS];
    for (int off = 16; off > 0; off >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, off);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = cnt;
    __syncthreads();
    long long t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s[w];
    __syncthreads();
    return t;
}

// Status of every entry into map: 1 active and kept, 2 halo of a kept cell
// (not kept, with a kept face neighbour), 0 dropped. The block's counts of
// both go to blk and blk2; the table slots of the current entries are emptied
// for the rehash (the table holds nothing else).
template <int N>
__device__ __forceinline__ void prune_count_body(const Model& m, const Bufs& b, const StepView& v) {
    const int* link = b.link[v.g];
    const unsigned short* om = b.om[v.g];
    const long long cap = m.cap;
    long long c0, c1;
    block_chunk(v.N, c0, c1, v.nb, v.bi);
    int na = 0, ng = 0;
    for (long long c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
        int st = 0;
        if (b.keep[c] && !is_halo(om, c)) {
            st = 1;
        } else {
            int L[2 * N];
            load_links<N>(link, cap, c, L);
#pragma unroll
            for (int d = 0; d < 2 * N; ++d)
                if (L[d] >= 0 && b.keep[L[d]] && !is_halo(om, L[d])) st = 2;
        }
        b.map[c] = st;
        na += st == 1;
        ng += st == 2;
    }
    const long long ta = block_count(na);
    const long long tg = block_count(ng);
    if (threadIdx.x == 0) {
        b.blk[v.bi] = ta;
        b.blk2[v.bi] = tg;
    }
    const unsigned int* slots = b.slot[v.g];
    for (long long c = c0 + threadIdx.x; c < c1; c += blockDim.x)
        reinterpret_cast<ulonglong2*>(b.table)[slots[c]] = make_ulonglong2(EMPTY_KEY, ~0ull);
}

// Offsets of this block's survivors in the new pool (active cells first, then
// halo cells) and the totals, read by every block from blk and blk2.
struct Survivors {
    long long base_a, base_g, total_a, total_g;
};
__device__ __forceinline__ Survivors block_offsets(const Bufs& b, int nb, int bi) {
    __shared__ long long s[4][WARPS];
    long long v[4] = {0, 0, 0, 0};  // offset a, total a, offset g, total g
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        const long long a = __ldcg(&b.blk[i]);
        const long long g = __ldcg(&b.blk2[i]);
        v[1] += a;
        v[3] += g;
        if (i < bi) {
            v[0] += a;
            v[2] += g;
        }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        for (int off = 16; off > 0; off >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], off);
        if ((threadIdx.x & 31) == 0) s[k][threadIdx.x >> 5] = v[k];
    }
    __syncthreads();
    long long t[4] = {0, 0, 0, 0};
#pragma unroll
    for (int k = 0; k < 4; ++k)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t[k] += s[k][w];
    __syncthreads();
    Survivors r;
    r.base_a = t[0];
    r.total_a = t[1];
    r.base_g = t[1] + t[2];
    r.total_g = t[3];
    return r;
}

// The face velocities and the CFL rate of entry c (generation g) move to nc of
// the other generation.
template <int N, typename T>
__device__ __forceinline__ void copy_velocities(const Model& m, const Bufs& b, int g, long long c, long long nc) {
    const T* U = static_cast<const T*>(b.u[g]);
    T* Uo = static_cast<T*>(b.u[g ^ 1]);
#pragma unroll
    for (int j = 0; j < N; ++j) Uo[j * m.cap + nc] = U[j * m.cap + c];
    b.rate[g ^ 1][nc] = b.rate[g][c];
}

// Stream compaction of the survivors in storage order into the other buffer
// set: the kept active cells at [0, total_a), the halo cells after them;
// map[c] = new index or -1. Values of active cells are rescaled by an exact
// power of two that brings the maximum into [1, 2) (their ratios do not
// change, and the exact sum stays in its window even after a very unlikely
// measurement); halo cells hold 0. Adds the active cells' digits, maximum and
// CFL rates.
template <int N, typename T>
__device__ __forceinline__ void prune_compact_body(const Model& m, const Bufs& b, const StepView& v, Survivors sv,
                                                   long long (&d)[NDIG], double& mx, double& rmax, int& err) {
    const T* Q = static_cast<const T*>(b.q[v.pb]);
    T* Qo = static_cast<T*>(b.q[v.pb ^ 1]);
    const unsigned long long* key = b.key[v.g];
    unsigned long long* keyo = b.key[v.g ^ 1];
    const unsigned short* om = b.om[v.g];
    unsigned short* omo = b.om[v.g ^ 1];
    const double mq = v.maxq;
    const double s2 = (mq > 0.0 && isfinite(mq)) ? ldexp(1.0, -ilogb(mq)) : 1.0;
    long long ba = sv.base_a, bg = sv.base_g;
    long long c0, c1;
    block_chunk(v.N, c0, c1, v.nb, v.bi);
    for (long long t0 = c0; t0 < c1; t0 += blockDim.x) {
        const long long c = t0 + threadIdx.x;
        const int st = (c < c1) ? b.map[c] : 0;
        int na, ng;
        const int pa = block_exclusive_scan(st == 1, na);
        const int pg = block_exclusive_scan(st == 2, ng);
        if (c < c1) {
            const unsigned long long k = key[c];
            if (st == 1) {
                const long long nc = ba + pa;
                const T val = (T)((double)Q[c] * s2);
                keyo[nc] = k;
                Qo[nc] = val;
                omo[nc] = (unsigned short)(om[c] & 0xfffu);
                copy_velocities<N, T>(m, b, v.g, c, nc);
                b.map[c] = (int)nc;
                acc_add(d, (double)val, err);
                mx = fmax(mx, (double)val);
                rmax = fmax(rmax, b.rate[v.g][c]);
            } else if (st == 2) {
                const long long nc = bg + pg;
                keyo[nc] = k;
                Qo[nc] = (T)0;
                omo[nc] = (unsigned short)((om[c] & 0xfffu) | OM_GHOST);
                copy_velocities<N, T>(m, b, v.g, c, nc);
                b.map[c] = (int)nc;
            } else {
                b.map[c] = -1;
            }
        }
        ba += na;
        bg += ng;
    }
}

// The compaction of the graph and direct paths: every survivor goes to the
// place map[c] that the prune's sort gave it (status in keep); the same
// values, rescaling and partials as prune_compact_body.
template <int N, typename T>
__device__ __forceinline__ void prune_compact_sorted_body(const Model& m, const Bufs& b, const StepView& v,
                                                          long long (&d)[NDIG], double& mx, double& rmax,
                                                          int& err) {
    const T* Q = static_cast<const T*>(b.q[v.pb]);
    T* Qo = static_cast<T*>(b.q[v.pb ^ 1]);
    const unsigned long long* key = b.key[v.g];
    unsigned long long* keyo = b.key[v.g ^ 1];
    const unsigned short* om = b.om[v.g];
    unsigned short* omo = b.om[v.g ^ 1];
    const double mq = v.maxq;
    const double s2 = (mq > 0.0 && isfinite(mq)) ? ldexp(1.0, -ilogb(mq)) : 1.0;
    for (WarpRuns r(v.N, v.nb, v.bi); r.next();) {
        const long long c = r.c;
        if (c >= v.N) continue;
        const int st = b.keep[c];
        if (st == 0) continue;
        const long long nc = b.map[c];
        const unsigned long long k = key[c];
        keyo[nc] = k;
        copy_velocities<N, T>(m, b, v.g, c, nc);
        if (st == 1) {
            const T val = (T)((double)Q[c] * s2);
            Qo[nc] = val;
            omo[nc] = (unsigned short)(om[c] & 0xfffu);
            acc_add(d, (double)val, err);
            mx = fmax(mx, (double)val);
            rmax = fmax(rmax, b.rate[v.g][c]);
        } else {
            Qo[nc] = (T)0;
            omo[nc] = (unsigned short)((om[c] & 0xfffu) | OM_GHOST);
        }
    }
}

// New links through the map, and the rehash of the survivors.
template <int N>
__device__ __forceinline__ void prune_relink_body(const Model& m, const Bufs& b, const StepView& v) {
    const int* link = b.link[v.g];
    int* linko = b.link[v.g ^ 1];
    const unsigned long long* keyo = b.key[v.g ^ 1];
    const long long cap = m.cap;
    for (WarpRuns r(v.N, v.nb, v.bi); r.next();) {
        const long long c = r.c;
        if (c >= v.N) continue;
        const int nc = b.map[c];
        if (nc < 0) continue;
        int L[2 * N];
        load_links<N>(link, cap, c, L);
#pragma unroll
        for (int d = 0; d < 2 * N; ++d) linko[(long long)d * cap + nc] = L[d] >= 0 ? b.map[L[d]] : -1;
        table_insert_new(m, b, keyo[nc], nc, b.slot[v.g ^ 1]);
    }
}

}  // namespace gbees
