// Device-side building blocks of the GBEES library: layout of the workspace,
// packed cell keys, the open-addressing hashtable, the drift models, the exact
// fixed-point accumulator and block reductions.
#pragma once

#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "gbees_keys.cuh"

namespace gbees {

namespace cg = cooperative_groups;

constexpr int MAXN = 6;
constexpr int THREADS = 256;
constexpr int WARPS = THREADS / 32;
constexpr int GRID_MAX = 8192;                       // blocks of the fixed launch grid (upper bound)
constexpr unsigned long long EMPTY_KEY = ~0ull;      // free hashtable slot

// Exact accumulator: NDIG signed 64-bit cells, each collecting 32-bit digits of a
// fixed-point number whose lowest bit weighs 2^ACC_LSB. The window
// [2^-128, 2^64) holds every density sum and moment of the workloads; terms
// below 2^-128 are truncated (deterministically), terms of 2^64 or more raise
// an error. Up to 2^31 terms per reduction need no carry.
constexpr int NDIG = 6;
constexpr int ACC_LSB = -128;

enum { DYN_CONSTANT = 0, DYN_LINEAR = 1, DYN_LORENZ63 = 2, DYN_LORENZ63_SHIFTED = 3, DYN_LORENZ96 = 4 };
enum { LIM_MC = 0, LIM_NONE = 1, LIM_LW = 2 };
enum {
    ST_OK = 0,
    ST_EINVAL = -1,
    ST_ECAPACITY = -2,
    ST_EKEYRANGE = -3,
    ST_EDEGENERATE = -4,
    ST_ECUDA = -5,
    ST_ETIMEOUT = -6,
    ST_ETABLE = -7
};

struct alignas(16) Slot {
    unsigned long long key;
    long long val;  // cell index (low 32 bits used)
};

// Scalars that live on the device so that a whole step needs no host round trip.
struct alignas(256) DevScalars {
    long long N;          // pool entries, active cells and halo cells (grows during grow)
    long long N_prev;     // pool entries before the current grow
    long long N_new;      // pool entries surviving the current prune
    long long NA;         // active cells
    long long NA_new;     // active cells surviving the current prune
    long long n_halo;     // halo cells appended by the current halo phase
    long long n_act;      // halo cells made active by the current grow (listed in map)
    long long n_glist;    // cells listed for the current grow (listed form)
    double t;             // time
    double t_target;      // end of the current propagate call
    double dt;            // last step
    unsigned long long maxrate_bits;      // max CFL rate over the cells (non-negative double bits)
    unsigned long long maxq_ord;          // order key of the running max of Q
    double maxq;          // max of Q after the last finalisation
    double w;             // (prod h) * sum Q at the last finalisation
    double scale;         // 1 / w, applied by the next step
    long long acc[NDIG];  // exact sum of Q
    long long step;       // steps since init
    long long steps_call; // steps of the current propagate call
    long long updates_call;  // cell updates of the current propagate call
    long long lookups_fallback;  // hashtable lookups of the flux update (none: every stencil cell is linked)
    int pbuf;             // current Q buffer
    int gen;              // current key/link buffer
    int done;             // t reached t_target
    int error;            // first error status (0 = none)
    int prune_now;        // the step just taken is a prune step
    unsigned int ticket;  // last-block election
    unsigned long long tmp_ord;  // scratch maximum (init)
    long long loop_iter;  // iterations of the device-side step loop in the current graph launch
    long long graph_kernels;  // kernels executed by graph launches (counted on the device)
    // grid barrier of a team of a batched launch: arrivals in the low 32 bits,
    // generation in the high 32 bits
    unsigned long long bar_word;
    // grid barrier of the persistent kernel: arrivals since the launch began
    // (cleared by the host before every persistent launch)
    unsigned long long bar_seq;
    // the step loop's running reductions, in global atomics: the largest CFL
    // rate of the current prune epoch (two epochs by parity), and the exact
    // sum and maximum of the apply phase (two steps by parity)
    unsigned long long loop_rate[2];
    long long loop_acc[2][NDIG];
    unsigned long long loop_maxq[2];
    // SM cycles spent by block 0 of the persistent kernel per phase (grow,
    // halo, link, faces, apply, prune, step scalars) and the steps they cover
    long long phase_cycles[8];
    long long phase_steps;
    // the current step (written by the last block of the link kernel)
    double step_dt;       // dt of the step being taken
    double step_t_new;    // time after it
    int step_last;        // the step lands on t_target
    int step_pad;
    double coef_dth[MAXN];  // dt / h_j
    double coef_ch[MAXN];   // dt / (2 h_j)
    long long mom[28][NDIG];     // exact sums for moments
    double mom_mean[MAXN];       // mean, input of the covariance pass
    double mom_out[28];          // moments times prod h
};

// Everything a kernel needs to know about the model and the grid (by value).
struct Model {
    int n;
    int dyn;
    int limiter;
    int key_bits;
    int prune_interval;
    int probe_width;
    int sort_order;              // storage order after a sorting prune (GBEES_ORDER_*)
    int bar_extra;               // arrivals a grid barrier waits for beyond its blocks (0; > 0 only to test the bounded wait)
    long long spin_limit;        // polls of a grid barrier before it gives up with ST_ETIMEOUT
    long long cap;               // cell capacity
    unsigned long long tmask;    // hashtable slots - 1
    double a[64];                // model parameters
    double h[MAXN];
    double x0[MAXN];
    double thr_rel;
    double cfl;
    double prod_h;
    double inv_h[MAXN];    // 1 / h_j
    double inv_2h[MAXN];   // 1 / (2 h_j)
    int h_pow2;            // bit j: h_j is a power of two
    // float copies for the FP32 update (no double-to-float conversion per use)
    float af[48];
    float hf[MAXN];
    float x0f[MAXN];
};

// Model parameter i in the arithmetic type of the caller.
template <typename R>
__device__ __forceinline__ R par(const Model& m, int i);
template <>
__device__ __forceinline__ double par<double>(const Model& m, int i) { return m.a[i]; }
template <>
__device__ __forceinline__ float par<float>(const Model& m, int i) { return m.af[i]; }

// One block's share of a grid-wide reduction, written without atomics and
// combined by whoever finishes the step (deterministic: integer digits, max).
struct alignas(64) Partial {
    long long acc[NDIG];           // exact-sum digits of the block's values
    unsigned long long maxq_ord;   // order key of the block's maximum value (0: none)
    unsigned long long rate_bits;  // the block's maximum CFL rate (non-negative double bits)
};

// Device buffers (by value). The pool holds the active cells and their halo:
// every face neighbour of an active cell that is not active itself is kept as
// a halo cell (p = 0, never updated, never counted), so that all cells of the
// update stencil (face neighbours, their face neighbours, the second
// neighbours) are reached through links. link[g] holds 2n direction-major
// int32 arrays of cap entries: link[g][(2j + s) * cap + c] is the index of the
// neighbour of entry c one step down (s = 0) or up (s = 1) in dimension j, or
// -1 when it is not in the pool (a warp's consecutive entries read one
// direction with one coalesced load).
//
// om[g][c]: bits 0..2n-1 are the outward directions of cell c (bit 2j+1: the
// flow leaves through the upper j-face, bit 2j: through the lower j-face),
// fixed at creation because the drift does not depend on time; bit 14 marks a
// halo cell; bit 15 marks an active cell whose downwind set is known to be
// active (cleared by every prune).
//
// Face velocities (storage type, dimension-major: u[g][j * cap + c]): f_j at
// the centre of the lower j-face of entry c (Eq. 7), evaluated once in FP64 when
// the entry is created (the drift does not depend on time) and carried along
// by the prune's compaction.
//
// Update scratch of the three-pass flux update (storage type, dimension-major:
// element d * cap + c, so that a warp's 32 consecutive entries read and write
// whole sectors): wl[d] the jump P_c - P_{c-e_d} across the lower d-face, wg[d]
// the d-direction wave entering the cell, tg the sum over d of wg[d] / (2 h_d)
// (one value per entry), fl[j] the flux through the lower j-face.
struct Bufs {
    unsigned long long* key[2];
    void* q[2];
    int* link[2];
    unsigned short* om[2];
    unsigned int* slot[2];  // hashtable slot of each cell
    unsigned char* keep;
    int* map;        // prune: status, then new index; grow: the halo cells it activated
    Slot* table;
    DevScalars* sc;
    long long* blk;  // per-block counts (active cells)
    long long* blk2; // per-block counts (halo cells)
    unsigned int* sorthist;  // digit histograms of the prune's radix sort
    void* u[2];  // face velocities (two generations, like the keys)
    double* rate[2];  // CFL rate sum_j |f_j(x_{c-e_j/2})| / h_j of every entry (Eq. 8, FP64, fixed at creation)
    void* wl;    // update scratch in the storage type
    void* wg;
    void* tg;
    void* fl;
    Partial* part;   // GRID_MAX per-block partials
};


constexpr unsigned short OM_COMPLETE = 0x8000;
constexpr unsigned short OM_GHOST = 0x4000;

// The kernels of one time step for one model and precision: those before the
// link phase, those after it, and the persistent step-loop kernel.
struct Kernels {
    void* pre[3];
    int npre;
    void* post[3];
    int npost;
    void* persist;
    void* batch;
    void* batch_teams;
};

// One grid of a batched propagation (k_batch): its model, its buffers (in its
// own workspace) and the time to propagate it to.
struct BatchItem {
    Model m;
    Bufs b;
    double t_end;
};

// Block of a team launch (k_batch_teams): the grid it works on (-1: none), the
// team's size and this block's index in the team.
struct TeamSlot {
    int item, nb, bi;
};



// ------------------------------------------------------------------ cell iteration
// Cells are handed out in runs of 32 consecutive cells (one warp, coalesced),
// consecutive runs to consecutive blocks, so that a small grid still spreads
// over every SM. The blocks that share the work of one grid are nb blocks of
// index bi (the whole launch, or one block when a launch runs many grids).
// Usage:
//   for (WarpRuns r(ncell, nb, bi); r.next();) { const long long c = r.c; if (c >= ncell) continue; ... }
struct WarpRuns {
    long long k, step, n, c;
    __device__ __forceinline__ WarpRuns(long long ncell, int nb, int bi)
        : k(bi + (long long)nb * (threadIdx.x >> 5) - (long long)nb * (blockDim.x >> 5)),
          step((long long)nb * (blockDim.x >> 5)),
          n(ncell),
          c(0) {}
    __device__ __forceinline__ explicit WarpRuns(long long ncell) : WarpRuns(ncell, gridDim.x, blockIdx.x) {}
    __device__ __forceinline__ bool next() {
        k += step;
        c = k * 32 + (threadIdx.x & 31);
        return k * 32 < n;
    }
};

// ------------------------------------------------------------------ keys

template <int N>
__device__ __forceinline__ bool pack_key(const Model& m, const int* I, unsigned long long& k) {
    return pack_key_bits<N>(m.key_bits, I, k);
}

template <int N>
__device__ __forceinline__ void unpack_key(const Model& m, unsigned long long k, int* I) {
    unpack_key_bits<N>(m.key_bits, k, I);
}

// ------------------------------------------------------------------ hashtable
// Open addressing with linear probing (Sec. 4.2); keys are claimed with
// atomicCAS (the concurrent insertion of Algorithm 2 without staging).

__device__ __forceinline__ int table_find(const Model& m, const Slot* __restrict__ T, unsigned long long key) {
    unsigned long long h = mix64(key) & m.tmask;
    for (unsigned long long probe = 0; probe <= m.tmask; ++probe) {
        ulonglong2 s = __ldcg(reinterpret_cast<const ulonglong2*>(T + h));
        if (s.x == key) return (int)(long long)s.y;
        if (s.x == EMPTY_KEY) return -1;
        h = (h + 1) & m.tmask;
    }
    return -1;
}

// Cooperative lookup: a tile of W lanes probes W consecutive slots per round
// (one coalesced load) and the lowest lane that sees the key or an empty slot
// decides. All lanes of the tile must call it with the same key.
template <int W>
__device__ __forceinline__ int table_find_tile(const Model& m, const Slot* __restrict__ T, unsigned long long key,
                                               cg::thread_block_tile<W> tile) {
    unsigned long long base = mix64(key) & m.tmask;
    const int lane = tile.thread_rank();
    for (unsigned long long probe = 0; probe <= m.tmask; probe += W) {
        unsigned long long h = (base + probe + lane) & m.tmask;
        ulonglong2 s = __ldcg(reinterpret_cast<const ulonglong2*>(T + h));
        unsigned hit = tile.ballot(s.x == key);
        unsigned emp = tile.ballot(s.x == EMPTY_KEY);
        if (hit | emp) {
            int first_hit = hit ? __ffs(hit) - 1 : W;
            int first_emp = emp ? __ffs(emp) - 1 : W;
            if (first_hit < first_emp) {
                long long v = tile.shfl((long long)s.y, first_hit);
                return (int)v;
            }
            return -1;
        }
    }
    return -1;
}

// Insert key if absent. Returns 1 and the slot when this thread claimed a new
// slot, 0 when the key is present, -1 when the table is full.
__device__ __forceinline__ int table_claim(const Model& m, Slot* T, unsigned long long key, unsigned long long* slot) {
    unsigned long long h = mix64(key) & m.tmask;
    for (unsigned long long probe = 0; probe <= m.tmask; ++probe) {
        unsigned long long k = *reinterpret_cast<volatile unsigned long long*>(&T[h].key);
        if (k == key) return 0;
        if (k == EMPTY_KEY) {
            unsigned long long old = atomicCAS(&T[h].key, EMPTY_KEY, key);
            if (old == EMPTY_KEY) {
                *slot = h;
                return 1;
            }
            if (old == key) return 0;
        }
        h = (h + 1) & m.tmask;
    }
    return -1;
}

// ------------------------------------------------------------------ errors

__device__ __forceinline__ void set_error(DevScalars* sc, int code) { atomicCAS(&sc->error, 0, code); }

__device__ __forceinline__ long long warp_aggregated_add(long long* counter, int count = 1) {
    cg::coalesced_group g = cg::coalesced_threads();
    long long base = 0;
    int total = g.size() * count;
    if (g.thread_rank() == 0) base = (long long)atomicAdd((unsigned long long*)counter, (unsigned long long)total);
    base = g.shfl(base, 0);
    return base + (long long)g.thread_rank() * count;
}

// ------------------------------------------------------------------ drift models

template <typename R>
struct Ar;  // IEEE operations without contraction into fused multiply-add

template <>
struct Ar<double> {
    static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
    static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
    static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
};
template <>
struct Ar<float> {
    static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
    static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
};

// f_j(y) with the evaluation order written out (no fused multiply-add), so that
// the FP64 velocities that take the grow / prune / CFL decisions are the IEEE
// values of the textbook expressions.
template <typename R, int N>
__device__ __forceinline__ R drift(const Model& m, int dyn, const R* y, int j) {
    using A = Ar<R>;
    switch (dyn) {
        case DYN_CONSTANT:
            return par<R>(m, j);
        case DYN_LINEAR: {
            R s = 0;
#pragma unroll
            for (int k = 0; k < N; ++k) s = A::add(s, A::mul(par<R>(m, j * N + k), y[k]));
            return A::add(s, par<R>(m, N * N + j));
        }
        case DYN_LORENZ63:
            if (N != 3) return 0;
            if (j == 0) return A::mul(par<R>(m, 0), A::sub(y[1], y[0]));
            if (j == 1) return A::sub(A::mul(y[0], A::sub(par<R>(m, 1), y[2 % N])), y[1]);
            return A::sub(A::mul(y[0], y[1]), A::mul(par<R>(m, 2), y[2 % N]));
        case DYN_LORENZ63_SHIFTED:
            if (N != 3) return 0;
            if (j == 0) return A::mul(par<R>(m, 0), A::sub(y[1], y[0]));
            if (j == 1) return A::sub(-y[1], A::mul(y[0], y[2 % N]));
            return A::sub(A::add(A::mul(-par<R>(m, 1), y[2 % N]), A::mul(y[0], y[1])),
                          A::mul(par<R>(m, 1), par<R>(m, 2)));
        case DYN_LORENZ96: {
            const int jp = (j + 1) % N, jm2 = (j + N - 2) % N, jm1 = (j + N - 1) % N;
            return A::add(A::sub(A::mul(A::sub(y[jp], y[jm2]), y[jm1]), y[j]), par<R>(m, 0));
        }
    }
    return 0;
}

// Centre coordinate x0_k + i_k h_k and lower-face coordinate x0_k + (i_k - 1/2) h_k,
// evaluated exactly as written (one rounded product, one rounded sum).
__device__ __forceinline__ double centre64(const Model& m, int k, int i) {
    return __dadd_rn(m.x0[k], __dmul_rn((double)i, m.h[k]));
}
__device__ __forceinline__ double lowface64(const Model& m, int k, int i) {
    return __dadd_rn(m.x0[k], __dmul_rn((double)i - 0.5, m.h[k]));
}

// FP64 face velocity f_j at the lower face of cell I in dimension j (Eq. 7).
template <int N>
__device__ __forceinline__ double face_velocity64(const Model& m, const int* I, int j) {
    double y[N];
#pragma unroll
    for (int k = 0; k < N; ++k) y[k] = (k == j) ? lowface64(m, k, I[k]) : centre64(m, k, I[k]);
    return drift<double, N>(m, m.dyn, y, j);
}

// x / h_j as the IEEE division rounds it. For a width that is a power of two
// the reciprocal is exact, so the product rounds the same real number: the
// same result for one FP64 multiplication instead of a division sequence.
__device__ __forceinline__ double div_h(const Model& m, double x, int j) {
    return ((m.h_pow2 >> j) & 1) ? __dmul_rn(x, m.inv_h[j]) : __ddiv_rn(x, m.h[j]);
}

// FP64 CFL rate sum_j |f_j(x_{i-e_j/2})| / h_j (Eq. 8 with |f|).
template <int N>
__device__ __forceinline__ double cfl_rate64(const Model& m, const int* I) {
    double r = 0.0;
#pragma unroll
    for (int j = 0; j < N; ++j) r = __dadd_rn(r, div_h(m, fabs(face_velocity64<N>(m, I, j)), j));
    return r;
}

// a * b + c rounded once, and the larger of two values, in the arithmetic
// type itself (explicit single-precision forms for float, so that nothing is
// widened to double).
__device__ __forceinline__ double fmadd(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fmadd(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double vmax(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ float vmax(float a, float b) { return fmaxf(a, b); }

// Sign tests, positive and negative parts. FP64 arithmetic is scarce on this
// chip, so for doubles they work on the bit pattern in the integer pipe (a
// finite double is > 0 exactly when its bits, read as a signed integer, are
// > 0; -0 reads as the smallest integer).
__device__ __forceinline__ bool gt0(double x) { return __double_as_longlong(x) > 0; }
__device__ __forceinline__ bool lt0(double x) {
    const long long b = __double_as_longlong(x);
    return b < 0 && (b << 1) != 0;
}
__device__ __forceinline__ bool gt0(float x) { return x > 0.0f; }
__device__ __forceinline__ bool lt0(float x) { return x < 0.0f; }
template <typename T>
__device__ __forceinline__ T pos_part(T x) { return gt0(x) ? x : (T)0; }
template <typename T>
__device__ __forceinline__ T neg_part(T x) { return lt0(x) ? x : (T)0; }
__device__ __forceinline__ double abs_bits(double x) {
    return __longlong_as_double(__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFll);
}
__device__ __forceinline__ float abs_bits(float x) { return fabsf(x); }
// min of two non-negative finite values (integer order of the bits for doubles)
__device__ __forceinline__ double min_nonneg(double a, double b) {
    return __longlong_as_double(min(__double_as_longlong(a), __double_as_longlong(b)));
}
__device__ __forceinline__ float min_nonneg(float a, float b) { return fminf(a, b); }

// The significance test p > p* (p* >= 0) of a stored value, decided exactly
// as (double)p > p* but without FP64 arithmetic: for doubles on the bit
// patterns (signed integer order equals the order of doubles when one side is
// non-negative), for floats against the largest float not above p*.
template <typename T>
struct Above;
template <>
struct Above<double> {
    long long pb;
    __device__ __forceinline__ explicit Above(double pstar) { pb = __double_as_longlong(pstar); }
    __device__ __forceinline__ bool operator()(double q) const { return __double_as_longlong(q) > pb; }
};
template <>
struct Above<float> {
    float pf;
    __device__ __forceinline__ explicit Above(double pstar) {
        pf = (float)pstar;
        if ((double)pf > pstar) pf = nextafterf(pf, -INFINITY);  // round towards -inf
    }
    __device__ __forceinline__ bool operator()(float q) const { return q > pf; }
};

// 2x and x/2 of a non-negative double with the results of IEEE x + x and
// x * 0.5 (round to nearest even), in integer operations only (no FP64 pipe):
// the exponent field moves by one; a subnormal or overflowing case is formed
// on the bit pattern directly.
__device__ __forceinline__ double twice_nonneg(double x) {
    const long long b = __double_as_longlong(x);
    const long long e = b >> 52;
    long long r = e == 0 ? (b << 1)                                   // subnormal (or 0): the significand doubles
                : e <= 2045 ? b + (1ll << 52)                         // one more in the exponent
                : e == 2046 ? 0x7FF0000000000000ll                    // overflow to +inf
                : b;                                                  // inf, NaN
    return __longlong_as_double(r);
}
__device__ __forceinline__ double half_nonneg(double x) {
    const long long b = __double_as_longlong(x);
    const long long e = b >> 52;
    if (e >= 2) return __longlong_as_double(b - (1ll << 52));         // one less in the exponent (inf, NaN stay)
    // the result is subnormal: halve the significand, ties to even
    const long long sig = e == 0 ? b : (b & 0xFFFFFFFFFFFFFll) | (1ll << 52);
    long long q = sig >> 1;
    if ((sig & 1) && (q & 1)) q += 1;
    return __longlong_as_double(q);
}
__device__ __forceinline__ float twice_nonneg(float x) { return x + x; }
__device__ __forceinline__ float half_nonneg(float x) { return 0.5f * x; }

template <typename T>
__device__ __forceinline__ T limited_wave(int lim, T W, T Wup) {
    if (lim == LIM_LW) return W;
    // MC limiter phi(theta) = max(0, min((1+theta)/2, 2, 2 theta)) with theta = Wup / W,
    // multiplied by W and written without the division: zero unless W and Wup
    // have the same sign, else sign(W) min(|W + Wup| / 2, 2 |W|, 2 |Wup|).
    if ((gt0(W) && gt0(Wup)) || (lt0(W) && lt0(Wup))) {
        const T aW = abs_bits(W), aU = abs_bits(Wup);
        const T v = min_nonneg(min_nonneg(half_nonneg(aW + aU), twice_nonneg(aW)), twice_nonneg(aU));
        return gt0(W) ? v : -v;
    }
    return (T)0;
}

// ------------------------------------------------------------------ exact accumulator

// Add x (a finite double) to the digits. Sets err on a non-finite or too
// large term.
__device__ __forceinline__ void acc_add(long long (&d)[NDIG], double x, int& err) {
    unsigned long long bits = (unsigned long long)__double_as_longlong(x);
    int ex = (int)((bits >> 52) & 0x7ff);
    unsigned long long mt = bits & 0xFFFFFFFFFFFFFull;
    if (ex == 0x7ff) { err = 1; return; }
    if (ex == 0) {
        if (mt == 0) return;
        ex = 1;
    } else {
        mt |= 1ull << 52;
    }
    int pos = ex - 1075 - ACC_LSB;  // x = mt * 2^(pos + ACC_LSB)
    if (pos < 0) {
        if (pos <= -64) return;
        mt >>= -pos;
        pos = 0;
        if (mt == 0) return;
    }
    if (pos > 32 * NDIG - 53 - 1) { err = 1; return; }
    const bool neg = (bits >> 63) != 0;
    const int k = pos >> 5, r = pos & 31;
    const unsigned long long lo = mt << r;
    const unsigned long long hi = r ? (mt >> (64 - r)) : 0ull;
    const long long d0 = (long long)(lo & 0xffffffffull), d1 = (long long)(lo >> 32), d2 = (long long)(hi & 0xffffffffull);
#pragma unroll
    for (int q = 0; q < NDIG; ++q) {
        long long v = (q == k) ? d0 : (q == k + 1) ? d1 : (q == k + 2) ? d2 : 0;
        d[q] += neg ? -v : v;
    }
}

// The same for a float (integer operations only; a float is exactly a double).
__device__ __forceinline__ void acc_add(long long (&d)[NDIG], float x, int& err) {
    const unsigned int bits = __float_as_uint(x);
    int ex = (int)((bits >> 23) & 0xff);
    unsigned long long mt = bits & 0x7FFFFFu;
    if (ex == 0xff) { err = 1; return; }
    if (ex == 0) {
        if (mt == 0) return;
        ex = 1;
    } else {
        mt |= 1u << 23;
    }
    int pos = ex - 150 - ACC_LSB;  // x = mt * 2^(pos + ACC_LSB)
    if (pos < 0) {
        if (pos <= -32) return;
        mt >>= -pos;
        pos = 0;
        if (mt == 0) return;
    }
    if (pos > 32 * NDIG - 24 - 1) { err = 1; return; }
    const bool neg = (bits >> 31) != 0;
    const int k = pos >> 5, r = pos & 31;
    const unsigned long long sh = mt << r;  // at most 55 bits
    const long long d0 = (long long)(sh & 0xffffffffull), d1 = (long long)(sh >> 32);
#pragma unroll
    for (int q = 0; q < NDIG; ++q) {
        long long v = (q == k) ? d0 : (q == k + 1) ? d1 : 0;
        d[q] += neg ? -v : v;
    }
}

// Round the exact value sum_q D[q] 2^(32 q + ACC_LSB) once to the nearest double.
__device__ inline double acc_to_double(const long long* D) {
    long long c[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) c[q] = q < NDIG ? D[q] : 0;
    for (int q = 0; q < 7; ++q) {
        long long carry = c[q] >> 32;  // floor division by 2^32
        c[q] -= carry * 4294967296ll;
        c[q + 1] += carry;
    }
    const bool neg = c[7] < 0;
    unsigned long long W[4];
    {
        unsigned int mag[8];
        unsigned long long carry = 1;
        for (int q = 0; q < 8; ++q) {
            unsigned int v = (unsigned int)(unsigned long long)c[q];
            if (neg) {
                unsigned long long s = (unsigned long long)(~v) + carry;
                mag[q] = (unsigned int)s;
                carry = s >> 32;
            } else {
                mag[q] = v;
            }
        }
        for (int q = 0; q < 4; ++q) W[q] = (unsigned long long)mag[2 * q] | ((unsigned long long)mag[2 * q + 1] << 32);
    }
    int top = -1;
    for (int q = 3; q >= 0; --q)
        if (W[q]) { top = q; break; }
    if (top < 0) return 0.0;
    const int msb = 64 * top + 63 - __clzll((long long)W[top]);
    auto extract = [&](int shift) -> unsigned long long {  // bits [shift, shift + 64)
        if (shift < 0) return W[0] << (-shift);
        int wq = shift >> 6, r = shift & 63;
        unsigned long long lo = wq < 4 ? W[wq] >> r : 0ull;
        unsigned long long hi = (r && wq + 1 < 4) ? W[wq + 1] << (64 - r) : 0ull;
        return lo | hi;
    };
    double result;
    if (msb < 53) {
        result = ldexp((double)W[0], ACC_LSB);
    } else {
        const int sh = msb - 53;  // the 54 bits [sh, msb] hold mantissa + round bit
        unsigned long long v54 = extract(sh) & ((1ull << 54) - 1);
        unsigned long long v = v54 >> 1;
        const unsigned long long round = v54 & 1ull;
        bool sticky = false;
        for (int q = 0; q < 4 && !sticky; ++q) {
            int lo_bit = 64 * q;
            if (lo_bit >= sh) break;
            int nb = sh - lo_bit;
            unsigned long long mask = nb >= 64 ? ~0ull : ((1ull << nb) - 1);
            sticky = (W[q] & mask) != 0;
        }
        if (round && (sticky || (v & 1ull))) v += 1;
        result = ldexp((double)v, msb - 52 + ACC_LSB);
    }
    return neg ? -result : result;
}

// Order-preserving map of doubles onto unsigned 64-bit keys (for atomicMax).
__device__ __forceinline__ unsigned long long ord_key(double x) {
    unsigned long long b = (unsigned long long)__double_as_longlong(x);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double ord_val(unsigned long long k) {
    unsigned long long b = (k >> 63) ? (k & 0x7FFFFFFFFFFFFFFFull) : ~k;
    return __longlong_as_double((long long)b);
}

// Block-wide reduction of the digits and of a maximum, then one atomic per
// digit into global memory. All threads of the block must call it.
__device__ __forceinline__ void block_reduce_acc_max(long long (&d)[NDIG], double mx, long long* g_acc,
                                                     unsigned long long* g_ord) {
    __shared__ long long s_acc[WARPS][NDIG];
    __shared__ double s_mx[WARPS];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NDIG; ++q) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) d[q] += __shfl_down_sync(0xffffffffu, d[q], off);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, off));
    if (lane == 0) {
#pragma unroll
        for (int q = 0; q < NDIG; ++q) s_acc[wid][q] = d[q];
        s_mx[wid] = mx;
    }
    __syncthreads();
    if (threadIdx.x < NDIG) {
        long long v = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += s_acc[w][threadIdx.x];
        if (v) atomicAdd((unsigned long long*)&g_acc[threadIdx.x], (unsigned long long)v);
    }
    if (threadIdx.x == 32 && g_ord) {
        double m = -INFINITY;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, s_mx[w]);
        if (m > -INFINITY) atomicMax(g_ord, ord_key(m));
    }
    __syncthreads();
}

__device__ __forceinline__ double block_max(double mx) {
    __shared__ double s_m[WARPS];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, off));
    if ((threadIdx.x & 31) == 0) s_m[threadIdx.x >> 5] = mx;
    __syncthreads();
    double m = -INFINITY;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, s_m[w]);
    __syncthreads();
    return m;
}

// True in every thread of exactly one block: the last one to arrive. One
// thread per block fences and takes a ticket (the block barrier before it
// orders the block's writes; fences are cumulative).
__device__ __forceinline__ bool last_block(DevScalars* sc) {
    __shared__ bool s_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        unsigned int t = atomicAdd(&sc->ticket, 1u);
        s_last = (t == gridDim.x - 1);
        if (s_last) __threadfence();
    }
    __syncthreads();
    return s_last;
}

// Normalisation scalars of a new grid from the exact sum and the running
// maximum. mode bit 2: keep w = 1 (cells loaded as given).
__device__ __forceinline__ void finalise_norm(const Model& m, DevScalars* sc, int mode) {
    sc->N_prev = sc->N;
    sc->maxq = sc->maxq_ord ? ord_val(sc->maxq_ord) : 0.0;
    if (mode & 2) {
        sc->w = 1.0;
        sc->scale = 1.0;
    } else {
        long long D[NDIG];
        for (int q = 0; q < NDIG; ++q) D[q] = *(volatile long long*)&sc->acc[q];
        double s = acc_to_double(D);
        double w = m.prod_h * s;
        sc->w = w;
        if (!(w > 0.0) || !isfinite(w)) {
            set_error(sc, ST_EDEGENERATE);
            sc->scale = 0.0;
        } else {
            sc->scale = 1.0 / w;
        }
    }
    for (int q = 0; q < NDIG; ++q) sc->acc[q] = 0;
    sc->maxq_ord = 0;
    sc->ticket = 0;
    if (sc->N == 0 && !(mode & 2)) set_error(sc, ST_EDEGENERATE);
}

// Write this block's partial (exact digits, maximum value, maximum rate).
// All threads of the block must call it; d, mx, rate are per thread. The
// maxima are reduced as order-preserving integer keys (integer pipe).
__device__ __forceinline__ void block_partial(Partial* part, long long (&d)[NDIG], double mx, double rate,
                                              int bi) {
    __shared__ long long s_acc[WARPS][NDIG];
    __shared__ unsigned long long s_mx[WARPS], s_rt[WARPS];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned long long mk = mx > -INFINITY ? ord_key(mx) : 0ull;
    unsigned long long rk = rate > 0.0 ? (unsigned long long)__double_as_longlong(rate) : 0ull;
#pragma unroll
    for (int q = 0; q < NDIG; ++q) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) d[q] += __shfl_down_sync(0xffffffffu, d[q], off);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        mk = max(mk, __shfl_down_sync(0xffffffffu, mk, off));
        rk = max(rk, __shfl_down_sync(0xffffffffu, rk, off));
    }
    if (lane == 0) {
#pragma unroll
        for (int q = 0; q < NDIG; ++q) s_acc[wid][q] = d[q];
        s_mx[wid] = mk;
        s_rt[wid] = rk;
    }
    __syncthreads();
    // one thread per digit and per maximum folds the warps' values
    const int q = threadIdx.x, nw = (int)(blockDim.x >> 5);
    if (q < NDIG) {
        long long a = 0;
        for (int w = 0; w < nw; ++w) a += s_acc[w][q];
        part[bi].acc[q] = a;
    } else if (q == NDIG) {
        unsigned long long mm = 0;
        for (int w = 0; w < nw; ++w) mm = max(mm, s_mx[w]);
        part[bi].maxq_ord = mm;
    } else if (q == NDIG + 1) {
        unsigned long long rr = 0;
        for (int w = 0; w < nw; ++w) rr = max(rr, s_rt[w]);
        part[bi].rate_bits = rr;
    }
    __syncthreads();
}
__device__ __forceinline__ void block_partial(Partial* part, long long (&d)[NDIG], double mx, double rate) {
    block_partial(part, d, mx, rate, blockIdx.x);
}

// The block's digits, maximum value and maximum rate folded into global
// accumulators with atomics (acc may be null: rate only). Integer sums and
// maxima: the totals do not depend on the order of the blocks.
__device__ __forceinline__ void block_atomics(long long* acc, unsigned long long* maxq, unsigned long long* rate,
                                              long long (&d)[NDIG], double mx, double r) {
    __shared__ long long s_acc[WARPS][NDIG];
    __shared__ unsigned long long s_mx[WARPS], s_rt[WARPS];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned long long mk = mx > -INFINITY ? ord_key(mx) : 0ull;
    unsigned long long rk = r > 0.0 ? (unsigned long long)__double_as_longlong(r) : 0ull;
    if (acc) {
#pragma unroll
        for (int q = 0; q < NDIG; ++q) {
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) d[q] += __shfl_down_sync(0xffffffffu, d[q], off);
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        mk = max(mk, __shfl_down_sync(0xffffffffu, mk, off));
        rk = max(rk, __shfl_down_sync(0xffffffffu, rk, off));
    }
    if (lane == 0) {
#pragma unroll
        for (int q = 0; q < NDIG; ++q) s_acc[wid][q] = d[q];
        s_mx[wid] = mk;
        s_rt[wid] = rk;
    }
    __syncthreads();
    const int q = threadIdx.x, nw = (int)(blockDim.x >> 5);
    if (q < NDIG) {
        if (acc) {
            long long a = 0;
            for (int w = 0; w < nw; ++w) a += s_acc[w][q];
            if (a) atomicAdd((unsigned long long*)&acc[q], (unsigned long long)a);
        }
    } else if (q == NDIG) {
        if (maxq) {
            unsigned long long mm = 0;
            for (int w = 0; w < nw; ++w) mm = max(mm, s_mx[w]);
            if (mm) atomicMax(maxq, mm);
        }
    } else if (q == NDIG + 1) {
        if (rate) {
            unsigned long long rr = 0;
            for (int w = 0; w < nw; ++w) rr = max(rr, s_rt[w]);
            if (rr) atomicMax(rate, rr);
        }
    }
    __syncthreads();
}

// Combine the partials of blocks [0, nblk) in every thread of the calling
// block (the same result everywhere): digit sums, maximum value, maximum rate.
struct Combined {
    long long acc[NDIG];
    unsigned long long maxq_ord;
    unsigned long long rate_bits;
};
__device__ __forceinline__ Combined combine_partials(const Partial* part, int nblk) {
    __shared__ long long s_acc[WARPS][NDIG];
    __shared__ unsigned long long s_mo[WARPS], s_rt[WARPS];
    long long d[NDIG] = {0, 0, 0, 0, 0, 0};
    unsigned long long mo = 0, rt = 0;
    for (int i = threadIdx.x; i < nblk; i += blockDim.x) {
        const Partial* p = part + i;
#pragma unroll
        for (int q = 0; q < NDIG; ++q) d[q] += __ldcg(&p->acc[q]);
        mo = max(mo, __ldcg(&p->maxq_ord));
        rt = max(rt, __ldcg(&p->rate_bits));
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NDIG; ++q)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) d[q] += __shfl_down_sync(0xffffffffu, d[q], off);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        mo = max(mo, __shfl_down_sync(0xffffffffu, mo, off));
        rt = max(rt, __shfl_down_sync(0xffffffffu, rt, off));
    }
    if (lane == 0) {
#pragma unroll
        for (int q = 0; q < NDIG; ++q) s_acc[wid][q] = d[q];
        s_mo[wid] = mo;
        s_rt[wid] = rt;
    }
    __syncthreads();
    // one thread per digit and per maximum folds the warps' values; every
    // thread then reads the results
    __shared__ unsigned long long s_fin[NDIG + 2];
    const int q = threadIdx.x, nw = (int)(blockDim.x >> 5);
    if (q < NDIG) {
        long long a = 0;
        for (int w = 0; w < nw; ++w) a += s_acc[w][q];
        s_fin[q] = (unsigned long long)a;
    } else if (q == NDIG) {
        unsigned long long mm = 0;
        for (int w = 0; w < nw; ++w) mm = max(mm, s_mo[w]);
        s_fin[q] = mm;
    } else if (q == NDIG + 1) {
        unsigned long long rr = 0;
        for (int w = 0; w < nw; ++w) rr = max(rr, s_rt[w]);
        s_fin[q] = rr;
    }
    __syncthreads();
    Combined c;
#pragma unroll
    for (int k = 0; k < NDIG; ++k) c.acc[k] = (long long)s_fin[k];
    c.maxq_ord = s_fin[NDIG];
    c.rate_bits = s_fin[NDIG + 1];
    __syncthreads();
    return c;
}

// Grid-wide barrier of a cooperative launch (all blocks resident). The wait is
// bounded: it gives up when another block has set an error or after
// spin_limit polls (BARRIER_SPIN_LIMIT by default: about two seconds), sets
// ST_ETIMEOUT, and returns false; callers then leave.
constexpr long long BARRIER_SPIN_LIMIT = 1ll << 26;

__device__ __forceinline__ unsigned long long atom_add_acq_rel_gpu(unsigned long long* p, unsigned long long v) {
    unsigned long long old;
    asm volatile("atom.add.acq_rel.gpu.u64 %0, [%1], %2;" : "=l"(old) : "l"(p), "l"(v) : "memory");
    return old;
}

__device__ __forceinline__ unsigned long long ld_acquire_gpu(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Barrier of the nb blocks that share the grid whose scalars are sc (the whole
// launch, or a team of a batched launch); every block of the team must be
// resident (cooperative launch). Bounded: gives up with ST_ETIMEOUT.
__device__ __forceinline__ bool grid_barrier(DevScalars* sc, int nb, long long spin_limit = BARRIER_SPIN_LIMIT) {
    __shared__ int s_ok;
    unsigned long long* word = &sc->bar_word;
    __syncthreads();
    if (threadIdx.x == 0) {
        // one release-acquire add per block: it publishes the block's writes
        // and counts the arrival; the last to arrive clears the count and opens
        // the next generation with a second add on the same word (a count of
        // nb plus 2^32 - nb carries into the generation), so the waiters'
        // acquire loads see every block's writes once the generation moves
        const unsigned long long old = atom_add_acq_rel_gpu(word, 1ull);
        const unsigned int gen = (unsigned int)(old >> 32);
        int ok = 1;
        if ((unsigned int)old == (unsigned int)nb - 1u) {
            atom_add_acq_rel_gpu(word, (1ull << 32) - (unsigned long long)(unsigned int)nb);
        } else {
            long long spins = 0;
            while ((unsigned int)(ld_acquire_gpu(word) >> 32) == gen) {
                if (*(volatile int*)&sc->error) { ok = 0; break; }
                if (++spins > spin_limit) {
                    set_error(sc, ST_ETIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(32);
            }
        }
        s_ok = ok && !*(volatile int*)&sc->error;
    }
    __syncthreads();
    return s_ok != 0;
}

// Barrier k (1, 2, ...) of a launch whose nb blocks all take part in every
// barrier, on a counter that was zero when the launch began: the barrier is
// complete once k * nb arrivals are counted. One release-acquire add per block
// and no reset, so the last arrival releases the waiters directly. Bounded like
// grid_barrier.
__device__ __forceinline__ bool grid_barrier_seq(DevScalars* sc, int nb, unsigned long long& k,
                                                 long long spin_limit = BARRIER_SPIN_LIMIT) {
    __shared__ int s_ok;
    unsigned long long* cnt = &sc->bar_seq;
    __syncthreads();
    k += 1;
    if (threadIdx.x == 0) {
        const unsigned long long target = k * (unsigned long long)(unsigned int)nb;
        const unsigned long long old = atom_add_acq_rel_gpu(cnt, 1ull);
        int ok = 1;
        if (old + 1ull < target) {
            long long spins = 0;
            while (ld_acquire_gpu(cnt) < target) {
                if (*(volatile int*)&sc->error) { ok = 0; break; }
                if (++spins > spin_limit) {
                    set_error(sc, ST_ETIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(32);
            }
        }
        s_ok = ok && !*(volatile int*)&sc->error;
    }
    __syncthreads();
    return s_ok != 0;
}

// Exclusive prefix of a 0/1 flag over the block (in thread order) and the total.
__device__ __forceinline__ int block_exclusive_scan(int flag, int& total) {
    __shared__ int s_w[WARPS];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned bal = __ballot_sync(0xffffffffu, flag);
    int in_warp = __popc(bal & ((1u << lane) - 1u));
    if (lane == 0) s_w[wid] = __popc(bal);
    __syncthreads();
    int before = 0, tot = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        int v = s_w[w];
        if (w < wid) before += v;
        tot += v;
    }
    __syncthreads();
    total = tot;
    return before + in_warp;
}

}  // namespace gbees
