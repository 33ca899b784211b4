// The flux update of one GBEES step: donor-cell upwind fluxes (Eq. 7), the
// corner-transport corrections of Algorithm 1 and the limited high-resolution
// correction, applied to every active cell in gather form, with the
// normalisation sum and maximum reduced in the epilogue and the step
// bookkeeping (time, dt of Eq. 8, buffers, prune schedule) done by the last
// block.
//
// Gather form of Algorithm 1. The corrections that Algorithm 1 scatters onto
// face (X, j) from the waves of the neighbouring faces add up to
//     -u_j(X) * sum_{d != j} dt/(2 h_d) * G_d(Y),
// where Y is the cell upwind of the face (X - e_j when u_j(X) > 0, X when
// u_j(X) < 0) and
//     G_d(Y) = max(u_d(Y), 0) (P_Y - P_{Y-e_d}) + min(u_d(Y+e_d), 0) (P_{Y+e_d} - P_Y)
// collects the d-direction waves entering Y (u_d(Y) is the velocity at the
// lower d-face of Y). Each cell therefore needs its face neighbours, the
// transverse neighbours of the upwind neighbour of each face (edge cells), and
// one cell two steps away per dimension for the limiter.
#pragma once

#include "gbees_device.cuh"

namespace gbees {

template <typename T>
struct CtuConsts {
    T h[MAXN];
    T dth[MAXN];  // dt / h_j
    T ch[MAXN];   // dt / (2 h_j)
};

template <int N, int DYN, typename T>
__device__ __forceinline__ T vel_at(const Model& m, const T* xc, const T* h, int js, int s, int d, int face) {
    T y[N];
#pragma unroll
    for (int k = 0; k < N; ++k) y[k] = xc[k];
    if (js >= 0) y[js] += (T)s * h[js];
    y[d] += (T)face * (T)0.5 * h[d];
    return drift<T, N>(m, DYN, y, d);
}

template <typename T>
__device__ __forceinline__ T limited_wave(int lim, T W, T Wup) {
    if (lim == LIM_LW) return W;
    // MC limiter phi(theta) = max(0, min((1+theta)/2, 2, 2 theta)) with theta = Wup / W,
    // multiplied by W and written without the division.
    if ((W > (T)0 && Wup > (T)0) || (W < (T)0 && Wup < (T)0)) {
        T aW = fabs(W), aU = fabs(Wup);
        T v = fmin(fmin((T)0.5 * (aW + aU), (T)2 * aW), (T)2 * aU);
        return W > (T)0 ? v : -v;
    }
    return (T)0;
}

template <int N, typename T>
__device__ __forceinline__ T q_or_zero(const T* __restrict__ Q, int i) {
    return i >= 0 ? Q[i] : (T)0;
}

template <int N, int DYN, typename T>
__global__ void __launch_bounds__(THREADS) k_ctu(const Model m, Bufs b) {
    DevScalars* sc = b.sc;
    if (*(volatile int*)&sc->done | *(volatile int*)&sc->error) return;
    const long long ncell = min(*(volatile long long*)&sc->N, m.cap);
    const int pb = *(volatile int*)&sc->pbuf, g = *(volatile int*)&sc->gen;
    const T* __restrict__ Q = static_cast<const T*>(b.q[pb]);
    T* __restrict__ Qn = static_cast<T*>(b.q[pb ^ 1]);
    const unsigned long long* __restrict__ key = b.key[g];
    const int* __restrict__ link = b.link[g];
    const long long cap = m.cap;
    const int lim = m.limiter;

    // Eq. 8: dt = CFL / max rate, clipped to land on the target time.
    const double rate = __longlong_as_double((long long)*(volatile unsigned long long*)&sc->maxrate_bits);
    const double t = *(volatile double*)&sc->t, tt = *(volatile double*)&sc->t_target;
    double dt = rate > 0.0 ? __ddiv_rn(m.cfl, rate) : (double)INFINITY;
    const double rem = __dsub_rn(tt, t);
    const bool last = dt >= rem;
    if (last) dt = rem;
    const T scale = (T)*(volatile double*)&sc->scale;
    CtuConsts<T> K;
#pragma unroll
    for (int j = 0; j < N; ++j) {
        K.h[j] = (T)m.h[j];
        K.dth[j] = (T)(dt / m.h[j]);
        K.ch[j] = (T)(dt / (2.0 * m.h[j]));
    }

    long long dacc[NDIG] = {0, 0, 0, 0, 0, 0};
    double mx = -INFINITY;
    int err = 0;
    long long fallback = 0;

    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell;
         c += (long long)gridDim.x * blockDim.x) {
        int I[N];
        unpack_key<N>(m, key[c], I);
        int L[2 * N];
#pragma unroll
        for (int d = 0; d < 2 * N; ++d) L[d] = link[(long long)d * cap + c];
        const T P0 = Q[c];
        T Pn[2 * N];
#pragma unroll
        for (int d = 0; d < 2 * N; ++d) Pn[d] = q_or_zero<N, T>(Q, L[d]);
        T xc[N];
#pragma unroll
        for (int k = 0; k < N; ++k) xc[k] = (T)m.x0[k] + (T)I[k] * K.h[k];
        T ulo[N], uhi[N];
#pragma unroll
        for (int j = 0; j < N; ++j) {
            ulo[j] = vel_at<N, DYN, T>(m, xc, K.h, -1, 0, j, -1);
            uhi[j] = vel_at<N, DYN, T>(m, xc, K.h, -1, 0, j, +1);
        }
        // d-direction waves entering c itself
        T Gc[N];
#pragma unroll
        for (int d = 0; d < N; ++d)
            Gc[d] = fmax(ulo[d], (T)0) * (P0 - Pn[2 * d]) + fmin(uhi[d], (T)0) * (Pn[2 * d + 1] - P0);

        // index of c + s e_j + t e_d, through the links or the hashtable
        auto edge = [&](int j, int sj, int d, int sd) -> int {
            int e = -2;
            const int a = L[2 * j + sj];
            if (a >= 0) {
                e = __ldg(link + (long long)(2 * d + sd) * cap + a);
            } else {
                const int bb = L[2 * d + sd];
                if (bb >= 0) e = __ldg(link + (long long)(2 * j + sj) * cap + bb);
            }
            if (e == -2) {
                int J[N];
#pragma unroll
                for (int k = 0; k < N; ++k) J[k] = I[k];
                J[j] += sj ? 1 : -1;
                J[d] += sd ? 1 : -1;
                unsigned long long kk;
                e = pack_key<N>(m, J, kk) ? table_find(m, b.table, kk) : -1;
                ++fallback;
            }
            return e;
        };
        // index of c + 2 s e_j
        auto second = [&](int j, int sj) -> int {
            const int a = L[2 * j + sj];
            if (a >= 0) return __ldg(link + (long long)(2 * j + sj) * cap + a);
            int J[N];
#pragma unroll
            for (int k = 0; k < N; ++k) J[k] = I[k];
            J[j] += sj ? 2 : -2;
            unsigned long long kk;
            ++fallback;
            return pack_key<N>(m, J, kk) ? table_find(m, b.table, kk) : -1;
        };
        // sum_{d != j} dt/(2 h_d) G_d(c + s e_j)
        auto trans_nb = [&](int j, int sj) -> T {
            const T PY = Pn[2 * j + sj];
            const int sgn = sj ? 1 : -1;
            T S = (T)0;
#pragma unroll
            for (int d = 0; d < N; ++d) {
                if (d == j) continue;
                const T Pm = q_or_zero<N, T>(Q, edge(j, sj, d, 0));
                const T Pp = q_or_zero<N, T>(Q, edge(j, sj, d, 1));
                const T ul = vel_at<N, DYN, T>(m, xc, K.h, j, sgn, d, -1);
                const T uh = vel_at<N, DYN, T>(m, xc, K.h, j, sgn, d, +1);
                S += K.ch[d] * (fmax(ul, (T)0) * (PY - Pm) + fmin(uh, (T)0) * (Pp - PY));
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
                            if (d != j) S += K.ch[d] * Gc[d];
                    } else {
                        S = trans_nb(j, side);  // upwind cell c - e_j (lower face) or c + e_j (upper face)
                    }
                    f -= u * S;  // Algorithm 1
                    const T W = PR - PL;
                    if (lim != LIM_NONE && W != (T)0) {
                        T Wup;
                        if (u > (T)0) Wup = side ? (P0 - Pn[2 * j]) : (Pn[2 * j] - q_or_zero<N, T>(Q, second(j, 0)));
                        else Wup = side ? (q_or_zero<N, T>(Q, second(j, 1)) - Pn[2 * j + 1]) : (Pn[2 * j + 1] - P0);
                        const T au = fabs(u);
                        f += (T)0.5 * au * ((T)1 - K.dth[j] * au) * limited_wave<T>(lim, W, Wup);
                    }
                }
                F[side] = f;
            }
            upd += K.dth[j] * (F[1] - F[0]);
        }
        const T qn = (P0 - upd) * scale;
        Qn[c] = qn;
        acc_add(dacc, (double)qn, err);
        mx = fmax(mx, (double)qn);
    }
    if (err) set_error(sc, ST_EDEGENERATE);
    block_reduce_acc_max(dacc, mx, sc->acc, &sc->maxq_ord);
    {
        __shared__ long long s_fb;
        if (threadIdx.x == 0) s_fb = 0;
        __syncthreads();
        if (fallback) atomicAdd((unsigned long long*)&s_fb, (unsigned long long)fallback);
        __syncthreads();
        if (threadIdx.x == 0 && s_fb) atomicAdd((unsigned long long*)&sc->lookups_fallback, (unsigned long long)s_fb);
    }
    if (last_block(sc) && threadIdx.x == 0) {
        sc->dt = dt;
        sc->t = last ? tt : __dadd_rn(t, dt);
        sc->step += 1;
        sc->steps_call += 1;
        sc->updates_call += ncell;
        sc->done = last;
        sc->pbuf = pb ^ 1;
        sc->prune_now = (m.prune_interval > 0 && (sc->step % m.prune_interval) == 0);
        finalise_norm(m, sc, 0);
    }
}

}  // namespace gbees
