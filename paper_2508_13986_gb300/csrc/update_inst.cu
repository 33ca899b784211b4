// Instantiations of the flux-update kernels and of the persistent step-loop
// kernel for one precision and one family of drift models. The build compiles
// this file once per (GBEES_PREC, GBEES_FAMILY) pair so that the instantiations
// compile in parallel:
//   GBEES_PREC   64 (FP64) or 32 (FP32 storage and fluxes)
//   GBEES_FAMILY 0 Lorenz '63 (both forms), 1 Lorenz '96 (n = 4..6),
//                2 linear n = 1..3, 3 linear n = 4..6, 4 constant n = 1..3,
//                5 constant n = 4..6
#include "gbees_persistent.cuh"

#ifndef GBEES_PREC
#error "GBEES_PREC must be 32 or 64"
#endif
#ifndef GBEES_FAMILY
#error "GBEES_FAMILY must be 0..5"
#endif

namespace gbees {

#if GBEES_PREC == 64
using Real = double;
#else
using Real = float;
#endif

// pre: the kernels before the link phase (grow, halo); post: after it (all
// take (Model, Bufs)).
template <int N, int DYN>
static void kernels_of(Kernels* k) {
    k->persist = (void*)k_persistent<N, DYN, Real>;
    k->batch = (void*)k_batch<N, DYN, Real>;
    k->batch_teams = (void*)k_batch_teams<N, DYN, Real>;
    k->pre[0] = (void*)k_waves_list<N, DYN, Real>;
    k->pre[1] = (void*)k_grow_list<N, Real>;
    k->pre[2] = (void*)k_halo<N, Real, 1>;
    k->npre = 3;
    k->post[0] = (void*)k_faces<N, DYN, Real>;
    k->post[1] = (void*)k_apply<N, Real>;
    k->npost = 2;
}

#define GBEES_JOIN2(a, b) a##b
#define GBEES_JOIN(a, b) GBEES_JOIN2(a, b)
#define GBEES_ENTRY GBEES_JOIN(GBEES_JOIN(update_kernels_p, GBEES_PREC), GBEES_JOIN(_f, GBEES_FAMILY))

// Kernels for dimension n and model dyn of this family; false when not covered.
bool GBEES_ENTRY(int n, int dyn, Kernels* k) {
#if GBEES_FAMILY == 0
    if (n != 3) return false;
    if (dyn == DYN_LORENZ63) { kernels_of<3, DYN_LORENZ63>(k); return true; }
    if (dyn == DYN_LORENZ63_SHIFTED) { kernels_of<3, DYN_LORENZ63_SHIFTED>(k); return true; }
    return false;
#elif GBEES_FAMILY == 1
    switch (n) {
        case 4: kernels_of<4, DYN_LORENZ96>(k); return true;
        case 5: kernels_of<5, DYN_LORENZ96>(k); return true;
        case 6: kernels_of<6, DYN_LORENZ96>(k); return true;
    }
    return false;
#elif GBEES_FAMILY == 2 || GBEES_FAMILY == 4
    constexpr int D = GBEES_FAMILY == 2 ? DYN_LINEAR : DYN_CONSTANT;
    switch (n) {
        case 1: kernels_of<1, D>(k); return true;
        case 2: kernels_of<2, D>(k); return true;
        case 3: kernels_of<3, D>(k); return true;
    }
    return false;
#else
    constexpr int D = GBEES_FAMILY == 3 ? DYN_LINEAR : DYN_CONSTANT;
    switch (n) {
        case 4: kernels_of<4, D>(k); return true;
        case 5: kernels_of<5, D>(k); return true;
        case 6: kernels_of<6, D>(k); return true;
    }
    return false;
#endif
}

}  // namespace gbees
