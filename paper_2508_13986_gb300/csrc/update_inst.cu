// Instantiations of the flux-update kernels and of the persistent step-loop
// kernel for one precision and one family of drift models. The build compiles
// this file once per (GBEES_PREC, GBEES_FAMILY) pair so that the instantiations
// compile in parallel:
//   GBEES_PREC   64 (three-pass FP64 update) or 32 (single-pass gather, FP32)
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

template <int N, int DYN>
static int kernels_of(void** f, void** persist) {
    *persist = (void*)k_persistent<N, DYN, Real>;
#if GBEES_PREC == 64
    f[0] = (void*)k_waves<N, DYN>;
    f[1] = (void*)k_faces<N, DYN>;
    f[2] = (void*)k_apply<N>;
    return 3;
#else
    f[0] = (void*)k_ctu<N, DYN, Real>;
    return 1;
#endif
}

#define GBEES_JOIN2(a, b) a##b
#define GBEES_JOIN(a, b) GBEES_JOIN2(a, b)
#define GBEES_ENTRY GBEES_JOIN(GBEES_JOIN(update_kernels_p, GBEES_PREC), GBEES_JOIN(_f, GBEES_FAMILY))

// Kernels for dimension n and model dyn of this family; 0 when not covered.
int GBEES_ENTRY(int n, int dyn, void** f, void** persist) {
#if GBEES_FAMILY == 0
    if (n != 3) return 0;
    if (dyn == DYN_LORENZ63) return kernels_of<3, DYN_LORENZ63>(f, persist);
    if (dyn == DYN_LORENZ63_SHIFTED) return kernels_of<3, DYN_LORENZ63_SHIFTED>(f, persist);
    return 0;
#elif GBEES_FAMILY == 1
    switch (n) {
        case 4: return kernels_of<4, DYN_LORENZ96>(f, persist);
        case 5: return kernels_of<5, DYN_LORENZ96>(f, persist);
        case 6: return kernels_of<6, DYN_LORENZ96>(f, persist);
    }
    return 0;
#elif GBEES_FAMILY == 2 || GBEES_FAMILY == 4
    constexpr int D = GBEES_FAMILY == 2 ? DYN_LINEAR : DYN_CONSTANT;
    switch (n) {
        case 1: return kernels_of<1, D>(f, persist);
        case 2: return kernels_of<2, D>(f, persist);
        case 3: return kernels_of<3, D>(f, persist);
    }
    return 0;
#else
    constexpr int D = GBEES_FAMILY == 3 ? DYN_LINEAR : DYN_CONSTANT;
    switch (n) {
        case 4: return kernels_of<4, D>(f, persist);
        case 5: return kernels_of<5, D>(f, persist);
        case 6: return kernels_of<6, D>(f, persist);
    }
    return 0;
#endif
}

}  // namespace gbees
