// FP32 instantiations of the flux-update kernel.
#include "gbees_ctu.cuh"

namespace gbees {

cudaError_t launch_ctu_f32(const Model& m, const Bufs& b, int grid, cudaStream_t s) {
    switch (m.dyn) {
        case DYN_LORENZ63:
            k_ctu<3, DYN_LORENZ63, float><<<grid, THREADS, 0, s>>>(m, b);
            break;
        case DYN_LORENZ63_SHIFTED:
            k_ctu<3, DYN_LORENZ63_SHIFTED, float><<<grid, THREADS, 0, s>>>(m, b);
            break;
        case DYN_LORENZ96:
            if (m.n == 4) k_ctu<4, DYN_LORENZ96, float><<<grid, THREADS, 0, s>>>(m, b);
            else if (m.n == 5) k_ctu<5, DYN_LORENZ96, float><<<grid, THREADS, 0, s>>>(m, b);
            else k_ctu<6, DYN_LORENZ96, float><<<grid, THREADS, 0, s>>>(m, b);
            break;
        case DYN_LINEAR:
            switch (m.n) {
                case 1: k_ctu<1, DYN_LINEAR, float><<<grid, THREADS, 0, s>>>(m, b); break;
                case 2: k_ctu<2, DYN_LINEAR, float><<<grid, THREADS, 0, s>>>(m, b); break;
                case 3: k_ctu<3, DYN_LINEAR, float><<<grid, THREADS, 0, s>>>(m, b); break;
                case 4: k_ctu<4, DYN_LINEAR, float><<<grid, THREADS, 0, s>>>(m, b); break;
                case 5: k_ctu<5, DYN_LINEAR, float><<<grid, THREADS, 0, s>>>(m, b); break;
                default: k_ctu<6, DYN_LINEAR, float><<<grid, THREADS, 0, s>>>(m, b); break;
            }
            break;
        default:
            switch (m.n) {
                case 1: k_ctu<1, DYN_CONSTANT, float><<<grid, THREADS, 0, s>>>(m, b); break;
                case 2: k_ctu<2, DYN_CONSTANT, float><<<grid, THREADS, 0, s>>>(m, b); break;
                case 3: k_ctu<3, DYN_CONSTANT, float><<<grid, THREADS, 0, s>>>(m, b); break;
                case 4: k_ctu<4, DYN_CONSTANT, float><<<grid, THREADS, 0, s>>>(m, b); break;
                case 5: k_ctu<5, DYN_CONSTANT, float><<<grid, THREADS, 0, s>>>(m, b); break;
                default: k_ctu<6, DYN_CONSTANT, float><<<grid, THREADS, 0, s>>>(m, b); break;
            }
            break;
    }
    return cudaGetLastError();
}

}  // namespace gbees
