// step_tma_f64.cu -- FP64 instantiations of the TMA-pipelined step.
#include "step_tma.cuh"

namespace fitgb {

template <>
cudaError_t launch_step_tma<double>(const StepArgs<double> &a, const TmaMaps &maps, Tile t, bool lossy,
                                    bool muarr, bool energy, cudaStream_t s) {
    using namespace tma;
#define FIT_T(TX, TY, S)                                                                    \
    if (t.tx == TX && t.ty == TY)                                                           \
        return lossy ? launch_one<double, TX, TY, S, true>(a, maps, muarr, energy, s)       \
                     : launch_one<double, TX, TY, S, false>(a, maps, muarr, energy, s);
    FIT_T(32, 8, 3)
    FIT_T(32, 4, 4)
#undef FIT_T
    return cudaErrorInvalidValue;
}

}  // namespace fitgb
