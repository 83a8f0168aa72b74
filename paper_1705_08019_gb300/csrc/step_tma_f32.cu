// step_tma_f32.cu -- FP32 instantiations of the TMA-pipelined step and the
// tensor-map encoder.
#include <cudaTypedefs.h>

#include "step_tma2.cuh"

namespace fitgb {

bool tma_tile_supported(int tx, int ty, int elem_bytes) {
    if (elem_bytes == 8) return tx == 32 && (ty == 4 || ty == 8);
    return (tx == 32 && (ty == 4 || ty == 8 || ty == 16)) || (tx == 64 && ty == 4);
}

bool step_grad_supported(Tile t) {
    if (!t.single) return (t.tx == 64 && t.ty == 4) || (t.tx == 32 && t.ty == 8);
    return (t.tx == 64 && t.ty == 4 && (t.stages == 0 || t.stages == 3)) ||
           (t.tx == 32 && t.ty == 8 && (t.stages == 0 || t.stages == 4));
}

// Tiles of the two-cells-per-thread kernels and their ring depths (the first
// listed for a tile is its default): (64, 4) 3 or 4, (32, 8) 4 or 3,
// (32, 16) 3, (32, 4) 4.
template <>
cudaError_t launch_step_tma<float>(const StepArgs<float> &a, const TmaMaps &maps, Tile t, bool lossy, bool muarr,
                                   bool energy, cudaStream_t s) {
    using namespace tma;
    if (!t.single) {
        if (a.gb || a.gd) {   // the adjoint step with the gradient fused in, or a forward step keeping e^{n+1}-e^n
            if (a.gb && a.gd) return cudaErrorInvalidValue;
            if (t.tx == 64 && t.ty == 4) {
                if (a.gd)
                    return lossy ? launch_two<64, 4, 3, true, kExtraDiff>(a, maps, muarr, energy, s)
                                 : launch_two<64, 4, 3, false, kExtraDiff>(a, maps, muarr, energy, s);
                return lossy ? launch_two<64, 4, 3, true, kExtraGrad>(a, maps, muarr, energy, s)
                             : launch_two<64, 4, 3, false, kExtraGrad>(a, maps, muarr, energy, s);
            }
            if (t.tx == 32 && t.ty == 8) {
                if (a.gd)
                    return lossy ? launch_two<32, 8, 4, true, kExtraDiff>(a, maps, muarr, energy, s)
                                 : launch_two<32, 8, 4, false, kExtraDiff>(a, maps, muarr, energy, s);
                return lossy ? launch_two<32, 8, 4, true, kExtraGrad>(a, maps, muarr, energy, s)
                             : launch_two<32, 8, 4, false, kExtraGrad>(a, maps, muarr, energy, s);
            }
            return cudaErrorInvalidValue;
        }
#define FIT_T2(TX, TY, S)                                                                  \
        if (t.tx == TX && t.ty == TY && (t.stages == 0 || t.stages == S))                  \
            return lossy ? launch_two<TX, TY, S, true>(a, maps, muarr, energy, s)          \
                         : launch_two<TX, TY, S, false>(a, maps, muarr, energy, s);
        FIT_T2(64, 4, 3)
        FIT_T2(64, 4, 4)
        FIT_T2(32, 8, 4)
        FIT_T2(32, 8, 3)
        FIT_T2(32, 16, 3)
        FIT_T2(32, 4, 4)
#undef FIT_T2
        return cudaErrorInvalidValue;
    }
    if (a.gd) return cudaErrorInvalidValue;   // the difference output is a two-cell kernel epilogue
    if (a.gb) {   // the adjoint step with the gradient accumulation fused in
        if (a.ge0 == nullptr) return cudaErrorInvalidValue;
        if (t.tx == 64 && t.ty == 4 && (t.stages == 0 || t.stages == 3))
            return lossy ? launch_one<float, 64, 4, 3, true, true>(a, maps, muarr, energy, s)
                         : launch_one<float, 64, 4, 3, false, true>(a, maps, muarr, energy, s);
        if (t.tx == 32 && t.ty == 8 && (t.stages == 0 || t.stages == 4))
            return lossy ? launch_one<float, 32, 8, 4, true, true>(a, maps, muarr, energy, s)
                         : launch_one<float, 32, 8, 4, false, true>(a, maps, muarr, energy, s);
        return cudaErrorInvalidValue;
    }
    if (t.stages != 0 && !((t.tx == 32 && t.ty == 8) || (t.tx == 64 && t.ty == 4)))
        t.stages = 0;   // a ring depth this tile has no variant for: its default
#define FIT_T(TX, TY, S)                                                                   \
    if (t.tx == TX && t.ty == TY && (t.stages == 0 || t.stages == S))                      \
        return lossy ? launch_one<float, TX, TY, S, true>(a, maps, muarr, energy, s)       \
                     : launch_one<float, TX, TY, S, false>(a, maps, muarr, energy, s);
    FIT_T(32, 8, 4)
    FIT_T(32, 8, 3)
    FIT_T(32, 16, 3)
    FIT_T(32, 4, 4)
    FIT_T(64, 4, 4)
    FIT_T(64, 4, 3)
#undef FIT_T
    return cudaErrorInvalidValue;
}

bool batched_tile_supported(int tx, int ty) {
    return (tx == 32 && (ty == 4 || ty == 8 || ty == 16)) || (tx == 64 && ty == 4);
}

cudaError_t launch_batched_f32(const BatchArgs<float> &b, Tile t, bool lossy, int ctas, cudaStream_t s) {
    using namespace tma;
    if (!t.single) {
#define FIT_T2(TX, TY, S)                                                                         \
        if (t.tx == TX && t.ty == TY && (t.stages == 0 || t.stages == S))                         \
            return lossy ? launch_batched_two<TX, TY, S, true>(b, ctas, s)                        \
                         : launch_batched_two<TX, TY, S, false>(b, ctas, s);
        FIT_T2(32, 8, 4)
        FIT_T2(32, 8, 3)
        FIT_T2(32, 16, 3)
        FIT_T2(32, 4, 4)
        FIT_T2(64, 4, 3)
        FIT_T2(64, 4, 4)
#undef FIT_T2
        return cudaErrorInvalidValue;
    }
    if (t.stages != 0 && !((t.tx == 32 && t.ty == 8) || (t.tx == 64 && t.ty == 4))) t.stages = 0;
#define FIT_T(TX, TY, S)                                                                          \
    if (t.tx == TX && t.ty == TY && (t.stages == 0 || t.stages == S))                             \
        return lossy ? launch_batched_one<float, TX, TY, S, true>(b, ctas, s)                     \
                     : launch_batched_one<float, TX, TY, S, false>(b, ctas, s);
    FIT_T(32, 8, 4)
    FIT_T(32, 8, 3)
    FIT_T(32, 16, 3)
    FIT_T(32, 4, 4)
    FIT_T(64, 4, 4)
    FIT_T(64, 4, 3)
#undef FIT_T
    return cudaErrorInvalidValue;
}

int batched_ctas_per_sm_f32(Tile t, bool lossy) {
    using namespace tma;
    if (!t.single) {
#define FIT_T2(TX, TY, S)                                                                         \
        if (t.tx == TX && t.ty == TY && (t.stages == 0 || t.stages == S))                         \
            return lossy ? batched_two_occupancy<TX, TY, S, true>() : batched_two_occupancy<TX, TY, S, false>();
        FIT_T2(32, 8, 4)
        FIT_T2(32, 8, 3)
        FIT_T2(32, 16, 3)
        FIT_T2(32, 4, 4)
        FIT_T2(64, 4, 3)
        FIT_T2(64, 4, 4)
#undef FIT_T2
        return 1;
    }
    if (t.stages != 0 && !((t.tx == 32 && t.ty == 8) || (t.tx == 64 && t.ty == 4))) t.stages = 0;
#define FIT_T(TX, TY, S)                                                                          \
    if (t.tx == TX && t.ty == TY && (t.stages == 0 || t.stages == S))                             \
        return lossy ? batched_occupancy<float, TX, TY, S, true>() : batched_occupancy<float, TX, TY, S, false>();
    FIT_T(32, 8, 4)
    FIT_T(32, 8, 3)
    FIT_T(32, 16, 3)
    FIT_T(32, 4, 4)
    FIT_T(64, 4, 4)
    FIT_T(64, 4, 3)
#undef FIT_T
    return 1;
}

namespace {
PFN_cuTensorMapEncodeTiled_v12000 encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    }
    return fn;
}
}  // namespace

bool encode_window_map(CUtensorMap *out, int eb, int nx, int ny, int nz, int pitch, const void *ptr, int ncomp,
                       int box_x, int box_y, int box_c) {
    PFN_cuTensorMapEncodeTiled_v12000 fn = encoder();
    if (!fn) return false;
    const CUtensorMapDataType dt = eb == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
    const cuuint64_t row = (cuuint64_t)pitch * eb;
    const cuuint64_t plane = row * ny;
    cuuint64_t dim[4] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz, (cuuint64_t)ncomp};
    cuuint64_t str[3] = {row, plane, plane * nz};
    cuuint32_t box[4] = {(cuuint32_t)box_x, (cuuint32_t)box_y, 1, (cuuint32_t)box_c};
    cuuint32_t ones[4] = {1, 1, 1, 1};
    return fn(out, dt, 4, const_cast<void *>(ptr), dim, str, box, ones, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
}

bool encode_tma_maps(TmaMaps *out, int eb, int nx, int ny, int nz, int pitch, void *state, int nblocks,
                     const void *coef, int ncoef, int tx, int ty, int nstate) {
    PFN_cuTensorMapEncodeTiled_v12000 fn = encoder();
    if (!fn) return false;
    const CUtensorMapDataType dt = eb == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
    const cuuint64_t row = (cuuint64_t)pitch * eb;
    const cuuint64_t plane = row * ny;
    const cuuint64_t comp = plane * nz;
    cuuint64_t sdim[5] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz, (cuuint64_t)nstate, (cuuint64_t)nblocks};
    cuuint64_t sstr[4] = {row, plane, comp, (cuuint64_t)nstate * comp};
    cuuint32_t sbox[5] = {(cuuint32_t)(tx + 8), (cuuint32_t)(ty + 2), 1, 3, 1};
    cuuint32_t ones[5] = {1, 1, 1, 1, 1};
    if (fn(&out->state, dt, 5, state, sdim, sstr, sbox, ones, CU_TENSOR_MAP_INTERLEAVE_NONE,
           CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
        CUDA_SUCCESS)
        return false;
    cuuint64_t cdim[4] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz, (cuuint64_t)ncoef};
    cuuint64_t cstr[3] = {row, plane, comp};
    cuuint32_t cbox[4] = {(cuuint32_t)tx, (cuuint32_t)ty, 1, (cuuint32_t)ncoef};
    if (fn(&out->coef, dt, 4, const_cast<void *>(coef), cdim, cstr, cbox, ones, CU_TENSOR_MAP_INTERLEAVE_NONE,
           CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
        CUDA_SUCCESS)
        return false;
    return true;
}

}  // namespace fitgb
