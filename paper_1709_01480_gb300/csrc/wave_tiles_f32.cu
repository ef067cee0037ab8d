// Wave-space tile kernels instantiated for float (launchers in wave_tiles_launch.cuh),
// and the float4 interpolation that only the FP32 operator has.
#include "wave_tiles_launch.cuh"

namespace fbim {

template <>
cudaError_t tile_set_smem<float>(const TileGeom& tg) {
    return wt::set_smem<float>(tg);
}

template <>
void tile_spread<float>(cudaStream_t st, const TileGeom& tg, float a, float g0, const int* tstart, const int2* tbase,
                        const void* tfrac, const void* mu_t, float* grid, float* ring) {
    wt::spread_tiles<float>(st, tg, a, g0, tstart, tbase, tfrac, mu_t, grid, ring);
}

template <>
void tile_interp<float>(cudaStream_t st, const TileGeom& tg, float a, float g0, const int* tstart, const int2* tbase,
                        const void* tfrac, const float* grid, void* v_t) {
    wt::interp_tiles<float>(st, tg, a, g0, tstart, tbase, tfrac, grid, v_t);
}

template <>
void warp_spread<float>(cudaStream_t st, int N, const TileGeom& tg, float a, float g0, const int2* tbase,
                        const void* tfrac, const float* wtab, const void* mu_t, const double2* mu, const int* tperm,
                        float* grid) {
    wt::spread_warp<float>(st, N, tg, a, g0, tbase, tfrac, wtab, mu_t, mu, tperm, grid);
}

// The float4 interpolation needs M % 4 == 0 (16-byte aligned chunks that never
// wrap), a 16-byte aligned grid and P <= 13 (4 chunks of 4 columns cover the window).
static bool vec_ok(const TileGeom& tg, const void* grid) {
    return tg.P <= 13 && tg.M % 4 == 0 && (reinterpret_cast<uintptr_t>(grid) & 15) == 0;
}

template <>
void warp_interp<float>(cudaStream_t st, int N, const TileGeom& tg, float a, float g0, const int2* tbase,
                        const void* tfrac, const float* wtab, const float* grid, void* v_t,
                        const InterpEpilogue<float>& ep) {
    if (!wtab && vec_ok(tg, grid)) {
        const float q2 = (float)std::exp(-2.0 * (double)a);
        k_interp_vec<<<(unsigned)(((size_t)N * 4 + 255) / 256), 256, 0, st>>>(N, tg.M, tg.P, tg.hw, a, q2, g0, tbase,
                                                                            (const float2*)tfrac, grid, (float2*)v_t, ep);
        return;
    }
    wt::interp_warp<float>(st, N, tg, a, g0, tbase, tfrac, wtab, grid, v_t, ep);
}

}  // namespace fbim
