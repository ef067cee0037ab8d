// Wave-space tile kernels instantiated for float.
#include <cmath>
#include <cstdint>

#include "wave_tiles.cuh"

namespace fbim {

// PMAX variants: the window loops unroll to PMAX with runtime P <= PMAX.
#define FBIM_PMAX_CASES(X) X(9) X(13) X(17) X(23)

static int pmax_for(int P) { return P <= 9 ? 9 : P <= 13 ? 13 : P <= 17 ? 17 : P <= 23 ? 23 : 0; }

// The kernels' dynamic shared-memory limit is a property of the kernel, not of a
// handle: it is raised to the device's opt-in maximum, and this handle's sizes are
// checked against that, so that handles of different sizes never lower it under one
// another's launches.
template <>
cudaError_t tile_set_smem<float>(const TileGeom& tg) {
    int dev = 0, optin = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err == cudaSuccess) err = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (err != cudaSuccess) return err;
    if ((int)spread_smem_bytes<float>(tg.TS, tg.P) > optin || (int)interp_smem_bytes<float>(tg.TS, tg.P) > optin)
        return cudaErrorInvalidValue;
    err = cudaErrorInvalidValue;
    switch (pmax_for(tg.P)) {
#define FBIM_SET(PM)                                                                                        \
    case PM:                                                                                                \
        err = cudaFuncSetAttribute(k_spread_tiles<float, PM>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin); \
        if (err == cudaSuccess)                                                                             \
            err = cudaFuncSetAttribute(k_interp_tiles<float, PM>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin); \
        break;
        FBIM_PMAX_CASES(FBIM_SET)
#undef FBIM_SET
    }
    return err;
}

template <>
void tile_spread<float>(cudaStream_t st, const TileGeom& tg, float a, float g0, const int* tstart, const int2* tbase,
                      const void* tfrac, const void* mu_t, float* grid, float* ring) {
    using T2 = typename V2<float>::type;
    const dim3 tiles(tg.n_tile, tg.n_tile);
    const size_t ss = spread_smem_bytes<float>(tg.TS, tg.P);
    const float q2 = (float)std::exp(-2.0 * (double)a);
    switch (pmax_for(tg.P)) {
#define FBIM_LAUNCH(PM)                                                                                   \
    case PM:                                                                                              \
        k_spread_tiles<float, PM><<<tiles, 256, ss, st>>>(tg, a, q2, g0, tstart, tbase, (const T2*)tfrac,      \
                                                        (const T2*)mu_t, grid, ring);                     \
        break;
        FBIM_PMAX_CASES(FBIM_LAUNCH)
#undef FBIM_LAUNCH
    }
    k_spread_fold<float><<<tiles, 256, 0, st>>>(tg, ring, grid);
}

template <>
void tile_interp<float>(cudaStream_t st, const TileGeom& tg, float a, float g0, const int* tstart, const int2* tbase,
                      const void* tfrac, const float* grid, void* v_t) {
    using T2 = typename V2<float>::type;
    const dim3 tiles(tg.n_tile, tg.n_tile);
    const size_t si = interp_smem_bytes<float>(tg.TS, tg.P);
    const float q2 = (float)std::exp(-2.0 * (double)a);
    switch (pmax_for(tg.P)) {
#define FBIM_LAUNCH(PM)                                                                                   \
    case PM:                                                                                              \
        k_interp_tiles<float, PM><<<tiles, 256, si, st>>>(tg, a, q2, g0, tstart, tbase, (const T2*)tfrac, grid,  \
                                                        (T2*)v_t);                                        \
        break;
        FBIM_PMAX_CASES(FBIM_LAUNCH)
#undef FBIM_LAUNCH
    }
}

static int warp_blocks(int N, int P) {
    const long long warps = P <= 16 ? (N + 1) / 2 : N;
    return (int)((warps * 32 + 255) / 256);
}

// The float4 interpolation needs M % 4 == 0 (16-byte aligned chunks that never
// wrap), a 16-byte aligned grid and P <= 13 (4 chunks of 4 columns cover the window).
static bool vec_ok(const TileGeom& tg, const void* grid) {
    return tg.P <= 13 && tg.M % 4 == 0 && (reinterpret_cast<uintptr_t>(grid) & 15) == 0;
}

template <>
void warp_spread<float>(cudaStream_t st, int N, const TileGeom& tg, float a, float g0, const int2* tbase,
                      const void* tfrac, const float* wtab, const void* mu_t, const double2* mu, const int* tperm,
                      float* grid) {
    using T2 = typename V2<float>::type;
    k_spread_warp<float><<<warp_blocks(N, tg.P), 256, 0, st>>>(N, tg.M, tg.P, tg.hw, a, g0, tbase, (const T2*)tfrac,
                                                            (const T2*)mu_t, mu, tperm, wtab, grid);
}

template <>
void warp_interp<float>(cudaStream_t st, int N, const TileGeom& tg, float a, float g0, const int2* tbase,
                      const void* tfrac, const float* wtab, const float* grid, void* v_t,
                      const InterpEpilogue<float>& ep) {
    using T2 = typename V2<float>::type;
    if (!wtab && vec_ok(tg, grid)) {
        const float q2 = (float)std::exp(-2.0 * (double)a);
        k_interp_vec<<<(unsigned)(((size_t)N * 4 + 255) / 256), 256, 0, st>>>(N, tg.M, tg.P, tg.hw, a, q2, g0, tbase,
                                                                            (const float2*)tfrac, grid, (float2*)v_t, ep);
        return;
    }
    k_interp_warp<float><<<warp_blocks(N, tg.P), 256, 0, st>>>(N, tg.M, tg.P, tg.hw, a, g0, tbase, (const T2*)tfrac,
                                                            wtab, grid, (T2*)v_t, ep);
}

}  // namespace fbim
