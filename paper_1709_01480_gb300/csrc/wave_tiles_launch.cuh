// Host-side launchers of the wave-space tile and warp kernels (wave_tiles.cuh), written
// once over the precision T.  Each of wave_tiles_f32.cu and wave_tiles_f64.cu includes
// this header and defines the specialisations that ewald_types.cuh declares for its own
// T, so the two precisions still compile as separate translation units.
#pragma once
#include <cmath>
#include <cstdint>

#include "wave_tiles.cuh"

namespace fbim {
namespace wt {

// PMAX variants: the window loops unroll to PMAX with runtime P <= PMAX.
#define FBIM_PMAX_CASES(X) X(9) X(13) X(17) X(23)

inline int pmax_for(int P) { return P <= 9 ? 9 : P <= 13 ? 13 : P <= 17 ? 17 : P <= 23 ? 23 : 0; }

// The kernels' dynamic shared-memory limit is a property of the kernel, not of a
// handle: it is raised to the device's opt-in maximum, and this handle's sizes are
// checked against that, so that handles of different sizes never lower it under one
// another's launches.
template <typename T>
cudaError_t set_smem(const TileGeom& tg) {
    int dev = 0, optin = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err == cudaSuccess) err = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (err != cudaSuccess) return err;
    if ((int)spread_smem_bytes<T>(tg.TS, tg.P) > optin || (int)interp_smem_bytes<T>(tg.TS, tg.P) > optin)
        return cudaErrorInvalidValue;
    err = cudaErrorInvalidValue;
    switch (pmax_for(tg.P)) {
#define FBIM_SET(PM)                                                                                    \
    case PM:                                                                                            \
        err = cudaFuncSetAttribute(k_spread_tiles<T, PM>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin); \
        if (err == cudaSuccess)                                                                         \
            err = cudaFuncSetAttribute(k_interp_tiles<T, PM>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin); \
        break;
        FBIM_PMAX_CASES(FBIM_SET)
#undef FBIM_SET
    }
    return err;
}

template <typename T>
void spread_tiles(cudaStream_t st, const TileGeom& tg, T a, T g0, const int* tstart, const int2* tbase,
                  const void* tfrac, const void* mu_t, T* grid, T* ring) {
    using T2 = typename V2<T>::type;
    const dim3 tiles(tg.n_tile, tg.n_tile);
    const size_t ss = spread_smem_bytes<T>(tg.TS, tg.P);
    const T q2 = (T)std::exp(-2.0 * (double)a);
    switch (pmax_for(tg.P)) {
#define FBIM_LAUNCH(PM)                                                                           \
    case PM:                                                                                      \
        k_spread_tiles<T, PM><<<tiles, 256, ss, st>>>(tg, a, q2, g0, tstart, tbase, (const T2*)tfrac, \
                                                      (const T2*)mu_t, grid, ring);               \
        break;
        FBIM_PMAX_CASES(FBIM_LAUNCH)
#undef FBIM_LAUNCH
    }
    k_spread_fold<T><<<tiles, 256, 0, st>>>(tg, ring, grid);
}

template <typename T>
void interp_tiles(cudaStream_t st, const TileGeom& tg, T a, T g0, const int* tstart, const int2* tbase,
                  const void* tfrac, const T* grid, void* v_t) {
    using T2 = typename V2<T>::type;
    const dim3 tiles(tg.n_tile, tg.n_tile);
    const size_t si = interp_smem_bytes<T>(tg.TS, tg.P);
    const T q2 = (T)std::exp(-2.0 * (double)a);
    switch (pmax_for(tg.P)) {
#define FBIM_LAUNCH(PM)                                                                                 \
    case PM:                                                                                            \
        k_interp_tiles<T, PM><<<tiles, 256, si, st>>>(tg, a, q2, g0, tstart, tbase, (const T2*)tfrac, grid, \
                                                      (T2*)v_t);                                        \
        break;
        FBIM_PMAX_CASES(FBIM_LAUNCH)
#undef FBIM_LAUNCH
    }
}

inline int warp_blocks(int N, int P) {
    const long long warps = P <= 16 ? (N + 1) / 2 : N;
    return (int)((warps * 32 + 255) / 256);
}

template <typename T>
void spread_warp(cudaStream_t st, int N, const TileGeom& tg, T a, T g0, const int2* tbase, const void* tfrac,
                 const T* wtab, const void* mu_t, const double2* mu, const int* tperm, T* grid) {
    using T2 = typename V2<T>::type;
    k_spread_warp<T><<<warp_blocks(N, tg.P), 256, 0, st>>>(N, tg.M, tg.P, tg.hw, a, g0, tbase, (const T2*)tfrac,
                                                           (const T2*)mu_t, mu, tperm, wtab, grid);
}

template <typename T>
void interp_warp(cudaStream_t st, int N, const TileGeom& tg, T a, T g0, const int2* tbase, const void* tfrac,
                 const T* wtab, const T* grid, void* v_t, const InterpEpilogue<T>& ep) {
    using T2 = typename V2<T>::type;
    k_interp_warp<T><<<warp_blocks(N, tg.P), 256, 0, st>>>(N, tg.M, tg.P, tg.hw, a, g0, tbase, (const T2*)tfrac,
                                                           wtab, grid, (T2*)v_t, ep);
}

}  // namespace wt
}  // namespace fbim
