// Wave-space tile kernels instantiated for double.
#include <cmath>

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
cudaError_t tile_set_smem<double>(const TileGeom& tg) {
    int dev = 0, optin = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err == cudaSuccess) err = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (err != cudaSuccess) return err;
    if ((int)spread_smem_bytes<double>(tg.TS, tg.P) > optin || (int)interp_smem_bytes<double>(tg.TS, tg.P) > optin)
        return cudaErrorInvalidValue;
    err = cudaErrorInvalidValue;
    switch (pmax_for(tg.P)) {
#define FBIM_SET(PM)                                                                                        \
    case PM:                                                                                                \
        err = cudaFuncSetAttribute(k_spread_tiles<double, PM>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin); \
        if (err == cudaSuccess)                                                                             \
            err = cudaFuncSetAttribute(k_interp_tiles<double, PM>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin); \
        break;
        FBIM_PMAX_CASES(FBIM_SET)
#undef FBIM_SET
    }
    return err;
}

template <>
void tile_spread<double>(cudaStream_t st, const TileGeom& tg, double a, double g0, const int* tstart, const int2* tbase,
                      const void* tfrac, const void* mu_t, double* grid, double* ring) {
    using T2 = typename V2<double>::type;
    const dim3 tiles(tg.n_tile, tg.n_tile);
    const size_t ss = spread_smem_bytes<double>(tg.TS, tg.P);
    const double q2 = (double)std::exp(-2.0 * (double)a);
    switch (pmax_for(tg.P)) {
#define FBIM_LAUNCH(PM)                                                                                   \
    case PM:                                                                                              \
        k_spread_tiles<double, PM><<<tiles, 256, ss, st>>>(tg, a, q2, g0, tstart, tbase, (const T2*)tfrac,      \
                                                        (const T2*)mu_t, grid, ring);                     \
        break;
        FBIM_PMAX_CASES(FBIM_LAUNCH)
#undef FBIM_LAUNCH
    }
    k_spread_fold<double><<<tiles, 256, 0, st>>>(tg, ring, grid);
}

template <>
void tile_interp<double>(cudaStream_t st, const TileGeom& tg, double a, double g0, const int* tstart, const int2* tbase,
                      const void* tfrac, const double* grid, void* v_t) {
    using T2 = typename V2<double>::type;
    const dim3 tiles(tg.n_tile, tg.n_tile);
    const size_t si = interp_smem_bytes<double>(tg.TS, tg.P);
    const double q2 = (double)std::exp(-2.0 * (double)a);
    switch (pmax_for(tg.P)) {
#define FBIM_LAUNCH(PM)                                                                                   \
    case PM:                                                                                              \
        k_interp_tiles<double, PM><<<tiles, 256, si, st>>>(tg, a, q2, g0, tstart, tbase, (const T2*)tfrac, grid,  \
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

template <>
void warp_spread<double>(cudaStream_t st, int N, const TileGeom& tg, double a, double g0, const int2* tbase,
                      const void* tfrac, const double* wtab, const void* mu_t, const double2* mu, const int* tperm,
                      double* grid) {
    using T2 = typename V2<double>::type;
    k_spread_warp<double><<<warp_blocks(N, tg.P), 256, 0, st>>>(N, tg.M, tg.P, tg.hw, a, g0, tbase, (const T2*)tfrac,
                                                            (const T2*)mu_t, mu, tperm, wtab, grid);
}

template <>
void warp_interp<double>(cudaStream_t st, int N, const TileGeom& tg, double a, double g0, const int2* tbase,
                      const void* tfrac, const double* wtab, const double* grid, void* v_t,
                      const InterpEpilogue<double>& ep) {
    using T2 = typename V2<double>::type;
    k_interp_warp<double><<<warp_blocks(N, tg.P), 256, 0, st>>>(N, tg.M, tg.P, tg.hw, a, g0, tbase, (const T2*)tfrac,
                                                            wtab, grid, (T2*)v_t, ep);
}

template <>
void node_weights<double>(cudaStream_t st, int N, const TileGeom& tg, double a, double g0, const void* tfrac,
                          double* wtab) {
    using T2 = typename V2<double>::type;
    const double q2 = std::exp(-2.0 * a);
    const unsigned nb = (unsigned)((N + 127) / 128);
    switch (pmax_for(tg.P)) {
#define FBIM_LAUNCH(PM)                                                                                       \
    case PM:                                                                                                  \
        k_node_weights<double, PM><<<nb, 128, 0, st>>>(N, tg.P, tg.hw, a, q2, g0, (const T2*)tfrac, wtab);   \
        break;
        FBIM_PMAX_CASES(FBIM_LAUNCH)
#undef FBIM_LAUNCH
    }
}

}  // namespace fbim
