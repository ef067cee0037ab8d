// Wave-space tile kernels instantiated for double (launchers in wave_tiles_launch.cuh),
// and the per-geometry window weights that only the FP64 operators use.
#include "wave_tiles_launch.cuh"

namespace fbim {

template <>
cudaError_t tile_set_smem<double>(const TileGeom& tg) {
    return wt::set_smem<double>(tg);
}

template <>
void tile_spread<double>(cudaStream_t st, const TileGeom& tg, double a, double g0, const int* tstart,
                         const int2* tbase, const void* tfrac, const void* mu_t, double* grid, double* ring) {
    wt::spread_tiles<double>(st, tg, a, g0, tstart, tbase, tfrac, mu_t, grid, ring);
}

template <>
void tile_interp<double>(cudaStream_t st, const TileGeom& tg, double a, double g0, const int* tstart,
                         const int2* tbase, const void* tfrac, const double* grid, void* v_t) {
    wt::interp_tiles<double>(st, tg, a, g0, tstart, tbase, tfrac, grid, v_t);
}

template <>
void warp_spread<double>(cudaStream_t st, int N, const TileGeom& tg, double a, double g0, const int2* tbase,
                         const void* tfrac, const double* wtab, const void* mu_t, const double2* mu,
                         const int* tperm, double* grid) {
    wt::spread_warp<double>(st, N, tg, a, g0, tbase, tfrac, wtab, mu_t, mu, tperm, grid);
}

template <>
void warp_interp<double>(cudaStream_t st, int N, const TileGeom& tg, double a, double g0, const int2* tbase,
                         const void* tfrac, const double* wtab, const double* grid, void* v_t,
                         const InterpEpilogue<double>& ep) {
    wt::interp_warp<double>(st, N, tg, a, g0, tbase, tfrac, wtab, grid, v_t, ep);
}

template <>
void node_weights<double>(cudaStream_t st, int N, const TileGeom& tg, double a, double g0, const void* tfrac,
                          double* wtab) {
    using T2 = typename V2<double>::type;
    const double q2 = std::exp(-2.0 * a);
    const unsigned nb = (unsigned)((N + 127) / 128);
    switch (wt::pmax_for(tg.P)) {
#define FBIM_LAUNCH(PM)                                                                                   \
    case PM:                                                                                              \
        k_node_weights<double, PM><<<nb, 128, 0, st>>>(N, tg.P, tg.hw, a, q2, g0, (const T2*)tfrac, wtab); \
        break;
        FBIM_PMAX_CASES(FBIM_LAUNCH)
#undef FBIM_LAUNCH
    }
}

}  // namespace fbim
