// Wave-space tile kernels instantiated for double (launchers in wave_tiles_launch.cuh),
// and the per-geometry window weights that only the FP64 operators use.
#include "dfloat.cuh"
#include "wave_tiles_launch.cuh"

namespace fbim {

namespace {

using dfl::df;

__device__ __forceinline__ df shfl_df(df v, int src) {
    return {__shfl_sync(0xffffffffu, v.hi, src), __shfl_sync(0xffffffffu, v.lo, src)};
}
__device__ __forceinline__ df shfl_xor_df(df v, int o, int width) {
    return {__shfl_xor_sync(0xffffffffu, v.hi, o, width), __shfl_xor_sync(0xffffffffu, v.lo, o, width)};
}

// The warp-per-node interpolation (k_interp_warp's layout: lane p = window column p,
// rows in turn, the row weight from lane q by shuffle) with float-float grid values
// and weights: products and sums in float-float on the FP32 pipes instead of two FP64
// FMAs per window point, the node's sum rounded to FP64 once.
__global__ void __launch_bounds__(256) k_interp_df(int N, int M, int P, int hw, const int2* __restrict__ tbase,
                                                   const float2* __restrict__ wdf, const float2* __restrict__ grid,
                                                   double2* __restrict__ v_t, InterpEpilogue<double> ep) {
    const int lane = threadIdx.x & 31;
    const int w = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    const bool two = P <= 16;
    const int sub = two ? (lane >> 4) : 0, p = two ? (lane & 15) : lane;
    const int i = w * (two ? 2 : 1) + sub;
    if (w * (two ? 2 : 1) >= N) return;  // warp-uniform
    const bool active = i < N && p < P;
    int2 b = make_int2(0, 0);
    df wx = {0.f, 0.f}, wy = {0.f, 0.f};
    if (active) {
        b = tbase[i];
        const float2 a = wdf[(size_t)i * 2 * P + p], c = wdf[(size_t)i * 2 * P + P + p];
        wx = {a.x, a.y};
        wy = {c.x, c.y};
    }
    int gx = b.x - hw + p;
    gx += (gx < 0) ? M : 0;
    gx -= (gx >= M) ? M : 0;
    int gy = b.y - hw;
    gy += (gy < 0) ? M : 0;
    const size_t MM = (size_t)M * M;
    const int src = two ? (sub << 4) : 0;
    df sx = {0.f, 0.f}, sy = {0.f, 0.f};
    for (int q = 0; q < P; ++q) {
        const df wq = shfl_df(wy, src + q);
        if (active) {
            const size_t g = (size_t)gy * M + gx;
            const float2 ux = __ldg(grid + g), uy = __ldg(grid + MM + g);
            sx = dfl::add_fast(sx, dfl::mul(wq, df{ux.x, ux.y}));
            sy = dfl::add_fast(sy, dfl::mul(wq, df{uy.x, uy.y}));
        }
        gy = (gy + 1 == M) ? 0 : gy + 1;
    }
    sx = dfl::mul(sx, wx);
    sy = dfl::mul(sy, wx);
    const int width = two ? 16 : 32;
    for (int o = width / 2; o > 0; o >>= 1) {
        sx = dfl::add(sx, shfl_xor_df(sx, o, width));
        sy = dfl::add(sy, shfl_xor_df(sy, o, width));
    }
    if (p == 0 && i < N) interp_store<double>(ep, v_t, i, dfl::to_double(sx), dfl::to_double(sy));
}

}  // namespace

void interp_df(cudaStream_t st, int N, const TileGeom& tg, const int2* tbase, const float2* wdf, const double* grid,
               void* v_t, const InterpEpilogue<double>& ep) {
    k_interp_df<<<wt::warp_blocks(N, tg.P), 256, 0, st>>>(N, tg.M, tg.P, tg.hw, tbase, wdf,
                                                         reinterpret_cast<const float2*>(grid), (double2*)v_t, ep);
}

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
                          double* wtab, float2* wdf) {
    using T2 = typename V2<double>::type;
    const double q2 = std::exp(-2.0 * a);
    const unsigned nb = (unsigned)((N + 127) / 128);
    switch (wt::pmax_for(tg.P)) {
#define FBIM_LAUNCH(PM)                                                                                   \
    case PM:                                                                                              \
        k_node_weights<double, PM><<<nb, 128, 0, st>>>(N, tg.P, tg.hw, a, q2, g0, (const T2*)tfrac, wtab, wdf); \
        break;
        FBIM_PMAX_CASES(FBIM_LAUNCH)
#undef FBIM_LAUNCH
    }
}

}  // namespace fbim
