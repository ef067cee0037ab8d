// Small device types and helpers shared by the Ewald operator translation units.
#pragma once
#include <cufft.h>
#include "fbim_internal.h"

namespace fbim {

template <typename T> struct V2;
template <> struct V2<double> { using type = double2; };
template <> struct V2<float> { using type = float2; };

template <typename T> struct Cplx;
template <> struct Cplx<double> { using type = cufftDoubleComplex; };
template <> struct Cplx<float> { using type = cufftComplex; };

__device__ __forceinline__ double dev_exp(double a) { return exp(a); }
__device__ __forceinline__ float dev_exp(float a) { return __expf(a); }
__device__ __forceinline__ double dev_log(double a) { return log(a); }
__device__ __forceinline__ float dev_log(float a) { return __logf(a); }
__device__ __forceinline__ double dev_div(double a, double b) { return a / b; }
__device__ __forceinline__ float dev_div(float a, float b) { return __fdividef(a, b); }

// E1(z)/2 - e^{-z} = S(z) - ln(z)/2 with S a Chebyshev series on [0, zmax] (Clenshaw).
template <typename T>
__device__ __forceinline__ T kernel_a(const ChebE1<T>& ce, T z) {
    T t = z * ce.scale - T(1);
    T t2 = t + t;
    T b1 = 0, b2 = 0;
    for (int k = ce.deg; k >= 1; --k) {
        T b0 = fma(t2, b1, ce.c[k] - b2);
        b2 = b1;
        b1 = b0;
    }
    T S = fma(t, b1, ce.c[0] - b2);
    return S - T(0.5) * dev_log(z);
}

struct TileGeom {
    int M, TS, n_tile, P, hw;
};

// Tile-kernel launchers, one translation unit per precision (wave_tiles_f32.cu,
// wave_tiles_f64.cu).  Return cudaSuccess or the attribute error.
template <typename T>
cudaError_t tile_set_smem(const TileGeom& tg);
template <typename T>
void tile_spread(cudaStream_t st, const TileGeom& tg, T a, T g0, const int* tstart, const int2* tbase,
                 const void* tfrac, const void* mu_t, T* grid);
template <typename T>
void tile_interp(cudaStream_t st, const TileGeom& tg, T a, T g0, const int* tstart, const int2* tbase,
                 const void* tfrac, const T* grid, void* v_t);
// Warp-per-node variants (grid zeroed by the caller before warp_spread).
template <typename T>
void warp_spread(cudaStream_t st, int N, const TileGeom& tg, T a, T g0, const int2* tbase, const void* tfrac,
                 const void* mu_t, T* grid);
template <typename T>
void warp_interp(cudaStream_t st, int N, const TileGeom& tg, T a, T g0, const int2* tbase, const void* tfrac,
                 const T* grid, void* v_t);

}  // namespace fbim
