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

// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds of
//   (hi0, lo0) = mulhilo(0xD2511F53, x0), (hi1, lo1) = mulhilo(0xCD9E8D57, x2),
//   x = (hi1 ^ x1 ^ k0, lo1, hi0 ^ x3 ^ k1, lo0),
// with the key bumped by (0x9E3779B9, 0xBB67AE85) between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 x, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        const unsigned hi0 = __umulhi(0xD2511F53u, x.x), lo0 = 0xD2511F53u * x.x;
        const unsigned hi1 = __umulhi(0xCD9E8D57u, x.z), lo1 = 0xCD9E8D57u * x.z;
        x = make_uint4(hi1 ^ x.y ^ k.x, lo1, hi0 ^ x.w ^ k.y, lo0);
    }
    return x;
}

// Two standard normals from block `idx` of (seed, stream, counter): 53-bit uniforms
// u1 = (x0, x1), u2 = (x2, x3) in (0, 1), Box-Muller in FP64.
__device__ __forceinline__ double2 philox_normals(unsigned long long seed, unsigned stream, unsigned counter,
                                                  unsigned long long idx) {
    uint4 c = make_uint4((unsigned)(idx & 0xffffffffull), (unsigned)(idx >> 32), stream, counter);
    uint2 k = make_uint2((unsigned)(seed & 0xffffffffull), (unsigned)(seed >> 32));
    uint4 x = philox4x32_10(c, k);
    const double u1 = ((double)(x.x >> 5) * 67108864.0 + (double)(x.y >> 6) + 0.5) * (1.0 / 9007199254740992.0);
    const double u2 = ((double)(x.z >> 5) * 67108864.0 + (double)(x.w >> 6) + 0.5) * (1.0 / 9007199254740992.0);
    const double rad = sqrt(-2.0 * log(u1));
    double s, c2;
    sincospi(2.0 * u2, &s, &c2);
    return make_double2(rad * c2, rad * s);
}

// The same pair from the same 53-bit uniforms, the logarithm, square root, sine and
// cosine in FP32: the noise of an FP32 operator (GB300's FP64 transcendentals run on
// its slow FP64 pipe).  Agrees with philox_normals to FP32 rounding.
__device__ __forceinline__ float2 philox_normals_f(unsigned long long seed, unsigned stream, unsigned counter,
                                                  unsigned long long idx) {
    uint4 c = make_uint4((unsigned)(idx & 0xffffffffull), (unsigned)(idx >> 32), stream, counter);
    uint2 k = make_uint2((unsigned)(seed & 0xffffffffull), (unsigned)(seed >> 32));
    uint4 x = philox4x32_10(c, k);
    const float two_m53 = 1.1102230246251565e-16f;  // 2^-53, exact
    const float u1 = ((float)(x.x >> 5) * 67108864.0f + ((float)(x.y >> 6) + 0.5f)) * two_m53;
    const float u2 = ((float)(x.z >> 5) * 67108864.0f + ((float)(x.w >> 6) + 0.5f)) * two_m53;
    const float rad = sqrtf(-2.0f * logf(u1));
    float s, c2;
    sincospif(2.0f * u2, &s, &c2);
    return make_float2(rad * c2, rad * s);
}

// Visit the sources s != t within r_c of cell-sorted target t over the 9 cells
// around t's cell; f(s, rx, ry, r2) gets the separation x_t - x_s.  Offsets are
// measured from each node's cell corner, so the periodic wrap is the cell shift.
template <typename T, typename F>
__device__ __forceinline__ void for_each_pair(int t, int n_box, T r_c, T rc2, const int* __restrict__ perm,
                                              const int* __restrict__ cell, const int* __restrict__ start,
                                              const typename V2<T>::type* __restrict__ off, F&& f) {
    int c = cell[perm[t]];
    int cx = c % n_box, cy = c / n_box;
    typename V2<T>::type ot = off[t];
    for (int dy = -1; dy <= 1; ++dy) {
        int ny = cy + dy;
        ny += (ny < 0) ? n_box : 0;
        ny -= (ny >= n_box) ? n_box : 0;
        T sy = ot.y - T(dy) * r_c;
        for (int dx = -1; dx <= 1; ++dx) {
            int nx = cx + dx;
            nx += (nx < 0) ? n_box : 0;
            nx -= (nx >= n_box) ? n_box : 0;
            T sx = ot.x - T(dx) * r_c;
            int nc = ny * n_box + nx;
            int lo = start[nc], hi = start[nc + 1];
            for (int s = lo; s < hi; ++s) {
                typename V2<T>::type os = off[s];
                T rx = sx - os.x, ry = sy - os.y;
                T r2 = rx * rx + ry * ry;
                if (r2 < rc2 && s != t) f(s, rx, ry, r2);
            }
        }
    }
}

struct TileGeom {
    int M, TS, n_tile, P, hw;
};

// Tile-kernel launchers, one translation unit per precision (wave_tiles_f32.cu,
// wave_tiles_f64.cu).  Return cudaSuccess or the attribute error.
template <typename T>
cudaError_t tile_set_smem(const TileGeom& tg);
// tile_spread writes every grid point (no zeroing needed); ring: the per-tile halo
// buffer of spread_ring_elems(TS, P, n_tile) elements.  Two launches.
template <typename T>
void tile_spread(cudaStream_t st, const TileGeom& tg, T a, T g0, const int* tstart, const int2* tbase,
                 const void* tfrac, const void* mu_t, T* grid, T* ring);
template <typename T>
void tile_interp(cudaStream_t st, const TileGeom& tg, T a, T g0, const int* tstart, const int2* tbase,
                 const void* tfrac, const T* grid, void* v_t);
// Fused end of the operator for the warp-per-node interpolation: instead of the wave
// part in tile order (v_t), write v[m] = (v_s[slot[m]] + v_band[m]) + wave_m in body
// order, m = tperm[i] -- the sum k_finish forms, in its order; v_s and v_band null: the
// wave part alone.  v null: the tile-order output.
template <typename T>
struct InterpEpilogue {
    double2* v = nullptr;
    const int* tperm = nullptr;
    const int* slot = nullptr;
    const typename V2<T>::type* v_s = nullptr;
    const double2* v_band = nullptr;
};

template <typename T>
__device__ __forceinline__ void interp_store(const InterpEpilogue<T>& ep, typename V2<T>::type* v_t, int i, T sx,
                                             T sy) {
    if (!ep.v) {
        v_t[i].x = sx;
        v_t[i].y = sy;
        return;
    }
    const int m = ep.tperm[i];
    double vx = 0.0, vy = 0.0;
    if (ep.v_s) {
        const typename V2<T>::type w = ep.v_s[ep.slot[m]];
        const double2 b = ep.v_band[m];
        vx = (double)w.x + b.x;
        vy = (double)w.y + b.y;
    }
    ep.v[m] = make_double2(vx + (double)sx, vy + (double)sy);
}

// Warp-per-node variants (grid zeroed by the caller before warp_spread); wtab: the
// node window weights of node_weights, or null (computed per lane).  The spread reads
// its forces as mu_t (tile order), or, when tperm is given, gathers them itself from
// the body-order FP64 forces mu: node i of the tile order is mu[tperm[i]].
template <typename T>
void warp_spread(cudaStream_t st, int N, const TileGeom& tg, T a, T g0, const int2* tbase, const void* tfrac,
                 const T* wtab, const void* mu_t, const double2* mu, const int* tperm, T* grid);
template <typename T>
void warp_interp(cudaStream_t st, int N, const TileGeom& tg, T a, T g0, const int2* tbase, const void* tfrac,
                 const T* wtab, const T* grid, void* v_t, const InterpEpilogue<T>& ep = InterpEpilogue<T>());
// wtab[N][2][P]: every node's column and (times g0) row window weights, and (wdf not
// null) the same as float-float pairs.  One launch.
template <typename T>
void node_weights(cudaStream_t st, int N, const TileGeom& tg, T a, T g0, const void* tfrac, T* wtab,
                  float2* wdf = nullptr);
// Interpolation of the FP64 operator of an FP32 handle in float-float arithmetic: the
// grid holds float-float pairs (wfft_inverse with df_out), the weights come from wdf;
// the warp-per-node layout of warp_interp, its output (tile order or the epilogue) in FP64.
void interp_df(cudaStream_t st, int N, const TileGeom& tg, const int2* tbase, const float2* wdf, const double* grid,
               void* v_t, const InterpEpilogue<double>& ep);

}  // namespace fbim
