// Real-space pair list and its product (Sec. 3.2, Eq. Mreal-decompose: the sum over
// node pairs within r_c).  The list is sliced ELL over list positions: the cell-sorted
// target rows are sorted by length within windows of 256 (row_of / pos_of), slices of
// 32 positions, entries [slice][k][32] of the 2x2 kernel value (xx, xy, yy) and the
// source slot.  Its own header so that the measured DRAM traffic of the product can be
// tied to this source.
#pragma once
#include "fbim_internal.h"
#include "ewald_types.cuh"

namespace fbim {

template <typename T> struct PairEntry;
template <> struct __align__(16) PairEntry<float> { float xx, xy, yy; int src; };
template <> struct __align__(16) PairEntry<double> { double xx, xy, yy; long long src; };
// An FP64-list entry of an FP32 handle in float-float form: the leading parts and the
// source in the first 16 bytes, the trailing parts in the second.
struct __align__(16) PairEntryDF { float xx_hi, xy_hi, yy_hi; int src; float xx_lo, xy_lo, yy_lo, pad; };

// One pair-list entry read with an evict-first hint: the list is streamed once per
// product and is larger than L2, where the gathered densities should stay.
__device__ __forceinline__ PairEntry<float> ld_entry(const PairEntry<float>* p) {
    const int4 v = __ldcs(reinterpret_cast<const int4*>(p));
    PairEntry<float> e;
    e.xx = __int_as_float(v.x);
    e.xy = __int_as_float(v.y);
    e.yy = __int_as_float(v.z);
    e.src = v.w;
    return e;
}
__device__ __forceinline__ PairEntry<double> ld_entry(const PairEntry<double>* p) {
    const double2 a = __ldcs(reinterpret_cast<const double2*>(p));
    const double2 b = __ldcs(reinterpret_cast<const double2*>(p) + 1);
    PairEntry<double> e;
    e.xx = a.x;
    e.xy = a.y;
    e.yy = b.x;
    e.src = __double_as_longlong(b.y);
    return e;
}

// v_s[row_of[p]] = sum_k pairs[p][k] mu_s[src] over list positions p (rows sorted by
// length within windows, so a slice's rows have nearly equal lengths): one block per
// 32-position slice, SPMV_P warps
// over each row's entries (warp p takes k = p, p + SPMV_P, ..., so that a warp still
// reads 32 consecutive entries), each thread taking its entries U at a time (U
// independent list loads, then U independent gathers) to keep several memory
// requests in flight; the SPMV_P partial sums are added in warp order.
constexpr int SPMV_P = 4;
template <typename T>
__global__ void __launch_bounds__(32 * SPMV_P) k_pair_spmv(int N, const int* __restrict__ slice_start,
                                                           const int* __restrict__ row_of,
                                                           const PairEntry<T>* __restrict__ pairs,
                                                           const typename V2<T>::type* __restrict__ mu_s,
                                                           typename V2<T>::type* __restrict__ v_s) {
    constexpr int U = sizeof(T) == 4 ? 8 : 4;
    using T2 = typename V2<T>::type;
    __shared__ T2 red[SPMV_P][32];
    const int sl = blockIdx.x, lane = threadIdx.x & 31, part = threadIdx.x >> 5;
    const int t = sl * 32 + lane;  // list position; the row is row_of[t]
    T ax = 0, ay = 0;
    if (t < N) {  // the slice's positions past N have no entries
        const int base = slice_start[sl], len = slice_start[sl + 1] - base;
        const PairEntry<T>* row = pairs + (size_t)base * 32 + lane;
        int k = part;
        for (; k + (U - 1) * SPMV_P < len; k += U * SPMV_P) {
            PairEntry<T> e[U];
            T2 m[U];
#pragma unroll
            for (int u = 0; u < U; ++u) e[u] = ld_entry(row + (size_t)(k + u * SPMV_P) * 32);
#pragma unroll
            for (int u = 0; u < U; ++u) m[u] = __ldg(mu_s + e[u].src);
#pragma unroll
            for (int u = 0; u < U; ++u) {
                ax = fma(e[u].xx, m[u].x, fma(e[u].xy, m[u].y, ax));
                ay = fma(e[u].xy, m[u].x, fma(e[u].yy, m[u].y, ay));
            }
        }
        for (; k < len; k += SPMV_P) {
            const PairEntry<T> e = ld_entry(row + (size_t)k * 32);
            const T2 m = __ldg(mu_s + e.src);
            ax = fma(e.xx, m.x, fma(e.xy, m.y, ax));
            ay = fma(e.xy, m.x, fma(e.yy, m.y, ay));
        }
    }
    red[part][lane].x = ax;
    red[part][lane].y = ay;
    __syncthreads();
    if (part == 0 && t < N) {
        T sx = red[0][lane].x, sy = red[0][lane].y;
#pragma unroll
        for (int p = 1; p < SPMV_P; ++p) {
            sx += red[p][lane].x;
            sy += red[p][lane].y;
        }
        const int r = row_of[t];
        v_s[r].x = sx;
        v_s[r].y = sy;
    }
}

}  // namespace fbim
