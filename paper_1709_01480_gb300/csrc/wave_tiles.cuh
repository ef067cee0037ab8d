// Wave-space tile kernels: Gaussian spreading and interpolation (Sec. 3.2, the
// operators S and S* of the spectral Ewald factorisation).  Included by one
// translation unit per precision so that the variants compile in parallel.
//
// The grid is cut into TS x TS tiles; a node belongs to the tile that holds its
// nearest grid point and its P x P window reaches at most (P-1)/2 points into
// the neighbouring tiles.  With a = 2 xi^2 h^2 / eta_s, g0 = 2 xi^2/(pi eta_s) and
// f the node's offset from its nearest grid point (in units of h), the window
// weights are separable:
//     wx_p = e^{-a (p - hw - f_x)^2},  wy_q = g0 e^{-a (q - hw - f_y)^2},  p, q = 0..P-1.
// Each weight is one exponential of a small argument near the window centre;
// the tail weights carry larger arguments but are correspondingly tiny, so the
// fast exponential keeps the window accurate to a few float ulps in absolute terms.
#pragma once
#include "fbim_internal.h"
#include "ewald_types.cuh"

namespace fbim {

// Weights of one window dimension into w[0..P-1] (registers when PMAX is unrolled).
template <typename T, int PMAX>
__device__ __forceinline__ void window_weights(int P, int hw, T f, T a, T scale, T* __restrict__ w) {
#pragma unroll
    for (int p = 0; p < PMAX; ++p) {
        const T d = T(p - hw) - f;
        w[p] = p < P ? scale * dev_exp(-a * d * d) : T(0);
    }
}

__device__ __forceinline__ float acc_exp(float x) { return expf(x); }
__device__ __forceinline__ double acc_exp(double x) { return exp(x); }

// The PMAX weights e^{-a (j - HW - f)^2}, j = 0..PMAX-1, HW = (PMAX-1)/2, by a
// two-sided recurrence from the centre: the ratio of neighbours is
// e^{-a (2 d + 1)} going up and e^{-a (1 - 2 d)} going down (d = j - HW - f), and
// each ratio is the previous one times q2 = e^{-2a}.  Three exponentials instead
// of PMAX; the tail weights, which carry the longest product chains, are the
// smallest.  A window of P < PMAX points uses j in [HW - hw, HW + hw].
template <typename T, int PMAX>
__device__ __forceinline__ void window_recur(T f, T a, T q2, T scale, T* __restrict__ w) {
    constexpr int HW = (PMAX - 1) / 2;
    w[HW] = scale * acc_exp(-a * f * f);
    T r = acc_exp(-a * (T(1) - T(2) * f));
#pragma unroll
    for (int j = HW; j < PMAX - 1; ++j) {
        w[j + 1] = w[j] * r;
        r *= q2;
    }
    r = acc_exp(-a * (T(1) + T(2) * f));
#pragma unroll
    for (int j = HW; j > 0; --j) {
        w[j - 1] = w[j] * r;
        r *= q2;
    }
}

// ---------------------------------------------------------------------------
// Spread.  One CTA per tile accumulates the windows of the tile's own nodes
// (nodes whose nearest grid point lies in the tile) into its extended region of
// W = TS + 2 hw points per side in shared memory, with shared-memory atomics:
// a half-warp (a warp when P > 16) takes a node, lane q < P its window row q.
// The core TS x TS points are then stored straight to the grid (plain stores: no
// zeroing, no global atomics) and the halo ring to a per-tile buffer; k_spread_fold adds the
// neighbours' rings to the border bands in a fixed order, so the result does
// not depend on scheduling.
// ---------------------------------------------------------------------------
template <typename T, int PMAX>
__global__ void __launch_bounds__(256) k_spread_tiles(TileGeom tg, T a, T q2, T g0, const int* __restrict__ tstart,
                                                     const int2* __restrict__ tbase,
                                                     const typename V2<T>::type* __restrict__ tfrac,
                                                     const typename V2<T>::type* __restrict__ mu_t,
                                                     T* __restrict__ grid, T* __restrict__ ring) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int HW = (PMAX - 1) / 2;
    const int P = tg.P, hw = tg.hw, TS = tg.TS, M = tg.M;
    const int W = TS + 2 * hw, pitch = W | 1, plane = W * pitch;
    T* acc = reinterpret_cast<T*>(smem_raw);  // [2][W][pitch]
    const int tx = blockIdx.x, ty = blockIdx.y, tile = ty * tg.n_tile + tx;
    for (int e = threadIdx.x; e < 2 * plane; e += blockDim.x) acc[e] = T(0);
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // a half-warp per node when the window has at most 16 rows, else a warp
    const bool half = P <= 16;
    const int per_warp = half ? 2 : 1;
    const int sub = half ? (lane >> 4) : 0;
    const int q = half ? (lane & 15) : lane;
    const int lo = tstart[tile], hi = tstart[tile + 1];
    const int shift = HW - hw;
    for (int i = lo + per_warp * warp + sub; i < hi; i += 8 * per_warp) {
        if (q >= P) continue;
        const int2 b = tbase[i];
        const typename V2<T>::type f = tfrac[i];
        const typename V2<T>::type mu = mu_t[i];
        T wx[PMAX];
        window_recur<T, PMAX>(f.x, a, q2, T(1), wx);
        const T dy = T(q - hw) - f.y;
        const T wyq = g0 * acc_exp(-a * dy * dy);
        const T cx = wyq * mu.x, cy = wyq * mu.y;
        // window origin (b - hw) relative to the extended region's origin (tile - hw)
        const int base = (b.y - ty * TS + q) * pitch + (b.x - tx * TS) - shift;
#pragma unroll
        for (int j = 0; j < PMAX; ++j) {
            if (j >= shift && j < shift + P) {
                atomicAdd(acc + base + j, wx[j] * cx);
                atomicAdd(acc + plane + base + j, wx[j] * cy);
            }
        }
    }
    __syncthreads();
    const size_t MM = (size_t)M * M;
    for (int e = threadIdx.x; e < TS * TS; e += blockDim.x) {
        const int ly = e / TS, lx = e - ly * TS;
        const size_t g = (size_t)(ty * TS + ly) * M + tx * TS + lx;
        const int s = (ly + hw) * pitch + lx + hw;
        grid[g] = acc[s];
        grid[MM + g] = acc[plane + s];
    }
    T* rt = ring + (size_t)tile * 2 * W * W;
    for (int e = threadIdx.x; e < W * W; e += blockDim.x) {
        const int ey = e / W, ex = e - ey * W;
        if (ey >= hw && ey < TS + hw && ex >= hw && ex < TS + hw) continue;
        rt[e] = acc[ey * pitch + ex];
        rt[W * W + e] = acc[plane + ey * pitch + ex];
    }
}

// Border bands of each tile: add the neighbours' halo rings (fixed neighbour order).
template <typename T>
__global__ void __launch_bounds__(256) k_spread_fold(TileGeom tg, const T* __restrict__ ring, T* __restrict__ grid) {
    const int hw = tg.hw, TS = tg.TS, M = tg.M, nt = tg.n_tile;
    const int W = TS + 2 * hw;
    const int tx = blockIdx.x, ty = blockIdx.y;
    const size_t MM = (size_t)M * M;
    for (int e = threadIdx.x; e < TS * TS; e += blockDim.x) {
        const int ly = e / TS, lx = e - ly * TS;
        if (ly >= hw && ly < TS - hw && lx >= hw && lx < TS - hw) continue;
        T sx = T(0), sy = T(0);
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                if (dx == 0 && dy == 0) continue;
                const int ex = lx - dx * TS + hw, ey = ly - dy * TS + hw;
                if (ex < 0 || ex >= W || ey < 0 || ey >= W) continue;
                int ntx = tx + dx, nty = ty + dy;
                ntx += (ntx < 0) ? nt : 0;
                ntx -= (ntx >= nt) ? nt : 0;
                nty += (nty < 0) ? nt : 0;
                nty -= (nty >= nt) ? nt : 0;
                const T* rt = ring + (size_t)(nty * nt + ntx) * 2 * W * W;
                sx += rt[ey * W + ex];
                sy += rt[W * W + ey * W + ex];
            }
        const size_t g = (size_t)(ty * TS + ly) * M + tx * TS + lx;
        grid[g] += sx;
        grid[MM + g] += sy;
    }
}

// ---------------------------------------------------------------------------
// Interpolation: v_t = sum_{P x P} g(x_t - y) U(y) (the h^2 weight is in k_scale).
// One CTA per tile loads the tile and a halo of hw points (periodic) into shared
// memory as interleaved (x, y) pairs with an odd row pitch; then each half-warp
// handles one node (lane q = window row q, one 8-byte load per point; P <= 16),
// or each warp one node when P > 16.  Rows are reduced across the lanes with
// shuffles.
// ---------------------------------------------------------------------------
template <typename T>
__host__ __device__ inline int interp_pitch(int W) { return W | 1; }

template <typename T, int PMAX>
__global__ void __launch_bounds__(256) k_interp_tiles(TileGeom tg, T a, T q2, T g0, const int* __restrict__ tstart,
                                                     const int2* __restrict__ tbase,
                                                     const typename V2<T>::type* __restrict__ tfrac,
                                                     const T* __restrict__ grid,
                                                     typename V2<T>::type* __restrict__ v_t) {
    using T2 = typename V2<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int HW = (PMAX - 1) / 2;
    const int P = tg.P, hw = tg.hw, TS = tg.TS, M = tg.M;
    const int W = TS + 2 * hw, pitch = interp_pitch<T>(W);
    T2* sg = reinterpret_cast<T2*>(smem_raw);  // [W][pitch] of (x, y)
    const int tx = blockIdx.x, ty = blockIdx.y;
    const int x0 = tx * TS - hw, y0 = ty * TS - hw;
    const size_t MM = (size_t)M * M;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int iy = warp; iy < W; iy += 8) {
        int gy = y0 + iy;
        gy += (gy < 0) ? M : 0;
        gy -= (gy >= M) ? M : 0;
        const T* srcx = grid + (size_t)gy * M;
        const T* srcy = srcx + MM;
        for (int ix = lane; ix < W; ix += 32) {
            int gx = x0 + ix;
            gx += (gx < 0) ? M : 0;
            gx -= (gx >= M) ? M : 0;
            T2 u;
            u.x = srcx[gx];
            u.y = srcy[gx];
            sg[iy * pitch + ix] = u;
        }
    }
    __syncthreads();
    const int tile = ty * tg.n_tile + tx;
    const int lo = tstart[tile], hi = tstart[tile + 1];
    const bool half = P <= 16;
    const int per_warp = half ? 2 : 1;
    const int sub = half ? (lane >> 4) : 0;
    const int q = half ? (lane & 15) : lane;
    const int shift = HW - hw;
    for (int i0 = lo + warp * per_warp; i0 < hi; i0 += 8 * per_warp) {
        const int i = i0 + sub;
        const bool have = i < hi;
        T ax = 0, ay = 0;
        if (have && q < P) {
            const int2 b = tbase[i];
            const typename V2<T>::type f = tfrac[i];
            T wx[PMAX];
            window_recur<T, PMAX>(f.x, a, q2, T(1), wx);
            const T dyq = T(q - hw) - f.y;
            const T wyq = g0 * acc_exp(-a * dyq * dyq);
            const int base = (b.y - ty * TS + q) * pitch + (b.x - tx * TS) - shift;
            T sx = 0, sy = 0;
#pragma unroll
            for (int j = 0; j < PMAX; ++j) {
                if (j >= shift && j < shift + P) {
                    const T2 u = sg[base + j];
                    sx = fma(wx[j], u.x, sx);
                    sy = fma(wx[j], u.y, sy);
                }
            }
            ax = wyq * sx;
            ay = wyq * sy;
        }
        const int width = half ? 16 : 32;
        for (int o = width / 2; o > 0; o >>= 1) {
            ax += __shfl_xor_sync(0xffffffffu, ax, o, width);
            ay += __shfl_xor_sync(0xffffffffu, ay, o, width);
        }
        if (have && q == 0) {
            v_t[i].x = ax;
            v_t[i].y = ay;
        }
    }
}


// ---------------------------------------------------------------------------
// Warp variants.  Lane p of a node's lane group owns window column p; the window
// rows are walked in a loop, so every step touches one contiguous row segment of
// P points per node (coalesced), and the row weights come from the lane that owns
// them by a shuffle.  Two nodes share a warp when P <= 16 (lanes 0-15, 16-31).
// Spreading reduces into the grid with fire-and-forget global atomic adds (the
// grid stays in L2); interpolation accumulates column sums, weights them by the
// column weights and reduces over the lane group.
// ---------------------------------------------------------------------------
// Window weights of every node, once per geometry: wtab[i][0][p] = w(p - hw - f_x) and
// wtab[i][1][p] = g0 w(p - hw - f_y), p < P, by the recurrence above (three
// exponentials per dimension).  The FP64 warp kernels read them instead of taking
// two FP64 exponentials per lane, which the FP64 pipe makes their largest cost.
// wdf (or null): the same weights as float-float pairs (hi = the FP32 rounding, lo =
// the FP32 rounding of the remainder), for the float-float interpolation.
template <typename T, int PMAX>
__global__ void k_node_weights(int N, int P, int hw, T a, T q2, T g0, const typename V2<T>::type* __restrict__ tfrac,
                               T* __restrict__ wtab, float2* __restrict__ wdf) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    constexpr int HW = (PMAX - 1) / 2;
    const int shift = HW - hw;
    const typename V2<T>::type f = tfrac[i];
    T w[PMAX];
    T* out = wtab + (size_t)i * 2 * P;
    window_recur<T, PMAX>(f.x, a, q2, T(1), w);
#pragma unroll
    for (int j = 0; j < PMAX; ++j)
        if (j >= shift && j < shift + P) out[j - shift] = w[j];
    window_recur<T, PMAX>(f.y, a, q2, g0, w);
#pragma unroll
    for (int j = 0; j < PMAX; ++j)
        if (j >= shift && j < shift + P) out[P + j - shift] = w[j];
    if (wdf) {
        float2* od = wdf + (size_t)i * 2 * P;
        for (int j = 0; j < 2 * P; ++j) {
            const double v = (double)out[j];
            const float hi = (float)v;
            od[j] = make_float2(hi, (float)(v - (double)hi));
        }
    }
}

// wtab: the node weights above, or null to compute them per lane.
template <typename T>
__global__ void __launch_bounds__(256) k_spread_warp(int N, int M, int P, int hw, T a, T g0,
                                                    const int2* __restrict__ tbase,
                                                    const typename V2<T>::type* __restrict__ tfrac,
                                                    const typename V2<T>::type* __restrict__ mu_t,
                                                    const double2* __restrict__ mu_n, const int* __restrict__ tperm,
                                                    const T* __restrict__ wtab, T* __restrict__ grid) {
    const int lane = threadIdx.x & 31;
    const int w = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    const bool two = P <= 16;
    const int sub = two ? (lane >> 4) : 0, p = two ? (lane & 15) : lane;
    const int i = w * (two ? 2 : 1) + sub;
    if (w * (two ? 2 : 1) >= N) return;  // warp-uniform
    const bool active = i < N && p < P;
    int2 b = make_int2(0, 0);
    typename V2<T>::type f = {T(0), T(0)}, mu = {T(0), T(0)};
    if (active) {
        b = tbase[i];
        if (!wtab) f = tfrac[i];
        if (tperm) {  // the gather into tile order, fused
            const double2 u = mu_n[tperm[i]];
            mu.x = (T)u.x;
            mu.y = (T)u.y;
        } else {
            mu = mu_t[i];
        }
    }
    T wx = T(0), wy = T(0);  // column weight of column p, row weight of row p
    if (active) {
        if (wtab) {
            wx = wtab[(size_t)i * 2 * P + p];
            wy = wtab[(size_t)i * 2 * P + P + p];
        } else {
            const T dx = T(p - hw) - f.x, dy = T(p - hw) - f.y;
            wx = acc_exp(-a * dx * dx);
            wy = g0 * acc_exp(-a * dy * dy);
        }
    }
    const T cx = wx * mu.x, cy = wx * mu.y;
    int gx = b.x - hw + p;
    gx += (gx < 0) ? M : 0;
    gx -= (gx >= M) ? M : 0;
    int gy = b.y - hw;
    gy += (gy < 0) ? M : 0;
    const size_t MM = (size_t)M * M;
    const int src = two ? (sub << 4) : 0;
    for (int q = 0; q < P; ++q) {
        const T wq = __shfl_sync(0xffffffffu, wy, src + q);
        if (active) {
            const size_t g = (size_t)gy * M + gx;
            atomicAdd(grid + g, wq * cx);
            atomicAdd(grid + MM + g, wq * cy);
        }
        gy = (gy + 1 == M) ? 0 : gy + 1;
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_interp_warp(int N, int M, int P, int hw, T a, T g0,
                                                    const int2* __restrict__ tbase,
                                                    const typename V2<T>::type* __restrict__ tfrac,
                                                    const T* __restrict__ wtab, const T* __restrict__ grid,
                                                    typename V2<T>::type* __restrict__ v_t, InterpEpilogue<T> ep) {
    const int lane = threadIdx.x & 31;
    const int w = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    const bool two = P <= 16;
    const int sub = two ? (lane >> 4) : 0, p = two ? (lane & 15) : lane;
    const int i = w * (two ? 2 : 1) + sub;
    if (w * (two ? 2 : 1) >= N) return;  // warp-uniform
    const bool active = i < N && p < P;
    int2 b = make_int2(0, 0);
    typename V2<T>::type f = {T(0), T(0)};
    if (active) {
        b = tbase[i];
        if (!wtab) f = tfrac[i];
    }
    T wx = T(0), wy = T(0);
    if (active) {
        if (wtab) {
            wx = wtab[(size_t)i * 2 * P + p];
            wy = wtab[(size_t)i * 2 * P + P + p];
        } else {
            const T dx = T(p - hw) - f.x, dy = T(p - hw) - f.y;
            wx = acc_exp(-a * dx * dx);
            wy = g0 * acc_exp(-a * dy * dy);
        }
    }
    int gx = b.x - hw + p;
    gx += (gx < 0) ? M : 0;
    gx -= (gx >= M) ? M : 0;
    int gy = b.y - hw;
    gy += (gy < 0) ? M : 0;
    const size_t MM = (size_t)M * M;
    const int src = two ? (sub << 4) : 0;
    T sx = 0, sy = 0;
    for (int q = 0; q < P; ++q) {
        const T wq = __shfl_sync(0xffffffffu, wy, src + q);
        if (active) {
            const size_t g = (size_t)gy * M + gx;
            sx = fma(wq, __ldg(grid + g), sx);
            sy = fma(wq, __ldg(grid + MM + g), sy);
        }
        gy = (gy + 1 == M) ? 0 : gy + 1;
    }
    sx *= wx;
    sy *= wx;
    const int width = two ? 16 : 32;
    for (int o = width / 2; o > 0; o >>= 1) {
        sx += __shfl_xor_sync(0xffffffffu, sx, o, width);
        sy += __shfl_xor_sync(0xffffffffu, sy, o, width);
    }
    if (p == 0 && i < N) interp_store<T>(ep, v_t, i, sx, sy);
}

// ---------------------------------------------------------------------------
// Vector interpolation (FP32, P <= 13, M a multiple of 4).  Four lanes take a node
// and eight nodes share a warp; lane c of a node owns grid columns
// [a0 + 4c, a0 + 4c + 4), a0 = the window's first column rounded down to a multiple
// of 4, so that 4 chunks cover the window (13 + 3 columns).  Every chunk is 16-byte
// aligned and never wraps (M is a multiple of 4), so each row costs one float4 load
// per chunk.  Row weights come from the two-sided recurrence in every lane.  (The
// same layout with float4 atomic adds made spreading slower than the scalar
// column-lane kernel, so spreading keeps that one.)
// ---------------------------------------------------------------------------
constexpr int kVecPMAX = 16;

static __device__ __forceinline__ void vec_setup(int i, int N, int lane, int P, int hw, float a, float q2, float g0, int M,
                                          const int2* __restrict__ tbase, const float2* __restrict__ tfrac,
                                          bool& active, int& gc, int& gy, float (&wx)[4], float (&wy)[kVecPMAX]) {
    constexpr int HW = (kVecPMAX - 1) / 2;
    active = i < N;
    int2 b = make_int2(0, 0);
    float2 f = make_float2(0.f, 0.f);
    if (active) {
        b = tbase[i];
        f = tfrac[i];
    }
    const int c = lane & 3;
    const int gx0 = b.x - hw;                 // window's first column (may be negative)
    const int off = ((gx0 % 4) + 4) % 4;      // columns before it in its aligned chunk
    int a0 = gx0 - off + 4 * c;               // this lane's chunk, a multiple of 4
    a0 += (a0 < 0) ? M : 0;
    a0 -= (a0 >= M) ? M : 0;
    gc = a0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int p = 4 * c + j - off;        // window column of chunk element j
        const float d = float(p - hw) - f.x;
        wx[j] = (active && p >= 0 && p < P) ? expf(-a * d * d) : 0.f;
    }
    window_recur<float, kVecPMAX>(f.y, a, q2, g0, wy);
    (void)HW;
    gy = b.y - hw;
    gy += (gy < 0) ? M : 0;
}

static __global__ void __launch_bounds__(256) k_interp_vec(int N, int M, int P, int hw, float a, float q2, float g0,
                                                   const int2* __restrict__ tbase, const float2* __restrict__ tfrac,
                                                   const float* __restrict__ grid, float2* __restrict__ v_t,
                                                   InterpEpilogue<float> ep) {
    constexpr int HW = (kVecPMAX - 1) / 2;
    const int lane = threadIdx.x & 31;
    const int i = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 2);
    bool active;
    int gc, gy;
    float wx[4], wy[kVecPMAX];
    vec_setup(i, N, lane, P, hw, a, q2, g0, M, tbase, tfrac, active, gc, gy, wx, wy);
    const size_t MM = (size_t)M * M;
    const int shift = HW - hw;
    float sx = 0.f, sy = 0.f;
    if (active) {
#pragma unroll
        for (int j = 0; j < kVecPMAX; ++j) {
            if (j >= shift && j < shift + P) {
                const float4 ux = __ldg(reinterpret_cast<const float4*>(grid + (size_t)gy * M + gc));
                const float4 uy = __ldg(reinterpret_cast<const float4*>(grid + MM + (size_t)gy * M + gc));
                sx = fmaf(wy[j], wx[0] * ux.x + wx[1] * ux.y + wx[2] * ux.z + wx[3] * ux.w, sx);
                sy = fmaf(wy[j], wx[0] * uy.x + wx[1] * uy.y + wx[2] * uy.z + wx[3] * uy.w, sy);
                gy = (gy + 1 == M) ? 0 : gy + 1;
            }
        }
    }
    // reduce over the node's four lanes (all lanes take part)
    sx += __shfl_xor_sync(0xffffffffu, sx, 1);
    sy += __shfl_xor_sync(0xffffffffu, sy, 1);
    sx += __shfl_xor_sync(0xffffffffu, sx, 2);
    sy += __shfl_xor_sync(0xffffffffu, sy, 2);
    if (active && (lane & 3) == 0) interp_store<float>(ep, v_t, i, sx, sy);
}

template <typename T>
inline size_t spread_smem_bytes(int TS, int P) {
    const int W = TS + (P - 1), pitch = W | 1;
    return 2 * (size_t)W * pitch * sizeof(T);
}

// per-tile halo rings of the spread: [n_tile^2][2][W][W]
inline size_t spread_ring_elems(int TS, int P, int n_tile) {
    const size_t W = TS + (P - 1);
    return (size_t)n_tile * n_tile * 2 * W * W;
}

template <typename T>
inline size_t interp_smem_bytes(int TS, int P) {
    const int W = TS + (P - 1), pitch = interp_pitch<T>(W);
    return 2 * (size_t)W * pitch * sizeof(T);
}

}  // namespace fbim
