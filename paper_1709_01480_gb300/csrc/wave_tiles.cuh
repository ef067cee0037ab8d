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

// ---------------------------------------------------------------------------
// Spread.  One CTA per tile, 8 warps.  Candidates (nodes of the 3 x 3 tile
// neighbourhood whose window meets this tile) are compacted in chunks into
// shared memory with their window weights (wy already multiplied by mu).  Warp
// w owns the rows [w RB, (w+1) RB) of the tile and lane l the columns l and
// l + 32; each warp accumulates its rows in registers over all candidates and
// writes them once.  No atomics: the sum over candidates runs in the compacted
// order, which is deterministic for a given node order.
// ---------------------------------------------------------------------------
template <typename T, int PMAX>
struct SpreadSmem {
    static constexpr int KMAX = 256;   // one raw chunk of 256 candidates at most
    int rx[KMAX], ry[KMAX];
    T wx[KMAX][PMAX];
    T wmx[KMAX][PMAX];   // wy * mu_x
    T wmy[KMAX][PMAX];   // wy * mu_y
    int warp_tot[8];
    int n_cand;
};

template <typename T, int PMAX>
__global__ void __launch_bounds__(256) k_spread_tiles(TileGeom tg, T a, T g0, const int* __restrict__ tstart,
                                                     const int2* __restrict__ tbase,
                                                     const typename V2<T>::type* __restrict__ tfrac,
                                                     const typename V2<T>::type* __restrict__ mu_t,
                                                     T* __restrict__ grid) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using S = SpreadSmem<T, PMAX>;
    S& sm = *reinterpret_cast<S*>(smem_raw);
    constexpr int KMAX = S::KMAX;
    const int P = tg.P, hw = tg.hw, TS = tg.TS, nt = tg.n_tile;
    const int tx = blockIdx.x, ty = blockIdx.y;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int RB = (TS + 7) / 8;
    const int r0 = warp * RB;

    // the nine neighbour lists, concatenated in a fixed order
    int lo[9], len[9], total = 0;
#pragma unroll
    for (int d = 0; d < 9; ++d) {
        int nty = ty + d / 3 - 1, ntx = tx + d % 3 - 1;
        nty += (nty < 0) ? nt : 0;
        nty -= (nty >= nt) ? nt : 0;
        ntx += (ntx < 0) ? nt : 0;
        ntx -= (ntx >= nt) ? nt : 0;
        int t = nty * nt + ntx;
        lo[d] = tstart[t];
        len[d] = tstart[t + 1] - lo[d];
        total += len[d];
    }

    T acc[2][8][2];
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int i = 0; i < 8; ++i) acc[c][i][0] = acc[c][i][1] = T(0);

    for (int base = 0; base < total; base += 256) {
        // ---- phase 1: test one raw candidate per thread, compact by a block scan ----
        const int j = base + threadIdx.x;
        int d = 0, off = j;
        bool valid = false;
        int rx = 0, ry = 0, idx = -1;
        if (j < total) {
            while (off >= len[d]) {
                off -= len[d];
                ++d;
            }
            idx = lo[d] + off;
            const int2 b = tbase[idx];
            const int dy = d / 3 - 1, dx = d % 3 - 1;
            int nty = ty + dy, ntx = tx + dx;
            nty += (nty < 0) ? nt : 0;
            nty -= (nty >= nt) ? nt : 0;
            ntx += (ntx < 0) ? nt : 0;
            ntx -= (ntx >= nt) ? nt : 0;
            // window origin relative to this tile, in the unwrapped frame of the neighbour
            rx = b.x - ntx * TS + dx * TS - hw;
            ry = b.y - nty * TS + dy * TS - hw;
            valid = !(rx + P <= 0 || rx >= TS || ry + P <= 0 || ry >= TS);
        }
        const unsigned bal = __ballot_sync(0xffffffffu, valid);
        if (lane == 0) sm.warp_tot[warp] = __popc(bal);
        __syncthreads();
        int before = 0, n_chunk = 0;
#pragma unroll
        for (int w = 0; w < 8; ++w) {
            before += (w < warp) ? sm.warp_tot[w] : 0;
            n_chunk += sm.warp_tot[w];
        }
        if (valid) {
            const int k = before + __popc(bal & ((1u << lane) - 1u));
            sm.rx[k] = rx;
            sm.ry[k] = ry;
            const typename V2<T>::type f = tfrac[idx];
            const typename V2<T>::type mu = mu_t[idx];
            T w[PMAX];
            window_weights<T, PMAX>(P, hw, f.x, a, T(1), w);
#pragma unroll
            for (int p = 0; p < PMAX; ++p) sm.wx[k][p] = w[p];
            window_weights<T, PMAX>(P, hw, f.y, a, g0, w);
#pragma unroll
            for (int p = 0; p < PMAX; ++p) {
                sm.wmx[k][p] = w[p] * mu.x;
                sm.wmy[k][p] = w[p] * mu.y;
            }
        }
        __syncthreads();
        // ---- phase 2: every warp accumulates its rows over the chunk ----
        for (int k = 0; k < n_chunk; ++k) {
            const int cy = sm.ry[k];
            if (cy >= r0 + RB || cy + P <= r0) continue;  // warp-uniform
            const int cx = sm.rx[k];
            const int p0 = lane - cx, p1 = lane + 32 - cx;
            const T wx0 = (p0 >= 0 && p0 < P) ? sm.wx[k][p0] : T(0);
            const T wx1 = (p1 >= 0 && p1 < P) ? sm.wx[k][p1] : T(0);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int q = r0 + i - cy;
                if (i < RB && q >= 0 && q < P) {
                    const T fx = sm.wmx[k][q], fy = sm.wmy[k][q];
                    acc[0][i][0] = fma(wx0, fx, acc[0][i][0]);
                    acc[0][i][1] = fma(wx1, fx, acc[0][i][1]);
                    acc[1][i][0] = fma(wx0, fy, acc[1][i][0]);
                    acc[1][i][1] = fma(wx1, fy, acc[1][i][1]);
                }
            }
        }
        __syncthreads();
    }
    const size_t MM = (size_t)tg.M * tg.M;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int r = r0 + i;
        if (i >= RB || r >= TS) continue;
        const size_t row = (size_t)(ty * TS + r) * tg.M + tx * TS;
        if (lane < TS) {
            grid[row + lane] = acc[0][i][0];
            grid[MM + row + lane] = acc[1][i][0];
        }
        if (lane + 32 < TS) {
            grid[row + lane + 32] = acc[0][i][1];
            grid[MM + row + lane + 32] = acc[1][i][1];
        }
    }
}

// ---------------------------------------------------------------------------
// Interpolation: v_t = sum_{P x P} g(x_t - y) U(y) (the h^2 weight is in k_scale).
// One CTA per tile loads the tile and a halo of hw points (periodic) into shared
// memory with an odd row pitch; then each half-warp handles one node (lane q =
// window row q; P <= 16), or each warp one node when P > 16.  Rows are reduced
// across the lanes with shuffles.
// ---------------------------------------------------------------------------
template <typename T>
__host__ __device__ inline int interp_pitch(int W) { return W | 1; }

template <typename T, int PMAX>
__global__ void __launch_bounds__(256) k_interp_tiles(TileGeom tg, T a, T g0, const int* __restrict__ tstart,
                                                     const int2* __restrict__ tbase,
                                                     const typename V2<T>::type* __restrict__ tfrac,
                                                     const T* __restrict__ grid,
                                                     typename V2<T>::type* __restrict__ v_t) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int P = tg.P, hw = tg.hw, TS = tg.TS, M = tg.M;
    const int W = TS + 2 * hw, pitch = interp_pitch<T>(W), plane = W * pitch;
    T* sg = reinterpret_cast<T*>(smem_raw);  // [2][W][pitch]
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
            sg[iy * pitch + ix] = srcx[gx];
            sg[plane + iy * pitch + ix] = srcy[gx];
        }
    }
    __syncthreads();
    const int tile = ty * tg.n_tile + tx;
    const int lo = tstart[tile], hi = tstart[tile + 1];
    const bool half = P <= 16;
    const int per_warp = half ? 2 : 1;
    const int sub = half ? (lane >> 4) : 0;
    const int q = half ? (lane & 15) : lane;
    const unsigned group = half ? (0xffffu << (16 * sub)) : 0xffffffffu;
    for (int i0 = lo + warp * per_warp; i0 < hi; i0 += 8 * per_warp) {
        const int i = i0 + sub;
        const bool have = i < hi;
        T ax = 0, ay = 0;
        if (have && q < P) {
            const int2 b = tbase[i];
            const int rx = b.x - tx * TS, ry = b.y - ty * TS;  // window origin (rx, ry) in sg
            const typename V2<T>::type f = tfrac[i];
            T wx[PMAX];
            window_weights<T, PMAX>(P, hw, f.x, a, T(1), wx);
            const T dyq = T(q - hw) - f.y;
            const T wyq = g0 * dev_exp(-a * dyq * dyq);
            const T* rowx = sg + (ry + q) * pitch + rx;
            const T* rowy = rowx + plane;
            T sx = 0, sy = 0;
#pragma unroll
            for (int p = 0; p < PMAX; ++p) {
                if (p < P) {
                    sx = fma(wx[p], rowx[p], sx);
                    sy = fma(wx[p], rowy[p], sy);
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
        (void)group;
        if (have && q == 0) {
            v_t[i].x = ax;
            v_t[i].y = ay;
        }
    }
}


// ---------------------------------------------------------------------------
// Warp-per-node variants.  A warp takes one node (tile-sorted order keeps
// consecutive warps on neighbouring grid regions); lane p < P computes the p-th
// weight of each dimension, and the P x P window is walked row-major, 32 points
// per step, so that each step touches a few short contiguous row segments.
// Spreading reduces into the grid with fire-and-forget global atomic adds (the
// grid stays in L2); interpolation gathers the same segments and reduces over
// the warp.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_spread_warp(int N, int M, int P, int hw, float invP, T a, T g0,
                                                    const int2* __restrict__ tbase,
                                                    const typename V2<T>::type* __restrict__ tfrac,
                                                    const typename V2<T>::type* __restrict__ mu_t,
                                                    T* __restrict__ grid) {
    const int lane = threadIdx.x & 31;
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= N) return;  // warp-uniform
    const int2 b = tbase[i];
    const typename V2<T>::type f = tfrac[i];
    const typename V2<T>::type mu = mu_t[i];
    const T dx = T(lane - hw) - f.x, dy = T(lane - hw) - f.y;
    const T wx = dev_exp(-a * dx * dx);
    const T wy = g0 * dev_exp(-a * dy * dy);
    const size_t MM = (size_t)M * M;
    const int PP = P * P;
    for (int k0 = 0; k0 < PP; k0 += 32) {
        const int k = k0 + lane;
        int q = (int)(((float)k + 0.5f) * invP);
        int p = k - q * P;
        const bool ok = k < PP;
        if (!ok) p = q = 0;
        const T w = __shfl_sync(0xffffffffu, wx, p) * __shfl_sync(0xffffffffu, wy, q);
        if (ok) {
            int gx = b.x + p - hw, gy = b.y + q - hw;
            gx += (gx < 0) ? M : 0;
            gx -= (gx >= M) ? M : 0;
            gy += (gy < 0) ? M : 0;
            gy -= (gy >= M) ? M : 0;
            const size_t g = (size_t)gy * M + gx;
            atomicAdd(grid + g, w * mu.x);
            atomicAdd(grid + MM + g, w * mu.y);
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_interp_warp(int N, int M, int P, int hw, float invP, T a, T g0,
                                                    const int2* __restrict__ tbase,
                                                    const typename V2<T>::type* __restrict__ tfrac,
                                                    const T* __restrict__ grid,
                                                    typename V2<T>::type* __restrict__ v_t) {
    const int lane = threadIdx.x & 31;
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= N) return;  // warp-uniform
    const int2 b = tbase[i];
    const typename V2<T>::type f = tfrac[i];
    const T dx = T(lane - hw) - f.x, dy = T(lane - hw) - f.y;
    const T wx = dev_exp(-a * dx * dx);
    const T wy = g0 * dev_exp(-a * dy * dy);
    const size_t MM = (size_t)M * M;
    const int PP = P * P;
    T ax = 0, ay = 0;
    for (int k0 = 0; k0 < PP; k0 += 32) {
        const int k = k0 + lane;
        int q = (int)(((float)k + 0.5f) * invP);
        int p = k - q * P;
        const bool ok = k < PP;
        if (!ok) p = q = 0;
        const T w = __shfl_sync(0xffffffffu, wx, p) * __shfl_sync(0xffffffffu, wy, q);
        if (ok) {
            int gx = b.x + p - hw, gy = b.y + q - hw;
            gx += (gx < 0) ? M : 0;
            gx -= (gx >= M) ? M : 0;
            gy += (gy < 0) ? M : 0;
            gy -= (gy >= M) ? M : 0;
            const size_t g = (size_t)gy * M + gx;
            ax = fma(w, __ldg(grid + g), ax);
            ay = fma(w, __ldg(grid + MM + g), ay);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        ax += __shfl_xor_sync(0xffffffffu, ax, o);
        ay += __shfl_xor_sync(0xffffffffu, ay, o);
    }
    if (lane == 0) {
        v_t[i].x = ax;
        v_t[i].y = ay;
    }
}

template <typename T, int PMAX>
inline size_t spread_smem_bytes() { return sizeof(SpreadSmem<T, PMAX>); }

template <typename T>
inline size_t interp_smem_bytes(int TS, int P) {
    const int W = TS + (P - 1), pitch = interp_pitch<T>(W);
    return 2 * (size_t)W * pitch * sizeof(T);
}

}  // namespace fbim
