// The positively split Ewald matvec v = M mu = (M(t) + M(a)_sym + M(w)) mu (Sec. 3.2).
//
//   real space   M(t): cell-list pair sum of G^(r)_xi over the 9 neighbour cells
//                (Sec. 3.2, Eqs. real-space-kernel, expint), r < r_c, m != n;
//                M(a): per-body band R_beta M(a)_ref R_beta^T, FP64 always.
//   wave space   M(w) = D* B D with D = C F S (Sec. 3.2, Eq. Mwave-factorization):
//                Gaussian spread S, forward FFT F, the Hasimoto tensor B with both
//                deconvolutions C folded in, inverse FFT, Gaussian interpolation S*.
//
// Layouts.  Real-space work runs in cell-sorted order (slot s holds node perm[s]).
// Per geometry, the pairs within r_c are found once from the cell list and their
// 2 x 2 kernel values stored in a sliced-ELL list (slices of 32 consecutive
// targets, entries interleaved so that a warp reads 32 consecutive entries); a
// matvec then streams the list once -- the real-space part is applied tens of
// times per geometry inside GMRES and Lanczos, so its transcendental work
// (E1, exp) is paid once.
// Wave-space work runs in grid-tile order (slot t holds node tperm[t]): the grid
// is cut into TS x TS tiles (TS divides M) and every node belongs to the tile of
// its nearest grid point.  Spreading is owner-computes: one CTA per tile
// accumulates, in shared memory, the Gaussians of the nodes of its own and its
// eight neighbouring tiles that reach into it (one thread per node, P unrolled),
// then writes its tile once -- no global atomics.  Interpolation loads the tile
// plus a halo of (P-1)/2 points into shared memory and gathers each of the
// tile's nodes from there.  The final kernel scatters both parts back to body
// order and adds the Alpert band.
//
// Templated on the operator precision T (double: parity path; float: fast path).
#include <cmath>

#include <type_traits>

#include "dfloat.cuh"
#include "fbim_internal.h"
#include "ewald_types.cuh"
#include "pair_spmv.cuh"

namespace fbim {

// ---------------------------------------------------------------------------
// Layout kernels
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_offsets(int N, const int* __restrict__ perm, const int* __restrict__ tperm,
                          const double* __restrict__ x, const int* __restrict__ cell,
                          const int2* __restrict__ gbase, int n_box, double r_c, double h,
                          typename V2<T>::type* __restrict__ off, int2* __restrict__ tbase,
                          typename V2<T>::type* __restrict__ tfrac) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= N) return;
    int m = perm[s];
    double px = x[2 * m], py = x[2 * m + 1];
    int c = cell[m];
    int cx = c % n_box, cy = c / n_box;
    off[s].x = (T)(px - cx * r_c);
    off[s].y = (T)(py - cy * r_c);
    int mt = tperm[s];
    double qx = x[2 * mt] / h, qy = x[2 * mt + 1] / h;
    tbase[s] = gbase[mt];
    tfrac[s].x = (T)(qx - rint(qx));
    tfrac[s].y = (T)(qy - rint(qy));
}

template <typename T>
__global__ void k_gather(int N, int n_p, const int* __restrict__ perm, const int* __restrict__ tperm, int want_s,
                         int want_t, const double* __restrict__ rot, const double2* __restrict__ mu,
                         typename V2<T>::type* __restrict__ mu_s, typename V2<T>::type* __restrict__ mu_t,
                         double2* __restrict__ mu_r, float4* __restrict__ mu_df, float4* __restrict__ mu_rdf) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= N) return;
    if (want_s) {
        double2 v = mu[perm[s]];
        mu_s[s].x = (T)v.x;
        mu_s[s].y = (T)v.y;
        if (mu_df) {
            const dfl::df a = dfl::from_double(v.x), b = dfl::from_double(v.y);
            mu_df[s] = make_float4(a.hi, a.lo, b.hi, b.lo);
        }
        // node s in body order, rotated into its body's frame for the Alpert band
        const int b = s / n_p;
        const double c = rot[2 * b], sn = rot[2 * b + 1];
        const double2 u = mu[s];
        const double rx = c * u.x + sn * u.y, ry = -sn * u.x + c * u.y;
        if (mu_rdf) {  // the float-float band's input
            const dfl::df a = dfl::from_double(rx), b = dfl::from_double(ry);
            mu_rdf[s] = make_float4(a.hi, a.lo, b.hi, b.lo);
        } else {
            mu_r[s] = make_double2(rx, ry);
        }
    }
    if (want_t) {
        double2 v = mu[tperm[s]];
        mu_t[s].x = (T)v.x;
        mu_t[s].y = (T)v.y;
    }
}

// ---------------------------------------------------------------------------
// Real space: v_t = sum_{n != t, r < r_c} G^(r)(x_t - x_n) mu_n over the 9 cells
// around t's cell.  The visit order below (cells dy, dx; slots ascending) is the
// column order of each row of the pair list.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(128) k_pair_count(int N, int n_box, T r_c, T rc2, const int* __restrict__ perm,
                                                   const int* __restrict__ cell, const int* __restrict__ start,
                                                   const typename V2<T>::type* __restrict__ off,
                                                   int* __restrict__ row_count, int* __restrict__ flags) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N) return;
    int n = 0;
    for_each_pair<T>(t, n_box, r_c, rc2, perm, cell, start, off, [&](int, T, T, T r2) {
        if (r2 == T(0))
            atomicOr(&flags[1], 1);
        else
            ++n;
    });
    row_count[t] = n;
}

// Rows sorted by length within windows of ROW_WINDOW consecutive (cell-sorted) rows, so
// that the 32 rows of a slice have nearly equal lengths and the sliced-ELL padding
// shrinks (sliced ELL with a sort window, "SELL-C-sigma").  One block per window: a
// bitonic sort of (length descending, row ascending) in shared memory; row_of[p] is the
// row at list position p (-1 past N), pos_of[t] the position of row t.  Positions p < N
// always hold rows: a window's missing rows sort last.
constexpr int ROW_WINDOW = 256;
inline size_t row_windows(size_t N) { return (N + ROW_WINDOW - 1) / ROW_WINDOW; }
__global__ void __launch_bounds__(ROW_WINDOW) k_sort_rows(int N, const int* __restrict__ row_count,
                                                         int* __restrict__ row_of, int* __restrict__ pos_of) {
    __shared__ unsigned long long key[ROW_WINDOW];
    const int i = threadIdx.x, t = blockIdx.x * ROW_WINDOW + i;
    const unsigned hi = t < N ? (1u << 30) - (unsigned)row_count[t] : 0xffffffffu;
    key[i] = ((unsigned long long)hi << 32) | (unsigned)t;
    __syncthreads();
    for (int k = 2; k <= ROW_WINDOW; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            const int q = i ^ j;
            if (q > i) {
                const unsigned long long a = key[i], b = key[q];
                const bool up = (i & k) == 0;
                if ((a > b) == up) {
                    key[i] = b;
                    key[q] = a;
                }
            }
            __syncthreads();
        }
    }
    const unsigned long long kv = key[i];
    const int p = blockIdx.x * ROW_WINDOW + i;
    const int row = (unsigned)(kv >> 32) == 0xffffffffu ? -1 : (int)(unsigned)(kv & 0xffffffffu);
    row_of[p] = row;
    if (row >= 0) pos_of[row] = p;
}

// slice_len[s] = longest row of the 32 positions in slice s (one warp per slice).
__global__ void k_slice_len(int n_slice, int N, const int* __restrict__ row_count, const int* __restrict__ row_of,
                            int* __restrict__ slice_len) {
    const int sl = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (sl >= n_slice) return;
    const int p = sl * 32 + lane;
    int v = p < N ? row_count[row_of[p]] : 0;
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) slice_len[sl] = v;
}

// Pass 2 of the list build: write each pair's separation (rx, ry in the xx, xy
// slots) and source; padding entries get a zero separation and the target itself.
template <typename T>
__global__ void __launch_bounds__(128) k_pair_fill(int N, int n_box, T r_c, T rc2, const int* __restrict__ perm,
                                                  const int* __restrict__ cell, const int* __restrict__ start,
                                                  const typename V2<T>::type* __restrict__ off,
                                                  const int* __restrict__ slice_start, const int* __restrict__ pos_of,
                                                  PairEntry<T>* __restrict__ pairs) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N) return;
    const int p = pos_of[t], sl = p >> 5, lane = p & 31;
    const int base = slice_start[sl], len = slice_start[sl + 1] - base;
    PairEntry<T>* row = pairs + (size_t)base * 32 + lane;
    int k = 0;
    for_each_pair<T>(t, n_box, r_c, rc2, perm, cell, start, off, [&](int s, T rx, T ry, T r2) {
        if (r2 == T(0)) return;
        PairEntry<T> e;
        e.xx = rx;
        e.xy = ry;
        e.yy = T(0);
        e.src = s;
        row[(size_t)k * 32] = e;
        ++k;
    });
    for (; k < len; ++k) {
        PairEntry<T> e;
        e.xx = e.xy = e.yy = T(0);
        e.src = t;
        row[(size_t)k * 32] = e;
    }
}

// The kernel G^(r)(r) / (4 pi eta) for separation (rx, ry): (a + b r r^T) with
// a = E1(z)/2 - e^{-z} (Chebyshev series of its entire part minus ln(z)/2) and
// b = e^{-z} / r^2, z = xi^2 r^2.
template <typename T>
__device__ __forceinline__ void pair_value(T rx, T ry, T xi2, T pref, const ChebE1<T>& ce, T& xx, T& xy, T& yy) {
    const T r2 = rx * rx + ry * ry;
    const T z = xi2 * r2;
    const T a = kernel_a<T>(ce, z);
    const T b = dev_div(dev_exp(-z), r2);
    xx = pref * (a + b * rx * rx);
    xy = pref * (b * rx * ry);
    yy = pref * (a + b * ry * ry);
}

// Pass 3: turn every stored separation into the kernel value in place.  One warp
// per target row, lane k on the row's k-th pair: only real pairs are evaluated, so
// the sliced-ELL padding idles no lane of the transcendental work.
template <typename T>
__global__ void __launch_bounds__(256) k_pair_eval_rows(int N, const int* __restrict__ slice_start,
                                                       const int* __restrict__ row_count,
                                                       const int* __restrict__ pos_of, T xi2, T pref,
                                                       ChebE1<T> ce, PairEntry<T>* __restrict__ pairs) {
    const int t = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (t >= N) return;
    const int n = row_count[t], p = pos_of[t];
    PairEntry<T>* row = pairs + (size_t)slice_start[p >> 5] * 32 + (p & 31);
    for (int k = lane; k < n; k += 32) {
        PairEntry<T> e = row[(size_t)k * 32];
        T xx, xy, yy;
        pair_value<T>(e.xx, e.xy, xi2, pref, ce, xx, xy, yy);
        e.xx = xx;
        e.xy = xy;
        e.yy = yy;
        row[(size_t)k * 32] = e;
    }
}

// FP64 list of a handle whose FP32 list is current: the same pairs in the same
// layout (so no FP64 neighbour search), each separation recomputed from the FP64
// cell offsets with the cell shift of its source (as the neighbour search forms it),
// then the kernel in float-float arithmetic (about 48 bits, ~1e-13 relative; the FP32
// pipes run it far faster than the FP64 pipe would).  Pairs within rounding of r_c
// may differ from an FP64 search; their kernel value is at the Ewald tolerance.
// The pair value in float-float from the piecewise tables in shared memory: S and
// e^{-z} by Horner in t = (z - zc[k]) inv_w on the piece k holding z, the logarithm
// of Sec. 3.2's a = S - ln(z)/2 by dfl::log.
__device__ __forceinline__ void pair_value_pw(dfl::df x, dfl::df y, dfl::df xi2, dfl::df pref,
                                              const float* __restrict__ zc, const float2* __restrict__ cS,
                                              const float2* __restrict__ cE, int K, float inv_w, float kscale,
                                              dfl::df& xx, dfl::df& xy, dfl::df& yy) {
    using namespace dfl;
    constexpr int D = kPwDeg;
    const df x2 = mul(x, x), y2 = mul(y, y), xy2 = mul(x, y);
    const df r2 = add(x2, y2);
    const df z = mul(xi2, r2);
    const int k = min(max((int)(z.hi * kscale), 0), K - 1);
    const df t = mul_f(add_f(z, -zc[k]), inv_w);
    const float2* s = cS + k * (D + 1);
    const float2* e = cE + k * (D + 1);
    df S = {s[D].x, s[D].y}, E = {e[D].x, e[D].y};
#pragma unroll
    for (int j = D - 1; j >= 0; --j) {
        S = add_fast(mul(S, t), df{s[j].x, s[j].y});
        E = add_fast(mul(E, t), df{e[j].x, e[j].y});
    }
    const df l = log(z);
    const df a = sub(S, df{0.5f * l.hi, 0.5f * l.lo});
    const df b = div(E, r2);
    xx = mul(pref, add(a, mul(b, x2)));
    xy = mul(pref, mul(b, xy2));
    yy = mul(pref, add(a, mul(b, y2)));
}

// One warp per target row, lanes over the row's entries; blocks loop over the rows
// (the tables are loaded into shared memory once per block).
__global__ void __launch_bounds__(256) k_pair_from32(int N, int n_box, dfl::df r_c, const int* __restrict__ perm,
                                                    const int* __restrict__ cell, const float4* __restrict__ off,
                                                    const int* __restrict__ slice_start,
                                                    const int* __restrict__ row_count,
                                                    const int* __restrict__ pos_of,
                                                    const PairEntry<float>* __restrict__ p32, dfl::df xi2,
                                                    dfl::df pref, const float* __restrict__ pw, int K, float inv_w,
                                                    float kscale, PairEntryDF* __restrict__ p64) {
    extern __shared__ float pw_s[];
    const int n_tab = K + 4 * K * (kPwDeg + 1);
    for (int i = threadIdx.x; i < n_tab; i += blockDim.x) pw_s[i] = pw[i];
    __syncthreads();
    const float* zc = pw_s;
    const float2* cS = reinterpret_cast<const float2*>(pw_s + K);
    const float2* cE = cS + K * (kPwDeg + 1);
    const int lane = threadIdx.x & 31, warps = blockDim.x >> 5;
    for (int t = blockIdx.x * warps + (threadIdx.x >> 5); t < N; t += gridDim.x * warps) {
        const int p = pos_of[t], sl = p >> 5, base = slice_start[sl], len = slice_start[sl + 1] - base;
        const int n = row_count[t];
        const int ct = cell[perm[t]], cxt = ct % n_box, cyt = ct / n_box;
        const float4 ot = off[t];
        const size_t r0 = (size_t)base * 32 + (p & 31);
        for (int k = lane; k < len; k += 32) {
            PairEntryDF e;
            if (k < n) {
                const int s = p32[r0 + (size_t)k * 32].src;
                const int cs = cell[perm[s]];
                int dx = cs % n_box - cxt, dy = cs / n_box - cyt;
                dx += (dx < -1) ? n_box : 0;
                dx -= (dx > 1) ? n_box : 0;
                dy += (dy < -1) ? n_box : 0;
                dy -= (dy > 1) ? n_box : 0;
                const float4 os = off[s];
                // (o_t - d r_c) - o_s with d in {-1, 0, 1}: d r_c is exact
                dfl::df rx = {ot.x, ot.y}, ry = {ot.z, ot.w};
                if (dx) rx = dfl::sub(rx, dx > 0 ? r_c : dfl::neg(r_c));
                if (dy) ry = dfl::sub(ry, dy > 0 ? r_c : dfl::neg(r_c));
                rx = dfl::sub(rx, dfl::df{os.x, os.y});
                ry = dfl::sub(ry, dfl::df{os.z, os.w});
                dfl::df xx, xy, yy;
                pair_value_pw(rx, ry, xi2, pref, zc, cS, cE, K, inv_w, kscale, xx, xy, yy);
                e = PairEntryDF{xx.hi, xy.hi, yy.hi, s, xx.lo, xy.lo, yy.lo, 0.0f};
            } else {
                e = PairEntryDF{0.0f, 0.0f, 0.0f, t, 0.0f, 0.0f, 0.0f, 0.0f};
            }
            p64[r0 + (size_t)k * 32] = e;
        }
    }
}

// Float-float copy of the FP64 cell offsets, one conversion per node.
__global__ void k_off_df(int N, const double2* __restrict__ off, float4* __restrict__ out) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= N) return;
    const double2 o = off[s];
    const dfl::df x = dfl::from_double(o.x), y = dfl::from_double(o.y);
    out[s] = make_float4(x.hi, x.lo, y.hi, y.lo);
}

// The FP64 real-space product of an FP32 handle on its float-float list: products
// and sums in float-float (about 2^-46 per operation, so ~1e-13 on a row sum),
// the sum rounded to FP64 once per row.  Same row order and U-wide batching as
// k_pair_spmv; nothing on the FP64 pipe but that final conversion.
__global__ void __launch_bounds__(256) k_pair_spmv_df(int N, const int* __restrict__ slice_start,
                                                     const int* __restrict__ row_of,
                                                     const PairEntryDF* __restrict__ pairs,
                                                     const float4* __restrict__ mu_df, double2* __restrict__ v_s) {
    constexpr int U = 4;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;  // list position
    if (p >= N) return;
    const int sl = p >> 5, lane = p & 31;
    const int base = slice_start[sl], len = slice_start[sl + 1] - base;
    const PairEntryDF* row = pairs + (size_t)base * 32 + lane;
    dfl::df ax = {0.0f, 0.0f}, ay = {0.0f, 0.0f};
    for (int k = 0; k < len; k += U) {
        int4 hi[U];
        float4 lo[U];
        float4 m[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (k + u < len) {
                const int4* q = reinterpret_cast<const int4*>(row + (size_t)(k + u) * 32);
                hi[u] = __ldcs(q);
                lo[u] = __ldcs(reinterpret_cast<const float4*>(q + 1));
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (k + u < len) m[u] = __ldg(mu_df + hi[u].w);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (k + u < len) {
                const dfl::df xx = {__int_as_float(hi[u].x), lo[u].x}, xy = {__int_as_float(hi[u].y), lo[u].y},
                              yy = {__int_as_float(hi[u].z), lo[u].z};
                const dfl::df mx = {m[u].x, m[u].y}, my = {m[u].z, m[u].w};
                ax = dfl::add_fast(dfl::add_fast(ax, dfl::mul(xy, my)), dfl::mul(xx, mx));
                ay = dfl::add_fast(dfl::add_fast(ay, dfl::mul(yy, my)), dfl::mul(xy, mx));
            }
        }
    }
    v_s[row_of[p]] = make_double2(dfl::to_double(ax), dfl::to_double(ay));
}

// ---------------------------------------------------------------------------
// Wave space
// ---------------------------------------------------------------------------
// Fourier scale between the FFTs: u(k) <- sc(k) (I - k k^T/k^2) u(k) with
//   sc = h^4 /(eta V) (1 + k^2/4xi^2) exp(-(1 - eta_s) k^2/4xi^2) / k^2,
// i.e. the Hasimoto tensor B (Sec. 3.2) times both Gaussian deconvolutions and
// the two grid quadrature weights h^2.  kappa = 0 and the Nyquist lines are zeroed
// (the grid is chosen so that they sit below the tolerance).
template <typename T>
__global__ void k_scale(int M, T twopi_L, T inv4xi2, T one_minus_eta, T pref,
                        typename Cplx<T>::type* __restrict__ spec) {
    const int Mh = M / 2 + 1;
    size_t n = (size_t)M * Mh;
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int r = (int)(i / Mh), c = (int)(i - (size_t)r * Mh);
    typename Cplx<T>::type* ux = spec;
    typename Cplx<T>::type* uy = spec + n;
    int ky_i = r < M / 2 ? r : r - M;
    if ((r == 0 && c == 0) || c == M / 2 || r == M / 2) {
        ux[i].x = ux[i].y = T(0);
        uy[i].x = uy[i].y = T(0);
        return;
    }
    T kx = twopi_L * T(c), ky = twopi_L * T(ky_i);
    T k2 = kx * kx + ky * ky;
    T ik2 = T(1) / k2;
    T q = k2 * inv4xi2;
    T sc = pref * (T(1) + q) * dev_exp(-one_minus_eta * q) * ik2;
    T pxx = T(1) - kx * kx * ik2, pyy = T(1) - ky * ky * ik2, pxy = -kx * ky * ik2;
    typename Cplx<T>::type a = ux[i], b = uy[i];
    ux[i].x = sc * (pxx * a.x + pxy * b.x);
    ux[i].y = sc * (pxx * a.y + pxy * b.y);
    uy[i].x = sc * (pxy * a.x + pyy * b.x);
    uy[i].y = sc * (pxy * a.y + pyy * b.y);
}

// Back to body order: v_m = v_s[slot[m]] + v_t[tslot[m]] + R_b A_ref[j] R_b^T mu (FP64 band).
// Alpert band (FP64): v_band_m = R_b sum_o A_ref[j][o] R_b^T mu_{b, j+o}, with mu_r the
// forces already rotated into their body's frame (k_gather), so each band entry costs
// four FP64 FMAs.  It depends on the forces alone, so it runs beside the wave space.
__global__ void k_band(int N, int n_p, int band, const double* __restrict__ rot, const double* __restrict__ A,
                       const double2* __restrict__ mu_r, double2* __restrict__ v_band) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= N) return;
    const int b = m / n_p, j = m - b * n_p;
    const double c = rot[2 * b], s = rot[2 * b + 1];
    double ax = 0, ay = 0;
    const int B = 2 * band + 1;
    const double2* ub = mu_r + (size_t)b * n_p;
    const double4_32a* a4 = reinterpret_cast<const double4_32a*>(A) + (size_t)j * B;
    for (int o = -band; o <= band; ++o) {
        int jj = j + o;
        jj += (jj < 0) ? n_p : 0;
        jj -= (jj >= n_p) ? n_p : 0;
        const double2 u = ub[jj];
        const double4_32a a = a4[o + band];
        ax += a.x * u.x + a.y * u.y;
        ay += a.z * u.x + a.w * u.y;
    }
    v_band[m] = make_double2(c * ax - s * ay, s * ax + c * ay);
}

// The same band product for the FP32 operator, in float-float arithmetic on the FP32
// pipes (about 2^-46 per operation, so the band velocities keep ~1e-14 of their size,
// FP64-class accuracy) instead of 84 FMAs per node on the FP64 pipe.  band_df holds
// each entry's four coefficients as float-float (a float4 of leading parts, one of
// trailing parts); mu_rdf the rotated forces (k_gather); the rotation back to the lab
// frame is in FP64.
__global__ void k_band_df(int N, int n_p, int band, const double* __restrict__ rot, const float4* __restrict__ A,
                          const float4* __restrict__ mu_rdf, double2* __restrict__ v_band) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= N) return;
    const int b = m / n_p, j = m - b * n_p;
    const int B = 2 * band + 1;
    const float4* ub = mu_rdf + (size_t)b * n_p;
    const float4* a2 = A + (size_t)j * B * 2;
    dfl::df ax = {0.f, 0.f}, ay = {0.f, 0.f};
    for (int o = -band; o <= band; ++o) {
        int jj = j + o;
        jj += (jj < 0) ? n_p : 0;
        jj -= (jj >= n_p) ? n_p : 0;
        const float4 u = ub[jj];
        const float4 hi = a2[2 * (o + band)], lo = a2[2 * (o + band) + 1];
        const dfl::df ux = {u.x, u.y}, uy = {u.z, u.w};
        ax = dfl::add_fast(ax, dfl::add_fast(dfl::mul({hi.x, lo.x}, ux), dfl::mul({hi.y, lo.y}, uy)));
        ay = dfl::add_fast(ay, dfl::add_fast(dfl::mul({hi.z, lo.z}, ux), dfl::mul({hi.w, lo.w}, uy)));
    }
    const double c = rot[2 * b], s = rot[2 * b + 1];
    const double bx = dfl::to_double(ax), by = dfl::to_double(ay);
    v_band[m] = make_double2(c * bx - s * by, s * bx + c * by);
}

// band_df from the FP64 band [n_p][B][4]: per entry (hi of the four, lo of the four)
__global__ void k_band_to_df(int n_entries, const double* __restrict__ A, float4* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_entries) return;
    dfl::df d[4];
    for (int q = 0; q < 4; ++q) d[q] = dfl::from_double(A[4 * (size_t)i + q]);
    out[2 * (size_t)i] = make_float4(d[0].hi, d[1].hi, d[2].hi, d[3].hi);
    out[2 * (size_t)i + 1] = make_float4(d[0].lo, d[1].lo, d[2].lo, d[3].lo);
}

// Back to body order: v_m = v_s[slot[m]] + v_band_m (real space) + v_t[tslot[m]] (wave space).
template <typename T>
__global__ void k_finish(int N, int with_real, int with_wave, const int* __restrict__ slot,
                         const int* __restrict__ tslot, const typename V2<T>::type* __restrict__ v_s,
                         const typename V2<T>::type* __restrict__ v_t, const double2* __restrict__ v_band,
                         double2* __restrict__ v) {
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= N) return;
    double vx = 0, vy = 0;
    if (with_real) {
        const typename V2<T>::type w = v_s[slot[m]];
        const double2 a = v_band[m];
        vx = (double)w.x + a.x;
        vy = (double)w.y + a.y;
    }
    if (with_wave) {
        const typename V2<T>::type w = v_t[tslot[m]];
        vx += (double)w.x;
        vy += (double)w.y;
    }
    v[m] = make_double2(vx, vy);
}

template <typename T> struct FftType;
template <> struct FftType<double> {
    static constexpr cufftType fwd = CUFFT_D2Z, inv = CUFFT_Z2D;
    static cufftResult f(cufftHandle p, double* in, cufftDoubleComplex* out) { return cufftExecD2Z(p, in, out); }
    static cufftResult i(cufftHandle p, cufftDoubleComplex* in, double* out) { return cufftExecZ2D(p, in, out); }
};
template <> struct FftType<float> {
    static constexpr cufftType fwd = CUFFT_R2C, inv = CUFFT_C2R;
    static cufftResult f(cufftHandle p, float* in, cufftComplex* out) { return cufftExecR2C(p, in, out); }
    static cufftResult i(cufftHandle p, cufftComplex* in, float* out) { return cufftExecC2R(p, in, out); }
};

template <typename T> static EwaldBuffers<T>& bufs(fbim_handle_s* h);
template <> EwaldBuffers<double>& bufs<double>(fbim_handle_s* h) { return h->e64; }
template <> EwaldBuffers<float>& bufs<float>(fbim_handle_s* h) { return h->e32; }
template <typename T> static const ChebE1<T>& cheb(fbim_handle_s* h);
template <> const ChebE1<double>& cheb<double>(fbim_handle_s* h) { return h->cheb64; }
template <> const ChebE1<float>& cheb<float>(fbim_handle_s* h) { return h->cheb32; }

// FP64 pair list from the current FP32 list (see k_pair_from32): no host sync.
static fbim_status build_pairs_from32(fbim_handle_s* h) {
    auto& e = h->e64;
    const auto& f = h->e32;
    const int N = h->N, n_slice = (N + 31) / 32;
    const size_t total = (size_t)(f.n_padded / 32);
    if (total > e.pair_cap) {
        cudaFree(e.pairs);
        e.pairs = nullptr;
        const size_t cap = total + total / 4 + 32;
        FBIM_CUDA_TRY(h, cudaMalloc(&e.pairs, cap * 32 * sizeof(PairEntry<double>)));
        e.pair_cap = cap;
        ++h->layout_version;
    }
    FBIM_CUDA_TRY(h, cudaMemcpyAsync(e.slice_start, f.slice_start, sizeof(int) * (n_slice + 1),
                                     cudaMemcpyDeviceToDevice, h->stream));
    // the same positions as the FP32 list (rows sorted by length within windows)
    FBIM_CUDA_TRY(h, cudaMemcpyAsync(e.row_of, f.row_of, sizeof(int) * (row_windows(N) * ROW_WINDOW + N),
                                     cudaMemcpyDeviceToDevice, h->stream));
    if (!e.off_df) {
        FBIM_CUDA_TRY(h, cudaMalloc(&e.off_df, (size_t)N * sizeof(float4)));
        FBIM_CUDA_TRY(h, cudaMalloc(&e.mu_df, (size_t)N * sizeof(float4)));
        ++h->layout_version;
    }
    k_off_df<<<(N + 255) / 256, 256, 0, h->stream>>>(N, (const double2*)e.off, e.off_df);
    if (!e.pw) {
        // piece half-width <= 0.09 keeps both series' truncation near 1e-15 at degree 8
        const int K = std::max(8, (int)std::ceil(h->zmax / 0.18));
        std::vector<float> zc;
        std::vector<double> cS, cE;
        float inv_w = 0.f;
        e1_piecewise(h->zmax, K, kPwDeg, zc, inv_w, cS, cE);
        std::vector<float> tab(zc);
        for (const auto* c : {&cS, &cE})
            for (double v : *c) {
                const dfl::df x = dfl::from_double(v);
                tab.push_back(x.hi);
                tab.push_back(x.lo);
            }
        // the kernel's limit, raised to the device maximum (shared by all handles)
        int dev = 0, optin = 0;
        FBIM_CUDA_TRY(h, cudaGetDevice(&dev));
        FBIM_CUDA_TRY(h, cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        if (tab.size() * sizeof(float) > (size_t)optin) {
            h->fail("piecewise pair-value tables exceed shared memory (xi r_c too large)");
            return FBIM_ERR_INVALID_ARG;
        }
        FBIM_CUDA_TRY(h, cudaMalloc(&e.pw, tab.size() * sizeof(float)));
        FBIM_CUDA_TRY(h, cudaMemcpy(e.pw, tab.data(), tab.size() * sizeof(float), cudaMemcpyHostToDevice));
        e.pw_K = K;
        e.pw_inv_w = inv_w;
        e.pw_kscale = (float)(K / h->zmax);
        FBIM_CUDA_TRY(h, cudaFuncSetAttribute(k_pair_from32, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    }
    const size_t smem = ((size_t)e.pw_K * (1 + 4 * (kPwDeg + 1))) * sizeof(float);
    int sms = 0, dev = 0;
    FBIM_CUDA_TRY(h, cudaGetDevice(&dev));
    FBIM_CUDA_TRY(h, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    int per_sm = 0;
    FBIM_CUDA_TRY(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pair_from32, 256, smem));
    const unsigned blocks = (unsigned)std::min<long long>(((long long)N + 7) / 8, (long long)std::max(per_sm, 1) * sms);
    k_pair_from32<<<blocks, 256, smem, h->stream>>>(
        N, h->n_box, dfl::from_double(h->r_c), h->perm, h->cell, e.off_df, f.slice_start, f.row_count,
        f.row_of + row_windows(N) * ROW_WINDOW, (const PairEntry<float>*)f.pairs, dfl::from_double(h->xi * h->xi),
        dfl::from_double(1.0 / (4.0 * M_PI * h->eta)), e.pw, e.pw_K, e.pw_inv_w, e.pw_kscale, (PairEntryDF*)e.pairs);
    h->launches += 2;
    FBIM_CUDA_TRY(h, cudaGetLastError());
    e.n_padded = f.n_padded;
    e.pairs_df = true;
    e.pairs_ready = true;
    e.pairs_geom = h->geom_version;
    return FBIM_OK;
}

// Real-space pair list for the current geometry: count, slice lengths, fill.
template <typename T>
static fbim_status build_pairs(fbim_handle_s* h) {
    if (std::is_same<T, double>::value && h->e32.ready && h->e32.pairs_ready && h->e32.pairs_geom == h->geom_version)
        return build_pairs_from32(h);
    auto& e = bufs<T>(h);
    using T2 = typename V2<T>::type;
    const int N = h->N, n_slice = (N + 31) / 32;
    const T rc = (T)h->r_c, rc2 = (T)(h->r_c * h->r_c);
    k_pair_count<T><<<(N + 127) / 128, 128, 0, h->stream>>>(N, h->n_box, rc, rc2, h->perm, h->cell, h->cell_start,
                                                            (const T2*)e.off, e.row_count, h->flags);
    // rows sorted by length within windows; slice lengths (one warp per slice) into
    // slice_start, then an exclusive scan in place
    int* pos_of = e.row_of + row_windows(N) * ROW_WINDOW;
    k_sort_rows<<<(unsigned)row_windows(N), ROW_WINDOW, 0, h->stream>>>(N, e.row_count, e.row_of, pos_of);
    k_slice_len<<<(unsigned)(((size_t)n_slice * 32 + 255) / 256), 256, 0, h->stream>>>(n_slice, N, e.row_count,
                                                                                        e.row_of, e.row_count + N);
    scan_exclusive(h->stream, e.row_count + N, n_slice, e.slice_start);
    int total = 0;
    FBIM_CUDA_TRY(h, cudaMemcpyAsync(&total, e.slice_start + n_slice, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    FBIM_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    if ((size_t)total > e.pair_cap) {
        cudaFree(e.pairs);
        e.pairs = nullptr;
        size_t cap = (size_t)total + total / 4 + 32;
        FBIM_CUDA_TRY(h, cudaMalloc(&e.pairs, cap * 32 * sizeof(PairEntry<T>)));
        e.pair_cap = cap;
        ++h->layout_version;
    }
    const T pref = (T)(1.0 / (4.0 * M_PI * h->eta));
    k_pair_fill<T><<<(N + 127) / 128, 128, 0, h->stream>>>(N, h->n_box, rc, rc2, h->perm, h->cell, h->cell_start,
                                                           (const T2*)e.off, e.slice_start, pos_of,
                                                           (PairEntry<T>*)e.pairs);
    k_pair_eval_rows<T><<<(unsigned)(((size_t)N * 32 + 255) / 256), 256, 0, h->stream>>>(
        N, e.slice_start, e.row_count, pos_of, (T)(h->xi * h->xi), pref, cheb<T>(h), (PairEntry<T>*)e.pairs);
    h->launches += 5;
    FBIM_CUDA_TRY(h, cudaGetLastError());
    e.n_padded = (long long)total * 32;
    e.pairs_df = false;
    e.pairs_ready = true;
    e.pairs_geom = h->geom_version;
    return FBIM_OK;
}

template <typename T>
fbim_status refresh_offsets(fbim_handle_s* h) {
    auto& e = bufs<T>(h);
    using T2 = typename V2<T>::type;
    const int tb = 256;
    k_offsets<T><<<(h->N + tb - 1) / tb, tb, 0, h->stream>>>(h->N, h->perm, h->tperm, h->x, h->cell, h->gbase,
                                                             h->n_box, h->r_c, h->h, (T2*)e.off, e.tbase,
                                                             (T2*)e.tfrac);
    h->launches += 1;
    if constexpr (std::is_same<T, double>::value) {
        if (e.wtab) {
            const TileGeom tg{h->M, h->TS, h->n_tile, e.P, (e.P - 1) / 2};
            const double alpha = 2.0 * h->xi * h->xi / e.eta_s;
            node_weights<double>(h->stream, h->N, tg, alpha * h->h * h->h, 2.0 * h->xi * h->xi / (M_PI * e.eta_s),
                                 e.tfrac, e.wtab, e.wtab_df);
            h->launches += 1;
        }
    }
    FBIM_CUDA_TRY(h, cudaGetLastError());
    return build_pairs<T>(h);
}

// Autotuner: time the spread and the interpolation of both kernel variants on the
// current geometry (forces = 1 on every node), each stage on its own (the spread
// variants leave the same grid), and keep the faster variant of each.
template <typename T>
static fbim_status autotune_wave(fbim_handle_s* h) {
    auto& e = bufs<T>(h);
    using T2 = typename V2<T>::type;
    const size_t M = h->M;
    const TileGeom tg{h->M, h->TS, h->n_tile, e.P, (e.P - 1) / 2};
    const double alpha = 2.0 * h->xi * h->xi / e.eta_s;
    const T ah2 = (T)(alpha * h->h * h->h);
    const T g0 = (T)(2.0 * h->xi * h->xi / (M_PI * e.eta_s));
    std::vector<T2> ones(h->N);
    for (auto& o : ones) o.x = o.y = T(1);
    FBIM_CUDA_TRY(h, cudaMemcpyAsync(e.mu_t, ones.data(), h->N * sizeof(T2), cudaMemcpyHostToDevice, h->stream));
    std::vector<double2> ones_n(h->N, make_double2(1.0, 1.0));  // the warp spread gathers from body order
    FBIM_CUDA_TRY(h, cudaMemcpyAsync(e.mu_r, ones_n.data(), h->N * sizeof(double2), cudaMemcpyHostToDevice, h->stream));
    FBIM_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    cudaEvent_t ev[2];
    for (auto& x : ev) FBIM_CUDA_TRY(h, cudaEventCreate(&x));
    auto spread = [&](int v) {
        if (v == 1) {
            cudaMemsetAsync(e.grid, 0, 2 * M * M * sizeof(T), h->stream);
            warp_spread<T>(h->stream, h->N, tg, ah2, g0, e.tbase, e.tfrac, e.wtab, nullptr, e.mu_r, h->tperm,
                           e.grid);
        } else {
            tile_spread<T>(h->stream, tg, ah2, g0, h->tile_start, e.tbase, e.tfrac, e.mu_t, e.grid, e.ring);
        }
    };
    auto interp = [&](int v) {
        if (v == 1)
            warp_interp<T>(h->stream, h->N, tg, ah2, g0, e.tbase, e.tfrac, e.wtab, e.grid, e.v_t);
        else
            tile_interp<T>(h->stream, tg, ah2, g0, h->tile_start, e.tbase, e.tfrac, e.grid, e.v_t);
    };
    for (int stage = 0; stage < 2; ++stage) {
        for (int v = 0; v < 2; ++v) {
            float tot = 0;
            for (int rep = 0; rep < 4; ++rep) {
                cudaEventRecord(ev[0], h->stream);
                if (stage == 0)
                    spread(v);
                else
                    interp(v);
                cudaEventRecord(ev[1], h->stream);
                cudaEventSynchronize(ev[1]);
                float ms = 0;
                cudaEventElapsedTime(&ms, ev[0], ev[1]);
                if (rep > 0) tot += ms;  // first repetition warms up
            }
            e.variant_ms[stage][v] = tot / 3;
        }
        (stage == 0 ? e.spread_variant : e.interp_variant) = e.variant_ms[stage][1] <= e.variant_ms[stage][0] ? 1 : 0;
    }
    for (auto& x : ev) cudaEventDestroy(x);
    FBIM_CUDA_TRY(h, cudaGetLastError());
    return FBIM_OK;
}

template <typename T>
fbim_status ensure_ewald(fbim_handle_s* h) {
    auto& e = bufs<T>(h);
    if (e.ready) return FBIM_OK;
    e.P = std::is_same<T, float>::value ? h->P32 : h->P;
    e.eta_s = std::is_same<T, float>::value ? h->eta_s32 : h->eta_s;
    using T2 = typename V2<T>::type;
    using C = typename Cplx<T>::type;
    const size_t N = h->N, M = h->M, Mh = h->M / 2 + 1;
    const size_t n_slice = (N + 31) / 32;
    FBIM_CUDA_TRY(h, cudaMalloc(&e.off, N * sizeof(T2)));
    FBIM_CUDA_TRY(h, cudaMalloc(&e.mu_s, N * sizeof(T2)));
    FBIM_CUDA_TRY(h, cudaMalloc(&e.v_s, N * sizeof(T2)));
    FBIM_CUDA_TRY(h, cudaMalloc(&e.tbase, N * sizeof(int2)));
    FBIM_CUDA_TRY(h, cudaMalloc(&e.tfrac, N * sizeof(T2)));
    FBIM_CUDA_TRY(h, cudaMalloc(&e.mu_t, N * sizeof(T2)));
    FBIM_CUDA_TRY(h, cudaMalloc(&e.v_t, N * sizeof(T2)));
    FBIM_CUDA_TRY(h, cudaMalloc(&e.mu_r, N * sizeof(double2)));
    FBIM_CUDA_TRY(h, cudaMalloc(&e.v_band, N * sizeof(double2)));
    {
        const size_t W = h->TS + e.P - 1;
        FBIM_CUDA_TRY(h, cudaMalloc(&e.ring, (size_t)h->n_tile * h->n_tile * 2 * W * W * sizeof(T)));
    }
    FBIM_CUDA_TRY(h, cudaMalloc(&e.grid, 2 * M * M * sizeof(T)));
    if (std::is_same<T, double>::value) FBIM_CUDA_TRY(h, cudaMalloc(&e.wtab, N * 2 * e.P * sizeof(T)));
    // the FP64 operator of an FP32 handle interpolates in float-float (weights as pairs)
    if (std::is_same<T, double>::value && h->precision == FBIM_FP32)
        FBIM_CUDA_TRY(h, cudaMalloc(&e.wtab_df, N * 2 * e.P * sizeof(float2)));
    FBIM_CUDA_TRY(h, cudaMalloc(&e.spec, 2 * M * Mh * sizeof(C)));
    FBIM_CUDA_TRY(h, cudaMalloc(&e.slice_start, scan_storage((int)n_slice) * sizeof(int)));
    FBIM_CUDA_TRY(h, cudaMalloc(&e.row_count, (n_slice * 33 + 1) * sizeof(int)));
    FBIM_CUDA_TRY(h, cudaMalloc(&e.row_of, (row_windows(N) * ROW_WINDOW + N) * sizeof(int)));
    int n[2] = {(int)M, (int)M};
    int inembed[2] = {(int)M, (int)M};
    int onembed[2] = {(int)M, (int)Mh};
    FBIM_CUFFT_TRY(h, cufftPlanMany(&e.plan_f, 2, n, inembed, 1, (int)(M * M), onembed, 1, (int)(M * Mh),
                                    FftType<T>::fwd, 2));
    FBIM_CUFFT_TRY(h, cufftPlanMany(&e.plan_i, 2, n, onembed, 1, (int)(M * Mh), inembed, 1, (int)(M * M),
                                    FftType<T>::inv, 2));
    FBIM_CUFFT_TRY(h, cufftSetStream(e.plan_f, h->stream));
    FBIM_CUFFT_TRY(h, cufftSetStream(e.plan_i, h->stream));
    FBIM_CUDA_TRY(h, tile_set_smem<T>(TileGeom{h->M, h->TS, h->n_tile, e.P, (e.P - 1) / 2}));
    if constexpr (std::is_same<T, double>::value) {
        if (h->precision == FBIM_FP32) FBIM_TRY(wfft_setup(h));
    } else {  // the FP32 operator's Alpert band in float-float
        const int n_ent = h->n_p * (2 * h->band + 1);
        FBIM_CUDA_TRY(h, cudaMalloc(&e.band_df, (size_t)n_ent * 2 * sizeof(float4)));
        FBIM_CUDA_TRY(h, cudaMalloc(&e.mu_rdf, N * sizeof(float4)));
        k_band_to_df<<<(n_ent + 255) / 256, 256, 0, h->stream>>>(n_ent, h->band_dev, e.band_df);
        h->launches += 1;
        FBIM_CUDA_TRY(h, cudaGetLastError());
    }
    e.ready = true;
    FBIM_TRY(refresh_offsets<T>(h));
    if (h->autotune == 1)
        FBIM_TRY(autotune_wave<T>(h));
    else
        e.spread_variant = e.interp_variant = h->autotune == 2 ? 1 : 0;
    return FBIM_OK;
}

// v_band = the Alpert band applied to the rotated forces: float-float for the FP32
// operator (band_df set), FP64 otherwise
template <typename T>
static void band_product(cudaStream_t st, fbim_handle_s* h, EwaldBuffers<T>& e) {
    const int N = h->N, tb = 256;
    if (e.band_df)
        k_band_df<<<(N + tb - 1) / tb, tb, 0, st>>>(N, h->n_p, h->band, h->rot, e.band_df, e.mu_rdf, e.v_band);
    else
        k_band<<<(N + tb - 1) / tb, tb, 0, st>>>(N, h->n_p, h->band, h->rot, h->band_dev, e.mu_r, e.v_band);
}

// v_s = (real-space pair list) mu_s, on the plain or the float-float list
template <typename T>
static void pair_product(cudaStream_t st, int N, EwaldBuffers<T>& e, bool df) {
    using T2 = typename V2<T>::type;
    if (df)
        k_pair_spmv_df<<<(N + 63) / 64, 64, 0, st>>>(N, e.slice_start, e.row_of, (const PairEntryDF*)e.pairs,
                                                     e.mu_df, (double2*)e.v_s);
    else
        k_pair_spmv<T><<<(N + 31) / 32, 32 * SPMV_P, 0, st>>>(N, e.slice_start, e.row_of,
                                                              (const PairEntry<T>*)e.pairs, (const T2*)e.mu_s,
                                                              (T2*)e.v_s);
}

template <typename T>
fbim_status apply_operator(fbim_handle_s* h, const double* mu, double* v, int which) {
    FBIM_TRY(ensure_ewald<T>(h));
    auto& e = bufs<T>(h);
    using T2 = typename V2<T>::type;
    using C = typename Cplx<T>::type;
    const int N = h->N, tb = 256;
    const bool real = which & 1, wave = which & 2;
    h->mark_begin();
    const bool df = real && e.pairs_df;  // float-float FP64 list (FP32 handles)
    // real space on the auxiliary stream, concurrent with the wave space (sequential
    // while the stage timers run, so that each stage is timed alone)
    const bool fork = real && wave && h->aux && !h->timing;
    // the warp spread gathers its forces itself; the warp interpolation writes the sum in
    // body order itself (after the real space has joined), so gather and finish drop out
    const bool spread_gathers = wave && e.spread_variant == 1;
    // the FP64 operator of an FP32 handle: float-float transforms and scale, and the
    // float-float interpolation from the transform's float-float output
    bool own_fft = false;
    if constexpr (std::is_same<T, double>::value) own_fft = wave && h->fft64.state == 1;
    const bool df_interp = own_fft && e.wtab_df;
    const bool fused_out = wave && (e.interp_variant == 1 || df_interp) && !h->timing && (fork || !real);
    const cudaStream_t rs = fork ? h->aux : h->stream;
    if (fork) {
        FBIM_CUDA_TRY(h, cudaEventRecord(h->ev_fork, h->stream));
        FBIM_CUDA_TRY(h, cudaStreamWaitEvent(h->aux, h->ev_fork, 0));
    }
    int n_launch = 0;
    if (real) {
        k_gather<T><<<(N + tb - 1) / tb, tb, 0, rs>>>(N, h->n_p, h->perm, h->tperm, 1, 0, h->rot,
                                                      (const double2*)mu, (T2*)e.mu_s, (T2*)e.mu_t, e.mu_r,
                                                      df ? e.mu_df : nullptr, e.mu_rdf);
        ++n_launch;
    }
    if (wave && !spread_gathers) {
        k_gather<T><<<(N + tb - 1) / tb, tb, 0, h->stream>>>(N, h->n_p, h->perm, h->tperm, 0, 1, h->rot,
                                                             (const double2*)mu, (T2*)e.mu_s, (T2*)e.mu_t, e.mu_r,
                                                             nullptr, nullptr);
        ++n_launch;
    }
    h->mark(FBIM_ST_GATHER);
    if (fork) {
        pair_product<T>(h->aux, N, e, df);
        band_product<T>(h->aux, h, e);
        FBIM_CUDA_TRY(h, cudaEventRecord(h->ev_join, h->aux));
    }
    const TileGeom tg{h->M, h->TS, h->n_tile, e.P, (e.P - 1) / 2};
    const double alpha = 2.0 * h->xi * h->xi / e.eta_s;
    const T ah2 = (T)(alpha * h->h * h->h);
    const T g0 = (T)(2.0 * h->xi * h->xi / (M_PI * e.eta_s));
    if (wave) {
        const size_t M = h->M, Mh = h->M / 2 + 1;
        if (e.spread_variant == 1) {
            FBIM_CUDA_TRY(h, cudaMemsetAsync(e.grid, 0, 2 * M * M * sizeof(T), h->stream));
            warp_spread<T>(h->stream, N, tg, ah2, g0, e.tbase, e.tfrac, e.wtab, nullptr, (const double2*)mu,
                           h->tperm, e.grid);
        } else {
            tile_spread<T>(h->stream, tg, ah2, g0, h->tile_start, e.tbase, e.tfrac, e.mu_t, e.grid, e.ring);
        }
        h->mark(FBIM_ST_SPREAD);
        if constexpr (std::is_same<T, double>::value) {
            if (own_fft) {
                wfft_forward(h, h->stream, e.grid);
                h->mark(FBIM_ST_FFT_F);
                wfft_scale(h, h->stream);
                h->mark(FBIM_ST_SCALE);
                wfft_inverse(h, h->stream, e.grid, df_interp);
                h->mark(FBIM_ST_FFT_I);
                h->launches += 2;
            }
        }
        if (!own_fft) {
            FBIM_CUFFT_TRY(h, FftType<T>::f(e.plan_f, e.grid, (C*)e.spec));
            h->mark(FBIM_ST_FFT_F);
            const double V = h->L * h->L;
            const double h4 = h->h * h->h * h->h * h->h;
            size_t ns = M * Mh;
            k_scale<T><<<(unsigned)((ns + tb - 1) / tb), tb, 0, h->stream>>>(
                (int)M, (T)(2.0 * M_PI / h->L), (T)(1.0 / (4.0 * h->xi * h->xi)), (T)(1.0 - e.eta_s),
                (T)(h4 / (h->eta * V)), (C*)e.spec);
            h->mark(FBIM_ST_SCALE);
            FBIM_CUFFT_TRY(h, FftType<T>::i(e.plan_i, (C*)e.spec, e.grid));
            h->mark(FBIM_ST_FFT_I);
        }
    }
    if (real && !fork) {
        pair_product<T>(h->stream, N, e, df);
        h->mark(FBIM_ST_PAIRS);
    }
    if (wave) {
        // warp interpolation, in float-float for the FP64 operator of an FP32 handle
        auto warp_interp_any = [&](const InterpEpilogue<T>& ep) {
            if constexpr (std::is_same<T, double>::value) {
                if (df_interp) {
                    interp_df(h->stream, N, tg, e.tbase, e.wtab_df, e.grid, e.v_t, ep);
                    return;
                }
            }
            warp_interp<T>(h->stream, N, tg, ah2, g0, e.tbase, e.tfrac, e.wtab, e.grid, e.v_t, ep);
        };
        if (fused_out) {
            if (fork) FBIM_CUDA_TRY(h, cudaStreamWaitEvent(h->stream, h->ev_join, 0));
            InterpEpilogue<T> ep;
            ep.v = (double2*)v;
            ep.tperm = h->tperm;
            if (real) {
                ep.slot = h->slot;
                ep.v_s = (const T2*)e.v_s;
                ep.v_band = e.v_band;
            }
            warp_interp_any(ep);
        } else if (df_interp) {
            warp_interp_any(InterpEpilogue<T>());
        } else if (e.interp_variant == 1) {
            warp_interp<T>(h->stream, N, tg, ah2, g0, e.tbase, e.tfrac, e.wtab, e.grid, e.v_t);
        } else {
            tile_interp<T>(h->stream, tg, ah2, g0, h->tile_start, e.tbase, e.tfrac, e.grid, e.v_t);
        }
        h->mark(FBIM_ST_INTERP);
    }
    if (!fused_out) {
        if (fork) FBIM_CUDA_TRY(h, cudaStreamWaitEvent(h->stream, h->ev_join, 0));
        if (real && !fork)
            band_product<T>(h->stream, h, e);
        k_finish<T><<<(N + tb - 1) / tb, tb, 0, h->stream>>>(N, real ? 1 : 0, wave ? 1 : 0, h->slot, h->tslot,
                                                             (const T2*)e.v_s, (const T2*)e.v_t, e.v_band,
                                                             (double2*)v);
        ++n_launch;
    }
    h->mark(FBIM_ST_FINISH);
    h->launches += n_launch + (wave ? (e.spread_variant == 1 ? 3 : 4) : 0) + (real ? 2 : 0);
    FBIM_CUDA_TRY(h, cudaGetLastError());
    h->collect();
    return FBIM_OK;
}


// ---------------------------------------------------------------------------
// Far-field noise (Sec. 3.3, Eq. sqrtMwave): (M(w))^1/2 W(w) = S* F* C* B^1/2 W(w).
// The half spectrum is filled directly with
//   u(k) = h^2 (eta V)^-1/2 (1 + k^2/4xi^2)^1/2 e^{-(1 - eta_s) k^2/8xi^2} / k (I - k k^T/k^2) W(kappa)
// (B^1/2 with one Gaussian deconvolution and the interpolation weight h^2), then
// inverse FFT and interpolation.  W(kappa) follows the Hermitian layout of the
// oracle: of each conjugate pair the member with the smaller index j_y M + j_x
// (j = kappa mod M) takes (Z[..][0] + i Z[..][1]) / sqrt 2, the other its conjugate;
// kappa = 0 and the Nyquist lines are zero (their Hasimoto weight is below the
// tolerance by the grid rule).  Z[j_y][j_x][comp][re/im] are standard normals,
// given by the caller or drawn from Philox stream 1 at index
// ((j_y M + j_x) 2 + comp) 2 + re/im.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_noise_spec(int M, T twopi_L, T inv4xi2, T one_minus_eta, T pref, const double* __restrict__ Z,
                             unsigned long long seed, unsigned counter, typename Cplx<T>::type* __restrict__ spec) {
    const int Mh = M / 2 + 1;
    const size_t n = (size_t)M * Mh;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int r = (int)(i / Mh), c = (int)(i - (size_t)r * Mh);
    typename Cplx<T>::type* ux = spec;
    typename Cplx<T>::type* uy = spec + n;
    if ((r == 0 && c == 0) || c == M / 2 || r == M / 2) {
        ux[i].x = ux[i].y = T(0);
        uy[i].x = uy[i].y = T(0);
        return;
    }
    // canonical member of the conjugate pair {(r, c), (-r mod M, -c mod M)}
    int jy = r, jx = c;
    double sg = 1.0;
    if (r > M / 2) {
        jy = M - r;
        jx = (M - c) % M;
        sg = -1.0;
    }
    double zr[2], zi[2];
    const size_t base = (size_t)jy * M + jx;
    if (Z) {
        const double* z = Z + base * 4;
        zr[0] = z[0];
        zi[0] = z[1];
        zr[1] = z[2];
        zi[1] = z[3];
    } else if constexpr (std::is_same<T, float>::value) {
        const float2 a = philox_normals_f(seed, 1u, counter, base * 2);
        const float2 b = philox_normals_f(seed, 1u, counter, base * 2 + 1);
        zr[0] = a.x;
        zi[0] = a.y;
        zr[1] = b.x;
        zi[1] = b.y;
    } else {
        double2 a = philox_normals(seed, 1u, counter, base * 2);
        double2 b = philox_normals(seed, 1u, counter, base * 2 + 1);
        zr[0] = a.x;
        zi[0] = a.y;
        zr[1] = b.x;
        zi[1] = b.y;
    }
    const double is2 = 0.70710678118654752440;
    const T wxr = (T)(zr[0] * is2), wxi = (T)(sg * zi[0] * is2);
    const T wyr = (T)(zr[1] * is2), wyi = (T)(sg * zi[1] * is2);
    const int ky_i = r < M / 2 ? r : r - M;
    const T kx = twopi_L * T(c), ky = twopi_L * T(ky_i);
    const T k2 = kx * kx + ky * ky;
    const T ik2 = T(1) / k2;
    const T q = k2 * inv4xi2;
    const T sc = pref * sqrt((T(1) + q) * ik2) * dev_exp(T(-0.5) * one_minus_eta * q);
    const T pxx = T(1) - kx * kx * ik2, pyy = T(1) - ky * ky * ik2, pxy = -kx * ky * ik2;
    ux[i].x = sc * (pxx * wxr + pxy * wyr);
    ux[i].y = sc * (pxx * wxi + pxy * wyi);
    uy[i].x = sc * (pxy * wxr + pyy * wyr);
    uy[i].y = sc * (pxy * wxi + pyy * wyi);
}

template <typename T>
fbim_status apply_noise(fbim_handle_s* h, const double* Z, unsigned long long seed, unsigned counter, double* out) {
    FBIM_TRY(ensure_ewald<T>(h));
    auto& e = bufs<T>(h);
    using T2 = typename V2<T>::type;
    using C = typename Cplx<T>::type;
    const int N = h->N, tb = 256;
    const size_t M = h->M, Mh = h->M / 2 + 1, ns = M * Mh;
    const double V = h->L * h->L;
    k_noise_spec<T><<<(unsigned)((ns + tb - 1) / tb), tb, 0, h->stream>>>(
        (int)M, (T)(2.0 * M_PI / h->L), (T)(1.0 / (4.0 * h->xi * h->xi)), (T)(1.0 - e.eta_s),
        (T)(h->h * h->h / std::sqrt(h->eta * V)), Z, seed, counter, (C*)e.spec);
    FBIM_CUFFT_TRY(h, FftType<T>::i(e.plan_i, (C*)e.spec, e.grid));
    const TileGeom tg{h->M, h->TS, h->n_tile, e.P, (e.P - 1) / 2};
    const double alpha = 2.0 * h->xi * h->xi / e.eta_s;
    const T ah2 = (T)(alpha * h->h * h->h);
    const T g0 = (T)(2.0 * h->xi * h->xi / (M_PI * e.eta_s));
    if (e.interp_variant == 1)
        warp_interp<T>(h->stream, N, tg, ah2, g0, e.tbase, e.tfrac, e.wtab, e.grid, e.v_t);
    else
        tile_interp<T>(h->stream, tg, ah2, g0, h->tile_start, e.tbase, e.tfrac, e.grid, e.v_t);
    k_finish<T><<<(N + tb - 1) / tb, tb, 0, h->stream>>>(N, 0, 1, h->slot, h->tslot, (const T2*)e.v_s,
                                                         (const T2*)e.v_t, e.v_band, (double2*)out);
    h->launches += 3;
    FBIM_CUDA_TRY(h, cudaGetLastError());
    return FBIM_OK;
}

template <typename T>
static void free_one(EwaldBuffers<T>& e) {
    cudaFree(e.off);
    cudaFree(e.mu_s);
    cudaFree(e.v_s);
    cudaFree(e.tbase);
    cudaFree(e.tfrac);
    cudaFree(e.mu_t);
    cudaFree(e.v_t);
    cudaFree(e.mu_r);
    cudaFree(e.v_band);
    cudaFree(e.ring);
    cudaFree(e.grid);
    cudaFree(e.wtab);
    cudaFree(e.wtab_df);
    cudaFree(e.spec);
    cudaFree(e.pairs);
    cudaFree(e.off_df);
    cudaFree(e.mu_df);
    cudaFree(e.band_df);
    cudaFree(e.mu_rdf);
    cudaFree(e.pw);
    cudaFree(e.slice_start);
    cudaFree(e.row_count);
    cudaFree(e.row_of);
    if (e.plan_f) cufftDestroy(e.plan_f);
    if (e.plan_i) cufftDestroy(e.plan_i);
    e = EwaldBuffers<T>();
}

void free_ewald(fbim_handle_s* h) {
    free_one(h->e64);
    free_one(h->e32);
    wfft_free(h);
}

template fbim_status ensure_ewald<double>(fbim_handle_s*);
template fbim_status ensure_ewald<float>(fbim_handle_s*);
template fbim_status refresh_offsets<double>(fbim_handle_s*);
template fbim_status refresh_offsets<float>(fbim_handle_s*);
template fbim_status apply_operator<double>(fbim_handle_s*, const double*, double*, int);
template fbim_status apply_operator<float>(fbim_handle_s*, const double*, double*, int);
template fbim_status apply_noise<double>(fbim_handle_s*, const double*, unsigned long long, unsigned, double*);
template fbim_status apply_noise<float>(fbim_handle_s*, const double*, unsigned long long, unsigned, double*);

}  // namespace fbim
