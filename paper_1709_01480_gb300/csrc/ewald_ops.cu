// The positively split Ewald matvec v = M mu = (M(t) + M(a)_sym + M(w)) mu (Sec. 3.2).
//
//   real space   M(t): cell-list pair sum of G^(r)_xi over the 9 neighbour cells
//                (Sec. 3.2, Eqs. real-space-kernel, expint), r < r_c, m != n;
//                M(a): per-body band R_beta M(a)_ref R_beta^T, FP64 always.
//   wave space   M(w) = D* B D with D = C F S (Sec. 3.2, Eq. Mwave-factorization):
//                Gaussian spread S, forward FFT F, the Hasimoto tensor B with both
//                deconvolutions C folded in, inverse FFT, Gaussian interpolation S*.
//
// All node-indexed work runs in cell-sorted order (slot s holds node perm[s]);
// the final kernel scatters back to body order and adds the Alpert band.
// Templated on the operator precision T (double: parity path; float: fast path).
#include <cmath>

#include "fbim_internal.h"

namespace fbim {

template <typename T> struct V2;
template <> struct V2<double> { using type = double2; };
template <> struct V2<float> { using type = float2; };

template <typename T> struct Cplx;
template <> struct Cplx<double> { using type = cufftDoubleComplex; };
template <> struct Cplx<float> { using type = cufftComplex; };

// ---------------------------------------------------------------------------
// E1(z) for z > 0 on the device: power series below z0, bottom-up continued
// fraction e^{-z}/(z + 1 - 1/(z + 3 - 4/(z + 5 - ...))) above (the classical
// expansions, Abramowitz & Stegun 5.1.11 and 5.1.22).  Term counts are fixed
// per precision: relative error <= 1e-13 (double) and <= 2e-7 (float).
// ---------------------------------------------------------------------------
template <typename T> struct E1Cfg;
template <> struct E1Cfg<double> { static constexpr double z0 = 3.0; static constexpr int ns = 36, nc = 26; };
template <> struct E1Cfg<float> { static constexpr float z0 = 2.0f; static constexpr int ns = 14, nc = 12; };

__device__ __forceinline__ double dev_exp(double a) { return exp(a); }
__device__ __forceinline__ float dev_exp(float a) { return __expf(a); }
__device__ __forceinline__ double dev_log(double a) { return log(a); }
__device__ __forceinline__ float dev_log(float a) { return __logf(a); }

template <typename T>
__device__ __forceinline__ T e1_times_half_minus_exp(T z, T& e_out) {
    // returns E1(z)/2 - e^{-z}; e_out = e^{-z}
    T e = dev_exp(-z);
    e_out = e;
    T r;
    if (z < E1Cfg<T>::z0) {
        T term = T(1), sum = T(0);
#pragma unroll
        for (int k = 1; k <= E1Cfg<T>::ns; ++k) {
            term *= -z / T(k);
            sum += term / T(k);
        }
        r = T(-0.57721566490153286061) - dev_log(z) - sum;
    } else {
        T f = z + T(2 * E1Cfg<T>::nc + 1);
#pragma unroll
        for (int k = E1Cfg<T>::nc; k >= 1; --k) f = z + T(2 * k - 1) - T(k * k) / f;
        r = e / f;
    }
    return T(0.5) * r - e;
}

// ---------------------------------------------------------------------------
// Layout kernels
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_offsets(int N, const int* __restrict__ perm, const double* __restrict__ x,
                          const int* __restrict__ cell, int n_box, double r_c, double h, int M,
                          typename V2<T>::type* __restrict__ off, int2* __restrict__ gbase,
                          typename V2<T>::type* __restrict__ gfrac) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= N) return;
    int m = perm[s];
    double px = x[2 * m], py = x[2 * m + 1];
    int c = cell[m];
    int cx = c % n_box, cy = c / n_box;
    off[s].x = (T)(px - cx * r_c);
    off[s].y = (T)(py - cy * r_c);
    double gx = px / h, gy = py / h;
    double bx = rint(gx), by = rint(gy);
    gbase[s] = make_int2(((int)bx) % M, ((int)by) % M);
    gfrac[s].x = (T)(gx - bx);
    gfrac[s].y = (T)(gy - by);
}

template <typename T>
__global__ void k_gather(int N, const int* __restrict__ perm, const double2* __restrict__ mu,
                         typename V2<T>::type* __restrict__ mu_s) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= N) return;
    double2 v = mu[perm[s]];
    mu_s[s].x = (T)v.x;
    mu_s[s].y = (T)v.y;
}

// ---------------------------------------------------------------------------
// Real space: v_t = sum_{n != t, r < r_c} G^(r)(x_t - x_n) mu_n over the 9 cells
// around t's cell.  One thread per target in cell-sorted order: neighbouring
// threads share most source cells, which stay in L1.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(128) k_pairs(int N, int n_box, T r_c, T rc2, T xi2, T pref,
                                              const int* __restrict__ perm, const int* __restrict__ cell,
                                              const int* __restrict__ start,
                                              const typename V2<T>::type* __restrict__ off,
                                              const typename V2<T>::type* __restrict__ mu_s,
                                              typename V2<T>::type* __restrict__ v_s, int* __restrict__ flags) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N) return;
    int c = cell[perm[t]];
    int cx = c % n_box, cy = c / n_box;
    typename V2<T>::type ot = off[t];
    T ax = 0, ay = 0;
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
                if (r2 < rc2 && s != t) {
                    if (r2 == T(0)) {
                        atomicOr(&flags[1], 1);
                        continue;
                    }
                    T e;
                    T a = e1_times_half_minus_exp<T>(xi2 * r2, e);
                    T b = e / r2;
                    typename V2<T>::type ms = mu_s[s];
                    T rm = rx * ms.x + ry * ms.y;
                    ax += a * ms.x + b * rx * rm;
                    ay += a * ms.y + b * ry * rm;
                }
            }
        }
    }
    v_s[t].x = pref * ax;
    v_s[t].y = pref * ay;
}

// ---------------------------------------------------------------------------
// Wave space
// ---------------------------------------------------------------------------
// Spread: grid_c(y) += g(y - x_n) mu_{n,c}, g(r) = (2 xi^2/(pi eta_s)) exp(-2 xi^2 r^2/eta_s),
// over the P x P grid points nearest to x_n (Sec. 3.2, the Gaussian spreading S).
template <typename T, int PMAX>
__global__ void __launch_bounds__(128) k_spread(int N, int M, int P, T alpha_h2, T g0,
                                               const int2* __restrict__ gbase,
                                               const typename V2<T>::type* __restrict__ gfrac,
                                               const typename V2<T>::type* __restrict__ mu_s,
                                               T* __restrict__ grid) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= N) return;
    int2 b = gbase[s];
    typename V2<T>::type f = gfrac[s];
    typename V2<T>::type mu = mu_s[s];
    const int hw = (P - 1) / 2;
    T wx[PMAX], wy[PMAX];
    for (int p = 0; p < P; ++p) {
        T dx = T(p - hw) - f.x, dy = T(p - hw) - f.y;
        wx[p] = dev_exp(-alpha_h2 * dx * dx);
        wy[p] = g0 * dev_exp(-alpha_h2 * dy * dy);
    }
    T* gx = grid;
    T* gy = grid + (size_t)M * M;
    for (int q = 0; q < P; ++q) {
        int iy = b.y + q - hw;
        iy += (iy < 0) ? M : 0;
        iy -= (iy >= M) ? M : 0;
        T wyq = wy[q];
        for (int p = 0; p < P; ++p) {
            int ix = b.x + p - hw;
            ix += (ix < 0) ? M : 0;
            ix -= (ix >= M) ? M : 0;
            T w = wyq * wx[p];
            size_t idx = (size_t)iy * M + ix;
            atomicAdd(&gx[idx], w * mu.x);
            atomicAdd(&gy[idx], w * mu.y);
        }
    }
}

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
    T q = k2 * inv4xi2;
    T sc = pref * (T(1) + q) * dev_exp(-one_minus_eta * q) / k2;
    T pxx = T(1) - kx * kx / k2, pyy = T(1) - ky * ky / k2, pxy = -kx * ky / k2;
    typename Cplx<T>::type a = ux[i], b = uy[i];
    ux[i].x = sc * (pxx * a.x + pxy * b.x);
    ux[i].y = sc * (pxx * a.y + pxy * b.y);
    uy[i].x = sc * (pxy * a.x + pyy * b.x);
    uy[i].y = sc * (pxy * a.y + pyy * b.y);
}

// Interpolation: v_t (+)= sum_{P x P} g(x_t - y) U(y) (the h^2 weight is in k_scale).
template <typename T, int PMAX>
__global__ void __launch_bounds__(128) k_interp(int N, int M, int P, T alpha_h2, T g0, int accumulate,
                                               const int2* __restrict__ gbase,
                                               const typename V2<T>::type* __restrict__ gfrac,
                                               const T* __restrict__ grid,
                                               typename V2<T>::type* __restrict__ v_s) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= N) return;
    int2 b = gbase[s];
    typename V2<T>::type f = gfrac[s];
    const int hw = (P - 1) / 2;
    T wx[PMAX], wy[PMAX];
    for (int p = 0; p < P; ++p) {
        T dx = T(p - hw) - f.x, dy = T(p - hw) - f.y;
        wx[p] = dev_exp(-alpha_h2 * dx * dx);
        wy[p] = g0 * dev_exp(-alpha_h2 * dy * dy);
    }
    const T* gx = grid;
    const T* gy = grid + (size_t)M * M;
    T ax = 0, ay = 0;
    for (int q = 0; q < P; ++q) {
        int iy = b.y + q - hw;
        iy += (iy < 0) ? M : 0;
        iy -= (iy >= M) ? M : 0;
        T rx = 0, ry = 0;
        for (int p = 0; p < P; ++p) {
            int ix = b.x + p - hw;
            ix += (ix < 0) ? M : 0;
            ix -= (ix >= M) ? M : 0;
            size_t idx = (size_t)iy * M + ix;
            rx += wx[p] * gx[idx];
            ry += wx[p] * gy[idx];
        }
        ax += wy[q] * rx;
        ay += wy[q] * ry;
    }
    if (accumulate) {
        v_s[s].x += ax;
        v_s[s].y += ay;
    } else {
        v_s[s].x = ax;
        v_s[s].y = ay;
    }
}

// Back to body order, plus the Alpert band: v_m = v_s[slot[m]] + R_b A_ref[j] R_b^T mu (FP64).
template <typename T>
__global__ void k_finish(int N, int n_p, int band, int with_alpert, const int* __restrict__ slot,
                         const typename V2<T>::type* __restrict__ v_s, const double* __restrict__ Q,
                         const double* __restrict__ A, const double2* __restrict__ mu,
                         double2* __restrict__ v) {
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= N) return;
    typename V2<T>::type w = v_s[slot[m]];
    double vx = (double)w.x, vy = (double)w.y;
    if (with_alpert) {
        int b = m / n_p, j = m - b * n_p;
        double c, s;
        sincos(Q[3 * b + 2], &s, &c);
        double ax = 0, ay = 0;
        const int B = 2 * band + 1;
        for (int o = -band; o <= band; ++o) {
            int jj = j + o;
            jj += (jj < 0) ? n_p : 0;
            jj -= (jj >= n_p) ? n_p : 0;
            double2 u = mu[b * n_p + jj];
            // rotate into the reference frame: R^T u
            double rx = c * u.x + s * u.y, ry = -s * u.x + c * u.y;
            const double* a = A + ((size_t)j * B + (o + band)) * 4;
            ax += a[0] * rx + a[1] * ry;
            ay += a[2] * rx + a[3] * ry;
        }
        vx += c * ax - s * ay;
        vy += s * ax + c * ay;
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

template <typename T>
fbim_status refresh_offsets(fbim_handle_s* h) {
    auto& e = bufs<T>(h);
    using T2 = typename V2<T>::type;
    const int tb = 256;
    k_offsets<T><<<(h->N + tb - 1) / tb, tb, 0, h->stream>>>(h->N, h->perm, h->x, h->cell, h->n_box, h->r_c, h->h,
                                                             h->M, (T2*)e.off, e.gbase, (T2*)e.gfrac);
    FBIM_CUDA_TRY(h, cudaGetLastError());
    return FBIM_OK;
}

template <typename T>
fbim_status ensure_ewald(fbim_handle_s* h) {
    auto& e = bufs<T>(h);
    if (e.ready) return FBIM_OK;
    using T2 = typename V2<T>::type;
    using C = typename Cplx<T>::type;
    const size_t N = h->N, M = h->M, Mh = h->M / 2 + 1;
    FBIM_CUDA_TRY(h, cudaMalloc(&e.off, N * sizeof(T2)));
    FBIM_CUDA_TRY(h, cudaMalloc(&e.gbase, N * sizeof(int2)));
    FBIM_CUDA_TRY(h, cudaMalloc(&e.gfrac, N * sizeof(T2)));
    FBIM_CUDA_TRY(h, cudaMalloc(&e.mu_s, N * sizeof(T2)));
    FBIM_CUDA_TRY(h, cudaMalloc(&e.v_s, N * sizeof(T2)));
    FBIM_CUDA_TRY(h, cudaMalloc(&e.grid, 2 * M * M * sizeof(T)));
    FBIM_CUDA_TRY(h, cudaMalloc(&e.spec, 2 * M * Mh * sizeof(C)));
    int n[2] = {(int)M, (int)M};
    int inembed[2] = {(int)M, (int)M};
    int onembed[2] = {(int)M, (int)Mh};
    FBIM_CUFFT_TRY(h, cufftPlanMany(&e.plan_f, 2, n, inembed, 1, (int)(M * M), onembed, 1, (int)(M * Mh),
                                    FftType<T>::fwd, 2));
    FBIM_CUFFT_TRY(h, cufftPlanMany(&e.plan_i, 2, n, onembed, 1, (int)(M * Mh), inembed, 1, (int)(M * M),
                                    FftType<T>::inv, 2));
    FBIM_CUFFT_TRY(h, cufftSetStream(e.plan_f, h->stream));
    FBIM_CUFFT_TRY(h, cufftSetStream(e.plan_i, h->stream));
    e.ready = true;
    return refresh_offsets<T>(h);
}

template <typename T, int PMAX>
static void launch_spread(fbim_handle_s* h, EwaldBuffers<T>& e, T ah2, T g0) {
    using T2 = typename V2<T>::type;
    const int tb = 128;
    k_spread<T, PMAX><<<(h->N + tb - 1) / tb, tb, 0, h->stream>>>(h->N, h->M, h->P, ah2, g0, e.gbase,
                                                                  (const T2*)e.gfrac, (const T2*)e.mu_s, e.grid);
}

template <typename T, int PMAX>
static void launch_interp(fbim_handle_s* h, EwaldBuffers<T>& e, T ah2, T g0, int acc) {
    using T2 = typename V2<T>::type;
    const int tb = 128;
    k_interp<T, PMAX><<<(h->N + tb - 1) / tb, tb, 0, h->stream>>>(h->N, h->M, h->P, ah2, g0, acc, e.gbase,
                                                                   (const T2*)e.gfrac, e.grid, (T2*)e.v_s);
}

template <typename T>
fbim_status apply_operator(fbim_handle_s* h, const double* mu, double* v, int which) {
    FBIM_TRY(ensure_ewald<T>(h));
    auto& e = bufs<T>(h);
    using T2 = typename V2<T>::type;
    using C = typename Cplx<T>::type;
    const int N = h->N, tb = 256;
    h->mark_begin();
    k_gather<T><<<(N + tb - 1) / tb, tb, 0, h->stream>>>(N, h->perm, (const double2*)mu, (T2*)e.mu_s);
    h->mark(FBIM_ST_GATHER);
    const bool real = which & 1, wave = which & 2;
    if (wave) {
        const size_t M = h->M, Mh = h->M / 2 + 1;
        FBIM_CUDA_TRY(h, cudaMemsetAsync(e.grid, 0, 2 * M * M * sizeof(T), h->stream));
        const double alpha = 2.0 * h->xi * h->xi / h->eta_s;
        const T ah2 = (T)(alpha * h->h * h->h);
        const T g0 = (T)(2.0 * h->xi * h->xi / (M_PI * h->eta_s));
        if (h->P <= 15)
            launch_spread<T, 15>(h, e, ah2, g0);
        else if (h->P <= 23)
            launch_spread<T, 23>(h, e, ah2, g0);
        else
            launch_spread<T, 31>(h, e, ah2, g0);
        h->mark(FBIM_ST_SPREAD);
        FBIM_CUFFT_TRY(h, FftType<T>::f(e.plan_f, e.grid, (C*)e.spec));
        h->mark(FBIM_ST_FFT_F);
        const double V = h->L * h->L;
        const double h4 = h->h * h->h * h->h * h->h;
        size_t ns = M * Mh;
        k_scale<T><<<(unsigned)((ns + tb - 1) / tb), tb, 0, h->stream>>>(
            (int)M, (T)(2.0 * M_PI / h->L), (T)(1.0 / (4.0 * h->xi * h->xi)), (T)(1.0 - h->eta_s),
            (T)(h4 / (h->eta * V)), (C*)e.spec);
        h->mark(FBIM_ST_SCALE);
        FBIM_CUFFT_TRY(h, FftType<T>::i(e.plan_i, (C*)e.spec, e.grid));
        h->mark(FBIM_ST_FFT_I);
    }
    if (real) {
        const T pref = (T)(1.0 / (4.0 * M_PI * h->eta));
        k_pairs<T><<<(N + 127) / 128, 128, 0, h->stream>>>(N, h->n_box, (T)h->r_c, (T)(h->r_c * h->r_c),
                                                           (T)(h->xi * h->xi), pref, h->perm, h->cell,
                                                           h->cell_start, (const T2*)e.off, (const T2*)e.mu_s,
                                                           (T2*)e.v_s, h->flags);
        h->mark(FBIM_ST_PAIRS);
    }
    if (wave) {
        const double alpha = 2.0 * h->xi * h->xi / h->eta_s;
        const T ah2 = (T)(alpha * h->h * h->h);
        const T g0 = (T)(2.0 * h->xi * h->xi / (M_PI * h->eta_s));
        int acc = real ? 1 : 0;
        if (h->P <= 15)
            launch_interp<T, 15>(h, e, ah2, g0, acc);
        else if (h->P <= 23)
            launch_interp<T, 23>(h, e, ah2, g0, acc);
        else
            launch_interp<T, 31>(h, e, ah2, g0, acc);
        h->mark(FBIM_ST_INTERP);
    }
    if (!real && !wave) FBIM_CUDA_TRY(h, cudaMemsetAsync(e.v_s, 0, N * sizeof(T2), h->stream));
    k_finish<T><<<(N + tb - 1) / tb, tb, 0, h->stream>>>(N, h->n_p, h->band, real ? 1 : 0, h->slot,
                                                         (const T2*)e.v_s, h->Q, h->band_dev,
                                                         (const double2*)mu, (double2*)v);
    h->mark(FBIM_ST_FINISH);
    FBIM_CUDA_TRY(h, cudaGetLastError());
    h->collect();
    return FBIM_OK;
}

template <typename T>
static void free_one(EwaldBuffers<T>& e) {
    cudaFree(e.off);
    cudaFree(e.gbase);
    cudaFree(e.gfrac);
    cudaFree(e.mu_s);
    cudaFree(e.v_s);
    cudaFree(e.grid);
    cudaFree(e.spec);
    if (e.plan_f) cufftDestroy(e.plan_f);
    if (e.plan_i) cufftDestroy(e.plan_i);
    e = EwaldBuffers<T>();
}

void free_ewald(fbim_handle_s* h) {
    free_one(h->e64);
    free_one(h->e32);
}

template fbim_status ensure_ewald<double>(fbim_handle_s*);
template fbim_status ensure_ewald<float>(fbim_handle_s*);
template fbim_status refresh_offsets<double>(fbim_handle_s*);
template fbim_status refresh_offsets<float>(fbim_handle_s*);
template fbim_status apply_operator<double>(fbim_handle_s*, const double*, double*, int);
template fbim_status apply_operator<float>(fbim_handle_s*, const double*, double*, int);

}  // namespace fbim
