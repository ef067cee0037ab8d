// Wave space of the FP64 residual operator of an FP32 handle in float-float
// arithmetic: the FFTs and the Fourier scale between them (Sec. 3.2), about 48-bit
// accurate, on the FP32 pipes (GB300 runs FP32 at ~74x its FP64 rate, where cuFFT's
// double transforms spend most of the residual's time).
//
// The two real grid components g0, g1 are packed into one complex field
// z = g0 + i g1 and transformed with one complex 2D FFT, Z = F z.  The scale
// u(k) = sc(k) (I - k k^T/k^2) g^(k) becomes, per pair (k, -k),
//     Z'(k) = s(k) [Z(k) - e^{2 i theta_k} conj(Z(-k))],   s = sc/2,
// where e^{i theta_k} = (k_x + i k_y)/|k| (the trace of I - k k^T/k^2 is 1 in 2D),
// and F^{-1} Z' = u0 + i u1.  k = 0 and the Nyquist lines are zeroed, as in the
// half-spectrum path.  Transforms are unnormalised, like cuFFT's.
//
// Three kernels, each owning two grid lines per CTA in shared memory:
//   x pass:  grid rows y            -> FFT over x -> T1[k_x][y]   (transposed store)
//   y pass:  T1 rows k_x and -k_x   -> FFT over y, scale, inverse FFT over y
//                                   -> T2[y][k_x]                 (transposed store)
//   x pass:  T2 rows y              -> inverse FFT over x -> grid rows y (FP64)
// Each 1D transform is a Stockham autosort FFT (radix 4, 2, 3, 5 passes, natural
// order in and out) between two shared-memory buffers; twiddles e^{-2 pi i m/M}
// come from a float-float table.  M must be even, 5-smooth and fit the shared
// memory (64 M bytes per CTA); otherwise the caller keeps cuFFT.
#include <cmath>
#include <vector>

#include "dfloat.cuh"
#include "fbim_internal.h"

namespace fbim {

namespace {

using dfl::df;

struct cdf {
    df re, im;
};

__device__ __forceinline__ cdf ldc(const float4 v) { return {{v.x, v.y}, {v.z, v.w}}; }
__device__ __forceinline__ float4 stc(const cdf a) { return make_float4(a.re.hi, a.re.lo, a.im.hi, a.im.lo); }
__device__ __forceinline__ cdf cadd(cdf a, cdf b) { return {dfl::add_fast(a.re, b.re), dfl::add_fast(a.im, b.im)}; }
__device__ __forceinline__ cdf csub(cdf a, cdf b) {
    return {dfl::add_fast(a.re, dfl::neg(b.re)), dfl::add_fast(a.im, dfl::neg(b.im))};
}
__device__ __forceinline__ cdf cmul(cdf a, cdf b) {
    return {dfl::add_fast(dfl::mul(a.re, b.re), dfl::neg(dfl::mul(a.im, b.im))),
            dfl::add_fast(dfl::mul(a.re, b.im), dfl::mul(a.im, b.re))};
}
__device__ __forceinline__ cdf cscale(cdf a, df c) { return {dfl::mul(a.re, c), dfl::mul(a.im, c)}; }
// exact scaling by a power of two
__device__ __forceinline__ cdf chalf(cdf a, float p2) {
    return {{a.re.hi * p2, a.re.lo * p2}, {a.im.hi * p2, a.im.lo * p2}};
}
// sg i a, sg = +-1
__device__ __forceinline__ cdf cmul_i(cdf a, float sg) { return {dfl::neg(dfl::df{a.im.hi * sg, a.im.lo * sg}), {a.re.hi * sg, a.re.lo * sg}}; }
__device__ __forceinline__ cdf cconj(cdf a) { return {a.re, dfl::neg(a.im)}; }

// sin(2 pi/3), cos and sin of 2 pi/5 and 4 pi/5 as float-float pairs
struct DfConst {
    float s3[2], c51[2], c52[2], s51[2], s52[2];
};
__constant__ DfConst kC;

__device__ __forceinline__ df dc(const float (&v)[2]) { return {v[0], v[1]}; }

// R-point DFT in place, sg = -1 forward, +1 inverse: y_q = sum_r v_r e^{sg 2 pi i r q / R}
template <int R>
__device__ __forceinline__ void dft(cdf* v, float sg);

template <>
__device__ __forceinline__ void dft<2>(cdf* v, float) {
    const cdf a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
}

template <>
__device__ __forceinline__ void dft<3>(cdf* v, float sg) {
    const cdf a = cadd(v[1], v[2]), b = csub(v[1], v[2]);
    const cdf t = cadd(v[0], chalf(a, -0.5f));
    const cdf u = cmul_i(cscale(b, dc(kC.s3)), sg);
    v[0] = cadd(v[0], a);
    v[1] = cadd(t, u);
    v[2] = csub(t, u);
}

template <>
__device__ __forceinline__ void dft<4>(cdf* v, float sg) {
    const cdf a = cadd(v[0], v[2]), b = csub(v[0], v[2]), c = cadd(v[1], v[3]), d = cmul_i(csub(v[1], v[3]), sg);
    v[0] = cadd(a, c);
    v[1] = cadd(b, d);
    v[2] = csub(a, c);
    v[3] = csub(b, d);
}

template <>
__device__ __forceinline__ void dft<5>(cdf* v, float sg) {
    const cdf a1 = cadd(v[1], v[4]), a2 = cadd(v[2], v[3]), b1 = csub(v[1], v[4]), b2 = csub(v[2], v[3]);
    const df c1 = dc(kC.c51), c2 = dc(kC.c52), s1 = dc(kC.s51), s2 = dc(kC.s52);
    const cdf t1 = cadd(v[0], cadd(cscale(a1, c1), cscale(a2, c2)));
    const cdf t2 = cadd(v[0], cadd(cscale(a1, c2), cscale(a2, c1)));
    const cdf u1 = cmul_i(cadd(cscale(b1, s1), cscale(b2, s2)), sg);
    const cdf u2 = cmul_i(csub(cscale(b1, s2), cscale(b2, s1)), sg);
    v[0] = cadd(v[0], cadd(a1, a2));
    v[1] = cadd(t1, u1);
    v[4] = csub(t1, u1);
    v[2] = cadd(t2, u2);
    v[3] = csub(t2, u2);
}

// One Stockham pass of radix R over `rows` lines of length M: src -> dst.
template <int R>
__device__ __forceinline__ void pass(const float4* __restrict__ src, float4* __restrict__ dst, int M, int Ns, int rows,
                                     const float4* __restrict__ tw, float sg) {
    const int nb = M / R, tws = M / (Ns * R);
    for (int t = threadIdx.x; t < rows * nb; t += blockDim.x) {
        const int row = t / nb, j = t - row * nb;
        const float4* s = src + row * M;
        float4* d = dst + row * M;
        const int jm = j % Ns;
        cdf v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = ldc(s[j + r * nb]);
        if (jm) {
#pragma unroll
            for (int r = 1; r < R; ++r) {
                cdf w = ldc(__ldg(tw + jm * r * tws));
                if (sg > 0.0f) w = cconj(w);
                v[r] = cmul(v[r], w);
            }
        }
        dft<R>(v, sg);
        const int base = (j / Ns) * Ns * R + jm;
#pragma unroll
        for (int r = 0; r < R; ++r) d[base + r * Ns] = stc(v[r]);
    }
}

// `rows` length-M transforms of the lines in b0 (b1 is scratch); returns the buffer
// holding the result.
__device__ float4* fft_lines(float4* b0, float4* b1, const DfFftPlan& p, int rows, const float4* __restrict__ tw,
                             float sg) {
    float4 *src = b0, *dst = b1;
    int Ns = 1;
    for (int k = 0; k < p.nr; ++k) {
        const int R = p.radix[k];
        switch (R) {
            case 2: pass<2>(src, dst, p.M, Ns, rows, tw, sg); break;
            case 3: pass<3>(src, dst, p.M, Ns, rows, tw, sg); break;
            case 4: pass<4>(src, dst, p.M, Ns, rows, tw, sg); break;
            default: pass<5>(src, dst, p.M, Ns, rows, tw, sg); break;
        }
        __syncthreads();
        float4* t = src;
        src = dst;
        dst = t;
        Ns *= R;
    }
    return src;
}

constexpr int kThreads = 256;

// grid rows y0, y0 + 1 (both components, FP64) -> FFT over x -> T1[k_x][y]
__global__ void __launch_bounds__(kThreads) k_dfft_x_fwd(DfFftPlan p, const float4* __restrict__ tw,
                                                        const double* __restrict__ grid, float4* __restrict__ T1) {
    extern __shared__ float4 sm[];
    const int M = p.M, y0 = 2 * blockIdx.x;
    const size_t MM = (size_t)M * M;
    float4* b0 = sm;
    float4* b1 = sm + 2 * M;
    for (int e = threadIdx.x; e < 2 * M; e += blockDim.x) {
        const size_t g = (size_t)y0 * M + e;  // rows y0, y0 + 1 are contiguous
        const df a = dfl::from_double(grid[g]), b = dfl::from_double(grid[MM + g]);
        b0[e] = make_float4(a.hi, a.lo, b.hi, b.lo);
    }
    __syncthreads();
    const float4* r = fft_lines(b0, b1, p, 2, tw, -1.0f);
    for (int e = threadIdx.x; e < 2 * M; e += blockDim.x) {
        const int kx = e >> 1, row = e & 1;
        T1[(size_t)kx * M + y0 + row] = r[row * M + kx];
    }
}

// T1 rows k_a = b and k_b = -b (b = 0 takes rows 0 and M/2) -> FFT over y -> scale
// -> inverse FFT over y -> T2[y][k_a], T2[y][k_b].  tab[b][k_y] holds (s, C = s e^{2 i theta})
// of k = (b, k_y) as 2 float4 (s hi, s lo, C_re hi, C_re lo), (C_im hi, C_im lo, -, -),
// zero where k = 0 or on a Nyquist line.
__global__ void __launch_bounds__(kThreads) k_dfft_y_scale(DfFftPlan p, const float4* __restrict__ tw,
                                                          const float4* __restrict__ tab,
                                                          const float4* __restrict__ T1, float4* __restrict__ T2) {
    extern __shared__ float4 sm[];
    const int M = p.M, b = blockIdx.x;
    const int ka = b, kb = b == 0 ? M / 2 : M - b;
    float4* b0 = sm;
    float4* b1 = sm + 2 * M;
    for (int e = threadIdx.x; e < 2 * M; e += blockDim.x) {
        const int row = e >= M, y = e - row * M;
        b0[e] = T1[(size_t)(row ? kb : ka) * M + y];
    }
    __syncthreads();
    float4* r = fft_lines(b0, b1, p, 2, tw, -1.0f);
    float4* r0 = r;
    float4* r1 = r + M;
    const float4* tb = tab + (size_t)b * M * 2;
    for (int ky = threadIdx.x; ky < M; ky += blockDim.x) {
        const float4 t0 = __ldg(tb + 2 * ky), t1 = __ldg(tb + 2 * ky + 1);
        const df s = {t0.x, t0.y};
        const cdf C = {{t0.z, t0.w}, {t1.x, t1.y}};
        if (b > 0) {
            const int kn = ky == 0 ? 0 : M - ky;
            const cdf A = ldc(r0[ky]), B = ldc(r1[kn]);
            r0[ky] = stc(csub(cscale(A, s), cmul(C, cconj(B))));
            r1[kn] = stc(csub(cscale(B, s), cmul(C, cconj(A))));
        } else {
            // row 0 pairs k_y with -k_y within itself (k_y = 0 and M/2 have s = C = 0);
            // row M/2 is a Nyquist line
            if (ky == 0 || ky == M / 2) {
                r0[ky] = make_float4(0.f, 0.f, 0.f, 0.f);
            } else if (ky < M / 2) {
                const int kn = M - ky;
                const cdf A = ldc(r0[ky]), B = ldc(r0[kn]);
                r0[ky] = stc(csub(cscale(A, s), cmul(C, cconj(B))));
                r0[kn] = stc(csub(cscale(B, s), cmul(C, cconj(A))));
            }
            r1[ky] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
    __syncthreads();
    const float4* q = fft_lines(r, r == b0 ? b1 : b0, p, 2, tw, 1.0f);
    for (int y = threadIdx.x; y < M; y += blockDim.x) {
        T2[(size_t)y * M + ka] = q[y];
        T2[(size_t)y * M + kb] = q[M + y];
    }
}

// T2 rows y0, y0 + 1 -> inverse FFT over x -> grid rows (real part -> component 0,
// imaginary part -> component 1), rounded to FP64
__global__ void __launch_bounds__(kThreads) k_dfft_x_inv(DfFftPlan p, const float4* __restrict__ tw,
                                                        const float4* __restrict__ T2, double* __restrict__ grid) {
    extern __shared__ float4 sm[];
    const int M = p.M, y0 = 2 * blockIdx.x;
    const size_t MM = (size_t)M * M;
    float4* b0 = sm;
    float4* b1 = sm + 2 * M;
    for (int e = threadIdx.x; e < 2 * M; e += blockDim.x) b0[e] = T2[(size_t)y0 * M + e];
    __syncthreads();
    const float4* r = fft_lines(b0, b1, p, 2, tw, 1.0f);
    for (int e = threadIdx.x; e < 2 * M; e += blockDim.x) {
        const float4 v = r[e];
        const size_t g = (size_t)y0 * M + e;
        grid[g] = dfl::to_double({v.x, v.y});
        grid[MM + g] = dfl::to_double({v.z, v.w});
    }
}

// Scale table in FP64, split into float-float (once per handle).
__global__ void k_dfft_table(int M, double twopi_L, double inv4xi2, double one_minus_eta, double pref,
                             float4* __restrict__ tab) {
    const size_t n = (size_t)(M / 2) * M;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int b = (int)(i / M), ky = (int)(i - (size_t)b * M);
    const int ky_i = ky < M / 2 ? ky : ky - M;
    double s = 0.0, cr = 0.0, ci = 0.0;
    if (!(b == 0 && ky == 0) && ky != M / 2) {
        const double kx = twopi_L * b, kyv = twopi_L * ky_i;
        const double k2 = kx * kx + kyv * kyv;
        const double q = k2 * inv4xi2;
        s = 0.5 * pref * (1.0 + q) * exp(-one_minus_eta * q) / k2;
        cr = s * (kx * kx - kyv * kyv) / k2;
        ci = s * 2.0 * kx * kyv / k2;
    }
    const df a = dfl::from_double(s), c = dfl::from_double(cr), d = dfl::from_double(ci);
    tab[2 * i] = make_float4(a.hi, a.lo, c.hi, c.lo);
    tab[2 * i + 1] = make_float4(d.hi, d.lo, 0.f, 0.f);
}

bool plan_radices(int M, DfFftPlan& p) {
    p.M = M;
    p.nr = 0;
    int m = M;
    auto take = [&](int r) {
        while (m % r == 0 && p.nr < kDfFftMaxPasses) {
            p.radix[p.nr++] = r;
            m /= r;
        }
    };
    take(4);
    take(2);
    take(3);
    take(5);
    return m == 1;
}

size_t smem_bytes(int M) { return (size_t)4 * M * sizeof(float4); }

}  // namespace

fbim_status dfft_setup(fbim_handle_s* h) {
    DfFft& d = h->dfft;
    if (d.state != 0) return FBIM_OK;
    d.state = -1;
    const int M = h->M;
    if (M % 2 != 0 || !plan_radices(M, d.plan)) return FBIM_OK;
    int dev = 0, optin = 0;
    FBIM_CUDA_TRY(h, cudaGetDevice(&dev));
    FBIM_CUDA_TRY(h, cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    const size_t sm = smem_bytes(M);
    if (sm > (size_t)optin) return FBIM_OK;
    for (const void* k : {(const void*)k_dfft_x_fwd, (const void*)k_dfft_y_scale, (const void*)k_dfft_x_inv})
        FBIM_CUDA_TRY(h, cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    {
        DfConst c;
        auto put = [](float (&dst)[2], double v) {
            const df x = dfl::from_double(v);
            dst[0] = x.hi;
            dst[1] = x.lo;
        };
        put(c.s3, std::sin(2.0 * M_PI / 3.0));
        put(c.c51, std::cos(2.0 * M_PI / 5.0));
        put(c.c52, std::cos(4.0 * M_PI / 5.0));
        put(c.s51, std::sin(2.0 * M_PI / 5.0));
        put(c.s52, std::sin(4.0 * M_PI / 5.0));
        FBIM_CUDA_TRY(h, cudaMemcpyToSymbolAsync(kC, &c, sizeof(c), 0, cudaMemcpyHostToDevice, h->stream));
    }
    std::vector<float4> tw(M);
    for (int m = 0; m < M; ++m) {
        const double ang = -2.0 * M_PI * (double)m / (double)M;
        const df c = dfl::from_double(std::cos(ang)), s = dfl::from_double(std::sin(ang));
        tw[m] = make_float4(c.hi, c.lo, s.hi, s.lo);
    }
    const size_t MM = (size_t)M * M, nt = (size_t)(M / 2) * M;
    FBIM_CUDA_TRY(h, cudaMalloc(&d.tw, M * sizeof(float4)));
    FBIM_CUDA_TRY(h, cudaMalloc(&d.tab, 2 * nt * sizeof(float4)));
    FBIM_CUDA_TRY(h, cudaMalloc(&d.T1, MM * sizeof(float4)));
    FBIM_CUDA_TRY(h, cudaMalloc(&d.T2, MM * sizeof(float4)));
    FBIM_CUDA_TRY(h, cudaMemcpyAsync(d.tw, tw.data(), M * sizeof(float4), cudaMemcpyHostToDevice, h->stream));
    const double V = h->L * h->L, h4 = h->h * h->h * h->h * h->h;
    k_dfft_table<<<(unsigned)((nt + 255) / 256), 256, 0, h->stream>>>(
        M, 2.0 * M_PI / h->L, 1.0 / (4.0 * h->xi * h->xi), 1.0 - h->eta_s, h4 / (h->eta * V), d.tab);
    FBIM_CUDA_TRY(h, cudaGetLastError());
    FBIM_CUDA_TRY(h, cudaStreamSynchronize(h->stream));  // tw is a host vector
    ++h->layout_version;
    d.state = 1;
    return FBIM_OK;
}

void dfft_free(fbim_handle_s* h) {
    DfFft& d = h->dfft;
    cudaFree(d.tw);
    cudaFree(d.tab);
    cudaFree(d.T1);
    cudaFree(d.T2);
    d = DfFft();
}

void dfft_forward(fbim_handle_s* h, cudaStream_t st, const double* grid) {
    const DfFft& d = h->dfft;
    const size_t sm = smem_bytes(d.plan.M);
    k_dfft_x_fwd<<<d.plan.M / 2, kThreads, sm, st>>>(d.plan, d.tw, grid, d.T1);
}

void dfft_scale(fbim_handle_s* h, cudaStream_t st) {
    const DfFft& d = h->dfft;
    const size_t sm = smem_bytes(d.plan.M);
    k_dfft_y_scale<<<d.plan.M / 2, kThreads, sm, st>>>(d.plan, d.tw, d.tab, d.T1, d.T2);
}

void dfft_inverse(fbim_handle_s* h, cudaStream_t st, double* grid) {
    const DfFft& d = h->dfft;
    const size_t sm = smem_bytes(d.plan.M);
    k_dfft_x_inv<<<d.plan.M / 2, kThreads, sm, st>>>(d.plan, d.tw, d.T2, grid);
}

}  // namespace fbim
