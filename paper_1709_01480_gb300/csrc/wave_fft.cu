// Wave-space transforms and Fourier scale (Sec. 3.2) of the FP64 residual operator
// of FP32 handles in float-float arithmetic (about 48-bit accurate, on the FP32
// pipes), replacing cuFFT's double transforms, which run on GB300's FP64 pipe at
// ~1/74 of its FP32 rate, and the separate scale kernel.  (The handle's own FP32
// operator keeps cuFFT: a plain-FP32 instance of these kernels measured about twice
// cuFFT's time, its index arithmetic and barriers outweighing the FP32 math.)
//
// The two real grid components g0, g1 are packed into one complex field
// z = g0 + i g1 and transformed with one complex 2D FFT, Z = F z.  The scale
// u(k) = sc(k) (I - k k^T/k^2) g^(k) becomes, per pair (k, -k),
//     Z'(k) = s(k) [Z(k) - e^{2 i theta_k} conj(Z(-k))],   s = sc/2,
// where e^{i theta_k} = (k_x + i k_y)/|k| (the trace of I - k k^T/k^2 is 1 in 2D),
// and F^{-1} Z' = u0 + i u1.  k = 0 and the Nyquist lines are zeroed, as in the
// half-spectrum path.  Transforms are unnormalised, like cuFFT's.
//
// Three kernels, each holding whole grid lines in shared memory:
//   x pass:  grid rows y (RB per CTA)   -> FFT over x      -> T1[k_x][y] (store of RB-long runs)
//   y pass:  T1 rows k_x and -k_x      -> FFT over y, scale, inverse FFT over y -> T2[k_x][y]
//   x pass:  T2 columns y (RB per CTA) -> inverse FFT over x -> grid rows y
// RB = 2 lines of 16-byte elements make 32-byte runs, so every global access moves
// whole sectors.  Each 1D transform is a Stockham autosort FFT (radix 4, 2, 3, 5
// passes, natural order in and out) between two shared-memory buffers, with
// twiddles e^{-2 pi i m/M} from a table.  The kernels are written over an
// arithmetic type A (complex value, storage, twiddle and grid types).  M must be a
// multiple of RB, 5-smooth and fit the shared memory (64 M bytes per CTA);
// otherwise the caller keeps cuFFT.
#include <cmath>
#include <vector>

#include "dfloat.cuh"
#include "fbim_internal.h"

namespace fbim {

namespace {

using dfl::df;

// sin(2 pi/3), cos and sin of 2 pi/5 and 4 pi/5 as float-float pairs
struct FftConst {
    float s3[2], c51[2], c52[2], s51[2], s52[2];
};
__constant__ FftConst kC;

// ---- float-float complex arithmetic ---------------------------------------------
struct cdf {
    df re, im;
};
struct ArD {
    using C = cdf;
    using S = float4;  // (re hi, re lo, im hi, im lo)
    using W = float4;
    using R = df;
    using G = double;
    static constexpr int RB = 2;
    __device__ static C ld(S v) { return {{v.x, v.y}, {v.z, v.w}}; }
    __device__ static S st(C a) { return make_float4(a.re.hi, a.re.lo, a.im.hi, a.im.lo); }
    __device__ static C ldw(W w) { return ld(w); }
    __device__ static C add(C a, C b) { return {dfl::add_fast(a.re, b.re), dfl::add_fast(a.im, b.im)}; }
    __device__ static C sub(C a, C b) {
        return {dfl::add_fast(a.re, dfl::neg(b.re)), dfl::add_fast(a.im, dfl::neg(b.im))};
    }
    __device__ static C mul(C a, C b) {
        return {dfl::add_fast(dfl::mul(a.re, b.re), dfl::neg(dfl::mul(a.im, b.im))),
                dfl::add_fast(dfl::mul(a.re, b.im), dfl::mul(a.im, b.re))};
    }
    __device__ static C scale(C a, R c) { return {dfl::mul(a.re, c), dfl::mul(a.im, c)}; }
    // exact scaling by a power of two
    __device__ static C pow2(C a, float p) { return {{a.re.hi * p, a.re.lo * p}, {a.im.hi * p, a.im.lo * p}}; }
    __device__ static C mul_i(C a, float sg) { return {{-sg * a.im.hi, -sg * a.im.lo}, {sg * a.re.hi, sg * a.re.lo}}; }
    __device__ static C conj(C a) { return {a.re, dfl::neg(a.im)}; }
    __device__ static R rc(const float (&v)[2]) { return {v[0], v[1]}; }
    __device__ static C zero() { return {{0.f, 0.f}, {0.f, 0.f}}; }
    __device__ static C from_grid(G a, G b) { return {dfl::from_double(a), dfl::from_double(b)}; }
    __device__ static void to_grid(C v, G& a, G& b) {
        a = dfl::to_double(v.re);
        b = dfl::to_double(v.im);
    }
    __device__ static void ldtab(const float4* tab, size_t i, R& s, C& c) {
        const float4 t0 = __ldg(tab + 2 * i), t1 = __ldg(tab + 2 * i + 1);
        s = {t0.x, t0.y};
        c = {{t0.z, t0.w}, {t1.x, t1.y}};
    }
};

// R-point DFT in place, sg = -1 forward, +1 inverse: y_q = sum_r v_r e^{sg 2 pi i r q / R}
template <typename A, int R>
struct Dft;

template <typename A>
struct Dft<A, 2> {
    __device__ static void run(typename A::C* v, float) {
        const typename A::C a = v[0], b = v[1];
        v[0] = A::add(a, b);
        v[1] = A::sub(a, b);
    }
};

template <typename A>
struct Dft<A, 3> {
    __device__ static void run(typename A::C* v, float sg) {
        using C = typename A::C;
        const C a = A::add(v[1], v[2]), b = A::sub(v[1], v[2]);
        const C t = A::add(v[0], A::pow2(a, -0.5f));
        const C u = A::mul_i(A::scale(b, A::rc(kC.s3)), sg);
        v[0] = A::add(v[0], a);
        v[1] = A::add(t, u);
        v[2] = A::sub(t, u);
    }
};

template <typename A>
struct Dft<A, 4> {
    __device__ static void run(typename A::C* v, float sg) {
        using C = typename A::C;
        const C a = A::add(v[0], v[2]), b = A::sub(v[0], v[2]), c = A::add(v[1], v[3]);
        const C d = A::mul_i(A::sub(v[1], v[3]), sg);
        v[0] = A::add(a, c);
        v[1] = A::add(b, d);
        v[2] = A::sub(a, c);
        v[3] = A::sub(b, d);
    }
};

template <typename A>
struct Dft<A, 5> {
    __device__ static void run(typename A::C* v, float sg) {
        using C = typename A::C;
        const C a1 = A::add(v[1], v[4]), a2 = A::add(v[2], v[3]), b1 = A::sub(v[1], v[4]), b2 = A::sub(v[2], v[3]);
        const typename A::R c1 = A::rc(kC.c51), c2 = A::rc(kC.c52), s1 = A::rc(kC.s51), s2 = A::rc(kC.s52);
        const C t1 = A::add(v[0], A::add(A::scale(a1, c1), A::scale(a2, c2)));
        const C t2 = A::add(v[0], A::add(A::scale(a1, c2), A::scale(a2, c1)));
        const C u1 = A::mul_i(A::add(A::scale(b1, s1), A::scale(b2, s2)), sg);
        const C u2 = A::mul_i(A::sub(A::scale(b1, s2), A::scale(b2, s1)), sg);
        v[0] = A::add(v[0], A::add(a1, a2));
        v[1] = A::add(t1, u1);
        v[4] = A::sub(t1, u1);
        v[2] = A::add(t2, u2);
        v[3] = A::sub(t2, u2);
    }
};

// One Stockham pass of radix R over `rows` lines of length M: src -> dst.
template <typename A, int R>
__device__ __forceinline__ void pass(const typename A::S* __restrict__ src, typename A::S* __restrict__ dst, int M,
                                     int Ns, int rows, const typename A::W* __restrict__ tw, float sg) {
    using C = typename A::C;
    const int nb = M / R, tws = M / (Ns * R);
    for (int t = threadIdx.x; t < rows * nb; t += blockDim.x) {
        const int row = t / nb, j = t - row * nb;
        const typename A::S* s = src + row * M;
        typename A::S* d = dst + row * M;
        const int jm = j % Ns;
        C v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = A::ld(s[j + r * nb]);
        if (jm) {
#pragma unroll
            for (int r = 1; r < R; ++r) {
                C w = A::ldw(__ldg(tw + jm * r * tws));
                if (sg > 0.0f) w = A::conj(w);
                v[r] = A::mul(v[r], w);
            }
        }
        Dft<A, R>::run(v, sg);
        const int base = (j / Ns) * Ns * R + jm;
#pragma unroll
        for (int r = 0; r < R; ++r) d[base + r * Ns] = A::st(v[r]);
    }
}

// `rows` length-M transforms of the lines in b0 (b1 is scratch); returns the buffer
// holding the result.
template <typename A>
__device__ typename A::S* fft_lines(typename A::S* b0, typename A::S* b1, const FftPlan& p, int rows,
                                    const typename A::W* __restrict__ tw, float sg) {
    typename A::S *src = b0, *dst = b1;
    int Ns = 1;
    for (int k = 0; k < p.nr; ++k) {
        const int R = p.radix[k];
        switch (R) {
            case 2: pass<A, 2>(src, dst, p.M, Ns, rows, tw, sg); break;
            case 3: pass<A, 3>(src, dst, p.M, Ns, rows, tw, sg); break;
            case 4: pass<A, 4>(src, dst, p.M, Ns, rows, tw, sg); break;
            default: pass<A, 5>(src, dst, p.M, Ns, rows, tw, sg); break;
        }
        __syncthreads();
        typename A::S* t = src;
        src = dst;
        dst = t;
        Ns *= R;
    }
    return src;
}

constexpr int kThreads = 256;

// grid rows y0 .. y0 + RB - 1 (both components) -> FFT over x -> T1[k_x][y]
template <typename A>
__global__ void __launch_bounds__(kThreads) k_fft_x_fwd(FftPlan p, const typename A::W* __restrict__ tw,
                                                       const typename A::G* __restrict__ grid,
                                                       typename A::S* __restrict__ T1) {
    using S = typename A::S;
    constexpr int RB = A::RB;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    S* b0 = reinterpret_cast<S*>(smem_raw);
    S* b1 = b0 + RB * p.M;
    const int M = p.M, y0 = RB * blockIdx.x;
    const size_t MM = (size_t)M * M;
    for (int e = threadIdx.x; e < RB * M; e += blockDim.x) {
        const size_t g = (size_t)y0 * M + e;  // the CTA's rows are contiguous
        b0[e] = A::st(A::from_grid(grid[g], grid[MM + g]));
    }
    __syncthreads();
    const S* r = fft_lines<A>(b0, b1, p, RB, tw, -1.0f);
    for (int e = threadIdx.x; e < RB * M; e += blockDim.x) {
        const int kx = e / RB, row = e - kx * RB;
        T1[(size_t)kx * M + y0 + row] = r[row * M + kx];
    }
}

// T1 rows k_a = b and k_b = -b (b = 0 takes rows 0 and M/2) -> FFT over y -> scale
// -> inverse FFT over y -> T2 rows k_a, k_b.  tab[b][k_y] holds (s, C = s e^{2 i theta})
// of k = (b, k_y), zero where k = 0 or on a Nyquist line.
template <typename A>
__global__ void __launch_bounds__(kThreads) k_fft_y_scale(FftPlan p, const typename A::W* __restrict__ tw,
                                                         const float4* __restrict__ tab,
                                                         const typename A::S* __restrict__ T1,
                                                         typename A::S* __restrict__ T2) {
    using S = typename A::S;
    using C = typename A::C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    S* b0 = reinterpret_cast<S*>(smem_raw);
    S* b1 = b0 + 2 * p.M;
    const int M = p.M, b = blockIdx.x;
    const int ka = b, kb = b == 0 ? M / 2 : M - b;
    for (int e = threadIdx.x; e < 2 * M; e += blockDim.x) {
        const int row = e >= M, y = e - row * M;
        b0[e] = T1[(size_t)(row ? kb : ka) * M + y];
    }
    __syncthreads();
    S* r = fft_lines<A>(b0, b1, p, 2, tw, -1.0f);
    S* r0 = r;
    S* r1 = r + M;
    const size_t t0 = (size_t)b * M;
    for (int ky = threadIdx.x; ky < M; ky += blockDim.x) {
        typename A::R s;
        C c;
        A::ldtab(tab, t0 + ky, s, c);
        if (b > 0) {
            const int kn = ky == 0 ? 0 : M - ky;
            const C za = A::ld(r0[ky]), zb = A::ld(r1[kn]);
            r0[ky] = A::st(A::sub(A::scale(za, s), A::mul(c, A::conj(zb))));
            r1[kn] = A::st(A::sub(A::scale(zb, s), A::mul(c, A::conj(za))));
        } else {
            // row 0 pairs k_y with -k_y within itself (k_y = 0 and M/2 have s = C = 0);
            // row M/2 is a Nyquist line
            if (ky == 0 || ky == M / 2) {
                r0[ky] = A::st(A::zero());
            } else if (ky < M / 2) {
                const int kn = M - ky;
                const C za = A::ld(r0[ky]), zb = A::ld(r0[kn]);
                r0[ky] = A::st(A::sub(A::scale(za, s), A::mul(c, A::conj(zb))));
                r0[kn] = A::st(A::sub(A::scale(zb, s), A::mul(c, A::conj(za))));
            }
            r1[ky] = A::st(A::zero());
        }
    }
    __syncthreads();
    const S* q = fft_lines<A>(r, r == b0 ? b1 : b0, p, 2, tw, 1.0f);
    for (int y = threadIdx.x; y < M; y += blockDim.x) {
        T2[(size_t)ka * M + y] = q[y];
        T2[(size_t)kb * M + y] = q[M + y];
    }
}

// T2 columns y0 .. y0 + RB - 1 -> inverse FFT over x -> grid rows (real part ->
// component 0, imaginary part -> component 1); df_out: each value stored as its
// float-float pair (hi, lo) in the grid value's 8 bytes instead of rounded to FP64
template <typename A>
__global__ void __launch_bounds__(kThreads) k_fft_x_inv(FftPlan p, const typename A::W* __restrict__ tw,
                                                       const typename A::S* __restrict__ T2,
                                                       typename A::G* __restrict__ grid, int df_out) {
    using S = typename A::S;
    constexpr int RB = A::RB;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    S* b0 = reinterpret_cast<S*>(smem_raw);
    S* b1 = b0 + RB * p.M;
    const int M = p.M, y0 = RB * blockIdx.x;
    const size_t MM = (size_t)M * M;
    for (int e = threadIdx.x; e < RB * M; e += blockDim.x) {
        const int kx = e / RB, row = e - kx * RB;
        b0[row * M + kx] = T2[(size_t)kx * M + y0 + row];
    }
    __syncthreads();
    const S* r = fft_lines<A>(b0, b1, p, RB, tw, 1.0f);
    for (int e = threadIdx.x; e < RB * M; e += blockDim.x) {
        const size_t g = (size_t)y0 * M + e;
        if (df_out) {
            const typename A::C v = A::ld(r[e]);
            float2* gf = reinterpret_cast<float2*>(grid);
            gf[g] = make_float2(v.re.hi, v.re.lo);
            gf[MM + g] = make_float2(v.im.hi, v.im.lo);
        } else {
            typename A::G a, c;
            A::to_grid(A::ld(r[e]), a, c);
            grid[g] = a;
            grid[MM + g] = c;
        }
    }
}

// Scale table (once per handle), computed in FP64 and stored in float-float.
template <typename A>
__global__ void k_fft_table(int M, double twopi_L, double inv4xi2, double one_minus_eta, double pref,
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

bool plan_radices(int M, FftPlan& p) {
    p.M = M;
    p.nr = 0;
    int m = M;
    auto take = [&](int r) {
        while (m % r == 0 && p.nr < kFftMaxPasses) {
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

template <typename A>
size_t smem_x(int M) {
    return (size_t)2 * A::RB * M * sizeof(typename A::S);
}
template <typename A>
size_t smem_y(int M) {
    return (size_t)4 * M * sizeof(typename A::S);
}


fbim_status upload_constants(fbim_handle_s* h) {
    FftConst c;
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
    return FBIM_OK;
}

}  // namespace

fbim_status wfft_setup(fbim_handle_s* h) {
    using A = ArD;
    WaveFft& d = h->fft64;
    if (d.state != 0) return FBIM_OK;
    d.state = -1;
    const int M = h->M;
    if (M % A::RB != 0 || M % 2 != 0 || !plan_radices(M, d.plan)) return FBIM_OK;
    int dev = 0, optin = 0;
    FBIM_CUDA_TRY(h, cudaGetDevice(&dev));
    FBIM_CUDA_TRY(h, cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    const size_t sx = smem_x<A>(M), sy = smem_y<A>(M);
    if (sx > (size_t)optin || sy > (size_t)optin) return FBIM_OK;
    // the limit belongs to the kernel, not the handle: the device maximum, so that
    // handles of other sizes never lower it under this one's launches
    FBIM_CUDA_TRY(h, cudaFuncSetAttribute(k_fft_x_fwd<A>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    FBIM_CUDA_TRY(h, cudaFuncSetAttribute(k_fft_x_inv<A>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    FBIM_CUDA_TRY(h, cudaFuncSetAttribute(k_fft_y_scale<A>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    FBIM_TRY(upload_constants(h));
    std::vector<typename A::W> tw(M);
    for (int m = 0; m < M; ++m) {
        const double ang = -2.0 * M_PI * (double)m / (double)M;
        const df a = dfl::from_double(std::cos(ang)), b = dfl::from_double(std::sin(ang));
        tw[m] = make_float4(a.hi, a.lo, b.hi, b.lo);
    }
    const size_t MM = (size_t)M * M, nt = (size_t)(M / 2) * M;
    FBIM_CUDA_TRY(h, cudaMalloc(&d.tw, M * sizeof(typename A::W)));
    FBIM_CUDA_TRY(h, cudaMalloc(&d.tab, 2 * nt * sizeof(float4)));
    FBIM_CUDA_TRY(h, cudaMalloc(&d.T1, MM * sizeof(typename A::S)));
    FBIM_CUDA_TRY(h, cudaMalloc(&d.T2, MM * sizeof(typename A::S)));
    FBIM_CUDA_TRY(h, cudaMemcpyAsync(d.tw, tw.data(), M * sizeof(typename A::W), cudaMemcpyHostToDevice, h->stream));
    const double V = h->L * h->L, h4 = h->h * h->h * h->h * h->h;
    k_fft_table<A><<<(unsigned)((nt + 255) / 256), 256, 0, h->stream>>>(
        M, 2.0 * M_PI / h->L, 1.0 / (4.0 * h->xi * h->xi), 1.0 - h->eta_s, h4 / (h->eta * V), (float4*)d.tab);
    FBIM_CUDA_TRY(h, cudaGetLastError());
    FBIM_CUDA_TRY(h, cudaStreamSynchronize(h->stream));  // tw is a host vector
    ++h->layout_version;
    d.state = 1;
    return FBIM_OK;
}

void wfft_free(fbim_handle_s* h) {
    WaveFft& d = h->fft64;
    cudaFree(d.tw);
    cudaFree(d.tab);
    cudaFree(d.T1);
    cudaFree(d.T2);
    d = WaveFft();
}

void wfft_forward(fbim_handle_s* h, cudaStream_t st, const double* grid) {
    using A = ArD;
    const WaveFft& d = h->fft64;
    const int M = d.plan.M;
    k_fft_x_fwd<A><<<M / A::RB, kThreads, smem_x<A>(M), st>>>(d.plan, (const A::W*)d.tw, grid, (A::S*)d.T1);
}

void wfft_scale(fbim_handle_s* h, cudaStream_t st) {
    using A = ArD;
    const WaveFft& d = h->fft64;
    const int M = d.plan.M;
    k_fft_y_scale<A><<<M / 2, kThreads, smem_y<A>(M), st>>>(d.plan, (const A::W*)d.tw, (const float4*)d.tab,
                                                             (const A::S*)d.T1, (A::S*)d.T2);
}

void wfft_inverse(fbim_handle_s* h, cudaStream_t st, double* grid, bool df_out) {
    using A = ArD;
    const WaveFft& d = h->fft64;
    const int M = d.plan.M;
    k_fft_x_inv<A><<<M / A::RB, kThreads, smem_x<A>(M), st>>>(d.plan, (const A::W*)d.tw, (const A::S*)d.T2, grid,
                                                             df_out ? 1 : 0);
}

}  // namespace fbim
