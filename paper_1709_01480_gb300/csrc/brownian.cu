// Random slip by the positively split Ewald sum (Sec. 3.3, Eq. sqrtM-split):
//     slip = sqrt(2 kT/dt) [ G^+ (G M(r) G^T)^1/2 W(r) + (M(w))^1/2 W(w) ]
// with the block-diagonal G_b = R_b G_ref R_b^T of Sec. 3.4 (Eqs.
// preconditioned-real-part, Gprecond-decomp, Gprecond-precompute).
//
// Near field: Lanczos iteration for f(A) w, f = sqrt, A = G M(r) G^T (the real-
// space operator in the handle's precision, G as one block operator over all bodies:
// on the tensor cores for FP32 handles), with full FP64 reorthogonalisation by the
// solver's fused classical Gram-Schmidt sweeps; each step runs on the device and the
// next is queued before the host reads the last one's alpha and beta.  After k steps
// y_k = |w| V_k f(T_k) e_1 and the iteration stops when |y_k - y_{k-1}| <= tol |y_k|,
// which needs only the small coefficient vectors because V_k is orthonormal.  Ritz
// values below zero (from the small negative eigenvalues the symmetrised Alpert block
// can leave) are clipped to zero.
// Far field: the wave-space noise pipeline (ewald_ops.cu).
#include <cublas_v2.h>

#include <algorithm>
#include <cmath>
#include <type_traits>
#include <vector>

#include "ewald_types.cuh"
#include "fbim_internal.h"
#include "lanczos_host.h"
#include "solver.cuh"

namespace fbim {

fbim_status ensure_solver(fbim_handle_s* h);

namespace {

// f32: the transform in FP32 (the near-field noise of an FP32 handle)
__global__ void k_philox_normals(size_t n, unsigned long long seed, unsigned stream, unsigned counter, int f32,
                                 double* __restrict__ out) {
    size_t blk = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (2 * blk >= n) return;
    double2 z;
    if (f32) {
        const float2 zf = philox_normals_f(seed, stream, counter, blk);
        z = make_double2(zf.x, zf.y);
    } else {
        z = philox_normals(seed, stream, counter, blk);
    }
    out[2 * blk] = z.x;
    if (2 * blk + 1 < n) out[2 * blk + 1] = z.y;
}

template <typename T>
__global__ void k_rot_in2(int N, int n_p, const double* __restrict__ rot, const double* __restrict__ in,
                          T* __restrict__ z) {
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= N) return;
    int b = m / n_p;
    double c = rot[2 * b], s = rot[2 * b + 1];
    double ux = in[2 * m], uy = in[2 * m + 1];
    z[2 * m] = (T)(c * ux + s * uy);
    z[2 * m + 1] = (T)(-s * ux + c * uy);
}

template <typename T>
__global__ void k_rot_out(int N, int n_p, const double* __restrict__ rot, const T* __restrict__ g,
                          double* __restrict__ out) {
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= N) return;
    int b = m / n_p;
    double c = rot[2 * b], s = rot[2 * b + 1];
    double gx = (double)g[2 * m], gy = (double)g[2 * m + 1];
    out[2 * m] = c * gx - s * gy;
    out[2 * m + 1] = s * gx + c * gy;
}

__global__ void k_combine(int n, double a, const double* __restrict__ x, double b, const double* __restrict__ y,
                          double* __restrict__ out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = a * x[i] + b * y[i];
}

// out_b = R_b B_ref R_b^T in_b for every body (B_ref = G_ref or G_ref^+), precision T.
template <typename T>
fbim_status block_apply(fbim_handle_s* h, const T* Bref, const double* in, double* out) {
    Solver* S = h->solver;
    const int N = h->N;
    if (std::is_same<T, float>::value && S->tc_G.ready) {  // the FP32 blocks on the tensor cores
        const TcBlock& tb = (const float*)Bref == S->G32 ? S->tc_G : S->tc_Gd;
        return tc_apply(h, tb, 0, in, out, nullptr, nullptr, nullptr, nullptr, S->tc_err);
    }
    T* z = (T*)S->zbuf;
    T* g = (T*)S->gbuf;
    k_rot_in2<T><<<(N + 255) / 256, 256, 0, h->stream>>>(N, h->n_p, h->rot, in, z);
    const int n2 = S->n2;
    cublasStatus_t st;
    if (std::is_same<T, float>::value) {
        const float one = 1.f, zero = 0.f;
        st = cublasSgemm(S->blas, CUBLAS_OP_N, CUBLAS_OP_N, n2, h->n_b, n2, &one, (const float*)Bref, n2,
                         (const float*)z, n2, &zero, (float*)g, n2);
    } else {
        const double one = 1.0, zero = 0.0;
        st = cublasDgemm(S->blas, CUBLAS_OP_N, CUBLAS_OP_N, n2, h->n_b, n2, &one, (const double*)Bref, n2,
                         (const double*)z, n2, &zero, (double*)g, n2);
    }
    if (st != CUBLAS_STATUS_SUCCESS) {
        h->fail("block_apply: GEMM failed");
        return FBIM_ERR_CUDA;
    }
    k_rot_out<T><<<(N + 255) / 256, 256, 0, h->stream>>>(N, h->n_p, h->rot, g, out);
    h->launches += 2;
    FBIM_CUDA_TRY(h, cudaGetLastError());
    return FBIM_OK;
}

template <typename T>
fbim_status near_field(fbim_handle_s* h, const double* W, double tol, int max_iter, double* y, int& iters) {
    Solver* S = h->solver;
    const int n = 2 * h->N;
    // basis rows V_0 .. V_{max_iter + 1} (a step queued past the last one writes one more)
    if (S->lanczos_max < max_iter + 2) {
        cudaFree(S->lz);
        cudaFree(S->lan_in);
        cudaFree(S->lan_w);
        cudaFree(S->lan_c);
        S->lz = S->lan_in = S->lan_w = S->lan_c = nullptr;
        S->lanczos_max = 0;
        FBIM_CUDA_TRY(h, cudaMalloc(&S->lz, sizeof(double) * (size_t)n * (max_iter + 2)));
        FBIM_CUDA_TRY(h, cudaMalloc(&S->lan_in, sizeof(double) * n));
        FBIM_CUDA_TRY(h, cudaMalloc(&S->lan_w, sizeof(double) * n));
        FBIM_CUDA_TRY(h, cudaMalloc(&S->lan_c, sizeof(double) * (max_iter + 1)));
        FBIM_TRY(cgs_alloc(h, S->lan, n, n, max_iter + 1));
        S->lanczos_max = max_iter + 2;
    }
    CgsState& c = S->lan;
    const T* G = std::is_same<T, float>::value ? (const T*)S->G32 : (const T*)S->G64;
    const T* Gd = std::is_same<T, float>::value ? (const T*)S->Gd32 : (const T*)S->Gd64;
    double* t1 = S->w;  // [>= n] scratch from the GMRES workspace
    double* t2 = S->r;
    // Start from W's projection G^+ G W onto the range of G: the component in the null
    // space of G (the near-null modes dropped from M(r)_ref, one normal mode per body at
    // coarse sampling) has f(0) = 0, and left in it would put a Ritz value at rounding
    // level under the square root (an error of sqrt(eps) that grows once the iteration
    // runs past convergence)
    // (W is first copied into the solver's workspace: the caller's vector need not have
    // the 16-byte alignment the tensor-core block operator's bulk copies require)
    FBIM_CUDA_TRY(h, cudaMemcpyAsync(t2, W, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->stream));
    FBIM_TRY(block_apply<T>(h, G, t2, t1));
    FBIM_TRY(block_apply<T>(h, Gd, t1, S->lan_w));
    W = S->lan_w;
    double wn = 0;
    FBIM_TRY(dev_norm2(h, n, W, wn));
    iters = 0;
    if (wn == 0) {
        FBIM_CUDA_TRY(h, cudaMemsetAsync(y, 0, sizeof(double) * n, h->stream));
        return FBIM_OK;
    }
    double* Vl = S->lz;
    cgs_start(h, c, 1.0 / wn, W, Vl, S->lan_in);
    // One step on the device: w = G M(r) G^T v_k (v_k in lan_in), full reorthogonalisation
    // against V_0..V_k (classical Gram-Schmidt, two passes, FP64), V_{k+1} = w / |w| into
    // the basis and lan_in.  The host reads alpha_k and beta_k from the step's history row.
    auto enqueue = [&](int k) -> fbim_status {
        FBIM_TRY(block_apply<T>(h, G, S->lan_in, t1));
        FBIM_TRY(apply_operator<T>(h, t1, t2, 1));
        FBIM_TRY(block_apply<T>(h, G, t2, S->lan_w));
        cgs_step(h, c, Vl, S->lan_w, true, S->lan_in);
        FBIM_CUDA_TRY(h, cudaGetLastError());
        FBIM_CUDA_TRY(h, cudaEventRecord(S->ev_step[k & 1], h->stream));
        return FBIM_OK;
    };
    const int hs = cgs_hist_stride(c.m), m = c.m;
    std::vector<double> alpha, beta, cprev, coef;
    double d_last = -1.0, d_prev = -1.0;  // the last two step-to-step changes of the iterate
    FBIM_TRY(enqueue(0));
    for (int k = 0; k < max_iter; ++k) {
        // queue the next step before reading this one, unless this one is predicted to
        // converge (the last change, shrunk by the last ratio of changes, within tol)
        bool ahead = k + 1 < max_iter;
        if (ahead && d_last >= 0.0 && d_prev > 0.0) ahead = d_last * std::min(d_last / d_prev, 1.0) > tol;
        if (ahead) FBIM_TRY(enqueue(k + 1));
        FBIM_CUDA_TRY(h, cudaEventSynchronize(S->ev_step[k & 1]));
        const double* row = c.hist_host + (size_t)k * hs;
        const double bn = std::sqrt(std::max(row[2 * (m + 1)], 0.0));
        alpha.push_back(row[k] + row[(m + 1) + k]);
        beta.push_back(bn);
        ++iters;
        coef = lanczos_sqrt_coeffs(alpha.data(), beta.data(), k + 1, wn);
        double dn = 0, cn = 0;
        for (int i = 0; i <= k; ++i) {
            const double prev = i < (int)cprev.size() ? cprev[i] : 0.0;
            dn += (coef[i] - prev) * (coef[i] - prev);
            cn += coef[i] * coef[i];
        }
        cprev = coef;
        if (!std::isfinite(bn) || !std::isfinite(cn)) {
            h->fail("Lanczos iterate is not finite");
            return FBIM_ERR_NONFINITE;
        }
        d_prev = d_last;
        d_last = cn > 0.0 ? std::sqrt(dn / cn) : 0.0;
        const bool converged = (k > 0 && std::sqrt(dn) <= tol * std::sqrt(cn)) || bn <= 1e-14 * wn;
        if (converged || k + 1 == max_iter) break;
        if (!ahead) FBIM_TRY(enqueue(k + 1));
    }
    // y = G^+ V c; a step queued past the last one read is complete before the combination
    const int k = (int)coef.size();
    FBIM_CUDA_TRY(h, cudaMemcpyAsync(S->lan_c, coef.data(), sizeof(double) * k, cudaMemcpyHostToDevice, h->stream));
    dev_combine(h, n, k, Vl, n, S->lan_c, 0.0, t1);
    FBIM_TRY(block_apply<T>(h, Gd, t1, y));
    return FBIM_OK;
}

}  // namespace

fbim_status lanczos_operator(fbim_handle_s* h, const double* in, double* out) {
    Solver* S = h->solver;
    if (h->precision == FBIM_FP32) {
        FBIM_TRY(block_apply<float>(h, S->G32, in, S->w));
        FBIM_TRY(apply_operator<float>(h, S->w, S->r, 1));
        return block_apply<float>(h, S->G32, S->r, out);
    }
    FBIM_TRY(block_apply<double>(h, S->G64, in, S->w));
    FBIM_TRY(apply_operator<double>(h, S->w, S->r, 1));
    return block_apply<double>(h, S->G64, S->r, out);
}

fbim_status gplus_apply(fbim_handle_s* h, const double* in, double* out) {
    Solver* S = h->solver;
    if (h->precision == FBIM_FP32) return block_apply<float>(h, S->Gd32, in, out);
    return block_apply<double>(h, S->Gd64, in, out);
}

fbim_status g_project(fbim_handle_s* h, const double* in, double* out) {
    Solver* S = h->solver;
    if (h->precision == FBIM_FP32) {
        FBIM_TRY(block_apply<float>(h, S->G32, in, S->w));
        return block_apply<float>(h, S->Gd32, S->w, out);
    }
    FBIM_TRY(block_apply<double>(h, S->G64, in, S->w));
    return block_apply<double>(h, S->Gd64, S->w, out);
}

fbim_status brownian_slip(fbim_handle_s* h, unsigned long long seed, unsigned long long counter, double kT, double dt,
                          const double* W_r, const double* Z_w, double tol, int max_iter, double* slip,
                          int* lanczos_iters) {
    FBIM_TRY(ensure_solver(h));
    Solver* S = h->solver;
    const int n = 2 * h->N;
    double* Wn = S->d;  // [>= n] scratch
    if (!W_r) {
        k_philox_normals<<<(unsigned)((n / 2 + 256) / 256), 256, 0, h->stream>>>(
            (size_t)n, seed, 0u, (unsigned)counter, h->precision == FBIM_FP32 ? 1 : 0, Wn);
        FBIM_CUDA_TRY(h, cudaGetLastError());
        h->launches += 1;
        W_r = Wn;
    }
    int it = 0;
    double* near = S->t;
    double* far = slip;
    if (h->precision == FBIM_FP32) {
        FBIM_TRY(near_field<float>(h, W_r, tol, max_iter, near, it));
        FBIM_TRY(apply_noise<float>(h, Z_w, seed, (unsigned)counter, far));
    } else {
        FBIM_TRY(near_field<double>(h, W_r, tol, max_iter, near, it));
        FBIM_TRY(apply_noise<double>(h, Z_w, seed, (unsigned)counter, far));
    }
    const double sc = std::sqrt(2.0 * kT / dt);
    k_combine<<<(n + 255) / 256, 256, 0, h->stream>>>(n, sc, near, sc, far, slip);
    h->launches += 1;
    FBIM_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    FBIM_TRY(tc_check(h));
    if (lanczos_iters) *lanczos_iters = it;
    return FBIM_OK;
}

}  // namespace fbim

extern "C" fbim_status fbim_brownian_slip(fbim_handle h, uint64_t seed, uint64_t counter, double kT, double dt,
                                          const double* W_r_dev, const double* Z_w_dev, double tol, int max_iter,
                                          double* slip_dev, int* lanczos_iters) {
    if (!h || !slip_dev || !(dt > 0) || !(kT >= 0) || !(tol > 0) || max_iter <= 0) return FBIM_ERR_INVALID_ARG;
    try {
        if (cudaSetDevice(h->device) != cudaSuccess) return FBIM_ERR_CUDA;
        return fbim::brownian_slip(h, seed, counter, kT, dt, W_r_dev, Z_w_dev, tol, max_iter, slip_dev,
                                   lanczos_iters);
    } catch (...) {
        h->fail("unexpected host exception in fbim_brownian_slip");
        return FBIM_ERR_SETUP;
    }
}

extern "C" fbim_status fbim_philox_normals(fbim_handle h, uint64_t seed, uint32_t stream, uint32_t counter,
                                           size_t n, double* out_dev) {
    if (!h || !out_dev) return FBIM_ERR_INVALID_ARG;
    if (cudaSetDevice(h->device) != cudaSuccess) return FBIM_ERR_CUDA;
    if (n == 0) return FBIM_OK;
    fbim::k_philox_normals<<<(unsigned)(((n + 1) / 2 + 255) / 256), 256, 0, h->stream>>>(n, seed, stream, counter, 0,
                                                                                    out_dev);
    FBIM_CUDA_TRY(h, cudaGetLastError());
    return FBIM_OK;
}

extern "C" fbim_status fbim_host_lanczos_sqrt(const double* alpha, const double* beta, int k, double wnorm,
                                              double* out) {
    if (!alpha || !out || k < 1 || (k > 1 && !beta)) return FBIM_ERR_INVALID_ARG;
    try {
        const std::vector<double> c = fbim::lanczos_sqrt_coeffs(alpha, beta, k, wnorm);
        std::copy(c.begin(), c.end(), out);
        return FBIM_OK;
    } catch (...) {
        return FBIM_ERR_SETUP;
    }
}
